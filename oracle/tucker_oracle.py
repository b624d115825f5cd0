"""FP64 CPU oracle: batch ST-HOSVD and the streaming ST-HOSVD update, written from the paper.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline, never by the product path. It shares no code with the CUDA library.

Paper: De, Li, Kolla, Phipps, "Efficient Computation of Tucker Decomposition for Streaming
Scientific Data Compression" (arXiv 2308.16395).

Conventions
-----------
* A d-way tensor is a NumPy array of shape (n_1, ..., n_d) indexed in paper order.
* The mode-k matricization X_(k) is column-major over the remaining modes (Sec. 2.1): the column
  index of X(i_1..i_d) is i_1 + n_1 (i_2 + n_2 (...)) with mode k skipped.
* ``k`` is 0-based in code (paper mode k+1).
* Everything is float64. Library primitives used as single steps: ``@`` (matmul),
  ``np.linalg.eigh`` (the eig of Alg. 1), ``np.linalg.qr`` (the QR of Alg. 3).

Readings of the paper where it is silent, garbled or ambiguous:
  R1 eigenvalues sorted descending, ties broken by the smaller index (Alg. 1);
  R2 ST-HOSVD keeps at least rank 1 per mode; Alg. 4's r'_k is clamped to n_k - r_k;
  R3 Alg. 1 returns singular values sqrt(lambda) (negative round-off eigenvalues clamped at 0
     for the square root; the tail sums use the eigenvalues as computed);
  R4 TruncatedSVD(S', 0) of Alg. 3 keeps the numerically nonzero part: eigenvalues of S'S'^T
     above m * u * lambda_1 (m = rows of S', u = 2^-53), and never more than S' has columns;
  R5 the orthogonality check of Alg. 3 tests the first column only, with eps_m = 1e-10;
  R6 the augmented spatial factors are not re-orthogonalised (Alg. 4 as printed);
  R7 the core update uses the explicit product U~_d(1:n_d,:)^T U_d (Alg. 5, last step);
  R8 the "<=" tests of Alg. 3 and Alg. 4 are taken literally;
  R9 index typos of Sec. 3.3 (P_{k-1}, L_{k-1} in the concatenation) read as P_k, L_k;
  R10 all-zero initial data is rejected (Assumption 1(c) needs S > 0);
  R11 re-compression (Sec. 5 observes over-estimated streamed ranks, Tables 1-2): Alg. 2 on the
      current representation, budget eps' = (tau_total ||X|| - b) / sqrt(d), new bound
      b + ||X^ - X^'|| (``recompress``);
  R12 orthogonality of U_d (Sec. 3.1 names the loss of orthogonality in U' U''): restored by the
      polar factor, C, S and V kept, the reconstruction's change added to the bound
      (``restore_orthogonality``);
  R13 block update (the Conclusions name several slices at once as future work): Alg. 4 on the
      block as one tensor with eps = tau ||Y_b|| / sqrt(d), then one Alg. 3 step per slice with
      eps / sqrt(B), so a block adds at most tau^2 ||Y_b||^2 (``block_update``).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

U64 = np.finfo(np.float64).eps / 2.0  # unit roundoff 2^-53


# ---------------------------------------------------------------------------------------------
# Tensor algebra (Sec. 2.1)
# ---------------------------------------------------------------------------------------------

def unfold(X: np.ndarray, k: int) -> np.ndarray:
    """Mode-k matricization X_(k) (n_k x prod_{l != k} n_l), column-major columns (Sec. 2.1)."""
    return np.moveaxis(X, k, 0).reshape(X.shape[k], -1, order="F")


def fold(M: np.ndarray, k: int, shape) -> np.ndarray:
    """Inverse of :func:`unfold`: the tensor of ``shape`` whose mode-k matricization is M."""
    shape = tuple(shape)
    rest = shape[:k] + shape[k + 1:]
    T = M.reshape((shape[k],) + rest, order="F")
    return np.moveaxis(T, 0, k)


def ttm(X: np.ndarray, A: np.ndarray, k: int) -> np.ndarray:
    """Tensor-times-matrix Y = X x_k A, defined by Y_(k) = A X_(k) (Sec. 2.1)."""
    shape = list(X.shape)
    shape[k] = A.shape[0]
    return fold(A @ unfold(X, k), k, shape)


def reconstruct(C: np.ndarray, Us) -> np.ndarray:
    """X^ = C x_1 U_1 ... x_d U_d (Eq. tucker_def, Sec. 2.2)."""
    X = C
    for k, U in enumerate(Us):
        X = ttm(X, U, k)
    return X


# ---------------------------------------------------------------------------------------------
# Alg. 1: truncated Gram SVD
# ---------------------------------------------------------------------------------------------

@dataclass
class TSVD:
    r: int
    U: np.ndarray          # m x r left singular vectors
    s: np.ndarray          # r singular values sqrt(lambda) (R3)
    lam: np.ndarray        # all m eigenvalues of A A^T, descending (R1)
    discarded: float       # lambda_{r+1} + ... + lambda_m (the squared error of the truncation)
    V: np.ndarray | None = None  # n x r right singular vectors A^T U S^-1 (optional)


def _tail_sums(lam: np.ndarray) -> np.ndarray:
    """tails[l] = lambda_{l+1} + ... + lambda_m for l = 0..m (tails[m] = 0)."""
    m = lam.shape[0]
    tails = np.zeros(m + 1)
    for l in range(m - 1, -1, -1):
        tails[l] = tails[l + 1] + lam[l]
    return tails


def truncated_svd(A: np.ndarray, eps: float, *, min_rank: int = 0, max_rank: int | None = None,
                  numerical: bool = False, want_v: bool = False) -> TSVD:
    """Alg. 1 (TruncatedSVD): Gram A A^T, eig, rank r = min{l : lambda_{l+1}+...+lambda_m <= eps^2}.

    ``numerical=True`` is the exact compact SVD "TruncatedSVD(S', 0)" of Alg. 3 under reading R4.
    ``min_rank`` / ``max_rank`` implement the clamps of reading R2.
    """
    m = A.shape[0]
    G = A @ A.T
    lam, P = np.linalg.eigh(G)
    order = np.argsort(-lam, kind="stable")  # descending; ties keep the smaller index first (R1)
    lam = lam[order]
    P = P[:, order]
    if numerical:
        cap = min(m, A.shape[1])
        thresh = m * U64 * lam[0] if m > 0 else 0.0
        r = int(np.sum(lam[:cap] > thresh)) if lam.size and lam[0] > 0 else 0
    else:
        tails = _tail_sums(lam)
        r = m
        for l in range(m + 1):
            if tails[l] <= eps * eps:
                r = l
                break
    r = max(r, min_rank)
    if max_rank is not None:
        r = min(r, max_rank)
    U = P[:, :r]
    s = np.sqrt(np.maximum(lam[:r], 0.0))
    discarded = float(np.sum(lam[r:]))
    V = None
    if want_v:
        V = (A.T @ U) / s[None, :]
    return TSVD(r=r, U=U, s=s, lam=lam, discarded=discarded, V=V)


# ---------------------------------------------------------------------------------------------
# Alg. 2: ST-HOSVD, plus the streaming-mode factorization of Assumption 1(c)
# ---------------------------------------------------------------------------------------------

@dataclass
class SthosvdResult:
    C: np.ndarray
    Us: list
    ranks: tuple
    S: np.ndarray              # r_d singular values of the last partial-core unfolding
    V: np.ndarray              # tensor of the shape of C with V_(d) = S^-1 C_(d) (row-orthonormal)
    discarded: list            # per-mode discarded energy lambda_{r+1}+... (Eq. partial_core_error)
    eps: float
    norm2: float


def sthosvd(X: np.ndarray, tau: float) -> SthosvdResult:
    """Alg. 2 with eps = tau ||X|| / sqrt(d); modes processed in order 1..d (streaming mode last).

    From the last mode's truncated Gram SVD, S = diag(sqrt(lambda_1..r_d)) and V_(d) = S^-1 C_(d),
    the core factorization of Assumption 1(c) (Sec. 3.2, Eq. tucker-core-factorization).
    """
    d = X.ndim
    norm2 = float(np.sum(X * X))
    if norm2 == 0.0:
        raise ValueError("all-zero initial data: Assumption 1(c) needs S > 0 (reading R10)")
    eps = tau * math.sqrt(norm2) / math.sqrt(d)
    C = X
    Us = []
    discarded = []
    last = None
    for k in range(d):
        res = truncated_svd(unfold(C, k), eps, min_rank=1)
        Us.append(res.U)
        discarded.append(res.discarded)
        C = ttm(C, res.U.T, k)
        last = res
    S = last.s.copy()
    Vd = unfold(C, d - 1) / S[:, None]
    V = fold(Vd, d - 1, C.shape)
    return SthosvdResult(C=C, Us=Us, ranks=tuple(C.shape), S=S, V=V, discarded=discarded,
                         eps=eps, norm2=norm2)


# ---------------------------------------------------------------------------------------------
# Alg. 3: incremental SVD (new row b appended to A ~ U S V^T)
# ---------------------------------------------------------------------------------------------

@dataclass
class IsvdInfo:
    p: np.ndarray
    q: float
    augmented: bool      # q > eps: new basis vector v added to V
    qr: bool             # re-orthogonalisation by QR happened
    ortho: float         # |V(:,1)^T v| (0 if not augmented)
    dropped: float       # energy of S' removed by the numerical-rank cut (R4)
    r_new: int


def isvd(U: np.ndarray, S: np.ndarray, V: np.ndarray, b: np.ndarray, eps: float,
         eps_m: float = 1e-10):
    """Alg. 3. U: m x r, S: r singular values, V: n x r, b: new row (n). Returns U~, S~, V~, info."""
    r = S.shape[0]
    p = V.T @ b
    e = b - V @ p
    q = float(np.linalg.norm(e))
    ortho = 0.0
    did_qr = False
    if q <= eps:
        Sp = np.vstack([np.diag(S), p[None, :]])              # (r+1) x r
        Vp = V
        augmented = False
    else:
        v = e / q
        Sp = np.zeros((r + 1, r + 1))
        Sp[:r, :r] = np.diag(S)
        Sp[r, :r] = p
        Sp[r, r] = q
        Vp = np.hstack([V, v[:, None]])
        augmented = True
        ortho = abs(float(V[:, 0] @ v)) if r > 0 else 0.0
        if ortho > eps_m:
            Q, R = np.linalg.qr(Vp)
            Vp = Q
            Sp = Sp @ R.T
            did_qr = True
    res = truncated_svd(Sp, 0.0, numerical=True, want_v=True)   # exact compact SVD (R4)
    U2, St, V2 = res.U, res.s, res.V
    Ut = np.vstack([U @ U2[:r, :], U2[r:r + 1, :]])
    Vt = Vp @ V2
    info = IsvdInfo(p=p, q=q, augmented=augmented, qr=did_qr, ortho=ortho,
                    dropped=res.discarded, r_new=res.r)
    return Ut, St, Vt, info


# ---------------------------------------------------------------------------------------------
# Alg. 4: non-streaming mode update
# ---------------------------------------------------------------------------------------------

@dataclass
class ModeInfo:
    k: int
    e_norm2: float       # ||E_k||_F^2
    grew: bool           # ||E_k|| > eps
    r_add: int           # r'_k
    discarded: float     # ||D*_{k-1} - D*_k x_k U~_k||^2 = ||E_k||^2 - sum of kept eigenvalues
    lam: np.ndarray | None = None


def _pad_zeros(T: np.ndarray, k: int, add: int) -> np.ndarray:
    """PadWithZeros: append ``add`` zero slices along mode k (Eqs. pad_core_with_zeros, pad_singular_vectors_with_zeros)."""
    if add == 0:
        return T
    shape = list(T.shape)
    shape[k] = add
    return np.concatenate([T, np.zeros(shape)], axis=k)


def non_streaming_update(k: int, Uk: np.ndarray, C: np.ndarray, D: np.ndarray, V: np.ndarray,
                         eps: float):
    """Alg. 4 for mode k (0-based): returns U~_k, C_k, D*_k, V_k, info."""
    P = ttm(D, Uk.T, k)                  # P_k = D*_{k-1} x_k U_k^T
    E = D - ttm(P, Uk, k)                # E_k = D*_{k-1} - P_k x_k U_k
    e2 = float(np.sum(E * E))
    if math.sqrt(e2) <= eps:             # R8
        return Uk, C, P, V, ModeInfo(k=k, e_norm2=e2, grew=False, r_add=0, discarded=e2)
    nk, rk = Uk.shape
    res = truncated_svd(unfold(E, k), eps, max_rank=nk - rk)     # R2 clamp
    W = res.U
    L = ttm(E, W.T, k)                   # L_k = E_k x_k W_k^T
    Ut = np.hstack([Uk, W])              # U~_k = [U_k W_k] (R6: no re-orthogonalisation)
    Ck = _pad_zeros(C, k, res.r)
    Dk = np.concatenate([P, L], axis=k)  # Concatenate(k, P_k, L_k) (R9)
    Vk = _pad_zeros(V, k, res.r)
    info = ModeInfo(k=k, e_norm2=e2, grew=True, r_add=res.r, discarded=res.discarded, lam=res.lam)
    return Ut, Ck, Dk, Vk, info


# ---------------------------------------------------------------------------------------------
# Streaming state and Alg. 5
# ---------------------------------------------------------------------------------------------

@dataclass
class StreamState:
    """The state of Assumption 1: core C, factors U_1..U_d, S, V with C = V x_d S."""

    C: np.ndarray
    Us: list
    S: np.ndarray
    V: np.ndarray
    tau: float
    eps_m: float = 1e-10
    err2: float = 0.0          # running squared-error bookkeeping (Prop. 1, Prop. 2, App. D)
    data_norm2: float = 0.0    # ||X~||_F^2 of all data seen
    log: list = field(default_factory=list)

    @property
    def d(self) -> int:
        return self.C.ndim

    @property
    def ranks(self) -> tuple:
        return tuple(self.C.shape)

    @property
    def n_d(self) -> int:
        return self.Us[-1].shape[0]


def init_stream(X: np.ndarray, tau: float, eps_m: float = 1e-10) -> StreamState:
    """Initial ST-HOSVD (Alg. 2) of the first slices X (n_1 x ... x n_{d-1} x n_init)."""
    res = sthosvd(X, tau)
    st = StreamState(C=res.C, Us=res.Us, S=res.S, V=res.V, tau=tau, eps_m=eps_m,
                     err2=float(sum(res.discarded)), data_norm2=res.norm2)
    st.log.append(dict(kind="init", ranks=res.ranks, eps=res.eps, discarded=res.discarded))
    return st


def stream_update(st: StreamState, Y: np.ndarray) -> StreamState:
    """Alg. 5: assimilate one slice Y (n_1 x ... x n_{d-1}) into the state, in place."""
    d = st.d
    y2 = float(np.sum(Y * Y))
    eps = st.tau * math.sqrt(y2) / math.sqrt(d)
    C = st.C
    D = Y.reshape(Y.shape + (1,), order="F")      # D*_0 = Y as an n_1 x ... x n_{d-1} x 1 tensor
    V = st.V
    Us = list(st.Us)
    modes = []
    for k in range(d - 1):
        Us[k], C, D, V, info = non_streaming_update(k, Us[k], C, D, V, eps)
        modes.append(info)
    dvec = D.reshape(-1, order="F")               # d = vec(D*_{d-1})
    rd = C.shape[-1]
    Vmat = V.reshape(-1, rd, order="F")           # V = V_{d-1,(d)}^T
    Ud = Us[-1]
    nd = Ud.shape[0]
    Ut, St, Vt, info = isvd(Ud, st.S, Vmat, dvec, eps, st.eps_m)
    rt = St.shape[0]
    spatial = C.shape[:-1]
    M = Ut[:nd, :].T @ Ud                         # U~_d(1:n_d,:)^T U_d            (R7)
    Cd = M @ unfold(C, d - 1) + np.outer(Ut[nd, :], dvec)
    st.C = fold(Cd, d - 1, spatial + (rt,))
    Us[-1] = Ut
    st.Us = Us
    st.S = St
    st.V = Vt.reshape(spatial + (rt,), order="F")
    disc = sum(m.discarded for m in modes)
    st.err2 += disc + (0.0 if info.augmented else info.q ** 2) + info.dropped
    st.data_norm2 += y2
    st.log.append(dict(kind="update", eps=eps, y2=y2, modes=modes, isvd=info, ranks=st.ranks))
    return st


def reconstruct_slices(st: StreamState, t0: int, t1: int) -> np.ndarray:
    """X^(:, ..., t) for t in [t0, t1): C x_1 U_1 ... x_{d-1} U_{d-1} x_d U_d(t0:t1, :)."""
    Us = list(st.Us[:-1]) + [st.Us[-1][t0:t1, :]]
    return reconstruct(st.C, Us)


# ---------------------------------------------------------------------------------------------
# Re-compression of a streaming state (batch ST-HOSVD of the current Tucker representation)
# ---------------------------------------------------------------------------------------------

def recompress(st: StreamState, tau_total: float) -> StreamState:
    """Re-truncate the Tucker representation of the state by the batch ST-HOSVD (Alg. 2), in place.

    The streaming ranks are over-estimates of what the data needs (Sec. 5, Tables 1-2); running
    Alg. 2 on the current representation X^ = C x_1 U_1 ... x_d U_d lowers them again. With every
    U_k orthonormal, the ST-HOSVD of X^ is the ST-HOSVD of the core C with the factors multiplied
    in: the mode-k Gram of X^'s partially projected unfolding is U_k G_k U_k^T for the
    corresponding Gram G_k of C's, so its eigenvectors are U_k Q_k with Q_k those of G_k. The
    budget: the running bound b (Prop. 1, Prop. 2) may grow to tau_total ||X||, and since
    ||X - X^'|| <= ||X - X^|| + ||X^ - X^'|| the re-compression may discard (tau_total ||X|| - b)^2
    in all, eps' = (tau_total ||X|| - b) / sqrt(d) per mode (Alg. 2's rule). The new bound is
    b + ||X^ - X^'||. The state keeps Assumption 1: S and V from the last mode's truncated SVD.
    """
    d = st.d
    b = math.sqrt(max(st.err2, 0.0))
    budget = tau_total * math.sqrt(st.data_norm2) - b
    if budget <= 0.0:
        raise ValueError("tau_total leaves no error budget beyond the running bound")
    eps = budget / math.sqrt(d)
    C = st.C
    Qs = []
    disc = 0.0
    last = None
    for k in range(d):
        res = truncated_svd(unfold(C, k), eps, min_rank=1)
        Qs.append(res.U)
        disc += res.discarded
        C = ttm(C, res.U.T, k)
        last = res
    st.Us = [U @ Q for U, Q in zip(st.Us, Qs)]
    st.C = C
    st.S = last.s.copy()
    st.V = fold(unfold(C, d - 1) / st.S[:, None], d - 1, C.shape)
    st.err2 = (b + math.sqrt(disc)) ** 2
    st.log.append(dict(kind="recompress", ranks=st.ranks, eps=eps, discarded=disc))
    return st


# ---------------------------------------------------------------------------------------------
# Orthogonality of the streaming factor (the loss the paper flags in the incremental SVD)
# ---------------------------------------------------------------------------------------------

def orthogonality_error(U: np.ndarray) -> float:
    """||U^T U - I||_F: how far a factor's columns are from orthonormal. Sec. 3.1 remarks that
    forming the new left singular vectors as a product U' U'' (Alg. 3) may lose orthogonality over
    many incremental updates."""
    r = U.shape[1]
    return float(np.linalg.norm(U.T @ U - np.eye(r)))


def restore_orthogonality(st: StreamState) -> float:
    """Replace the streaming factor U_d by its nearest matrix with orthonormal columns (the polar
    factor W Z^T of U_d = W Sigma Z^T, from numpy's SVD), in place, keeping C, S, V (Assumption 1
    is untouched). The reconstruction changes by (U_d' - U_d) C_(d), of norm ||(U_d' - U_d) S||_F
    since V_(d) is row-orthonormal; that amount is added to the running bound (triangle
    inequality). Returns it."""
    U = st.Us[-1]
    W, _, Zt = np.linalg.svd(U, full_matrices=False)
    Un = W @ Zt
    change = float(np.linalg.norm((Un - U) * st.S[None, :]))
    st.Us[-1] = Un
    b = math.sqrt(max(st.err2, 0.0))
    st.err2 = (b + change) ** 2
    st.log.append(dict(kind="restore_orthogonality", change=change))
    return change


# ---------------------------------------------------------------------------------------------
# Several slices at once (the block update the Conclusions name as future work)
# ---------------------------------------------------------------------------------------------

def block_update(st: StreamState, Yb: np.ndarray) -> StreamState:
    """Assimilate B slices Yb (n_1 x ... x n_{d-1} x B) at once, in place.

    The spatial modes see the block as one tensor with a trailing mode of size B: Alg. 4 for each
    k with eps = tau ||Yb|| / sqrt(d) (Alg. 5's rule applied to the block), so a mode's residual
    Gram, rank cut and augmentation cover all B slices together. The streaming mode then takes
    the B projected slices as B new rows, one incremental SVD step (Alg. 3) each, in slice order,
    with the streaming share of the block's budget split evenly: eps_r = eps / sqrt(B) per row.
    The block's added squared error is then at most (d - 1) eps^2 + B eps_r^2 = tau^2 ||Yb||^2,
    Alg. 5's guarantee for the block (reading of the future-work sentence; B = 1 is Alg. 5).
    """
    d = st.d
    B = Yb.shape[-1]
    y2 = float(np.sum(Yb * Yb))
    eps = st.tau * math.sqrt(y2) / math.sqrt(d)
    C = st.C
    D = Yb                                        # D*_0: the block, n_1 x ... x n_{d-1} x B
    V = st.V
    Us = list(st.Us)
    modes = []
    for k in range(d - 1):
        Us[k], C, D, V, info = non_streaming_update(k, Us[k], C, D, V, eps)
        modes.append(info)
    eps_r = eps / math.sqrt(B)
    spatial = C.shape[:-1]
    S = st.S
    err = sum(m.discarded for m in modes)
    rows = []
    for b in range(B):
        dvec = D[..., b].reshape(-1, order="F")  # slice b of D*_{d-1}
        rd = C.shape[-1]
        Vmat = V.reshape(-1, rd, order="F")
        Ud = Us[-1]
        nd = Ud.shape[0]
        Ut, St, Vt, info = isvd(Ud, S, Vmat, dvec, eps_r, st.eps_m)
        rt = St.shape[0]
        M = Ut[:nd, :].T @ Ud                     # U~_d(1:n_d,:)^T U_d            (R7)
        Cd = M @ unfold(C, d - 1) + np.outer(Ut[nd, :], dvec)
        C = fold(Cd, d - 1, spatial + (rt,))
        Us[-1] = Ut
        S = St
        V = Vt.reshape(spatial + (rt,), order="F")
        err += (0.0 if info.augmented else info.q ** 2) + info.dropped
        rows.append(info)
    st.C, st.Us, st.S, st.V = C, Us, S, V
    st.err2 += err
    st.data_norm2 += y2
    st.log.append(dict(kind="block", eps=eps, eps_row=eps_r, y2=y2, modes=modes, rows=rows,
                       ranks=st.ranks, added=err))
    return st
