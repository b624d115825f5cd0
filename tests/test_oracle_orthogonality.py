"""CPU pins of the oracle's orthogonality measure and restoration of the streaming factor.

The restoration replaces U_d by its polar factor; the pins check it against what the
mathematics fixes: the result has orthonormal columns, no matrix with orthonormal columns is
closer to U_d (compared with the QR factor and with random orthonormal perturbations of the
result), the reconstruction moves by exactly the amount added to the bound, Assumption 1(c) is
untouched, and an already orthonormal factor is left as it is."""

import math

import numpy as np

import oracle as O
from workloads import LowRankStream


def _state(T=40, seed=7, upto=None):
    """A stream of T slices, streamed up to slice upto (default T)."""
    s = LowRankStream((12, 10, 8), (3, 3, 2, 4), T, 1e-3, seed=seed)
    X = s.tensor(0, T)
    st = O.init_stream(X[..., :6].copy(order="F"), 2e-3)
    for t in range(6, T if upto is None else upto):
        O.stream_update(st, X[..., t].copy(order="F"))
    return st, X


def _perturbed(st, rng, size=1e-6):
    """The state with U_d pushed off orthonormality (as accumulated rounding would)."""
    U = st.Us[-1]
    st.Us[-1] = U + size * rng.standard_normal(U.shape)
    return st


def test_measure_is_zero_for_orthonormal_and_sees_a_perturbation():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((50, 6)))
    assert O.orthogonality_error(Q) < 1e-14
    E = 1e-7 * rng.standard_normal((50, 6))
    G = (Q + E).T @ (Q + E) - np.eye(6)
    assert abs(O.orthogonality_error(Q + E) - np.linalg.norm(G)) < 1e-20
    assert O.orthogonality_error(Q + E) > 1e-8


def test_restoration_is_the_nearest_orthonormal_factor():
    rng = np.random.default_rng(2)
    st, _ = _state()
    st = _perturbed(st, rng)
    U0 = st.Us[-1].copy()
    O.restore_orthogonality(st)
    U1 = st.Us[-1]
    assert O.orthogonality_error(U1) < 1e-13
    d1 = np.linalg.norm(U1 - U0)
    # the QR factor (signs matched) and nearby orthonormal matrices are no closer
    Qr, R = np.linalg.qr(U0)
    Qr = Qr * np.sign(np.diag(R))[None, :]
    assert d1 <= np.linalg.norm(Qr - U0) * (1 + 1e-9)
    for _ in range(20):
        A = rng.standard_normal((U1.shape[1], U1.shape[1])) * 1e-4
        Rot = np.linalg.qr(np.eye(U1.shape[1]) + (A - A.T))[0]
        Rot = Rot * np.sign(np.diag(np.linalg.qr(np.eye(U1.shape[1]) + (A - A.T))[1]))[None, :]
        assert d1 <= np.linalg.norm(U1 @ Rot - U0) * (1 + 1e-9)


def test_bound_grows_by_the_reconstruction_change_and_assumption_1_holds():
    rng = np.random.default_rng(3)
    st, X = _state()
    st = _perturbed(st, rng)
    Xh0 = O.reconstruct(st.C, st.Us)
    b0 = math.sqrt(st.err2)
    C0, S0, V0 = st.C.copy(), st.S.copy(), st.V.copy()
    change = O.restore_orthogonality(st)
    Xh1 = O.reconstruct(st.C, st.Us)
    assert abs(np.linalg.norm(Xh1 - Xh0) - change) <= 1e-12 * np.linalg.norm(Xh0)
    assert math.sqrt(st.err2) == b0 + change
    # C, S and V (so Assumption 1(c) as it held) are left exactly as they were
    assert np.array_equal(st.C, C0) and np.array_equal(st.S, S0) and np.array_equal(st.V, V0)


def test_orthonormal_factor_is_left_alone_and_the_stream_goes_on():
    st, X = _state(T=40, upto=30)
    e0 = O.orthogonality_error(st.Us[-1])
    assert e0 < 1e-12       # FP64 streaming keeps U_d orthonormal to rounding here
    U0 = st.Us[-1].copy()
    change = O.restore_orthogonality(st)
    assert np.linalg.norm(st.Us[-1] - U0) < 1e-12 and change < 1e-10
    for t in range(30, 40):
        O.stream_update(st, X[..., t].copy(order="F"))
    assert np.linalg.norm(X - O.reconstruct(st.C, st.Us)) <= math.sqrt(st.err2) * (1 + 1e-12)
