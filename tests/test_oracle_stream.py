"""Pins of the oracle's streaming update (Alg. 4, Alg. 5) against the paper's invariants and
closed forms: exact-rank recovery, Prop. 2, the ST-HOSVD error split of the new slice, the error
bound of Alg. 5, Assumption 1 carried across updates, and the d = 2 (matrix) special case."""

import json
import math
import os

import numpy as np
import pytest

import oracle as O
from workloads import CONFIG1, LowRankStream, SineWave, config1_tensor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def c1_run():
    s = config1_tensor()
    X = s.tensor(0, CONFIG1["steps"])
    st = O.init_stream(X[..., :CONFIG1["n_init"]], CONFIG1["tau"])
    snaps = []
    for t in range(CONFIG1["n_init"], CONFIG1["steps"]):
        O.stream_update(st, X[..., t])
        Xh = O.reconstruct(st.C, st.Us)
        Xs = X[..., : t + 1]
        snaps.append(dict(ranks=st.ranks, true2=float(np.sum((Xs - Xh) ** 2)),
                          bound2=st.err2, norm2=float(np.sum(Xs * Xs)), data_norm2=st.data_norm2,
                          Us=[U.copy() for U in st.Us], S=st.S.copy(), V=st.V.copy(), C=st.C.copy(),
                          log=st.log[-1]))
    return X, st, snaps


def test_config1_exact_ranks_every_step(c1_run):
    """Exact multilinear rank (4,4,3,6) + 1e-4 noise, tau = 1e-3: the ranks never move."""
    _, st, snaps = c1_run
    assert st.log[0]["ranks"] == (4, 4, 3, 6)
    for s in snaps:
        assert s["ranks"] == (4, 4, 3, 6)


def test_config1_error_bound_every_step(c1_run):
    """Alg. 5 guarantee ||X~ - X^~|| <= tau ||X~|| after every slice; the bookkeeping (Prop. 1,
    App. D) is an upper bound of the true error, and the error sits at the noise level."""
    _, _, snaps = c1_run
    tau = CONFIG1["tau"]
    for s in snaps:
        assert math.sqrt(s["true2"]) <= tau * math.sqrt(s["norm2"])
        assert s["true2"] <= s["bound2"] * (1 + 1e-9)
        assert abs(s["data_norm2"] - s["norm2"]) <= 1e-12 * s["norm2"]
    rel = math.sqrt(snaps[-1]["true2"] / snaps[-1]["norm2"])
    assert 0.5e-4 < rel < 2e-4


def test_config1_invariants_every_step(c1_run):
    """Assumption 1 after each update: orthonormal U_k, row-orthonormal V_(d), S > 0."""
    _, _, snaps = c1_run
    for s in snaps:
        for U in s["Us"]:
            np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-10)
        d = s["C"].ndim
        Vd = O.unfold(s["V"], d - 1)
        np.testing.assert_allclose(Vd @ Vd.T, np.eye(Vd.shape[0]), atol=1e-10)
        assert np.all(s["S"] > 0)
        if s["log"]["isvd"].augmented:
            # c8: C = V x_d S holds exactly on steps whose residual e was used
            np.testing.assert_allclose(O.ttm(s["V"], np.diag(s["S"]), d - 1), s["C"],
                                       atol=1e-9 * np.linalg.norm(s["C"]))


def test_streaming_vs_batch_sthosvd(c1_run):
    """The batch ST-HOSVD of all 40 slices at the same tau finds the same exact ranks."""
    X, st, _ = c1_run
    res = O.sthosvd(X, CONFIG1["tau"])
    assert res.ranks == st.ranks


def _growth_case():
    """A stream whose spatial ranks must grow: the first slices avoid part of the mode-1 basis."""
    rng = np.random.default_rng(11)
    n = (9, 8, 7)
    A = [np.linalg.qr(rng.standard_normal((m, 4)))[0] for m in n]
    T = 14
    X = np.zeros(n + (T,), order="F")
    for t in range(T):
        r_use = 2 if t < 6 else 4
        G = rng.standard_normal((r_use, r_use, r_use))
        X[..., t] = O.reconstruct(G, [a[:, :r_use] for a in A])
    X += 1e-6 * rng.standard_normal(X.shape)
    return X


def test_prop2_and_slice_pythagoras_on_rank_growth():
    """Prop. 2: the spatial updates keep C x U unchanged (C_k x_k U~_k = C_{k-1} x_k U_k);
    D*_k = D*_{k-1} x_k U~_k^T; ||Y - D*_{d-1} x U~||^2 = sum_k ||D*_{k-1} - D*_k x_k U~_k||^2."""
    X = _growth_case()
    st = O.init_stream(X[..., :6], 1e-3)
    assert st.ranks[:3] == (2, 2, 2)
    Y = X[..., 6]
    d = st.d
    eps = st.tau * np.linalg.norm(Y) / math.sqrt(d)
    C, V, D = st.C, st.V, Y.reshape(Y.shape + (1,), order="F")
    Us = list(st.Us)
    old = O.reconstruct(st.C, st.Us)
    disc = 0.0
    grew = False
    for k in range(d - 1):
        Uk_old = Us[k]
        Uk, Ck, Dk, Vk, info = O.non_streaming_update(k, Us[k], C, D, V, eps)
        grew |= info.grew
        np.testing.assert_allclose(O.ttm(Ck, Uk, k), O.ttm(C, Uk_old, k), atol=1e-12)
        np.testing.assert_allclose(Dk, O.ttm(D, Uk.T, k), atol=1e-10)
        np.testing.assert_allclose(Uk.T @ Uk, np.eye(Uk.shape[1]), atol=1e-9)
        piece = float(np.sum((D - O.ttm(Dk, Uk, k)) ** 2))
        assert abs(piece - info.discarded) <= 1e-9 * np.sum(Y * Y)
        assert piece <= eps ** 2 * (1 + 1e-9)
        disc += piece
        Us[k], C, D, V = Uk, Ck, Dk, Vk
    assert grew
    np.testing.assert_allclose(O.reconstruct(C, Us), old, atol=1e-10)
    Yh = O.reconstruct(D, Us[:-1] + [np.ones((1, 1))])
    assert abs(float(np.sum((Y.reshape(Yh.shape, order="F") - Yh) ** 2)) - disc) <= 1e-9 * np.sum(Y * Y)


def test_rank_growth_stream_meets_bound():
    X = _growth_case()
    tau = 1e-3
    st = O.init_stream(X[..., :6], tau)
    prev = st.ranks
    for t in range(6, X.shape[-1]):
        O.stream_update(st, X[..., t])
        assert all(a >= b for a, b in zip(st.ranks[:-1], prev[:-1]))   # spatial ranks only grow
        assert st.ranks[-1] >= prev[-1] - 0
        prev = st.ranks
        Xh = O.reconstruct(st.C, st.Us)
        Xs = X[..., : t + 1]
        assert np.linalg.norm(Xs - Xh) <= tau * np.linalg.norm(Xs)
    assert st.ranks[:3] == (4, 4, 4)


def test_matrix_stream_d2_matches_svd():
    """d = 2: Alg. 5 reduces to column-basis growth + Brand's ISVD; with tiny tau on an exact
    rank-5 matrix it reproduces the singular values and the matrix."""
    rng = np.random.default_rng(12)
    n, T, r = 20, 30, 5
    A = rng.standard_normal((n, r)) @ rng.standard_normal((r, T))
    st = O.init_stream(A[:, :3].copy(order="F"), 1e-6)
    for t in range(3, T):
        O.stream_update(st, A[:, t].copy())
    sv = np.linalg.svd(A, compute_uv=False)
    assert st.ranks == (5, 5)
    Ah = O.reconstruct(st.C, st.Us)
    np.testing.assert_allclose(Ah, A, atol=1e-8 * np.linalg.norm(A))
    core_sv = np.linalg.svd(st.C, compute_uv=False)
    np.testing.assert_allclose(core_sv, sv[:5], rtol=1e-8)


def test_zero_slice_changes_nothing_but_adds_a_zero_row():
    s = LowRankStream((6, 5, 4), (2, 2, 2, 3), 8, 1e-3, seed=3)
    X = s.tensor(0, 8)
    st = O.init_stream(X[..., :5], 1e-2)
    before = O.reconstruct(st.C, st.Us)
    ranks = st.ranks
    O.stream_update(st, np.zeros(X.shape[:-1], order="F"))
    assert st.ranks == ranks
    after = O.reconstruct(st.C, st.Us)
    np.testing.assert_allclose(after[..., :-1], before, atol=1e-12)
    np.testing.assert_allclose(after[..., -1], 0.0, atol=1e-14)


def test_slice_in_span_needs_no_new_basis():
    s = LowRankStream((6, 5, 4), (2, 2, 2, 3), 8, 0.0, seed=4)
    X = s.tensor(0, 8)
    st = O.init_stream(X[..., :5], 1e-4)
    Y = 0.3 * X[..., 1] - 1.2 * X[..., 3]
    O.stream_update(st, Y)
    lg = st.log[-1]
    assert not any(m.grew for m in lg["modes"])
    assert lg["isvd"].q < 1e-10 * np.linalg.norm(Y)


def test_golden_sine_wave_batch_ranks_table1():
    """Table 1: batch ST-HOSVD of the noisy sine-wave tensor at tau = 1e-2 gives ranks (11,11,15);
    the streaming run from an initial ST-HOSVD meets the same tolerance with ranks >= those.
    Reduced streaming length (the exact ranks do not depend on it)."""
    with open(os.path.join(GOLDEN, "table1_sine_wave.json")) as f:
        g = json.load(f)
    sw = SineWave(n=tuple(g["n"]), steps_each=g["steps_each_reduced"], freqs_a=tuple(g["freqs_a"]),
                  freqs_b=tuple(g["freqs_b"]), noise=g["noise"])
    X = np.stack([sw.slice(t) for t in range(sw.steps)], axis=-1)
    res = O.sthosvd(X, g["tau"])
    assert list(res.ranks) == g["batch_ranks"]
    st = O.init_stream(X[..., : g["n_init_reduced"]], g["tau"])
    for t in range(g["n_init_reduced"], sw.steps):
        O.stream_update(st, X[..., t])
    assert all(a >= b for a, b in zip(st.ranks, res.ranks))
    Xh = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(X - Xh) <= g["tau"] * np.linalg.norm(X)
