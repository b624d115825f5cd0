"""CPU pins of the oracle's re-compression (the batch ST-HOSVD of Alg. 2 run again on a streaming
state's Tucker representation).

The pins do not reuse the oracle's own route: the re-compressed state is checked against an
ST-HOSVD of the full reconstruction written here from numpy's SVD, against the error bound on
the data, against Assumption 1(c), and by streaming on after it.
"""

import math

import numpy as np
import pytest

import oracle as O
from workloads import LowRankStream


def _svd_sthosvd(X, eps):
    """ST-HOSVD by truncated SVDs of the unfoldings (numpy.linalg.svd): ranks, reconstruction."""
    C = X
    Us = []
    for k in range(X.ndim):
        M = np.moveaxis(C, k, 0).reshape(C.shape[k], -1, order="F")
        u, s, _ = np.linalg.svd(M, full_matrices=False)
        tails = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])
        r = next(l for l in range(len(s) + 1) if tails[l] <= eps * eps)
        r = max(r, 1)
        Us.append(u[:, :r])
        C = O.ttm(C, u[:, :r].T, k)
    Xh = C
    for k, U in enumerate(Us):
        Xh = O.ttm(Xh, U, k)
    return tuple(C.shape), Xh


def _overfit_state(seed=3, T=30, upto=None):
    """A stream whose ranks the updates over-estimate: exact rank (3, 3, 2, 4) plus noise at a
    tight tolerance, so the updates also pick up noise directions. Streams slices 0..upto-1."""
    s = LowRankStream((14, 12, 10), (3, 3, 2, 4), T, 3e-3, seed=seed)
    X = s.tensor(0, T)
    st = O.init_stream(X[..., :6].copy(order="F"), 2e-3)
    for t in range(6, T if upto is None else upto):
        O.stream_update(st, X[..., t].copy(order="F"))
    return st, X


def test_recompress_equals_svd_sthosvd_of_the_reconstruction():
    st, X = _overfit_state()
    Xh = O.reconstruct(st.C, st.Us)
    b = math.sqrt(st.err2)
    tau_total = 2.0 * b / math.sqrt(st.data_norm2)
    eps = (tau_total * math.sqrt(st.data_norm2) - b) / math.sqrt(st.d)
    ranks_ref, Xh_ref = _svd_sthosvd(Xh, eps)
    O.recompress(st, tau_total)
    assert st.ranks == ranks_ref
    Xh_new = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(Xh_new - Xh_ref) <= 1e-10 * np.linalg.norm(Xh_ref)


def test_recompress_bound_covers_the_true_error_and_ranks_shrink():
    st, X = _overfit_state()
    before = st.ranks
    tau_total = 1.5 * math.sqrt(st.err2 / st.data_norm2)
    O.recompress(st, tau_total)
    assert all(a <= b for a, b in zip(st.ranks, before))
    assert st.ranks != before                      # the over-estimated ranks come down
    Xh = O.reconstruct(st.C, st.Us)
    true = np.linalg.norm(X - Xh)
    assert true <= math.sqrt(st.err2) * (1 + 1e-12)
    assert math.sqrt(st.err2) <= tau_total * math.sqrt(st.data_norm2) * (1 + 1e-12)


def test_recompress_keeps_assumption_1_and_the_stream_goes_on():
    st, X = _overfit_state(T=30, upto=24)
    O.recompress(st, 1.5 * math.sqrt(st.err2 / st.data_norm2))
    d = st.d
    Cd = O.unfold(st.C, d - 1)
    Vd = O.unfold(st.V, d - 1)
    np.testing.assert_allclose(Cd, st.S[:, None] * Vd, atol=1e-12 * np.abs(Cd).max())
    np.testing.assert_allclose(Vd @ Vd.T, np.eye(Vd.shape[0]), atol=1e-10)
    for U in st.Us:
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-10)
    for t in range(24, 30):
        O.stream_update(st, X[..., t].copy(order="F"))
    Xh = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(X - Xh) <= math.sqrt(st.err2) * (1 + 1e-12)


def test_recompress_without_budget_is_refused():
    st, _ = _overfit_state(T=12)
    with pytest.raises(ValueError):
        O.recompress(st, 0.5 * math.sqrt(st.err2 / st.data_norm2))
