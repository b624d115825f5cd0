"""CPU pins of the oracle's block update (several slices at once, the Conclusions' future work):
a block of one slice is Alg. 5 exactly; an exact-rank stream keeps its ranks; the running bound
covers the true error; every block adds at most tau^2 ||Yb||^2 (the reading's guarantee); the
result stays within tau of the data; block and slice-by-slice streams agree in their accuracy."""

import math

import numpy as np
import pytest

import oracle as O
from workloads import LowRankStream


def _stream(T=40, seed=8, noise=1e-4, ranks=(4, 4, 3, 6), n=(24, 20, 16)):
    s = LowRankStream(n, ranks, T, noise, seed=seed)
    return s.tensor(0, T)


def test_block_of_one_slice_is_alg5():
    X = _stream()
    a = O.init_stream(X[..., :10].copy(order="F"), 1e-3)
    b = O.init_stream(X[..., :10].copy(order="F"), 1e-3)
    for t in range(10, 25):
        O.stream_update(a, X[..., t].copy(order="F"))
        O.block_update(b, X[..., t:t + 1].copy(order="F"))
        assert a.ranks == b.ranks
    np.testing.assert_allclose(O.reconstruct(b.C, b.Us), O.reconstruct(a.C, a.Us),
                               atol=1e-12 * np.abs(X).max())
    np.testing.assert_allclose(b.S, a.S, rtol=1e-12)
    assert b.err2 == pytest.approx(a.err2, rel=1e-12, abs=1e-300)
    assert b.data_norm2 == pytest.approx(a.data_norm2, rel=1e-14)


@pytest.mark.parametrize("B", [2, 3, 5])
def test_exact_rank_stream_keeps_its_ranks_in_blocks(B):
    X = _stream(T=40, noise=0.0)
    st = O.init_stream(X[..., :10].copy(order="F"), 1e-3)
    assert st.ranks == (4, 4, 3, 6)
    for t0 in range(10, 40, B):
        O.block_update(st, X[..., t0:min(t0 + B, 40)].copy(order="F"))
        assert st.ranks[:3] == (4, 4, 3) and st.ranks[3] <= 6
    Xh = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(X - Xh) <= 1e-10 * np.linalg.norm(X)


@pytest.mark.parametrize("B", [2, 4])
def test_bound_covers_the_error_and_each_block_stays_in_budget(B):
    X = _stream(T=42, noise=3e-3, seed=9)      # noise above tau: ranks grow, both branches of Alg. 3
    tau = 2e-3
    st = O.init_stream(X[..., :6].copy(order="F"), tau)
    grew = 0
    for t0 in range(6, 42, B):
        Yb = X[..., t0:t0 + B].copy(order="F")
        before = st.err2
        O.block_update(st, Yb)
        lg = st.log[-1]
        grew += sum(m.grew for m in lg["modes"])
        assert st.err2 - before <= tau ** 2 * float(np.sum(Yb * Yb)) * (1 + 1e-12)
        assert lg["added"] == pytest.approx(st.err2 - before, rel=1e-12, abs=1e-300)
        Xh = O.reconstruct(st.C, st.Us)
        true = np.linalg.norm(X[..., :t0 + B] - Xh)
        assert true <= math.sqrt(st.err2) * (1 + 1e-10)
    assert grew > 0
    assert math.sqrt(st.err2) <= tau * math.sqrt(st.data_norm2) * (1 + 1e-12)
    # Assumption 1(c) after the last block
    d = st.d
    np.testing.assert_allclose(O.unfold(st.C, d - 1), st.S[:, None] * O.unfold(st.V, d - 1),
                               atol=1e-10 * np.abs(st.C).max())


def test_blocks_and_single_slices_reach_the_same_accuracy():
    X = _stream(T=40, noise=1e-4, seed=10)
    tau = 1e-3
    a = O.init_stream(X[..., :10].copy(order="F"), tau)
    b = O.init_stream(X[..., :10].copy(order="F"), tau)
    for t in range(10, 40):
        O.stream_update(a, X[..., t].copy(order="F"))
    for t0 in range(10, 40, 5):
        O.block_update(b, X[..., t0:t0 + 5].copy(order="F"))
    ea = np.linalg.norm(X - O.reconstruct(a.C, a.Us)) / np.linalg.norm(X)
    eb = np.linalg.norm(X - O.reconstruct(b.C, b.Us)) / np.linalg.norm(X)
    assert ea <= tau and eb <= tau
    assert a.ranks[:3] == b.ranks[:3] == (4, 4, 3)
