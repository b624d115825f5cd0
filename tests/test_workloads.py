"""CPU pins of the seeded synthetic inputs that both the oracle and the CUDA path consume
(workloads/synth.py): each generator produces what its stated recipe says, so that a mistake in a
generator cannot hide behind agreement between the two sides that read the same wrong data."""

import math

import numpy as np
import pytest

from workloads import BlobField, LowRankStream, batched_streams


def _blob_brute(bf, t, i, j, k, v):
    """The advected-blob field at grid point (i, j, k), variable v, step t, written out from the
    recipe: sum_b a_{b,v} exp(-1/2 delta^T Sigma_b^{-1} delta), delta = x - c_b - v_b t with the
    periodic minimum image on [0, 1)^3."""
    x = np.array([i / bf.grid[0], j / bf.grid[1], k / bf.grid[2]])
    s = 0.0
    for b in range(bf.nblobs):
        d = x - (bf.centres[b] + bf.vel[b] * t)
        d = d - np.round(d)
        s += bf.amp[b, v] * math.exp(-0.5 * float(d @ bf.prec[b] @ d))
    return s


def test_blob_field_signal_is_the_recipe_at_sampled_points():
    bf = BlobField(grid=(20, 16, 12), nvar=3, nblobs=7, noise=1e-5, seed=3)
    rng = np.random.default_rng(0)
    for t in (0, 5, 40):
        sig = bf.signal_torch(t).numpy()                 # (nvar, n3, n2, n1)
        for _ in range(25):
            i, j, k = (int(rng.integers(0, n)) for n in bf.grid)
            v = int(rng.integers(0, bf.nvar))
            assert sig[v, k, j, i] == pytest.approx(_blob_brute(bf, t, i, j, k, v), rel=1e-12, abs=1e-14)


def test_blob_covariances_are_rotated_diagonals_in_the_stated_range():
    bf = BlobField(grid=(8, 8, 8), nvar=2, nblobs=20, seed=9)
    assert np.all((bf.sig >= 0.02) & (bf.sig <= 0.10))
    assert np.all(np.abs(bf.vel) <= 0.5 / bf.vel_div)
    for b in range(bf.nblobs):
        P = bf.prec[b]
        np.testing.assert_allclose(P, P.T, rtol=1e-14, atol=1e-12)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(P)), np.sort(1.0 / bf.sig[b] ** 2),
                                   rtol=1e-10)


def test_blob_slices_carry_the_stated_noise_in_both_generators():
    import torch

    bf = BlobField(grid=(24, 20, 8), nvar=2, nblobs=6, noise=1e-3, seed=4)
    t = 3
    sig = bf.signal_torch(t).numpy().T                   # paper order (n1, n2, n3, nvar)
    y = bf.slice(t, dtype=np.float64)
    assert y.shape == bf.spatial and y.flags.f_contiguous
    assert np.linalg.norm(y - sig) == pytest.approx(1e-3 * np.linalg.norm(sig), rel=1e-10)
    yt = bf.slice_torch(t, "cpu", dtype=torch.float64)   # row-major (nvar, n3, n2, n1)
    assert tuple(reversed(yt.shape)) == bf.spatial and yt.is_contiguous()
    d = yt.numpy().T - sig
    assert np.linalg.norm(d) == pytest.approx(1e-3 * np.linalg.norm(sig), rel=1e-10)
    # the same slice twice is the same slice (seeded by the step)
    assert np.array_equal(bf.slice(t, dtype=np.float64), y)
    assert torch.equal(bf.slice_torch(t, "cpu", dtype=torch.float64), yt)


def test_exact_rank_stream_has_its_multilinear_ranks_and_tensor_noise_scale():
    ranks = (4, 3, 2, 5)
    s = LowRankStream((12, 10, 8), ranks, 30, 0.0, seed=6)
    X = s.tensor(0, 30)
    for k, r in enumerate(ranks):
        sv = np.linalg.svd(np.moveaxis(X, k, 0).reshape(X.shape[k], -1), compute_uv=False)
        assert sv[r - 1] > 1e-8 * sv[0] and (len(sv) == r or sv[r] < 1e-12 * sv[0]), (k, sv[:r + 1])
    # noise over the whole tensor: ||N|| = eta ||Xbar||
    sn = LowRankStream((12, 10, 8), ranks, 30, 1e-2, seed=6, noise_scope="tensor")
    Xn = sn.tensor(0, 30)
    assert np.linalg.norm(Xn - X) == pytest.approx(1e-2 * np.linalg.norm(X), rel=1e-10)
    # per slice: ||N_t|| = eta ||Xbar_t||
    ss = LowRankStream((12, 10, 8), ranks, 30, 1e-2, seed=6)
    for t in (0, 17):
        assert np.linalg.norm(ss.slice(t) - s.slice(t)) == pytest.approx(
            1e-2 * np.linalg.norm(s.slice(t)), rel=1e-10)


def test_exact_rank_factors_are_orthonormal():
    s = LowRankStream((12, 10, 8), (4, 3, 2, 5), 30, 0.0, seed=2)
    for F in s.factors:
        np.testing.assert_allclose(F.T @ F, np.eye(F.shape[1]), atol=1e-12)


def test_batched_streams_follow_their_stated_ranges_and_are_reproducible():
    a = batched_streams(nstreams=16, steps=20)
    b = batched_streams(nstreams=16, steps=20)
    for (sa, ta), (sb, tb) in zip(a, b):
        assert sa.spatial == sb.spatial and sa.ranks == sb.ranks and ta == tb
        assert np.array_equal(sa.slice(3), sb.slice(3))
        assert all(32 <= n <= 160 for n in sa.spatial)
        assert all(1 <= r <= 24 for r in sa.ranks)
        assert all(r >= 4 or r == n for r, n in zip(sa.ranks[:3], sa.spatial))
        assert ta in (1e-2, 1e-3, 1e-4)
        assert sa.slice(0).dtype == np.float32
    assert len({s.spatial for s, _ in a}) > 1 and len({t for _, t in a}) > 1
