"""Pins of the oracle's Alg. 1 (truncated Gram SVD) and Alg. 2 (ST-HOSVD)."""

import math

import numpy as np
import pytest

import oracle as O
from workloads import SineWave


def _with_singular_values(m, n, s, seed):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((m, len(s))))[0]
    V = np.linalg.qr(rng.standard_normal((n, len(s))))[0]
    return U @ np.diag(s) @ V.T, U, V


@pytest.mark.parametrize("eps,r_expect", [
    (0.0, 5),                 # nothing may be dropped
    (math.sqrt(1.0) - 1e-9, 5),   # tail {1} = 1 > eps^2
    (math.sqrt(1.0) + 1e-9, 4),   # drop sigma=1 (lambda=1)
    (math.sqrt(5.0) + 1e-9, 3),   # drop lambdas 4+1
    (math.sqrt(14.0) + 1e-9, 2),  # 9+4+1
    (math.sqrt(55.0) + 1e-9, 0),  # everything (25+16+9+4+1)
])
def test_rank_rule_on_known_spectrum(eps, r_expect):
    """Alg. 1: r = min{l : lambda_{l+1} + ... + lambda_m <= eps^2} with lambda = sigma^2."""
    s = np.array([5.0, 4.0, 3.0, 2.0, 1.0])
    A, U, V = _with_singular_values(7, 9, s, 1)
    res = O.truncated_svd(A, eps, want_v=True)
    assert res.r == r_expect
    np.testing.assert_allclose(res.lam[:5], s ** 2, rtol=1e-12)
    np.testing.assert_allclose(res.s, s[:r_expect], rtol=1e-12)
    # U spans the top-r left singular subspace; V = A^T U S^-1 are the right singular vectors
    if r_expect:
        P = res.U @ res.U.T
        np.testing.assert_allclose(P @ U[:, :r_expect], U[:, :r_expect], atol=1e-12)
        np.testing.assert_allclose(res.V.T @ res.V, np.eye(r_expect), atol=1e-12)
        approx = res.U @ np.diag(res.s) @ res.V.T
    else:
        approx = np.zeros_like(A)
    err2 = np.linalg.norm(A - approx) ** 2
    assert abs(err2 - res.discarded) < 1e-10
    assert err2 <= eps ** 2 + 1e-10


def test_gram_svd_vs_direct_svd():
    """Singular values of the Gram route agree with numpy's direct SVD on random small matrices."""
    rng = np.random.default_rng(2)
    for m, n in [(2, 3), (5, 5), (12, 7), (9, 20)]:
        A = rng.standard_normal((m, n))
        res = O.truncated_svd(A, 0.0)
        sv = np.linalg.svd(A, compute_uv=False)
        k = min(m, n)
        np.testing.assert_allclose(np.sqrt(np.maximum(res.lam[:k], 0)), sv, rtol=1e-10)


def test_descending_order_and_ties():
    """Reading R1: eigenvalues sorted descending."""
    A = np.diag([1.0, 3.0, 2.0, 3.0])
    res = O.truncated_svd(A, 0.0)
    np.testing.assert_allclose(res.lam, [9.0, 9.0, 4.0, 1.0])


def _lowrank_tensor(shape, ranks, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal(ranks)
    Us = [np.linalg.qr(rng.standard_normal((n, r)))[0] for n, r in zip(shape, ranks)]
    return O.reconstruct(C, Us), C, Us


def test_sthosvd_recovers_exact_ranks():
    X, _, _ = _lowrank_tensor((6, 7, 8, 9), (2, 3, 4, 2), 3)
    # tau above sqrt(u): the Gram route cannot resolve squared singular values below u ||X||^2
    res = O.sthosvd(X, 1e-6)
    assert res.ranks == (2, 3, 4, 2)
    Xh = O.reconstruct(res.C, res.Us)
    assert np.linalg.norm(X - Xh) <= 1e-10 * np.linalg.norm(X)


def test_sthosvd_error_split_and_bound():
    """Eq. partial_core_error: ||X - X^||^2 = sum_k ||C*_{k-1} - C*_k x_k U_k||^2 <= tau^2 ||X||^2."""
    rng = np.random.default_rng(4)
    X, _, _ = _lowrank_tensor((8, 9, 10), (3, 3, 3), 5)
    X = X + 0.02 * rng.standard_normal(X.shape) * np.linalg.norm(X) / math.sqrt(X.size)
    tau = 0.05
    res = O.sthosvd(X, tau)
    Xh = O.reconstruct(res.C, res.Us)
    err2 = np.linalg.norm(X - Xh) ** 2
    assert abs(err2 - sum(res.discarded)) <= 1e-9 * np.sum(X * X)
    for dk in res.discarded:
        assert dk <= res.eps ** 2 * (1 + 1e-12)
    assert math.sqrt(err2) <= tau * np.linalg.norm(X)
    # Pythagoras with orthonormal factors: ||X||^2 = ||C||^2 + ||X - X^||^2
    assert abs(np.sum(X * X) - np.sum(res.C ** 2) - err2) <= 1e-9 * np.sum(X * X)


def test_sthosvd_core_factorization_assumption_1c():
    """Assumption 1(c): C = V x_d S, V_(d) row-orthonormal, S > 0."""
    rng = np.random.default_rng(6)
    X = rng.standard_normal((5, 6, 7))
    res = O.sthosvd(X, 0.3)
    d = X.ndim
    Vd = O.unfold(res.V, d - 1)
    np.testing.assert_allclose(Vd @ Vd.T, np.eye(Vd.shape[0]), atol=1e-10)
    assert np.all(res.S > 0) and np.all(np.diff(res.S) <= 0)
    np.testing.assert_allclose(O.ttm(res.V, np.diag(res.S), d - 1), res.C, atol=1e-12)


def test_sthosvd_against_independent_svd_implementation():
    """An ST-HOSVD written here with np.linalg.svd of explicit unfoldings (not the Gram route)."""
    rng = np.random.default_rng(7)
    X, _, _ = _lowrank_tensor((3, 4, 5), (2, 2, 3), 8)
    X = X + 1e-6 * rng.standard_normal(X.shape)
    tau = 1e-3
    eps2 = (tau * np.linalg.norm(X)) ** 2 / 3
    C = X.copy()
    Us = []
    for k in range(3):
        Ck = np.moveaxis(C, k, 0)
        M = Ck.reshape(Ck.shape[0], -1)        # column order is irrelevant for the left singular vectors
        u, s, _ = np.linalg.svd(M, full_matrices=False)
        tails = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])
        r = int(np.argmax(tails <= eps2))
        r = max(r, 1)
        Us.append(u[:, :r])
        C = np.moveaxis(np.tensordot(u[:, :r].T, np.moveaxis(C, k, 0), axes=1), 0, k)
    Xh_ref = C
    for k, U in enumerate(Us):
        Xh_ref = np.moveaxis(np.tensordot(U, np.moveaxis(Xh_ref, k, 0), axes=1), 0, k)
    res = O.sthosvd(X, tau)
    assert res.ranks == tuple(U.shape[1] for U in Us)
    np.testing.assert_allclose(O.reconstruct(res.C, res.Us), Xh_ref, atol=1e-9)


def test_sine_wave_exact_rank_closed_form():
    """Sec. 5.1: the noiseless sine-wave tensor has exact mode-k rank 2 f_k + 1."""
    sw = SineWave(n=(30, 26), steps_each=20, freqs_a=(2, 3, 4), freqs_b=(2, 3, 6), noise=0.0)
    X = np.stack([sw.slice(t) for t in range(20)], axis=-1)      # first block only
    res = O.sthosvd(X, 1e-6)
    assert res.ranks == (5, 7, 9)
    # both blocks: the second block adds the |j_3| in {5, 6} terms, 4 more streaming-mode directions
    X = np.stack([sw.slice(t) for t in range(40)], axis=-1)
    res = O.sthosvd(X, 1e-6)
    assert res.ranks == (5, 7, 13)


def test_zero_tensor_rejected():
    with pytest.raises(ValueError):
        O.sthosvd(np.zeros((3, 3, 3)), 0.1)
