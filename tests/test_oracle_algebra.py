"""Pins of the oracle's tensor algebra (Sec. 2.1) against definitions written out by brute force."""

import itertools

import numpy as np
import pytest

import oracle as O


def _rand(shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 4, 3), (5, 1, 2)])
def test_unfold_matches_index_formula(shape):
    """X_(k)(i_k, 1 + sum_{l != k} (i_l - 1) prod_{l' < l, l' != k} n_l') = X(i_1..i_d), Sec. 2.1."""
    X = _rand(shape)
    d = len(shape)
    for k in range(d):
        M = O.unfold(X, k)
        assert M.shape == (shape[k], X.size // shape[k])
        for idx in itertools.product(*[range(n) for n in shape]):
            col = 0
            for l in range(d):
                if l == k:
                    continue
                stride = 1
                for lp in range(l):
                    if lp != k:
                        stride *= shape[lp]
                col += idx[l] * stride
            assert M[idx[k], col] == X[idx]
        np.testing.assert_array_equal(O.fold(M, k, shape), X)


def test_ttm_brute_force():
    """Y = X x_2 A: Y(i1, j, i3) = sum_i2 A(j, i2) X(i1, i2, i3)."""
    X = _rand((3, 4, 5), 1)
    A = _rand((2, 4), 2)
    Y = O.ttm(X, A, 1)
    assert Y.shape == (3, 2, 5)
    ref = np.zeros((3, 2, 5))
    for i1 in range(3):
        for j in range(2):
            for i3 in range(5):
                ref[i1, j, i3] = sum(A[j, i2] * X[i1, i2, i3] for i2 in range(4))
    np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-13)


def test_ttm_commutes():
    """TTMs along different modes commute (Sec. 2.1)."""
    X = _rand((3, 4, 5), 3)
    A = _rand((6, 3), 4)
    B = _rand((2, 5), 5)
    np.testing.assert_allclose(O.ttm(O.ttm(X, A, 0), B, 2), O.ttm(O.ttm(X, B, 2), A, 0), rtol=1e-12)


def test_kronecker_form_of_ttm_chain():
    """Eq. tucker_matrix: Y_(k) = A_k X_(k) (A_d kron ... A_{k+1} kron A_{k-1} ... kron A_1)^T."""
    shape = (2, 3, 4)
    X = _rand(shape, 6)
    As = [_rand((m, n), 7 + i) for i, (m, n) in enumerate([(3, 2), (2, 3), (5, 4)])]
    Y = X
    for k, A in enumerate(As):
        Y = O.ttm(Y, A, k)
    for k in range(3):
        others = [As[l] for l in reversed(range(3)) if l != k]
        K = others[0]
        for M in others[1:]:
            K = np.kron(K, M)
        np.testing.assert_allclose(O.unfold(Y, k), As[k] @ O.unfold(X, k) @ K.T, rtol=1e-12, atol=1e-12)


def test_reconstruct_is_ttm_chain_and_norm_preserving():
    """With orthonormal factors, ||C x_1 U_1 ... x_d U_d|| = ||C|| (Sec. 2.2)."""
    rng = np.random.default_rng(8)
    C = rng.standard_normal((2, 3, 2))
    Us = [np.linalg.qr(rng.standard_normal((n, r)))[0] for n, r in [(5, 2), (4, 3), (6, 2)]]
    X = O.reconstruct(C, Us)
    assert X.shape == (5, 4, 6)
    assert abs(np.linalg.norm(X) - np.linalg.norm(C)) < 1e-12 * np.linalg.norm(C)
    # brute force element
    i = (4, 1, 3)
    v = sum(C[a, b, c] * Us[0][i[0], a] * Us[1][i[1], b] * Us[2][i[2], c]
            for a in range(2) for b in range(3) for c in range(2))
    assert abs(X[i] - v) < 1e-13
