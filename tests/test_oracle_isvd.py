"""Pins of the oracle's incremental SVD (Alg. 3, Prop. 1)."""

import numpy as np
import pytest

import oracle as O


def _svd_r(A, r):
    u, s, vt = np.linalg.svd(A, full_matrices=False)
    return u[:, :r], s[:r], vt[:r, :].T


def test_isvd_row_by_row_reproduces_batch_svd():
    """Appending the rows of an exact rank-4 matrix with eps ~ 0 yields its SVD (Sec. 3.1)."""
    rng = np.random.default_rng(0)
    m, n, r = 30, 12, 4
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    U, S, V = _svd_r(A[:5], 4)
    for i in range(5, m):
        U, S, V, info = O.isvd(U, S, V, A[i], 1e-9 * np.linalg.norm(A[i]))
    np.testing.assert_allclose(S, np.linalg.svd(A, compute_uv=False)[:len(S)], rtol=1e-9)
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, A, atol=1e-9 * np.linalg.norm(A))
    np.testing.assert_allclose(U.T @ U, np.eye(len(S)), atol=1e-10)
    np.testing.assert_allclose(V.T @ V, np.eye(len(S)), atol=1e-10)


@pytest.mark.parametrize("ignore", [True, False])
def test_prop1_error_evolution(ignore):
    """Prop. 1: the squared error grows by exactly ||e||^2 when e is ignored, by 0 otherwise."""
    rng = np.random.default_rng(1)
    m, n = 10, 15
    A = rng.standard_normal((m, n))
    U, S, V = _svd_r(A, 5)
    err0 = np.linalg.norm(A - U @ np.diag(S) @ V.T) ** 2
    b = rng.standard_normal(n)
    e = b - V @ (V.T @ b)
    qn = np.linalg.norm(e)
    eps = qn * (1.0 + 1e-6) if ignore else qn * (1.0 - 1e-6)
    Ut, St, Vt, info = O.isvd(U, S, V, b, eps)
    assert info.augmented == (not ignore)
    At = np.vstack([A, b[None, :]])
    err1 = np.linalg.norm(At - Ut @ np.diag(St) @ Vt.T) ** 2
    expect = err0 + (qn ** 2 if ignore else 0.0)
    assert abs(err1 - expect) <= 1e-10 * np.sum(At * At)
    assert len(St) == (5 if ignore else 6)


def test_qr_branch_leaves_result_unchanged():
    """Reading R5: the QR re-orthogonalisation changes V' and S' but not U~ S~ V~^T (exact arithmetic)."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((8, 20))
    U, S, V = _svd_r(A, 6)
    b = rng.standard_normal(20)
    r1 = O.isvd(U, S, V, b, 1e-3, eps_m=1.0)    # never QR
    r2 = O.isvd(U, S, V, b, 1e-3, eps_m=0.0)    # always QR
    assert not r1[3].qr and r2[3].qr
    np.testing.assert_allclose(r1[1], r2[1], rtol=1e-12)
    np.testing.assert_allclose(r1[0] @ np.diag(r1[1]) @ r1[2].T, r2[0] @ np.diag(r2[1]) @ r2[2].T, atol=1e-12)


def test_zero_row_keeps_singular_values():
    """A zero row: q = 0 <= eps, S~ = S, and U~ gains a zero row."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 9))
    U, S, V = _svd_r(A, 4)
    Ut, St, Vt, info = O.isvd(U, S, V, np.zeros(9), 0.0)
    assert not info.augmented and info.q == 0.0
    np.testing.assert_allclose(St, S, rtol=1e-12)
    np.testing.assert_allclose(Ut[-1], 0.0, atol=1e-14)
    np.testing.assert_allclose(Ut[:-1] @ np.diag(St) @ Vt.T, U @ np.diag(S) @ V.T, atol=1e-12)


def test_row_in_span_has_zero_residual():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((6, 9))
    U, S, V = _svd_r(A, 4)
    b = V @ rng.standard_normal(4)
    Ut, St, Vt, info = O.isvd(U, S, V, b, 1e-8)
    assert info.q < 1e-13 and not info.augmented
    At = np.vstack([U @ np.diag(S) @ V.T, b[None, :]])
    np.testing.assert_allclose(Ut @ np.diag(St) @ Vt.T, At, atol=1e-12)


def test_numerical_rank_of_compact_svd():
    """Reading R4: with q <= eps, S' = [S; p^T] has r columns, so the rank stays r."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((7, 11))
    U, S, V = _svd_r(A, 3)
    b = V @ rng.standard_normal(3) + 1e-6 * rng.standard_normal(11)
    Ut, St, Vt, info = O.isvd(U, S, V, b, 1e-3)
    assert len(St) == 3 and info.r_new == 3
