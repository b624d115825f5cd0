"""Pins of the oracle's projection / reconstruction adjoints (oracle/tucker_adjoint.py).

Each check is independent of the formulas it tests: central finite differences of the forward
maps, torch.autograd through an einsum restatement of the forward maps, brute-force loops, and
the adjoint identity between projection and reconstruction.
"""

import itertools

import numpy as np
import pytest

from oracle import tucker_adjoint as A


def _case(n, r, seed, orthonormal=False):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal(n)
    if orthonormal:
        Us = [np.linalg.qr(rng.standard_normal((nk, rk)))[0] for nk, rk in zip(n, r)]
    else:
        Us = [rng.standard_normal((nk, rk)) / np.sqrt(nk) for nk, rk in zip(n, r)]
    T = rng.standard_normal(n)
    return rng, Y, Us, T


def test_project_by_brute_force():
    _, Y, Us, _ = _case((3, 4, 2), (2, 3, 2), 0)
    G = A.project(Y, Us)
    ref = np.zeros((2, 3, 2))
    for a, b, c in itertools.product(range(2), range(3), range(2)):
        for i, j, k in itertools.product(range(3), range(4), range(2)):
            ref[a, b, c] += Y[i, j, k] * Us[0][i, a] * Us[1][j, b] * Us[2][k, c]
    np.testing.assert_allclose(G, ref, rtol=1e-13, atol=1e-14)
    Yh = A.expand(ref, Us)
    ref2 = np.zeros((3, 4, 2))
    for i, j, k in itertools.product(range(3), range(4), range(2)):
        for a, b, c in itertools.product(range(2), range(3), range(2)):
            ref2[i, j, k] += ref[a, b, c] * Us[0][i, a] * Us[1][j, b] * Us[2][k, c]
    np.testing.assert_allclose(Yh, ref2, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("n,r", [((6, 5, 4), (3, 2, 2)), ((7, 3), (2, 3)), ((4, 3, 5, 2), (2, 2, 3, 1))])
def test_projection_and_reconstruction_are_mutual_adjoints(n, r):
    rng, Y, Us, _ = _case(n, r, 1)
    Gbar = rng.standard_normal(r)
    lhs = np.sum(A.project(Y, Us) * Gbar)
    rhs = np.sum(Y * A.expand(Gbar, Us))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def _fd(f, x, h=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = x[i]
        x[i] = old + h
        fp = f()
        x[i] = old - h
        fm = f()
        x[i] = old
        g[i] = (fp - fm) / (2 * h)
    return g


def test_composite_gradient_against_central_differences():
    """16 x 16 x 8, ranks (4, 4, 3): every entry of Y and of each U_n, h = 1e-6."""
    _, Y, Us, T = _case((16, 16, 8), (4, 4, 3), 2)
    Ybar, Ubar = A.composite_grad(Y, Us, T)
    f = lambda: A.composite_loss(Y, Us, T)  # noqa: E731
    gY = _fd(f, Y)
    scale = np.max(np.abs(Ybar))
    assert np.max(np.abs(gY - Ybar)) <= 1e-6 * scale
    for n in range(3):
        gU = _fd(f, Us[n])
        assert np.max(np.abs(gU - Ubar[n])) <= 1e-6 * np.max(np.abs(Ubar[n])), n


def test_single_chain_adjoints_against_central_differences():
    """L = <P(Y;U), Gbar> and L = <R(G;U), Ybar> separately (each term of the factor gradient)."""
    rng, Y, Us, _ = _case((7, 5, 4), (3, 2, 3), 3)
    Gbar = rng.standard_normal((3, 2, 3))
    Ybar, Ubar = A.project_adjoint(Y, Us, Gbar)
    f = lambda: float(np.sum(A.project(Y, Us) * Gbar))  # noqa: E731
    np.testing.assert_allclose(_fd(f, Y), Ybar, atol=1e-7)
    for n in range(3):
        np.testing.assert_allclose(_fd(f, Us[n]), Ubar[n], atol=1e-7)
    G = rng.standard_normal((3, 2, 3))
    Yhbar = rng.standard_normal((7, 5, 4))
    Gbar2, Ubar2 = A.expand_adjoint(G, Us, Yhbar)
    f2 = lambda: float(np.sum(A.expand(G, Us) * Yhbar))  # noqa: E731
    np.testing.assert_allclose(_fd(f2, G), Gbar2, atol=1e-7)
    for n in range(3):
        np.testing.assert_allclose(_fd(f2, Us[n]), Ubar2[n], atol=1e-7)


def _einsum_loss(torch, Y, Us, T):
    d = Y.dim()
    full = "ijklmnop"[:d]
    core = "abcdefgh"[:d]
    ops = ",".join(f"{full[k]}{core[k]}" for k in range(d))
    G = torch.einsum(f"{full},{ops}->{core}", Y, *Us)
    Yh = torch.einsum(f"{core},{ops}->{full}", G, *Us)
    return ((Yh - T) ** 2).sum()


@pytest.mark.parametrize("n,r", [((16, 16, 8), (4, 4, 3)), ((9, 6), (3, 2)), ((5, 4, 6, 3), (2, 3, 2, 2)),
                                 ((6, 5, 4), (6, 5, 4)), ((6, 5, 4), (1, 1, 1))])
def test_composite_gradient_against_torch_autograd(n, r):
    torch = pytest.importorskip("torch")
    _, Y, Us, T = _case(n, r, 4)
    Ybar, Ubar = A.composite_grad(Y, Us, T)
    Yt = torch.tensor(Y, requires_grad=True)
    Ut = [torch.tensor(U, requires_grad=True) for U in Us]
    L = _einsum_loss(torch, Yt, Ut, torch.tensor(T))
    L.backward()
    assert abs(L.item() - A.composite_loss(Y, Us, T)) <= 1e-12 * L.item()
    np.testing.assert_allclose(Yt.grad.numpy(), Ybar, rtol=1e-10, atol=1e-11 * np.max(np.abs(Ybar)))
    for k in range(len(n)):
        np.testing.assert_allclose(Ut[k].grad.numpy(), Ubar[k], rtol=1e-10,
                                   atol=1e-11 * np.max(np.abs(Ubar[k])))


def test_in_span_data_is_a_stationary_point():
    """Orthonormal U, Y inside their span and T = Y: the loss is 0 and every gradient vanishes."""
    rng, _, Us, _ = _case((8, 6, 5), (3, 2, 2), 5, orthonormal=True)
    Y = A.expand(rng.standard_normal((3, 2, 2)), Us)
    Ybar, Ubar = A.composite_grad(Y, Us, Y.copy())
    assert A.composite_loss(Y, Us, Y) < 1e-26
    assert np.max(np.abs(Ybar)) < 1e-12
    for U in Ubar:
        assert np.max(np.abs(U)) < 1e-12
