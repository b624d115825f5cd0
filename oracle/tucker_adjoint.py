"""FP64 CPU oracle of the Tucker projection and reconstruction chains and of their adjoints.

TEST INFRASTRUCTURE ONLY -- imported by tests/ and bench.py's CPU legs, never by the product
path. It shares no code with the CUDA library.

Definitions (Sec. 2.1-2.2 of the paper: the mode-k product X x_k A defined by
(X x_k A)_(k) = A X_(k), and the Tucker model X^ = G x_1 U_1 ... x_d U_d):

  projection      G  = P(Y; U)  = Y x_1 U_1^T x_2 U_2^T ... x_d U_d^T      (the core of Y)
  reconstruction  Y^ = R(G; U)  = G x_1 U_1 x_2 U_2 ... x_d U_d

Both are linear in their tensor argument and multilinear in the factors. With the Kronecker form
of the Tucker model (Sec. 2.2),

  R(G; U)_(n) = U_n G_(n) (U_d (x) ... (x) U_{n+1} (x) U_{n-1} (x) ... (x) U_1)^T,
  P(Y; U)_(n) = U_n^T Y_(n) (U_d (x) ... (x) U_{n+1} (x) U_{n-1} (x) ... (x) U_1),

so for a scalar loss with upstream gradients Gbar = dL/dG and Ybar^ = dL/dY^:

  projection adjoint
    dL/dY   = R(Gbar; U)                                   (P and R are mutual adjoints in Y, G)
    dL/dU_n = [Y x_{m != n} U_m^T]_(n)  Gbar_(n)^T          (n_n x r_n)
  reconstruction adjoint
    dL/dG   = P(Ybar^; U)
    dL/dU_n = [Ybar^ x_{m != n} U_m^T]_(n)  G_(n)^T         (n_n x r_n)

Each formula is evaluated here literally, one mode product at a time, with nothing shared
between the terms (the CUDA path reuses common prefixes of the chains; the oracle does not).
The factors are treated as unconstrained matrices (Euclidean gradients). The composite loss
L(Y, U) = || R(P(Y; U); U) - T ||_F^2 is the differentiation workload.

Pinned in tests/test_oracle_adjoint.py against central finite differences of the forward maps,
against torch.autograd through an einsum restatement, and against the adjoint identity
<P(Y), Gbar> = <Y, R(Gbar)>.
"""

from __future__ import annotations

import numpy as np

from .tucker_oracle import ttm, unfold


def project(Y: np.ndarray, Us) -> np.ndarray:
    """G = Y x_1 U_1^T ... x_d U_d^T."""
    G = Y
    for k, U in enumerate(Us):
        G = ttm(G, U.T, k)
    return G


def expand(G: np.ndarray, Us) -> np.ndarray:
    """Y^ = G x_1 U_1 ... x_d U_d."""
    Y = G
    for k, U in enumerate(Us):
        Y = ttm(Y, U, k)
    return Y


def project_all_but(X: np.ndarray, Us, n: int) -> np.ndarray:
    """X x_{m != n} U_m^T (mode n keeps its size)."""
    Z = X
    for m, U in enumerate(Us):
        if m != n:
            Z = ttm(Z, U.T, m)
    return Z


def project_adjoint(Y: np.ndarray, Us, Gbar: np.ndarray):
    """(dL/dY, [dL/dU_n]) of G = P(Y; U) given Gbar = dL/dG."""
    Ybar = expand(Gbar, Us)
    Ubar = [unfold(project_all_but(Y, Us, n), n) @ unfold(Gbar, n).T for n in range(len(Us))]
    return Ybar, Ubar


def expand_adjoint(G: np.ndarray, Us, Yhbar: np.ndarray):
    """(dL/dG, [dL/dU_n]) of Y^ = R(G; U) given Yhbar = dL/dY^."""
    Gbar = project(Yhbar, Us)
    Ubar = [unfold(project_all_but(Yhbar, Us, n), n) @ unfold(G, n).T for n in range(len(Us))]
    return Gbar, Ubar


def composite_loss(Y: np.ndarray, Us, T: np.ndarray) -> float:
    """L = || R(P(Y; U); U) - T ||_F^2."""
    D = expand(project(Y, Us), Us) - T
    return float(np.sum(D * D))


def composite_grad(Y: np.ndarray, Us, T: np.ndarray):
    """(dL/dY, [dL/dU_n]) of the composite loss: reconstruction adjoint, then projection adjoint;
    the factor gradients of the two chains add."""
    G = project(Y, Us)
    Yh = expand(G, Us)
    Yhbar = 2.0 * (Yh - T)
    Gbar, Ubar_r = expand_adjoint(G, Us, Yhbar)
    Ybar, Ubar_p = project_adjoint(Y, Us, Gbar)
    return Ybar, [a + b for a, b in zip(Ubar_r, Ubar_p)]
