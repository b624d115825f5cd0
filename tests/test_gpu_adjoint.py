"""GPU parity of the projection / reconstruction chains and their adjoints (include/tucker_ttm.h)
against the FP64 oracle (oracle/tucker_adjoint.py, pinned by finite differences and autograd).

Bars: FP64 -- 1e-12 relative (elementwise against the largest entry); FP32 -- 1e-5 relative to
the largest entry (FP32 storage and FMA accumulation over at most a few hundred terms per dot
product: ~1e-6 expected, the 1e-5 bar of the mixed form).
"""

import numpy as np
import pytest

from oracle import tucker_adjoint as A

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def ag():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_16395_gb300 import build as b

    b.build()
    import paper_2308_16395_gb300 as p

    p.load_library()
    from paper_2308_16395_gb300 import autograd

    return autograd


def _dev(x, dtype, ag):
    """numpy (paper order) -> column-major CUDA tensor in paper order."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x.T)).to(device="cuda", dtype=dtype)
    return t.permute(*reversed(range(t.dim())))


def _np(t):
    return t.detach().double().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _case(n, r, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal(n)
    Us = [np.linalg.qr(rng.standard_normal((nk, rk)))[0] for nk, rk in zip(n, r)]
    T = rng.standard_normal(n)
    return rng, Y, Us, T


def _composite(ag, Y, Us, T, dtype):
    import torch

    Yt = _dev(Y, dtype, ag).requires_grad_(True)
    Ut = [_dev(U, dtype, ag).requires_grad_(True) for U in Us]
    Tt = _dev(T, dtype, ag)
    G = ag.project(Yt, Ut)
    Yh = ag.reconstruct(G, Ut)
    L = ((Yh - Tt) ** 2).sum()
    L.backward()
    torch.cuda.synchronize()
    return L.item(), _np(Yt.grad), [_np(U.grad) for U in Ut], _np(G), _np(Yh)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_fd_instance_16x16x8(ag, dt):
    """The finite-difference instance: 16 x 16 x 8, ranks (4, 4, 3)."""
    import torch

    _, Y, Us, T = _case((16, 16, 8), (4, 4, 3), 1)
    dtype = torch.float64 if dt == "f64" else torch.float32
    if dt == "f32":  # both sides see the same rounded inputs
        Y, T = Y.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
        Us = [U.astype(np.float32).astype(np.float64) for U in Us]
    L, Yb, Ub, G, Yh = _composite(ag, Y, Us, T, dtype)
    Yb_o, Ub_o = A.composite_grad(Y, Us, T)
    assert abs(L - A.composite_loss(Y, Us, T)) <= 10 * TOL[dt] * abs(L)
    assert _rel(G, A.project(Y, Us)) <= TOL[dt]
    assert _rel(Yb, Yb_o) <= TOL[dt]
    for k in range(3):
        assert _rel(Ub[k], Ub_o[k]) <= TOL[dt], k
    if dt == "f64":
        # central differences (h = 1e-6) of the FP64 loss on sampled entries
        rng = np.random.default_rng(0)
        for _ in range(12):
            i = tuple(int(rng.integers(0, s)) for s in Y.shape)
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i] += 1e-6
            Ym[i] -= 1e-6
            fd = (A.composite_loss(Yp, Us, T) - A.composite_loss(Ym, Us, T)) / 2e-6
            assert abs(fd - Yb[i]) <= 1e-6 * np.max(np.abs(Yb))
        for k in range(3):
            for _ in range(4):
                i = (int(rng.integers(0, Us[k].shape[0])), int(rng.integers(0, Us[k].shape[1])))
                Up = [U.copy() for U in Us]
                Um = [U.copy() for U in Us]
                Up[k][i] += 1e-6
                Um[k][i] -= 1e-6
                fd = (A.composite_loss(Y, Up, T) - A.composite_loss(Y, Um, T)) / 2e-6
                assert abs(fd - Ub[k][i]) <= 1e-6 * np.max(np.abs(Ub[k]))


def test_config3_full_size_fp32(ag):
    """128 x 128 x 64 FP32, ranks (20, 20, 12): gradients within 1e-5 of the FP64 oracle."""
    import torch

    _, Y, Us, T = _case((128, 128, 64), (20, 20, 12), 3)
    Y, T = Y.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    Us = [U.astype(np.float32).astype(np.float64) for U in Us]
    L, Yb, Ub, G, Yh = _composite(ag, Y, Us, T, torch.float32)
    Yb_o, Ub_o = A.composite_grad(Y, Us, T)
    assert _rel(Yh, A.expand(A.project(Y, Us), Us)) <= TOL["f32"]
    assert _rel(Yb, Yb_o) <= TOL["f32"]
    for k in range(3):
        assert _rel(Ub[k], Ub_o[k]) <= TOL["f32"], k


@pytest.mark.parametrize("n,r", [((37, 29, 11), (5, 4, 3)), ((50,), (7,)), ((33, 17), (33, 1)),
                                 ((9, 7, 5, 6), (3, 7, 2, 1)), ((6, 5, 4), (6, 5, 4)),
                                 ((300, 3, 40), (9, 2, 5))])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_single_chain_adjoints_ragged(ag, n, r, dt):
    """Each entry point on its own, ragged sizes, m = 1..4, full and unit ranks."""
    import torch

    import paper_2308_16395_gb300 as pkg

    rng, Y, Us, _ = _case(n, r, 7)
    Us = [rng.standard_normal(U.shape) for U in Us]          # unconstrained factors
    Gbar = rng.standard_normal(r)
    Yhbar = rng.standard_normal(n)
    G0 = rng.standard_normal(r)
    dtype = torch.float64 if dt == "f64" else torch.float32
    if dt == "f32":
        rd = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
        Y, Gbar, Yhbar, G0 = rd(Y), rd(Gbar), rd(Yhbar), rd(G0)
        Us = [rd(U) for U in Us]
    Ut = [_dev(U, dtype, ag) for U in Us]
    desc = pkg.ttm_desc(n, r, dt)
    nb = pkg.tucker_ttm_workspace_bytes(desc)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    up = [U.data_ptr() for U in Ut]
    s = torch.cuda.current_stream().cuda_stream
    # forward maps
    Yd, Gd = _dev(Y, dtype, ag), _dev(G0, dtype, ag)
    Gout = ag.empty_colmajor(r, dtype, "cuda")
    pkg.tucker_ttm_project(desc, up, Yd.data_ptr(), Gout.data_ptr(), work.data_ptr(), nb, s)
    Yout = ag.empty_colmajor(n, dtype, "cuda")
    pkg.tucker_ttm_reconstruct(desc, up, Gd.data_ptr(), Yout.data_ptr(), work.data_ptr(), nb, s)
    torch.cuda.synchronize()
    assert _rel(_np(Gout), A.project(Y, Us)) <= TOL[dt]
    assert _rel(_np(Yout), A.expand(G0, Us)) <= TOL[dt]
    # projection adjoint, every output
    Ybar_o, Ubar_o = A.project_adjoint(Y, Us, Gbar)
    Yb = ag.empty_colmajor(n, dtype, "cuda")
    Ub = [ag.empty_colmajor(U.shape, dtype, "cuda") for U in Us]
    pkg.tucker_ttm_project_adjoint(desc, up, Yd.data_ptr(), _dev(Gbar, dtype, ag).data_ptr(),
                                   Yb.data_ptr(), [u.data_ptr() for u in Ub], work.data_ptr(), nb, s)
    torch.cuda.synchronize()
    assert _rel(_np(Yb), Ybar_o) <= TOL[dt]
    for k in range(len(n)):
        assert _rel(_np(Ub[k]), Ubar_o[k]) <= TOL[dt], k
    # reconstruction adjoint with only the last factor's gradient and dL/dG requested
    Gbar_o, Ubar2_o = A.expand_adjoint(G0, Us, Yhbar)
    Gb = ag.empty_colmajor(r, dtype, "cuda")
    Ub2 = [None] * (len(n) - 1) + [ag.empty_colmajor(Us[-1].shape, dtype, "cuda")]
    pkg.tucker_ttm_reconstruct_adjoint(desc, up, Gd.data_ptr(), _dev(Yhbar, dtype, ag).data_ptr(),
                                       Gb.data_ptr(), [u.data_ptr() if u is not None else 0 for u in Ub2],
                                       work.data_ptr(), nb, s)
    torch.cuda.synchronize()
    assert _rel(_np(Gb), Gbar_o) <= TOL[dt]
    assert _rel(_np(Ub2[-1]), Ubar2_o[-1]) <= TOL[dt]


def test_matches_torch_einsum_autograd(ag):
    """The composite gradient equals torch.autograd through an einsum restatement (FP64, GPU)."""
    import torch

    _, Y, Us, T = _case((24, 20, 10), (6, 5, 3), 11)
    L, Yb, Ub, _, _ = _composite(ag, Y, Us, T, torch.float64)
    Yt = torch.tensor(Y, device="cuda", requires_grad=True)
    Ut = [torch.tensor(U, device="cuda", requires_grad=True) for U in Us]
    G = torch.einsum("ijk,ia,jb,kc->abc", Yt, *Ut)
    Yh = torch.einsum("abc,ia,jb,kc->ijk", G, *Ut)
    Le = ((Yh - torch.tensor(T, device="cuda")) ** 2).sum()
    Le.backward()
    assert _rel(Yb, _np(Yt.grad)) <= 1e-12
    for k in range(3):
        assert _rel(Ub[k], _np(Ut[k].grad)) <= 1e-12


def test_non_colmajor_inputs_and_partial_grads(ag):
    """Row-major inputs are accepted (converted), and only requested gradients are formed."""
    import torch

    _, Y, Us, T = _case((12, 10, 6), (3, 3, 2), 13)
    Yt = torch.tensor(Y, device="cuda")                       # row-major
    Ut = [torch.tensor(U, device="cuda") for U in Us]
    Ut[1].requires_grad_(True)
    G = ag.project(Yt, Ut)
    (G ** 2).sum().backward()
    _, Ubar_o = A.project_adjoint(Y, Us, 2 * A.project(Y, Us))
    assert Yt.grad is None and Ut[0].grad is None
    assert _rel(_np(Ut[1].grad), Ubar_o[1]) <= 1e-12
