"""torch.autograd Functions over the Tucker projection and reconstruction chains.

    G  = project(Y, Us)      = Y x_1 U_1^T ... x_m U_m^T
    Y^ = reconstruct(G, Us)  = G x_1 U_1 ... x_m U_m

Forward and backward passes are single C-ABI calls (``include/tucker_ttm.h``): the backward of
``project`` is ``tucker_ttm_project_adjoint`` (dL/dY and dL/dU_k), the backward of
``reconstruct`` is ``tucker_ttm_reconstruct_adjoint`` (dL/dG and dL/dU_k). Only the inputs are
saved for backward; the partial products Y x_{k!=n} U_k^T are recomputed by the adjoint calls.
The factors are unconstrained matrices (Euclidean gradients).

Tensors are in paper index order, e.g. Y of shape (n_1, ..., n_m) and U_k of shape (n_k, r_k), on
a CUDA device, all float32 or all float64. The library works on column-major data (mode 1
fastest): a tensor whose memory is not column-major is copied into that layout first (a layout
conversion of the argument, no arithmetic). :func:`empty_colmajor` and :func:`as_colmajor` give
tensors that need no copy.
"""

from __future__ import annotations

import torch

from . import (tucker_ttm_project, tucker_ttm_project_adjoint, tucker_ttm_reconstruct,
               tucker_ttm_reconstruct_adjoint, tucker_ttm_workspace_bytes, ttm_desc)


def _rev(t):
    return tuple(reversed(range(t.dim())))


def is_colmajor(t: torch.Tensor) -> bool:
    return t.permute(*_rev(t)).is_contiguous()


def as_colmajor(t: torch.Tensor) -> torch.Tensor:
    """t itself if its memory is column-major, else a column-major copy (same shape)."""
    if is_colmajor(t):
        return t
    p = _rev(t)
    return t.permute(*p).contiguous().permute(*p)


def empty_colmajor(shape, dtype, device) -> torch.Tensor:
    shape = tuple(int(s) for s in shape)
    t = torch.empty(tuple(reversed(shape)), dtype=dtype, device=device)
    return t.permute(*reversed(range(len(shape))))


def _check(X, Us):
    if not X.is_cuda or any(not U.is_cuda for U in Us):
        raise ValueError("tensors must be on a CUDA device")
    if X.dtype not in (torch.float32, torch.float64) or any(U.dtype != X.dtype for U in Us):
        raise ValueError("all tensors must be float32 or all float64")
    if len(Us) != X.dim():
        raise ValueError("one factor per mode")


def _desc(n, r, dtype):
    return ttm_desc(n, r, "f32" if dtype == torch.float32 else "f64")


def _work(desc, device):
    nb = tucker_ttm_workspace_bytes(desc)
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device), nb


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return t.data_ptr() if t is not None else 0


class TuckerProject(torch.autograd.Function):
    """G = Y x_1 U_1^T ... x_m U_m^T; backward: tucker_ttm_project_adjoint."""

    @staticmethod
    def forward(ctx, Y, *Us):
        _check(Y, Us)
        n = tuple(Y.shape)
        r = tuple(U.shape[1] for U in Us)
        for k, U in enumerate(Us):
            if U.shape[0] != n[k]:
                raise ValueError(f"U_{k + 1} must be {n[k]} x r")
        Yc = as_colmajor(Y)
        Uc = [as_colmajor(U) for U in Us]
        desc = _desc(n, r, Y.dtype)
        work, nb = _work(desc, Y.device)
        G = empty_colmajor(r, Y.dtype, Y.device)
        tucker_ttm_project(desc, [U.data_ptr() for U in Uc], Yc.data_ptr(), G.data_ptr(),
                           work.data_ptr(), nb, _stream())
        ctx.save_for_backward(Yc, *Uc)
        ctx.shape = (n, r)
        return G

    @staticmethod
    def backward(ctx, Gbar):
        Yc, *Uc = ctx.saved_tensors
        n, r = ctx.shape
        need = ctx.needs_input_grad
        Gb = as_colmajor(Gbar)
        desc = _desc(n, r, Yc.dtype)
        work, nb = _work(desc, Yc.device)
        Ybar = empty_colmajor(n, Yc.dtype, Yc.device) if need[0] else None
        Ubar = [empty_colmajor((n[k], r[k]), Yc.dtype, Yc.device) if need[1 + k] else None
                for k in range(len(n))]
        if Ybar is not None or any(u is not None for u in Ubar):
            tucker_ttm_project_adjoint(desc, [U.data_ptr() for U in Uc], Yc.data_ptr(), Gb.data_ptr(),
                                       _ptr(Ybar), [_ptr(u) for u in Ubar], work.data_ptr(), nb,
                                       _stream())
        return (Ybar, *Ubar)


class TuckerReconstruct(torch.autograd.Function):
    """Y^ = G x_1 U_1 ... x_m U_m; backward: tucker_ttm_reconstruct_adjoint."""

    @staticmethod
    def forward(ctx, G, *Us):
        _check(G, Us)
        r = tuple(G.shape)
        n = tuple(U.shape[0] for U in Us)
        for k, U in enumerate(Us):
            if U.shape[1] != r[k]:
                raise ValueError(f"U_{k + 1} must be n x {r[k]}")
        Gc = as_colmajor(G)
        Uc = [as_colmajor(U) for U in Us]
        desc = _desc(n, r, G.dtype)
        work, nb = _work(desc, G.device)
        Yh = empty_colmajor(n, G.dtype, G.device)
        tucker_ttm_reconstruct(desc, [U.data_ptr() for U in Uc], Gc.data_ptr(), Yh.data_ptr(),
                               work.data_ptr(), nb, _stream())
        ctx.save_for_backward(Gc, *Uc)
        ctx.shape = (n, r)
        return Yh

    @staticmethod
    def backward(ctx, Yhbar):
        Gc, *Uc = ctx.saved_tensors
        n, r = ctx.shape
        need = ctx.needs_input_grad
        Yb = as_colmajor(Yhbar)
        desc = _desc(n, r, Gc.dtype)
        work, nb = _work(desc, Gc.device)
        Gbar = empty_colmajor(r, Gc.dtype, Gc.device) if need[0] else None
        Ubar = [empty_colmajor((n[k], r[k]), Gc.dtype, Gc.device) if need[1 + k] else None
                for k in range(len(n))]
        if Gbar is not None or any(u is not None for u in Ubar):
            tucker_ttm_reconstruct_adjoint(desc, [U.data_ptr() for U in Uc], Gc.data_ptr(),
                                           Yb.data_ptr(), _ptr(Gbar), [_ptr(u) for u in Ubar],
                                           work.data_ptr(), nb, _stream())
        return (Gbar, *Ubar)


def project(Y, Us):
    """G = Y x_1 U_1^T ... x_m U_m^T (differentiable in Y and every U_k)."""
    return TuckerProject.apply(Y, *Us)


def reconstruct(G, Us):
    """Y^ = G x_1 U_1 ... x_m U_m (differentiable in G and every U_k)."""
    return TuckerReconstruct.apply(G, *Us)
