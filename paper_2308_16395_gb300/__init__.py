"""Python binding of the GB300 streaming ST-HOSVD library (arXiv 2308.16395).

Argument marshalling only: every function forwards to the C ABI declared in
``include/tucker_stream.h`` (same names). Tensors are passed as device pointers; PyTorch supplies
device memory and streams. Raises ``RuntimeError`` when the CUDA library is missing -- there is no
CPU fallback.

Layout: a column-major (mode-1 fastest) tensor n_1 x ... x n_m is a row-major torch tensor of
shape (n_m, ..., n_1); :func:`paper_order` gives the view with the shape in paper order.
"""

from __future__ import annotations

import ctypes
import os

from .build import LIB as _LIB_PATH

MAX_MODES = 8
TUCKER_F32, TUCKER_F64 = 0, 1
TUCKER_PREC_FP64, TUCKER_PREC_MIXED = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECAPACITY", 4: "ENUMERIC", 5: "ETIMEOUT",
          6: "ECUDA", 7: "ESTATE"}
EXPORTS = ["tucker_init_sthosvd", "tucker_stream_update", "tucker_reconstruct",
           "tucker_error_norm", "tucker_get_ranks", "tucker_get_step_info", "tucker_copy_factor",
           "tucker_copy_core", "tucker_copy_sv", "tucker_last_error", "tucker_destroy",
           "tucker_version", "tucker_profile_enable", "tucker_profile_read",
           "tucker_reconstruct_noalloc", "tucker_ttm_workspace_bytes", "tucker_ttm_project",
           "tucker_ttm_reconstruct", "tucker_ttm_project_adjoint", "tucker_ttm_reconstruct_adjoint",
           "tucker_batch_create", "tucker_batch_update", "tucker_batch_kernels", "tucker_batch_destroy",
           "tucker_graph_kernels", "tucker_block_graph_kernels", "tucker_error_norm_async", "tucker_set_launch_plan",
           "tucker_get_launch_plan", "tucker_stream_update_host", "tucker_get_step_log",
           "tucker_replay_next", "tucker_stream_update_batched", "tucker_recompress",
           "tucker_test_stall_next", "tucker_orthogonality_error", "tucker_restore_orthogonality",
           "tucker_stream_update_block"]
NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024   # TUCKER_NOALLOC_SCRATCH_BYTES
NPHASES = 6


class TuckerConfig(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dtype", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("block_cap", ctypes.c_int32), ("n", ctypes.c_int64 * MAX_MODES),
                ("rank_cap", ctypes.c_int64 * MAX_MODES), ("steps_cap", ctypes.c_int64),
                ("core_cap", ctypes.c_int64), ("tau", ctypes.c_double), ("eps_m", ctypes.c_double)]


class TtmDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("n", ctypes.c_int64 * MAX_MODES), ("r", ctypes.c_int64 * MAX_MODES)]


class LaunchPlan(ctypes.Structure):
    _fields_ = [("grid_proj", ctypes.c_int32), ("grid_tc", ctypes.c_int32),
                ("grid_isvd", ctypes.c_int32), ("grid_cv", ctypes.c_int32)]


class StepInfo(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("y_norm2", ctypes.c_double),
                ("e_norm2", ctypes.c_double * MAX_MODES), ("grew", ctypes.c_int32 * MAX_MODES),
                ("r_add", ctypes.c_int32 * MAX_MODES), ("q", ctypes.c_double),
                ("augmented", ctypes.c_int32), ("r_stream", ctypes.c_int32),
                ("discarded", ctypes.c_double)]


class StepRecord(ctypes.Structure):
    _fields_ = [("n_d", ctypes.c_int64), ("ranks", ctypes.c_int32 * MAX_MODES),
                ("grew", ctypes.c_int32 * MAX_MODES), ("r_add", ctypes.c_int32 * MAX_MODES),
                ("eig_path", ctypes.c_int32 * MAX_MODES), ("eig_iters", ctypes.c_int32 * MAX_MODES),
                ("augmented", ctypes.c_int32), ("replayed", ctypes.c_int32),
                ("eps", ctypes.c_double), ("y_norm2", ctypes.c_double),
                ("e_norm2", ctypes.c_double * MAX_MODES), ("tail_cut", ctypes.c_double * MAX_MODES),
                ("tail_prev", ctypes.c_double * MAX_MODES), ("q", ctypes.c_double),
                ("discarded", ctypes.c_double)]


class Replay(ctypes.Structure):
    _fields_ = [("grow", ctypes.c_int32 * MAX_MODES), ("augment", ctypes.c_int32)]


class RecompressInfo(ctypes.Structure):
    _fields_ = [("ranks", ctypes.c_int64 * MAX_MODES), ("discarded", ctypes.c_double),
                ("err_bound", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NPHASES), ("bytes", ctypes.c_double * NPHASES),
                ("launches", ctypes.c_int64), ("updates", ctypes.c_int64),
                ("ms_slice_pass", ctypes.c_double)]


class TuckerError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libtucker_stream.so (built by ``paper_2308_16395_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.tucker_init_sthosvd.argtypes = [ctypes.POINTER(TuckerConfig), vp, i64, vp, ctypes.POINTER(vp)]
    lib.tucker_stream_update.argtypes = [vp, vp, vp]
    lib.tucker_stream_update_host.argtypes = [vp, vp, vp]
    lib.tucker_stream_update_block.argtypes = [vp, vp, ctypes.c_int32, vp]
    lib.tucker_reconstruct.argtypes = [vp, i64, i64, vp, vp]
    lib.tucker_reconstruct_noalloc.argtypes = [vp, i64, i64, vp, vp]
    lib.tucker_error_norm.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.tucker_get_ranks.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.tucker_get_step_info.argtypes = [vp, ctypes.POINTER(StepInfo)]
    lib.tucker_get_step_log.argtypes = [vp, i64, i64, ctypes.POINTER(StepRecord)]
    lib.tucker_replay_next.argtypes = [vp, ctypes.POINTER(Replay)]
    lib.tucker_copy_factor.argtypes = [vp, i32, vp]
    lib.tucker_copy_core.argtypes = [vp, vp]
    lib.tucker_copy_sv.argtypes = [vp, vp, vp]
    lib.tucker_recompress.argtypes = [vp, ctypes.c_double, vp, ctypes.POINTER(RecompressInfo)]
    lib.tucker_test_stall_next.argtypes = [vp]
    lib.tucker_orthogonality_error.argtypes = [vp, vp]
    lib.tucker_restore_orthogonality.argtypes = [vp, vp, vp]
    lib.tucker_last_error.argtypes = [vp]
    lib.tucker_last_error.restype = ctypes.c_char_p
    lib.tucker_destroy.argtypes = [vp]
    lib.tucker_destroy.restype = None
    lib.tucker_version.restype = ctypes.c_char_p
    lib.tucker_profile_enable.argtypes = [vp, i32]
    lib.tucker_profile_read.argtypes = [vp, ctypes.POINTER(Profile)]
    lib.tucker_batch_create.argtypes = [vp, vp, i32, ctypes.POINTER(vp)]
    lib.tucker_batch_create.restype = ctypes.c_int
    lib.tucker_batch_update.argtypes = [vp, vp]
    lib.tucker_stream_update_batched.argtypes = [vp, vp, i32, vp]
    lib.tucker_stream_update_batched.restype = ctypes.c_int
    lib.tucker_batch_update.restype = ctypes.c_int
    lib.tucker_set_launch_plan.argtypes = [vp, ctypes.POINTER(LaunchPlan)]
    lib.tucker_set_launch_plan.restype = ctypes.c_int
    lib.tucker_get_launch_plan.argtypes = [vp, ctypes.POINTER(LaunchPlan)]
    lib.tucker_get_launch_plan.restype = ctypes.c_int
    lib.tucker_error_norm_async.argtypes = [vp, vp, vp]
    lib.tucker_error_norm_async.restype = ctypes.c_int
    lib.tucker_graph_kernels.argtypes = [vp]
    lib.tucker_graph_kernels.restype = i64
    lib.tucker_block_graph_kernels.argtypes = [vp, i32]
    lib.tucker_block_graph_kernels.restype = i64
    lib.tucker_batch_kernels.argtypes = [vp]
    lib.tucker_batch_kernels.restype = i64
    lib.tucker_batch_destroy.argtypes = [vp]
    lib.tucker_batch_destroy.restype = None
    pdesc = ctypes.POINTER(TtmDesc)
    lib.tucker_ttm_workspace_bytes.argtypes = [pdesc]
    lib.tucker_ttm_workspace_bytes.restype = i64
    lib.tucker_ttm_project.argtypes = [pdesc, vp, vp, vp, vp, i64, vp]
    lib.tucker_ttm_reconstruct.argtypes = [pdesc, vp, vp, vp, vp, i64, vp]
    lib.tucker_ttm_project_adjoint.argtypes = [pdesc, vp, vp, vp, vp, vp, vp, i64, vp]
    lib.tucker_ttm_reconstruct_adjoint.argtypes = [pdesc, vp, vp, vp, vp, vp, vp, i64, vp]
    for name in ("tucker_ttm_project", "tucker_ttm_reconstruct", "tucker_ttm_project_adjoint",
                 "tucker_ttm_reconstruct_adjoint"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("tucker_profile_enable", "tucker_profile_read", "tucker_init_sthosvd", "tucker_stream_update",
                 "tucker_stream_update_host", "tucker_reconstruct",
                 "tucker_reconstruct_noalloc", "tucker_error_norm", "tucker_get_ranks", "tucker_get_step_info",
                 "tucker_get_step_log", "tucker_replay_next", "tucker_copy_factor", "tucker_copy_core", "tucker_copy_sv",
                 "tucker_recompress", "tucker_test_stall_next", "tucker_orthogonality_error",
                 "tucker_restore_orthogonality", "tucker_stream_update_block"):
        getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _check(code: int, handle=None):
    if code != 0:
        msg = ""
        if handle:
            msg = load_library().tucker_last_error(handle).decode()
        raise TuckerError(code, msg)


def make_config(n, tau, *, dtype="f32", precision="mixed", rank_cap=None, steps_cap=0,
                core_cap=0, eps_m=0.0, block_cap=0) -> TuckerConfig:
    """n: spatial sizes n_1..n_{d-1}; rank_cap: d entries (0 = default)."""
    c = TuckerConfig()
    c.block_cap = int(block_cap)
    c.ndim = len(n) + 1
    c.dtype = TUCKER_F32 if dtype in ("f32", "float32") else TUCKER_F64
    c.precision = TUCKER_PREC_MIXED if precision == "mixed" else TUCKER_PREC_FP64
    for i, v in enumerate(n):
        c.n[i] = int(v)
    if rank_cap is not None:
        for i, v in enumerate(rank_cap):
            c.rank_cap[i] = int(v)
    c.steps_cap = int(steps_cap)
    c.core_cap = int(core_cap)
    c.tau = float(tau)
    c.eps_m = float(eps_m)
    return c


# --- C ABI, same names ------------------------------------------------------------------------

def tucker_init_sthosvd(cfg: TuckerConfig, X_ptr: int, n_init: int, stream: int = 0) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.tucker_init_sthosvd(ctypes.byref(cfg), ctypes.c_void_p(X_ptr), int(n_init),
                                   ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def tucker_stream_update(h: int, Y_ptr: int, stream: int = 0) -> None:
    _check(load_library().tucker_stream_update(h, ctypes.c_void_p(Y_ptr), ctypes.c_void_p(stream)), h)


def tucker_stream_update_block(h: int, Y_ptr: int, nslices: int, stream: int = 0) -> None:
    """B slices at once (contiguous, slice after slice): the block update."""
    _check(load_library().tucker_stream_update_block(h, ctypes.c_void_p(Y_ptr), int(nslices),
                                                     ctypes.c_void_p(stream)), h)


def tucker_stream_update_host(h: int, Y_host_ptr: int, stream: int = 0) -> None:
    _check(load_library().tucker_stream_update_host(h, ctypes.c_void_p(Y_host_ptr), ctypes.c_void_p(stream)), h)


def tucker_reconstruct(h: int, t0: int, t1: int, out_ptr: int, stream: int = 0) -> None:
    _check(load_library().tucker_reconstruct(h, int(t0), int(t1), ctypes.c_void_p(out_ptr),
                                             ctypes.c_void_p(stream)), h)


def tucker_reconstruct_noalloc(h: int, t0: int, t1: int, out_ptr: int, stream: int = 0) -> None:
    """Allocation-free reconstruction (temporaries in the library's fixed device array)."""
    _check(load_library().tucker_reconstruct_noalloc(h, int(t0), int(t1), ctypes.c_void_p(out_ptr),
                                                     ctypes.c_void_p(stream)), h)


def tucker_error_norm(h: int) -> tuple[float, float]:
    e, n = ctypes.c_double(), ctypes.c_double()
    _check(load_library().tucker_error_norm(h, ctypes.byref(e), ctypes.byref(n)), h)
    return e.value, n.value


def tucker_error_norm_async(h: int, out_ptr: int, stream: int = 0) -> None:
    """Enqueue a copy of (err^2, ||X||^2) into host memory at out_ptr (2 doubles); no sync."""
    _check(load_library().tucker_error_norm_async(h, ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream)), h)


def tucker_get_ranks(h: int, d: int) -> tuple[tuple, int]:
    arr = (ctypes.c_int64 * MAX_MODES)()
    nd = ctypes.c_int64()
    _check(load_library().tucker_get_ranks(h, arr, ctypes.byref(nd)), h)
    return tuple(int(arr[i]) for i in range(d)), int(nd.value)


def tucker_get_step_info(h: int, d: int) -> dict:
    s = StepInfo()
    _check(load_library().tucker_get_step_info(h, ctypes.byref(s)), h)
    m = d - 1
    return dict(eps=s.eps, y_norm2=s.y_norm2, e_norm2=[s.e_norm2[i] for i in range(m)],
                grew=[bool(s.grew[i]) for i in range(m)], r_add=[s.r_add[i] for i in range(m)],
                q=s.q, augmented=bool(s.augmented), r_stream=s.r_stream, discarded=s.discarded)


def tucker_get_step_log(h: int, d: int, first: int, count: int) -> list[dict]:
    """Records [first, first + count) of the per-update log, one dict per update."""
    arr = (StepRecord * max(count, 1))()
    _check(load_library().tucker_get_step_log(h, int(first), int(count), arr), h)
    m = d - 1
    out = []
    for i in range(count):
        r = arr[i]
        out.append(dict(n_d=int(r.n_d), ranks=tuple(int(r.ranks[k]) for k in range(d)),
                        grew=[bool(r.grew[k]) for k in range(m)], r_add=[int(r.r_add[k]) for k in range(m)],
                        eig_path=[int(r.eig_path[k]) for k in range(m)],
                        eig_iters=[int(r.eig_iters[k]) for k in range(m)],
                        augmented=bool(r.augmented), replayed=bool(r.replayed), eps=r.eps,
                        y_norm2=r.y_norm2, e_norm2=[r.e_norm2[k] for k in range(m)],
                        tail_cut=[r.tail_cut[k] for k in range(m)],
                        tail_prev=[r.tail_prev[k] for k in range(m)], q=r.q, discarded=r.discarded))
    return out


def tucker_replay_next(h: int, grow, augment: int = -1) -> None:
    """Test hook: force the decisions of the next update (grow[k]: -1 own, 0 none, r > 0)."""
    rp = Replay()
    for k in range(MAX_MODES):
        rp.grow[k] = -1
    for k, v in enumerate(grow):
        rp.grow[k] = int(v)
    rp.augment = int(augment)
    _check(load_library().tucker_replay_next(h, ctypes.byref(rp)), h)


def tucker_copy_factor(h: int, mode: int, dst_ptr: int) -> None:
    _check(load_library().tucker_copy_factor(h, int(mode), ctypes.c_void_p(dst_ptr)), h)


def tucker_copy_core(h: int, dst_ptr: int) -> None:
    _check(load_library().tucker_copy_core(h, ctypes.c_void_p(dst_ptr)), h)


def tucker_copy_sv(h: int, S_ptr: int, V_ptr: int) -> None:
    _check(load_library().tucker_copy_sv(h, ctypes.c_void_p(S_ptr), ctypes.c_void_p(V_ptr)), h)


def tucker_orthogonality_error(h: int, d: int) -> list:
    """||U_k^T U_k - I||_F for every factor (FP64, on the device)."""
    out = (ctypes.c_double * d)()
    _check(load_library().tucker_orthogonality_error(h, out), h)
    return [float(v) for v in out]


def tucker_restore_orthogonality(h: int, stream: int = 0) -> float:
    """Replace U_d by its polar factor; returns the reconstruction change added to the bound."""
    ch = ctypes.c_double()
    _check(load_library().tucker_restore_orthogonality(h, ctypes.c_void_p(stream), ctypes.byref(ch)), h)
    return ch.value


def tucker_test_stall_next(h: int) -> None:
    """Test hook: the next update's mode-1 tensor-core pass withholds its loads (its waits run
    out, TUCKER_ETIMEOUT latches)."""
    _check(load_library().tucker_test_stall_next(h), h)


def tucker_recompress(h: int, d: int, tau_total: float, stream: int = 0) -> dict:
    """Batch ST-HOSVD (Alg. 2) of the current representation within tau_total ||X||."""
    info = RecompressInfo()
    _check(load_library().tucker_recompress(h, float(tau_total), ctypes.c_void_p(stream),
                                            ctypes.byref(info)), h)
    return {"ranks": tuple(int(info.ranks[k]) for k in range(d)), "discarded": info.discarded,
            "err_bound": info.err_bound}


def tucker_profile_enable(h: int, on: int = 1) -> None:
    _check(load_library().tucker_profile_enable(h, int(on)), h)


def tucker_profile_read(h: int) -> dict:
    p = Profile()
    _check(load_library().tucker_profile_read(h, ctypes.byref(p)), h)
    return dict(ms=[p.ms[i] for i in range(NPHASES)], bytes=[p.bytes[i] for i in range(NPHASES)],
                launches=int(p.launches), updates=int(p.updates), ms_slice_pass=p.ms_slice_pass)


# --- batched form -----------------------------------------------------------------------------

def tucker_batch_create(handles, slot_ptrs) -> int:
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*handles)
    ys = (ctypes.c_void_p * n)(*slot_ptrs)
    b = ctypes.c_void_p()
    _check(load_library().tucker_batch_create(hs, ys, n, ctypes.byref(b)))
    return b.value


def tucker_batch_update(b: int, stream: int = 0) -> None:
    _check(load_library().tucker_batch_update(b, ctypes.c_void_p(stream)))


def tucker_stream_update_batched(handles, slice_ptrs, stream: int = 0) -> None:
    """One update of each state from its own device slice, one graph launch (cached per list)."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*handles)
    ys = (ctypes.c_void_p * n)(*slice_ptrs)
    _check(load_library().tucker_stream_update_batched(hs, ys, n, ctypes.c_void_p(stream)))


def tucker_batch_kernels(b: int) -> int:
    return int(load_library().tucker_batch_kernels(b))


def tucker_batch_destroy(b: int) -> None:
    if b:
        load_library().tucker_batch_destroy(b)


class TuckerBatch:
    """Independent TuckerStream states advanced together, one CUDA-graph launch per time step.

    ``slots[i]`` is the device tensor the graph reads state i's next slice from (allocated here,
    shape and dtype of that stream's slices): write the time step's slices into the slots, then
    call :meth:`update`.
    """

    def __init__(self, streams, stream=None):
        import torch

        self.streams = list(streams)
        self.slots = [torch.empty(tuple(reversed(s.n)), dtype=s.dtype, device="cuda") for s in self.streams]
        self._stream = stream
        self.b = tucker_batch_create([s.h for s in self.streams], [y.data_ptr() for y in self.slots])

    def _sp(self) -> int:
        import torch

        s = self._stream if self._stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    @property
    def kernels(self) -> int:
        return tucker_batch_kernels(self.b)

    def update(self) -> None:
        tucker_batch_update(self.b, self._sp())
        for s in self.streams:
            s._stream = self._stream

    def close(self) -> None:
        if getattr(self, "b", None):
            tucker_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- projection / reconstruction chains and adjoints (include/tucker_ttm.h) --------------------

def ttm_desc(n, r, dtype="f32") -> TtmDesc:
    d = TtmDesc()
    d.ndim = len(n)
    d.dtype = TUCKER_F32 if dtype in ("f32", "float32") else TUCKER_F64
    for i, (a, b) in enumerate(zip(n, r)):
        d.n[i] = int(a)
        d.r[i] = int(b)
    return d


def _ptrs(ps):
    """Host array of device pointers (NULL entries allowed)."""
    if ps is None:
        return None
    arr = (ctypes.c_void_p * MAX_MODES)()
    for i, p in enumerate(ps):
        arr[i] = p or None
    return arr


def tucker_ttm_workspace_bytes(desc: TtmDesc) -> int:
    v = load_library().tucker_ttm_workspace_bytes(ctypes.byref(desc))
    if v < 0:
        raise TuckerError(1, "invalid ttm descriptor")
    return int(v)


def tucker_ttm_project(desc, U_ptrs, Y_ptr, G_ptr, work_ptr, work_bytes, stream=0) -> None:
    _check(load_library().tucker_ttm_project(ctypes.byref(desc), _ptrs(U_ptrs), ctypes.c_void_p(Y_ptr),
                                             ctypes.c_void_p(G_ptr), ctypes.c_void_p(work_ptr),
                                             int(work_bytes), ctypes.c_void_p(stream)))


def tucker_ttm_reconstruct(desc, U_ptrs, G_ptr, Y_ptr, work_ptr, work_bytes, stream=0) -> None:
    _check(load_library().tucker_ttm_reconstruct(ctypes.byref(desc), _ptrs(U_ptrs), ctypes.c_void_p(G_ptr),
                                                 ctypes.c_void_p(Y_ptr), ctypes.c_void_p(work_ptr),
                                                 int(work_bytes), ctypes.c_void_p(stream)))


def tucker_ttm_project_adjoint(desc, U_ptrs, Y_ptr, Gbar_ptr, Ybar_ptr, Ubar_ptrs, work_ptr,
                               work_bytes, stream=0) -> None:
    _check(load_library().tucker_ttm_project_adjoint(
        ctypes.byref(desc), _ptrs(U_ptrs), ctypes.c_void_p(Y_ptr), ctypes.c_void_p(Gbar_ptr),
        ctypes.c_void_p(Ybar_ptr), _ptrs(Ubar_ptrs), ctypes.c_void_p(work_ptr), int(work_bytes),
        ctypes.c_void_p(stream)))


def tucker_ttm_reconstruct_adjoint(desc, U_ptrs, G_ptr, Yhbar_ptr, Gbar_ptr, Ubar_ptrs, work_ptr,
                                   work_bytes, stream=0) -> None:
    _check(load_library().tucker_ttm_reconstruct_adjoint(
        ctypes.byref(desc), _ptrs(U_ptrs), ctypes.c_void_p(G_ptr), ctypes.c_void_p(Yhbar_ptr),
        ctypes.c_void_p(Gbar_ptr), _ptrs(Ubar_ptrs), ctypes.c_void_p(work_ptr), int(work_bytes),
        ctypes.c_void_p(stream)))


def tucker_set_launch_plan(h: int, grid_proj=0, grid_tc=0, grid_isvd=0, grid_cv=0) -> None:
    p = LaunchPlan(int(grid_proj), int(grid_tc), int(grid_isvd), int(grid_cv))
    _check(load_library().tucker_set_launch_plan(h, ctypes.byref(p)), h)


def tucker_get_launch_plan(h: int) -> dict:
    p = LaunchPlan()
    _check(load_library().tucker_get_launch_plan(h, ctypes.byref(p)), h)
    return dict(grid_proj=p.grid_proj, grid_tc=p.grid_tc, grid_isvd=p.grid_isvd, grid_cv=p.grid_cv)


def tucker_graph_kernels(h: int) -> int:
    return int(load_library().tucker_graph_kernels(h))


def tucker_block_graph_kernels(h: int, nslices: int) -> int:
    return int(load_library().tucker_block_graph_kernels(h, int(nslices)))


def tucker_last_error(h: int) -> str:
    return load_library().tucker_last_error(h).decode()


def tucker_destroy(h: int) -> None:
    if h:
        load_library().tucker_destroy(h)


def tucker_version() -> str:
    return load_library().tucker_version().decode()


def paper_order(t):
    """View of a row-major torch tensor as the column-major tensor in paper index order."""
    return t.permute(*reversed(range(t.dim())))


class TuckerStream:
    """Streaming Tucker state on the current CUDA device (torch tensors in, torch tensors out).

    ``X`` holds the first slices as a row-major tensor of shape (n_init, n_{d-1}, ..., n_1)
    (i.e. column-major n_1 x ... x n_{d-1} x n_init). Every method calls the C ABI.
    """

    def __init__(self, X, tau, *, precision="mixed", rank_cap=None, steps_cap=0, core_cap=0,
                 eps_m=0.0, block_cap=0, stream=None):
        import torch

        if not X.is_cuda:
            raise ValueError("X must be a CUDA tensor")
        X = X.contiguous()
        self.n = tuple(reversed(X.shape[1:]))
        self.d = len(self.n) + 1
        self.dtype = X.dtype
        dt = "f32" if X.dtype == torch.float32 else "f64"
        self.cfg = make_config(self.n, tau, dtype=dt, precision=precision, rank_cap=rank_cap,
                               steps_cap=steps_cap, core_cap=core_cap, eps_m=eps_m,
                               block_cap=block_cap)
        self._stream = stream
        self.n_init = int(X.shape[0])
        self.h = tucker_init_sthosvd(self.cfg, X.data_ptr(), X.shape[0], self._sp())

    def _sp(self) -> int:
        import torch

        s = self._stream if self._stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    def update(self, Y) -> None:
        if tuple(reversed(Y.shape)) != self.n or Y.dtype != self.dtype or not Y.is_contiguous():
            raise ValueError("slice shape/dtype/layout mismatch")
        tucker_stream_update(self.h, Y.data_ptr(), self._sp())

    def update_block(self, Yb) -> None:
        """B slices at once: Yb row-major (B, n_{d-1}, ..., n_1), contiguous on the device."""
        if tuple(reversed(Yb.shape[1:])) != self.n or Yb.dtype != self.dtype or not Yb.is_contiguous():
            raise ValueError("block shape/dtype/layout mismatch")
        tucker_stream_update_block(self.h, Yb.data_ptr(), int(Yb.shape[0]), self._sp())

    def update_host(self, Y) -> None:
        """Update from a slice in host memory (a CPU tensor, pinned for overlap): the library
        copies it into a staging buffer on its own copy stream and updates after the copy."""
        if (Y.device.type != "cpu" or tuple(reversed(Y.shape)) != self.n or Y.dtype != self.dtype
                or not Y.is_contiguous()):
            raise ValueError("host slice shape/dtype/layout mismatch")
        tucker_stream_update_host(self.h, Y.data_ptr(), self._sp())

    @property
    def ranks(self) -> tuple:
        return tucker_get_ranks(self.h, self.d)[0]

    @property
    def n_d(self) -> int:
        return tucker_get_ranks(self.h, self.d)[1]

    def error_norm(self) -> tuple[float, float]:
        return tucker_error_norm(self.h)

    def step_info(self) -> dict:
        return tucker_get_step_info(self.h, self.d)

    def step_log(self, first: int = 0, count: int | None = None) -> list[dict]:
        """Per-update records (decisions, norms, tails) of updates [first, first + count)."""
        if count is None:
            count = self.n_d - self.n_init - first
        return tucker_get_step_log(self.h, self.d, first, count)

    def replay_next(self, grow, augment: int = -1) -> None:
        """Test hook: force the next update's decisions (see tucker_replay_next)."""
        tucker_replay_next(self.h, grow, augment)

    def orthogonality_error(self) -> list:
        """||U_k^T U_k - I||_F for every factor (see tucker_orthogonality_error)."""
        return tucker_orthogonality_error(self.h, self.d)

    def restore_orthogonality(self) -> float:
        """Polar factor of U_d (see tucker_restore_orthogonality)."""
        return tucker_restore_orthogonality(self.h, self._sp())

    def recompress(self, tau_total: float) -> dict:
        """Re-compress within tau_total ||X|| (see tucker_recompress)."""
        return tucker_recompress(self.h, self.d, tau_total, self._sp())

    def reconstruct(self, t0: int, t1: int):
        import torch

        out = torch.empty((t1 - t0,) + tuple(reversed(self.n)), dtype=self.dtype, device="cuda")
        tucker_reconstruct(self.h, t0, t1, out.data_ptr(), self._sp())
        return out

    def factor(self, k: int):
        """U_k as an FP64 (rows x r_k) tensor."""
        import torch

        ranks, nd = tucker_get_ranks(self.h, self.d)
        rows = self.n[k] if k < self.d - 1 else nd
        buf = torch.empty((ranks[k], rows), dtype=torch.float64, device="cuda")
        tucker_copy_factor(self.h, k, buf.data_ptr())
        return buf.t()

    def core(self):
        """C as an FP64 tensor in paper index order (r_1, ..., r_d)."""
        import torch

        ranks = self.ranks
        buf = torch.empty(tuple(reversed(ranks)), dtype=torch.float64, device="cuda")
        tucker_copy_core(self.h, buf.data_ptr())
        return paper_order(buf)

    def sv(self):
        """(S, V) with V in paper index order."""
        import torch

        ranks = self.ranks
        S = torch.empty((ranks[-1],), dtype=torch.float64, device="cuda")
        V = torch.empty(tuple(reversed(ranks)), dtype=torch.float64, device="cuda")
        tucker_copy_sv(self.h, S.data_ptr(), V.data_ptr())
        return S, paper_order(V)

    def close(self) -> None:
        if getattr(self, "h", None):
            tucker_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
