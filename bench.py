#!/usr/bin/env python
"""Benchmark of the streaming ST-HOSVD update on one GB300 (or N independent replicas).

Default workload (``--workload stream``): the large advected-blob stream, 4-way slices
384 x 384 x 256 x 4 (x, y, z, variable) of 80 advected anisotropic Gaussian blobs, FP32 storage
(604 MB per slice), tau = 1e-4, initial ST-HOSVD on the first 10 slices, then one update (Alg. 5)
per step with the full mixed-precision path. Every step assimilates a new slice larger than the
129 MB L2; all slices are resident in HBM before the timed region. ``--workload stream192``: the
192 x 192 x 96 x 12 stream of 40 blobs (170 MB slices), with the plain FP64 GPU form beside it.
Prints one JSON line (rank 0), with the parity of the timed updates against the FP64 CPU oracle
(run over exactly the same stream in the CPU-baseline leg).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload stream|stream192|stream64|batched|adjoint|sine|block]
                  [--precision mixed|fp64] [--block B]

--impl reference times the FP64 CPU oracle (the reference arm of this build) on the host cores.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "slices/s and GB/s ingested at ≤1e-5 rel. error vs FP64 oracle; % of roofline"
N_INIT = 10
# single-stream workloads: (grid, variables, blobs, seed, tau)
STREAMS = {
    "stream": dict(grid=(384, 384, 256), nvar=4, nblobs=80, seed=5, tau=1e-4,
                   name="advected-blob stream 384x384x256x4 fp32 slices (80 blobs, 604 MB per slice)"),
    "stream192": dict(grid=(192, 192, 96), nvar=12, nblobs=40, seed=2, tau=1e-4,
                      name="advected-blob stream 192x192x96x12 fp32 slices (40 blobs, 170 MB per slice)"),
    # the 384 x 384 x 256 x 4 stream cut to 64 planes: the small case the kernel captures run on
    # (151 MB slices, above L2, a few GB on the device)
    "stream64": dict(grid=(384, 384, 64), nvar=4, nblobs=80, seed=5, tau=1e-4,
                     name="advected-blob stream 384x384x64x4 fp32 slices (80 blobs, 151 MB per slice)"),
}
DELTA_DEC = 3e-2    # relative distance of a near-cutoff decision from eps^2 (mixed form)
PHASES = ["mode-1 projection + residual (k_tc_pass16)", "k_ttm_proj (modes 2..d-1)", "growth (gram/eig/append)",
          "isvd (k_isvd_p/k_isvd_e/secular)", "factor (k_ud_update/k_core_m)", "k_cv_update (C and V)"]
KERNEL_OF_PHASE = ["k_tc_pass16<1, 0>", "k_tc_pass16", "k_resid_gram", "k_isvd_e", "k_core_m", "k_cv_update"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6780.7), "measured"
    return 6800.0, "fallback"


def _traffic_table():
    """Per-launch DRAM bytes of the kernels, from the committed ncu summary (profiles/)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)   # the first sample lands inside the timed region
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _blobfield(wl: str):
    from workloads import BlobField

    c = STREAMS[wl]
    return BlobField(grid=c["grid"], nvar=c["nvar"], nblobs=c["nblobs"], noise=1e-5, seed=c["seed"])


def _host64(y):
    """A device slice (row-major (n_{d-1}, ..., n_1)) as a Fortran-ordered FP64 NumPy array."""
    import numpy as np

    return y.cpu().numpy().T.astype(np.float64)


# ---------------------------------------------------------------------------------------------
# CPU-baseline leg: the FP64 oracle over the same stream, timed, and the parity of the GPU run
# ---------------------------------------------------------------------------------------------

def _oracle_margins(rec, eps2):
    """Relative distances |stat - eps^2| / eps^2 of one oracle update's decisions."""
    import numpy as np

    out = {}
    for m in rec["modes"]:
        out[f"branch{m.k + 1}"] = abs(m.e_norm2 - eps2) / eps2
        if m.grew and m.lam is not None:
            lam = np.asarray(m.lam)
            tails = np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])
            r = m.r_add
            out[f"cut{m.k + 1}"] = min(abs(tails[r] - eps2), abs(tails[r - 1] - eps2)) / eps2
    out["isvd"] = abs(rec["isvd"].q ** 2 - eps2) / eps2
    return out


def oracle_leg(wl: str, slices, W: int, K: int, snap: dict | None):
    """Run the FP64 oracle (host cores) over the initial slices, the W warm-up updates and the K
    timed updates of the GPU run; time the K timed updates; compare with the GPU snapshot."""
    import numpy as np

    import oracle as O

    tau = STREAMS[wl]["tau"]
    X0 = np.asfortranarray(np.stack([_host64(slices[t]) for t in range(N_INIT)], axis=-1))
    st = O.init_stream(X0, tau)
    del X0
    for t in range(N_INIT, N_INIT + W):
        O.stream_update(st, _host64(slices[t]))
    dt = 0.0
    for t in range(N_INIT + W, N_INIT + W + K):
        Y = _host64(slices[t])
        t0 = time.perf_counter()
        O.stream_update(st, Y)
        dt += time.perf_counter() - t0
    cpu = {"value": K / dt, "unit": "slices/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"FP64 NumPy oracle on the same stream: initial ST-HOSVD of {N_INIT} slices and "
                     f"{W} warm-up updates (untimed), then the {K} timed updates of the GPU run"}
    if snap is None:
        return cpu, None, st.ranks
    par = {"delta_dec": DELTA_DEC}
    upd = [r for r in st.log if r["kind"] == "update"]
    gl = snap["log"]
    trace_equal, first_flip = True, None
    for i, (ro, rg) in enumerate(zip(upd, gl)):
        if tuple(ro["ranks"]) != tuple(rg["ranks"]):
            trace_equal = False
            marg = _oracle_margins(ro, ro["eps"] ** 2)
            first_flip = {"update": i, "t": N_INIT + i, "oracle_ranks": list(ro["ranks"]),
                          "gpu_ranks": list(rg["ranks"]), "smallest_margin": min(marg.values()),
                          "margins": {k: float(v) for k, v in marg.items()}}
            break
    par["updates_compared"] = len(gl)
    par["rank_trace_equal"] = trace_equal
    par["first_flip"] = first_flip
    if first_flip is not None:
        par["flip_within_delta_dec"] = first_flip["smallest_margin"] < DELTA_DEC
    par["oracle_final_ranks"] = list(st.ranks)
    par["gpu_final_ranks"] = list(snap["ranks"])
    if trace_equal:
        # reconstructions of the sampled slices (invariant to sign and rotation freedom)
        rd = []
        for t, xg in snap["recon"].items():
            xo = O.reconstruct_slices(st, t, t + 1)[..., 0]
            rd.append(float(np.linalg.norm(xg.astype(np.float64) - xo) / np.linalg.norm(xo)))
        par["recon_slices"] = sorted(snap["recon"].keys())
        par["recon_rel_diff_max"] = max(rd)
        # largest principal angle between the oracle's and the GPU's factor subspaces
        sines = []
        for k, Ug in enumerate(snap["factors"]):
            Uo = st.Us[k]
            Pg = Ug - Uo @ (Uo.T @ Ug)
            sines.append(float(np.linalg.norm(Pg, 2)))
        par["subspace_sin_max"] = sines
        # core after aligning the column signs of every factor
        Cg = snap["core"]
        for k, Ug in enumerate(snap["factors"]):
            sg = np.sign(np.sum(st.Us[k] * Ug, axis=0))
            sg[sg == 0] = 1.0
            shape = [1] * Cg.ndim
            shape[k] = -1
            Cg = Cg * sg.reshape(shape)
        par["core_rel_diff_aligned"] = float(np.linalg.norm(Cg - st.C) / np.linalg.norm(st.C))
        par["recon_within_1e-5"] = par["recon_rel_diff_max"] <= 1e-5
    par["gpu_true_rel_error"] = snap["true_rel"]
    par["gpu_bound_rel"] = snap["bound_rel"]
    par["oracle_bound_rel"] = math.sqrt(st.err2 / st.data_norm2)
    par["tau"] = tau
    par["error_within_tau"] = snap["true_rel"] <= tau
    return cpu, par, st.ranks


def gpu_snapshot(pkg, ts, slices, t_end: int, samples):
    """State of the GPU run for the parity leg: update log, ranks, factors and core (FP64), the
    reconstruction of a few slices, and the true error over every slice seen."""
    import torch

    d = ts.d
    snap = {"log": ts.step_log(0, t_end - N_INIT), "ranks": ts.ranks}
    snap["factors"] = [ts.factor(k).cpu().numpy() for k in range(d)]
    snap["core"] = ts.core().cpu().numpy()
    snap["recon"] = {}
    err2 = tot2 = 0.0
    for t in range(t_end):
        xh = ts.reconstruct(t, t + 1)[0]
        err2 += float(torch.sum((xh.double() - slices[t].double()) ** 2))
        tot2 += float(torch.sum(slices[t].double() ** 2))
        if t in samples:
            snap["recon"][t] = xh.cpu().numpy().T.copy()
        del xh
    snap["true_rel"] = math.sqrt(err2 / tot2)
    eb, dn = ts.error_norm()
    snap["bound_rel"] = eb / dn
    return snap


def _reference_line(args, rate, unit, workload, sample, extra=None, dtype="f64", hib=True):
    line = {
        "metric": METRIC, "value": rate, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 / rate, "higher_is_better": hib,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "impl": "reference", "config": {"workload": workload, "parallelism": "host cores (numpy)"},
        "cpu_baseline": {"value": rate, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    line.update(extra or {})
    print(json.dumps(line), flush=True)


def run_reference_other(args):
    """The FP64 oracle on the host cores for the sine, block, adjoint and batched workloads: a
    bounded sample of each, on the workload, metric and unit of this build's line for it."""
    import numpy as np

    import oracle as O

    K = max(1, min(args.steps, 40))
    wl = args.workload
    if wl == "sine":
        from workloads import SineWave

        sw = SineWave()
        n_init, tau = 200, 1e-2
        xs = [sw.slice(t) for t in range(n_init + K)]
        st = O.init_stream(np.asfortranarray(np.stack(xs[:n_init], axis=-1)), tau)
        t0 = time.perf_counter()
        for t in range(n_init, n_init + K):
            O.stream_update(st, xs[t])
        rate = K / (time.perf_counter() - t0)
        _reference_line(args, rate, "slices/s",
                        "sine-wave stream (Sec. 5.1): 100x100 spatial, 5000 steps, rank bump at "
                        "2500, eta=1e-3, tau=1e-2, n_init=200",
                        f"FP64 oracle: initial ST-HOSVD of 200 slices (untimed), {K} timed updates",
                        {"final_ranks": list(st.ranks)})
    elif wl == "block":
        from workloads import LowRankStream

        B = args.block
        ne, tau = 10, 1e-3
        nb = max(1, min(K, 30))
        lrs = LowRankStream((24, 20, 16), (4, 4, 3, 6), ne + B * nb, 1e-4, seed=1, noise_scope="tensor")
        X = lrs.tensor(0, ne + B * nb)
        st = O.init_stream(np.asfortranarray(X[..., :ne]), tau)
        t0 = time.perf_counter()
        for i in range(nb):
            O.block_update(st, np.asfortranarray(X[..., ne + i * B:ne + (i + 1) * B]))
        rate = nb * B / (time.perf_counter() - t0)
        _reference_line(args, rate, "slices/s",
                        f"block update (B = {B} slices per call); the oracle's block update on the "
                        "exact-rank 24x20x16 stream",
                        f"FP64 oracle block update, {nb} blocks of {B} after an untimed initial "
                        "ST-HOSVD of 10 slices", {"final_ranks": list(st.ranks)})
    elif wl == "adjoint":
        import oracle.tucker_adjoint as OA

        rng = np.random.default_rng(230816395 + 3)
        n, r = (128, 128, 64), (20, 20, 12)
        Y = rng.standard_normal(n)
        T = rng.standard_normal(n)
        Us = [np.linalg.qr(rng.standard_normal((nk, rk)))[0] for nk, rk in zip(n, r)]
        reps = max(1, min(K, 3))
        t0 = time.perf_counter()
        for _ in range(reps):
            OA.composite_grad(Y, Us, T)
        rate = reps / (time.perf_counter() - t0)
        _reference_line(args, rate, "slices/s",
                        "adjoint: gradient of ||(Y x U^T) x U - T||^2 w.r.t. Y and U_n, "
                        "128x128x64, ranks (20,20,12)",
                        f"FP64 oracle gradient (oracle/tucker_adjoint.py), {reps} evaluations")
    else:   # batched
        from workloads import batched_streams

        specs = batched_streams(nstreams=64, steps=100)
        n_up, dt, n_sl = max(1, min(K, 5)), 0.0, 0
        for s, tau in specs[:3]:
            xs = [s.slice(t).astype(np.float64) for t in range(N_INIT + n_up)]
            st = O.init_stream(np.asfortranarray(np.stack(xs[:N_INIT], axis=-1)), tau)
            t0 = time.perf_counter()
            for t in range(N_INIT, N_INIT + n_up):
                O.stream_update(st, np.asfortranarray(xs[t]))
            dt += time.perf_counter() - t0
            n_sl += n_up
        _reference_line(args, n_sl / dt, "slices/s",
                        "batched: 64 independent streams, sizes U{32..160}^3, ranks 4..24, "
                        "noise 1e-4, tau in {1e-2,1e-3,1e-4}",
                        f"FP64 oracle, streams 0-2 of the 64 (their own sizes), {n_up} updates each "
                        "after an untimed initial ST-HOSVD")


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    if args.workload in ("sine", "block", "adjoint", "batched"):
        run_reference_other(args)
        return
    import torch

    wl = args.workload if args.workload in STREAMS else "stream"
    K = max(1, min(args.steps, 40))
    W = min(args.warmup, 5)
    bf = _blobfield(wl)
    slices = [bf.slice_torch(t, "cuda") for t in range(N_INIT + W + K)]
    torch.cuda.synchronize()
    cpu, _, ranks = oracle_leg(wl, slices, W, K, None)
    rate = cpu["value"]
    line = {
        "metric": METRIC, "value": rate, "unit": "slices/s", "n_gpus": args.gpus, "steps": K,
        "warmup": W, "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": STREAMS[wl]["name"] + f", tau={STREAMS[wl]['tau']:g}, n_init={N_INIT}",
                   "parallelism": "host cores (numpy)"},
        "cpu_baseline": dict(cpu),
        "e2e": {"value": rate, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "final_ranks": list(ranks),
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import paper_2308_16395_gb300 as pkg

    wl = args.workload
    conf = STREAMS[wl]
    tau = conf["tau"]
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    bf = _blobfield(wl)
    K, W = args.steps, args.warmup
    KP = min(K, 8)                   # profiled updates (launch by launch, phase events)
    KE = 0 if args.no_e2e else min(K, 10)   # end-to-end updates (host slices in)
    T_timed = N_INIT + W + K
    T = T_timed + KP + KE
    dev = torch.device("cuda", local)
    slices = [bf.slice_torch(t, dev) for t in range(T)]         # row-major (nvar, n3, n2, n1) FP32
    torch.cuda.synchronize()
    slice_bytes = slices[0].numel() * slices[0].element_size()
    # the streaming rank never exceeds the number of slices seen, so that bounds its capacity
    # (and the row stride of the core and V)
    caps = [0, 0, 0, 0, min(256, (T + 4 + 7) // 8 * 8)]
    kw = dict(precision=args.precision, rank_cap=caps, steps_cap=T + 4, core_cap=4 << 20)

    X0 = torch.stack(slices[:N_INIT]).contiguous()
    ts = pkg.TuckerStream(X0, tau, **kw)
    del X0
    torch.cuda.synchronize()
    for t in range(N_INIT, N_INIT + W):
        ts.update(slices[t])   # the first update captures the graph
    ts.ranks  # synchronizes, surfaces latched errors

    # ---- device-resident timed region (graph form of the update) ----
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(N_INIT + W, T_timed):
        ts.update(slices[t])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    graph_kernels = pkg.tucker_graph_kernels(ts.h)
    ranks = ts.ranks
    eb, dn = ts.error_norm()
    log = ts.step_log(0, T_timed - N_INIT)
    grown = sum(sum(r["grew"]) for r in log[W:])
    if dist:
        t_ = torch.tensor([ms], device=dev)
        dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        ms = float(t_.item())
    snap = None
    want_parity = rank == 0 and ws == 1 and not args.no_cpu
    if want_parity:
        samples = {N_INIT + W, (N_INIT + W + T_timed - 1) // 2, T_timed - 1}
        snap = gpu_snapshot(pkg, ts, slices, T_timed, samples)

    # ---- the next KP updates of the same stream launch by launch, CUDA events around each
    # phase and around the slice-pass kernel (phase breakdown, roofline of the slice pass) ----
    pkg.tucker_profile_enable(ts.h, 1)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for t in range(T_timed, T_timed + KP):
        ts.update(slices[t])
    p1.record(stream)
    torch.cuda.synchronize()
    ms_eager = p0.elapsed_time(p1)
    prof = pkg.tucker_profile_read(ts.h)
    pkg.tucker_profile_enable(ts.h, 0)

    # ---- end to end: the next KE slices from pinned host memory through the library's
    # host-input update (tucker_stream_update_host: copy on the library's copy stream into
    # alternating staging buffers, update after the copy, so slice t+1's copy overlaps update
    # t), and the step's result (error bound and data norm) out every step into pinned host
    # memory ----
    e2e = None
    if KE:
        t_e = T_timed + KP
        host = [slices[t].cpu().pin_memory() for t in range(t_e, t_e + KE)]
        # each pinned buffer goes to the device once before the timed region: the first
        # device access to freshly pinned pages on this host runs at about half the link's rate
        # (the pages are mapped for the GPU on first use), which a streaming application's reused
        # ring of pinned buffers pays once
        scratch = torch.empty_like(slices[0])
        for h in host:
            scratch.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        del scratch
        res = torch.zeros((KE, 2), dtype=torch.float64).pin_memory()
        # the first host-input call allocates the staging buffers: outside the timed region
        ts.update_host(host[0])
        pkg.tucker_error_norm_async(ts.h, res[0].data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(1, KE):
            ts.update_host(host[i])
            pkg.tucker_error_norm_async(ts.h, res[i].data_ptr(), stream.cuda_stream)
        f1.record(stream)
        torch.cuda.synchronize()
        ms2 = f0.elapsed_time(f1)
        eb2 = ts.error_norm()[0]
        assert abs(float(res[KE - 1, 0]) ** 0.5 - eb2) <= 1e-12 * (1 + eb2)
        if dist:
            t_ = torch.tensor([ms2], device=dev)
            dist.all_reduce(t_, op=dist.ReduceOp.MAX)
            ms2 = float(t_.item())
        n_e = KE - 1
        e2e = {"value": ws * n_e / (ms2 / 1e3), "unit": "slices/s", "h2d_bytes_per_step": slice_bytes,
               "d2h_bytes_per_step": 16, "steps": n_e,
               "api": "tucker_stream_update_host + tucker_error_norm_async",
               "pipeline": "H2D of slice t+1 (library copy stream) overlaps update t",
               "host_buffers": "one pinned buffer per timed slice, each copied to the device once before the timed region (first-use page mapping, as a reused ring pays once)",
               "ms_per_step": ms2 / n_e}
        del host
    ts.close()

    # ---- the plain FP64 GPU form on the same slices (a few updates, graph form) ----
    fp64_form = None
    if args.precision == "mixed" and not args.no_fp64 and wl == "stream192":
        K64 = min(K, 5)
        kw64 = dict(kw, precision="fp64")
        X0 = torch.stack(slices[:N_INIT]).contiguous()
        t64 = pkg.TuckerStream(X0, tau, **kw64)
        del X0
        for t in range(N_INIT, N_INIT + W):
            t64.update(slices[t])
        t64.ranks
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for t in range(N_INIT + W, N_INIT + W + K64):
            t64.update(slices[t])
        q1.record(stream)
        torch.cuda.synchronize()
        ms64 = q0.elapsed_time(q1) / K64
        fp64_form = {"ms_per_step": ms64, "slices_per_s": 1e3 / ms64, "steps": K64,
                     "ranks": list(t64.ranks),
                     "note": "every step FP64 (SIMT contractions, FP64 eigensolves), same slices"}
        t64.close()
    elif wl == "stream":
        fp64_form = {"skipped": "the FP64 form's eigensolves of 384 x 384 Grams run for seconds each "
                                "on this part (FP64 is a small fraction of the FP32 rate); "
                                "--workload stream192 carries the comparison"}

    # ---- roofline of the pass over the slice (live CUDA events, library byte accounting) ----
    peak, peak_src = _peaks()
    ph = 0
    ms_k = prof["ms_slice_pass"]
    nprof = max(prof["updates"], 1)
    achieved = prof["bytes"][ph] / (ms_k / 1e3) / 1e9 if ms_k > 0 else 0.0
    traffic = _traffic_table().get(f"{KERNEL_OF_PHASE[ph]}@{wl}")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": KERNEL_OF_PHASE[ph] + " (" + PHASES[ph] + ")",
                "kernel_ms_per_launch": ms_k / nprof,
                "algorithmic_bytes_per_launch": prof["bytes"][ph] / nprof,
                "peak_source": peak_src,
                "profiled_updates": f"t={T_timed}..{T_timed + KP - 1} (the updates after the timed ones)",
                "phases_ms_per_step": {PHASES[i]: prof["ms"][i] / nprof for i in range(len(PHASES))},
                "phases_gbs": {PHASES[i]: (prof["bytes"][i] / (prof["ms"][i] / 1e3) / 1e9
                                           if prof["ms"][i] > 0 else 0.0) for i in range(len(PHASES))},
                "launch_sequence_ms_per_step": ms_eager / max(KP, 1)}

    value = ws * K / (ms / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": conf["name"] + f", tau={tau:g}, n_init={N_INIT}, "
                               f"timed updates t={N_INIT + W}..{T_timed - 1}",
                   "precision": args.precision, "parallelism": "replicas" if ws > 1 else "1 gpu",
                   "l2": f"inputs larger than L2: every step reads a new {slice_bytes / 1e6:.0f} MB slice"},
        "gbs_ingested": value * slice_bytes / 1e9,
        "final_ranks": list(ranks), "rel_error_bound": eb / dn,
        "grown_modes_in_timed_updates": grown,
        "gpu_launches": int(graph_kernels) * K,
        "gpu_launches_note": "kernel nodes of the update graph (conditional growth bodies included, an upper bound) x steps",
        "roofline": roofline,
        "clocks": ck,
        "e2e": e2e,
        "fp64_form": fp64_form,
    }
    del slices[T_timed:]
    if want_parity:
        try:
            cpu, par, _ = oracle_leg(wl, slices, W, K, snap)
            out["cpu_baseline"] = cpu
            out["parity"] = par
        except Exception as e:  # report, do not fail the GPU line
            out["cpu_baseline"] = {"value": None, "error": str(e)[:300]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_adjoint(args):
    """Gradient evaluations of L = ||(Y x_n U_n^T) x_n U_n - T||^2 with respect to Y and every
    U_n: 128 x 128 x 64 FP32 slices, ranks (20, 20, 12); forward and backward through the C ABI
    (tucker_ttm_*), timed eagerly and as one captured CUDA graph per evaluation."""
    import torch

    from paper_2308_16395_gb300 import autograd as ag

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, r = (128, 128, 64), (20, 20, 12)
    g = torch.Generator(device="cpu").manual_seed(230816395 + 3)
    Yh_host = torch.randn(tuple(reversed(n)), generator=g).pin_memory()
    Th_host = torch.randn(tuple(reversed(n)), generator=g).pin_memory()
    Us = []
    for nk, rk in zip(n, r):
        q, _ = torch.linalg.qr(torch.randn(nk, rk, generator=g, dtype=torch.float64))
        Us.append(q.float().t().contiguous().to(dev).t().requires_grad_(True))   # column-major
    Y = Yh_host.to(dev).permute(2, 1, 0).requires_grad_(True)
    T = Th_host.to(dev).permute(2, 1, 0)

    def step():
        G = ag.project(Y, Us)
        L = ((ag.reconstruct(G, Us) - T) ** 2).sum()
        L.backward()
        return L

    for _ in range(max(args.warmup, 3)):
        Y.grad = None
        for U in Us:
            U.grad = None
        step()
    torch.cuda.synchronize()
    K = args.steps
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(K):
        Y.grad = None
        for U in Us:
            U.grad = None
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms_eager = e0.elapsed_time(e1) / K
    # one CUDA graph per gradient evaluation
    side = torch.cuda.Stream()
    side.wait_stream(st)
    with torch.cuda.stream(side):
        for _ in range(3):
            Y.grad = None
            for U in Us:
                U.grad = None
            step()
    st.wait_stream(side)
    Y.grad = None
    for U in Us:
        U.grad = None
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        Ls = step()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0.record(st)
    for _ in range(K):
        graph.replay()
    e1.record(st)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms_graph = e0.elapsed_time(e1) / K
    # end to end: host Y and T copied in, the loss read back, every evaluation
    Yin = Y.detach()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(st)
    for _ in range(K):
        Yin.permute(2, 1, 0).copy_(Yh_host, non_blocking=True)
        T.permute(2, 1, 0).copy_(Th_host, non_blocking=True)
        graph.replay()
        float(Ls.item())
    f1.record(st)
    torch.cuda.synchronize()
    ms_e2e = f0.elapsed_time(f1) / K
    N = n[0] * n[1] * n[2]
    # algorithmic bytes of one evaluation: Y and T read, dL/dY written, each mode product over a
    # full-size operand reads or writes N values (3 forward, 3 for dL/dG, 2 partial chains of the
    # factor gradients, 3 for dL/dY), FP32
    alg_bytes = 4 * N * (3 + 11)
    line = {
        "metric": METRIC, "value": 1e3 / ms_graph, "unit": "slices/s", "n_gpus": 1, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "adjoint: gradient of ||(Y x U^T) x U - T||^2 w.r.t. Y and U_n, "
                               "128x128x64 fp32, ranks (20,20,12)", "parallelism": "1 gpu",
                   "l2": "8 MB working set, L2-resident (latency-bound by design)"},
        "eager_ms_per_eval": ms_eager, "graph_ms_per_eval": ms_graph,
        "gbs_effective": alg_bytes / (ms_graph / 1e3) / 1e9,
        "e2e": {"value": 1e3 / ms_e2e, "unit": "slices/s", "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 4},
        "clocks": ck,
    }
    peak, src = _peaks()
    gbs = alg_bytes / (ms_graph / 1e3) / 1e9
    line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                        "frac": gbs / peak, "traffic": None, "peak_source": src,
                        "kernel": "one gradient evaluation (the k_ttm_mode / k_ttm_gram chain)",
                        "algorithmic_bytes_per_eval": alg_bytes,
                        "note": "the 8 MB working set stays in L2, so the HBM copy bandwidth is a "
                                "nominal denominator; ~20 dependent launches set the time"}
    if not args.no_cpu:
        import numpy as np

        import oracle.tucker_adjoint as OA

        Yn = Y.detach().double().cpu().numpy()
        Tn = T.detach().double().cpu().numpy()
        Un = [U.detach().double().cpu().numpy() for U in Us]
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            gY, gU = OA.composite_grad(Yn, Un, Tn)
        dt = (time.perf_counter() - t0) / reps
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "slices/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"FP64 oracle gradient (oracle/tucker_adjoint.py), {reps} "
                                          "evaluations on the same Y, T, U_n"}
        # parity of the graph's last evaluation (same inputs) against the FP64 oracle
        rY = float(np.linalg.norm(Y.grad.double().cpu().numpy() - gY) / np.linalg.norm(gY))
        rU = max(float(np.linalg.norm(U.grad.double().cpu().numpy() - g) / np.linalg.norm(g))
                 for U, g in zip(Us, gU))
        line["parity"] = {"grad_Y_rel": rY, "grad_U_rel_max": rU,
                          "loss_rel": abs(float(Ls.item()) - OA.composite_loss(Yn, Un, Tn))
                          / OA.composite_loss(Yn, Un, Tn)}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """64 independent low-rank-plus-noise streams, spatial sizes uniform in 32..160 per mode, ranks
    4..24, noise 1e-4, tau from {1e-2, 1e-3, 1e-4}, FP32 slices, mixed form; initial ST-HOSVD on
    10 slices each, then one graph launch (tucker_batch_update) per time step updates all 64."""
    import torch

    import paper_2308_16395_gb300 as pkg
    from workloads import batched_streams

    from paper_2308_16395_gb300.sharding import assign_streams, max_over_ranks, stream_cost

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2308_16395_gb300.autotune import CANDIDATES, tune_batch

    K, W = args.steps, max(args.warmup, 3)
    W_TUNE = 2 * len(CANDIDATES)          # launch-shape tuning steps (untimed, before warm-up)
    T = N_INIT + W_TUNE + W + K
    all_specs = batched_streams(nstreams=64, steps=100)
    # independent streams: each rank updates its own balanced share (no data-path collective)
    mine = assign_streams([stream_cost(s.spatial) for s, _ in all_specs], ws)[rank]
    specs = [all_specs[i] for i in mine]
    gens = []
    for i, (s, tau) in zip(mine, specs):
        # the stream's Tucker factors (drawn by the generator) and a per-stream noise generator
        core = torch.tensor(s.core, device=dev)
        facs = [torch.tensor(f, device=dev) for f in s.factors]
        g = torch.Generator(device=dev)
        g.manual_seed(230816395 + 4000 + i)
        gens.append((s, tau, core, facs, g))

    def make_slice(gi, t, out=None):
        s, tau, core, facs, g = gens[gi]
        x = torch.einsum("abcd,ia,jb,kc,d->ijk", core, facs[0], facs[1], facs[2], facs[3][t])
        z = torch.randn(x.shape, generator=g, device=dev, dtype=torch.float64)
        x = x + (s.noise * torch.linalg.norm(x) / torch.linalg.norm(z)) * z
        y = x.permute(2, 1, 0).float()                   # row-major (n3, n2, n1) = column-major
        if out is None:
            return y.contiguous()
        out.copy_(y)

    states = []
    for gi, (s, tau, _, _, _) in enumerate(gens):
        X0 = torch.stack([make_slice(gi, t) for t in range(N_INIT)]).contiguous()
        states.append(pkg.TuckerStream(X0, tau, precision="mixed", steps_cap=T + 4,
                                       rank_cap=[0, 0, 0, (T + 4 + 7) // 8 * 8]))
        del X0
    # per-stream launch shapes: the share multiplier is tuned on the streams' next time steps
    tstep = [N_INIT]

    def feed(b):
        for gi, slot in enumerate(b.slots):
            make_slice(gi, tstep[0], slot)
        tstep[0] += 1

    best_c, tune_ms = tune_batch(states, feed)
    batch = pkg.TuckerBatch(states)
    stream = torch.cuda.current_stream()
    for t in range(N_INIT + W_TUNE, N_INIT + W_TUNE + W):
        for gi, slot in enumerate(batch.slots):
            make_slice(gi, t, slot)
        batch.update()
    torch.cuda.synchronize()
    slice_bytes = sum(slot.numel() * 4 for slot in batch.slots)
    clocks = ClockSampler(local)
    clocks.start()
    ms = 0.0
    for t in range(N_INIT + W_TUNE + W, T):
        for gi, slot in enumerate(batch.slots):
            make_slice(gi, t, slot)                 # new slices land in the slots (untimed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.update()
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    ck = clocks.stop()
    ranks = [st.ranks for st in states]
    ms = max_over_ranks(ms, dev)
    if ws > 1:
        import torch.distributed as dist

        t_ = torch.tensor([float(sum(slot.numel() * 4 for slot in batch.slots))], device=dev)
        dist.all_reduce(t_)
        slice_bytes = float(t_.item())
    value = len(all_specs) * K / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "slices/s", "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched: 64 independent streams, sizes U{32..160}^3, ranks 4..24, "
                               "noise 1e-4, tau in {1e-2,1e-3,1e-4}, fp32, mixed form; one graph "
                               "launch per time step", "parallelism": "1 gpu",
                   "l2": "216 MB of new slices per step (larger than L2)",
                   "sharding": f"{ws} rank(s), streams split by slice size (longest first)"},
        "gbs_ingested": slice_bytes * K / (ms / 1e3) / 1e9,
        "time_steps_per_s": K / (ms / 1e3),
        "graph_kernels_per_step": batch.kernels,
        "launch_shape": {"share_multiplier": best_c,
                         "tuning_ms_per_step": {str(c): round(v, 3) for c, v in tune_ms.items()}},
        "gpu_launches": batch.kernels,
        "rank_range": [min(min(r[:3]) for r in ranks), max(max(r[:3]) for r in ranks),
                       min(r[3] for r in ranks), max(r[3] for r in ranks)],
        "clocks": ck,
    }
    peak, src = _peaks()
    gbs = slice_bytes * K / (ms / 1e3) / 1e9
    line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                        "frac": gbs / peak, "traffic": None, "peak_source": src,
                        "kernel": "one batched time step (all states' update chains in one graph)",
                        "note": "slice bytes ingested per step / step time; the step is a chain of "
                                "short dependent launches per stream (latency-bound), so this is "
                                "far from the bandwidth bound"}
    batch.close()
    for st in states:
        st.close()
    if not args.no_fp64 and ws == 1:
        # the plain FP64 GPU form on the same 64 streams (fresh noise draws, same structure and
        # tolerances), one graph launch per time step, launch shapes tuned the same way
        K64 = min(K, 10)
        T64 = N_INIT + W_TUNE + W + K64
        st64 = []
        for gi, (s, tau, _, _, _) in enumerate(gens):
            X0 = torch.stack([make_slice(gi, t) for t in range(N_INIT)]).contiguous()
            st64.append(pkg.TuckerStream(X0, tau, precision="fp64", steps_cap=T64 + 4,
                                         rank_cap=[0, 0, 0, (T64 + 4 + 7) // 8 * 8]))
            del X0
        tstep[0] = N_INIT
        best64, tune64 = tune_batch(st64, feed)
        b64 = pkg.TuckerBatch(st64)
        for t in range(N_INIT + W_TUNE, N_INIT + W_TUNE + W):
            for gi, slot in enumerate(b64.slots):
                make_slice(gi, t, slot)
            b64.update()
        torch.cuda.synchronize()
        ms64 = 0.0
        for t in range(N_INIT + W_TUNE + W, T64):
            for gi, slot in enumerate(b64.slots):
                make_slice(gi, t, slot)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b64.update()
            e1.record(stream)
            e1.synchronize()
            ms64 += e0.elapsed_time(e1)
        line["fp64_form"] = {"value": len(all_specs) * K64 / (ms64 / 1e3), "unit": "slices/s",
                             "ms_per_step": ms64 / K64, "steps": K64,
                             "share_multiplier": best64,
                             "tuning_ms_per_step": {str(c): round(v, 3) for c, v in tune64.items()},
                             "note": "plain FP64 GPU form, same streams and tolerances, time steps "
                                     f"{N_INIT + W_TUNE + W}..{T64 - 1}, launch shapes tuned as for "
                                     "the mixed form"}
        b64.close()
        for st in st64:
            st.close()
    if not args.no_cpu and rank == 0:
        # the FP64 oracle on the host over a bounded sample: the first three streams, initial
        # ST-HOSVD untimed, then five updates each
        import numpy as np

        import oracle as O

        n_up, t_cpu, n_sl = 5, 0.0, 0
        for gi in range(3):
            s, tau = gens[gi][0], gens[gi][1]
            xs = [make_slice(gi, t).permute(2, 1, 0).double().cpu().numpy() for t in range(N_INIT + n_up)]
            so = O.init_stream(np.asfortranarray(np.stack(xs[:N_INIT], axis=-1)), tau)
            t0 = time.perf_counter()
            for t in range(N_INIT, N_INIT + n_up):
                O.stream_update(so, np.asfortranarray(xs[t]))
            t_cpu += time.perf_counter() - t0
            n_sl += n_up
        line["cpu_baseline"] = {"value": n_sl / t_cpu, "unit": "slices/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": "FP64 oracle, streams 0-2 of the 64 (their own sizes), "
                                          "5 updates each after an untimed initial ST-HOSVD"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_sine(args):
    """The sine-wave stream of Sec. 5.1 at the paper's size: f = sum_j c_j sin(pi j . x) on a
    100 x 100 spatial grid, 5000 time steps, time-mode frequency bound 5 for the first 2500 steps
    and 7 after (the rank bump), eta = 1e-3, tau = 1e-2, initial ST-HOSVD on 200 slices, then
    4800 single-slice updates (graph form), slices resident in HBM (FP64 slices for the FP64
    form, as in the paper; FP32 for the mixed form). Reports slices/s over all updates, the time
    per update over the first and the last 480 updates (the cost per update grows with n_d),
    the final ranks (Table 1: (11, 11, 18) with the paper's coefficients) and the relative error
    of the reconstruction of all 5000 slices."""
    import numpy as np
    import torch

    import paper_2308_16395_gb300 as pkg
    from workloads import SineWave

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sw = SineWave()
    n_init, tau = 200, 1e-2
    T = sw.steps
    tdt = torch.float64 if args.precision == "fp64" else torch.float32
    host = np.stack([sw.slice(t) for t in range(T)], axis=0)          # (T, n1, n2) paper order
    Xg = torch.from_numpy(np.ascontiguousarray(host.transpose(0, 2, 1))).to(dev, tdt)   # (T, n2, n1)
    del host
    X0 = Xg[:n_init].contiguous()
    ts = pkg.TuckerStream(X0, tau, precision=args.precision, rank_cap=[0, 0, 64], steps_cap=T + 8)
    del X0
    st = torch.cuda.current_stream()
    # warm-up: the first update captures the graph
    ts.update(Xg[n_init])
    ts.ranks
    K = T - n_init - 1
    blk = K // 10
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    ev[0].record(st)
    for i, t in enumerate(range(n_init + 1, T)):
        if i == blk:
            ev[1].record(st)
        if i == K - blk:
            ev[2].record(st)
        ts.update(Xg[t])
    ev[3].record(st)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev[0].elapsed_time(ev[3])
    first = ev[0].elapsed_time(ev[1]) / blk
    last = ev[2].elapsed_time(ev[3]) / blk
    ranks = ts.ranks
    R = ts.reconstruct(0, T)
    rel = float(torch.linalg.norm((R.double() - Xg.double()).flatten()) / torch.linalg.norm(Xg.double().flatten()))
    eb, dn = ts.error_norm()
    # Sec. 3.1's concern for long streams: the streaming factor's distance from orthonormal at
    # n_d = 5000, before and after tucker_restore_orthogonality (outside the timed region)
    orth = {"n_d": T, "before": ts.orthogonality_error()[-1]}
    orth["bound_change"] = ts.restore_orthogonality()
    orth["after"] = ts.orthogonality_error()[-1]
    ts.close()
    line = {
        "metric": METRIC, "value": K / (ms / 1e3), "unit": "slices/s", "n_gpus": 1, "steps": K,
        "warmup": 1, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": "sine-wave stream (Sec. 5.1): 100x100 spatial, 5000 steps, rank bump "
                               "at 2500, eta=1e-3, tau=1e-2, n_init=200",
                   "precision": args.precision, "parallelism": "1 gpu",
                   "l2": "80 KB slices: L2-resident, latency-bound by design"},
        "ms_per_update_first_10pct": first, "ms_per_update_last_10pct": last,
        "final_ranks": list(ranks), "paper_stream_ranks": [11, 11, 18],
        "rel_error_true": rel, "rel_error_bound": eb / dn,
        "ud_orthogonality": orth,
        "clocks": ck,
    }
    if not args.no_cpu:
        import oracle as O

        Xs = [sw.slice(t) for t in range(n_init + 20)]
        so = O.init_stream(np.asfortranarray(np.stack(Xs[:n_init], axis=-1)), tau)
        t0 = time.perf_counter()
        for t in range(n_init, n_init + 20):
            O.stream_update(so, Xs[t])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 20 / dt, "unit": "slices/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": "FP64 oracle: init on 200 slices (untimed), 20 timed updates"}
    print(json.dumps(line), flush=True)


def _block_case(pkg, torch, Xg, n_init, tau, prec, B, caps, eager=False):
    """One stream through blocks of B slices (B = 1: tucker_stream_update), graph form, slices
    resident: a warm-up block (captures the graph), then as many whole blocks as fit, timed with
    CUDA events. Returns the state, the timed slice count, the time in ms and the blocks' kernel
    nodes."""
    T = Xg.shape[0]
    ts = pkg.TuckerStream(Xg[:n_init].contiguous(), tau, precision=prec, rank_cap=caps,
                          steps_cap=T + 8, block_cap=max(B, 1))
    if eager:
        pkg.tucker_profile_enable(ts.h, 1)   # launch by launch, so that a profiler lists kernels
    st = torch.cuda.current_stream()

    def step(t):
        if B == 1:
            ts.update(Xg[t])
        else:
            ts.update_block(Xg[t:t + B])

    step(n_init)
    ts.ranks
    nblk = (T - n_init - B) // B
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for i in range(nblk):
        step(n_init + B + i * B)
    e1.record(st)
    torch.cuda.synchronize()
    if eager:
        kern = pkg.tucker_profile_read(ts.h)["launches"] // max(nblk + 1, 1)
    else:
        kern = pkg.tucker_graph_kernels(ts.h) if B == 1 else pkg.tucker_block_graph_kernels(ts.h, B)
    return ts, nblk * B, e0.elapsed_time(e1), kern * nblk


def run_block(args):
    """Block updates (several slices per call, the Conclusions' future work) beside single-slice
    updates, on the small-slice workloads where an update's chain of dependent launches, not the
    slice's bytes, sets the time: the exact-rank 24 x 20 x 16 stream of ranks (4, 4, 3, 6)
    (noise 1e-4, tau = 1e-3, n_init = 10; extended from 40 to 490 steps so that the timed region
    is long enough; FP64 form, FP64 slices) and the 100 x 100 sine-wave stream of Sec. 5.1
    (5000 steps, tau = 1e-2, n_init = 200, mixed form, FP32 slices). For each block size B
    (B = 1 is tucker_stream_update) and each stream: slices/s over the timed blocks (graph form,
    slices resident in HBM), the final ranks, the true relative error of the reconstruction and
    the running bound. The exact-rank stream also runs through the oracle's block update at every
    B (parity: equal ranks after every block, reconstruction against the oracle's). ``value`` is
    the sine-wave stream's slices/s at B = --block."""
    import numpy as np
    import torch

    import paper_2308_16395_gb300 as pkg
    from workloads import LowRankStream, SineWave

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes = sorted({int(x) for x in args.block_sizes.split(",")} | {args.block})
    which = set(args.block_cases.split(","))
    # exact-rank stream (the FP64 workload's recipe, 490 steps)
    Te, ne, taue = 490, 10, 1e-3
    lrs = LowRankStream((24, 20, 16), (4, 4, 3, 6), Te, 1e-4, seed=1, noise_scope="tensor")
    Xe = lrs.tensor(0, Te)                                            # paper order, FP64
    Xeg = torch.from_numpy(np.ascontiguousarray(np.moveaxis(Xe, -1, 0).transpose(0, 3, 2, 1))).to(dev)
    # sine wave (Sec. 5.1)
    sw = SineWave()
    Ts, ns, taus = sw.steps, 200, 1e-2
    hs = np.stack([sw.slice(t) for t in range(Ts)], axis=0)
    Xsg = torch.from_numpy(np.ascontiguousarray(hs.transpose(0, 2, 1))).to(dev, torch.float32)
    del hs
    clocks = ClockSampler(local)
    clocks.start()
    cases = {"exact_rank_24x20x16_fp64": [], "sine_100x100_mixed": []}
    sizes_e = sizes if "exact" in which else []
    sizes_s = sizes if "sine" in which else []
    launches = 0
    import oracle as O
    oracle_ms = None
    for B in sizes_e:
        ts, n, ms, kern = _block_case(pkg, torch, Xeg, ne, taue, "fp64", B, None, args.eager)
        launches += kern
        used = ne + B + n
        R = pkg.paper_order(ts.reconstruct(0, used)).cpu().numpy()
        eb, dn = ts.error_norm()
        rec = {"B": B, "slices_per_s": n / (ms / 1e3), "ms_per_slice": ms / n, "timed_slices": n,
               "ranks": list(ts.ranks),
               "rel_error_true": float(np.linalg.norm(Xe[..., :used] - R) / np.linalg.norm(Xe[..., :used])),
               "rel_error_bound": eb / dn}
        if not args.no_cpu:
            # the oracle over the same slices in the same blocks
            so = O.init_stream(np.asfortranarray(Xe[..., :ne]), taue)
            t0 = time.perf_counter()
            ranks_ok = True
            log = ts.step_log()
            t = ne
            while t < used:
                b = min(B, used - t)
                if B == 1:
                    O.stream_update(so, np.asfortranarray(Xe[..., t]))
                else:
                    O.block_update(so, np.asfortranarray(Xe[..., t:t + b]))
                t += b
                ranks_ok &= tuple(log[t - ne - 1]["ranks"]) == so.ranks
            dt = time.perf_counter() - t0
            if B == args.block:
                oracle_ms = dt * 1e3 / (used - ne)
            Ro = O.reconstruct(so.C, so.Us)
            rec["parity"] = {"ranks_equal_every_block": bool(ranks_ok),
                             "recon_rel_diff": float(np.linalg.norm(R - Ro) / np.linalg.norm(Ro))}
        ts.close()
        cases["exact_rank_24x20x16_fp64"].append(rec)
    for B in sizes_s:
        ts, n, ms, kern = _block_case(pkg, torch, Xsg, ns, taus, "mixed", B, [0, 0, 64], args.eager)
        launches += kern
        used = ns + B + n
        R = ts.reconstruct(0, used).double()
        X = Xsg[:used].double()
        eb, dn = ts.error_norm()
        cases["sine_100x100_mixed"].append({
            "B": B, "slices_per_s": n / (ms / 1e3), "ms_per_slice": ms / n, "timed_slices": n,
            "ranks": list(ts.ranks),
            "rel_error_true": float(torch.linalg.norm((R - X).flatten()) / torch.linalg.norm(X.flatten())),
            "rel_error_bound": eb / dn})
        ts.close()
    ck = clocks.stop()
    main = next(r for r in (cases["sine_100x100_mixed"] or cases["exact_rank_24x20x16_fp64"])
                if r["B"] == args.block)
    line = {
        "metric": METRIC, "value": main["slices_per_s"], "unit": "slices/s", "n_gpus": 1,
        "steps": main["timed_slices"] // args.block, "warmup": 1,
        "ms_per_step": main["ms_per_slice"] * args.block, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"block update (B = {args.block} slices per call) of the 100x100 "
                               "sine-wave stream (Sec. 5.1), beside the exact-rank 24x20x16 stream; "
                               "B = 1 is the single-slice update",
                   "parallelism": "1 gpu", "l2": "small slices: L2-resident, latency-bound"},
        "cases": cases,
        "gpu_launches": int(launches),
        "gpu_launches_note": "kernel nodes of the block graphs (conditional bodies included) x blocks, all cases",
        "clocks": ck,
    }
    if oracle_ms is not None:
        line["cpu_baseline"] = {"value": 1e3 / oracle_ms, "unit": "slices/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"FP64 oracle block update (B = {args.block}) over the "
                                          "exact-rank 24x20x16 stream's timed slices"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="stream",
                    choices=["stream", "stream192", "stream64", "adjoint", "batched", "sine", "block"])
    ap.add_argument("--block", type=int, default=16, help="slices per block (--workload block)")
    ap.add_argument("--block-sizes", default="1,4,8,16,32", help="block sizes compared (--workload block)")
    ap.add_argument("--block-cases", default="exact,sine", help="streams of --workload block: exact, sine")
    ap.add_argument("--eager", action="store_true",
                    help="--workload block: launch by launch (phase profiling on), for kernel listings")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle leg (CPU baseline and parity)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU form comparison")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "sine":
        run_sine(args)
    elif args.workload == "block":
        run_block(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
