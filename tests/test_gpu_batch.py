"""Batched form: independent streams of uneven sizes, ranks and tolerances advanced by one
CUDA-graph launch per time step (tucker_batch_*), against the same states updated one by one
through tucker_stream_update and against the FP64 oracle."""

import numpy as np
import pytest

import oracle as O
from tests.parity import replay_for, to_device
from workloads import LowRankStream, batched_streams

pytestmark = pytest.mark.gpu

# relative distance of a near-cutoff decision from eps^2 (see tests/test_gpu_parity.py)
DELTA_DEC = {"mixed": 3e-2, "fp64": 1e-8}
DELTA_Q = {"mixed": 1.5e-1, "fp64": 1e-8}


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_16395_gb300 as p
    from paper_2308_16395_gb300 import build as b

    b.build()
    p.load_library()
    return p


def _small_streams():
    """Five uneven mixed-form FP32 streams (sizes 8..40, ranks 2..6, tau from {1e-2, 1e-3, 1e-4})
    plus one FP64-form stream of FP64 slices."""
    out = [(s, tau, "mixed", "f32") for s, tau in
           batched_streams(nstreams=5, steps=16, size_range=(8, 40), rank_range=(2, 6), seed=21)]
    out.append((LowRankStream((20, 13, 9), (3, 4, 2, 3), 16, 1e-4, seed=22), 1e-3, "fp64", "f64"))
    return out


def _bench_streams():
    """Six streams drawn like the benchmark's 64 (sizes 32..160 per mode, ranks 4..24, noise
    1e-4, tau from {1e-2, 1e-3, 1e-4}), mixed form, FP32 slices."""
    return [(s, tau, "mixed", "f32") for s, tau in batched_streams(nstreams=6, steps=16, seed=4)]


@pytest.mark.parametrize("which", ["small", "bench_sizes"])
def test_batch_matches_single_updates_and_oracle(pkg, which):
    """Every state of the batch equals the same state updated one by one (to 1e-12) and follows
    the oracle at every step (near-cutoff decisions replayed into both library states)."""
    import torch

    n_init, T = 5, 16
    streams = _small_streams() if which == "small" else _bench_streams()
    entries = []
    for s, tau, prec, dt in streams:
        tdt = torch.float32 if dt == "f32" else torch.float64
        X = s.tensor(0, T).astype(np.float64)
        Xs = X.astype(np.float32).astype(np.float64) if dt == "f32" else X
        Xg = to_device(Xs, tdt)
        kw = dict(precision=prec, steps_cap=T + 4)
        a = pkg.TuckerStream(Xg[:n_init].contiguous(), tau, **kw)
        b = pkg.TuckerStream(Xg[:n_init].contiguous(), tau, **kw)
        st = O.init_stream(Xs[..., :n_init].copy(order="F"), tau)
        assert a.ranks == st.ranks
        entries.append(dict(a=a, b=b, st=st, Xg=Xg, Xs=Xs, prec=prec, tau=tau))
    batch = pkg.TuckerBatch([e["a"] for e in entries])
    assert batch.kernels > 0
    replays = 0
    for t in range(n_init, T):
        for e in entries:
            O.stream_update(e["st"], e["Xs"][..., t].copy(order="F"))
            rp = replay_for(e["st"].log[-1], DELTA_DEC[e["prec"]], DELTA_Q[e["prec"]])
            if rp is not None:
                e["a"].replay_next(*rp)
                e["b"].replay_next(*rp)
                replays += 1
        for e, slot in zip(entries, batch.slots):
            slot.copy_(e["Xg"][t])
        batch.update()
        for e in entries:
            e["b"].update(e["Xg"][t].contiguous())
        for e in entries:
            ra, rb = e["a"].ranks, e["b"].ranks
            assert ra == rb, (t, ra, rb)
            assert ra == e["st"].ranks, (t, ra, e["st"].ranks)
    for e in entries:
        Ra = e["a"].reconstruct(0, T).double()
        Rb = e["b"].reconstruct(0, T).double()
        assert float(torch.linalg.norm(Ra - Rb) / torch.linalg.norm(Rb)) <= 1e-12
        Xh = O.reconstruct(e["st"].C, e["st"].Us)
        rel = np.linalg.norm(pkg.paper_order(Ra).cpu().numpy() - Xh) / np.linalg.norm(Xh)
        assert rel < (1e-5 if e["prec"] == "mixed" else 1e-9), rel
        ea, da = e["a"].error_norm()
        eb, db = e["b"].error_norm()
        assert abs(ea - eb) <= 1e-12 * max(eb, 1e-300) and abs(da - db) <= 1e-12 * db
    print(f"PARITY batch {which}: {len(entries)} streams, {replays} replayed updates")
    batch.close()
    for e in entries:
        e["a"].close()
        e["b"].close()


def test_batch_error_latches_in_one_state(pkg):
    import torch

    s1 = LowRankStream((16, 12, 10), (3, 3, 2, 4), 12, 1e-4, seed=5)
    s2 = LowRankStream((14, 11, 9), (2, 3, 2, 3), 12, 1e-4, seed=6)
    X1 = to_device(s1.tensor(0, 12), torch.float64)
    X2 = to_device(s2.tensor(0, 12), torch.float64)
    a = pkg.TuckerStream(X1[:6].contiguous(), 1e-3, precision="fp64", steps_cap=7)   # room for 1 update
    b = pkg.TuckerStream(X2[:6].contiguous(), 1e-3, precision="fp64", steps_cap=16)
    ref = pkg.TuckerStream(X2[:6].contiguous(), 1e-3, precision="fp64", steps_cap=16)
    batch = pkg.TuckerBatch([a, b])
    for t in range(6, 9):
        batch.slots[0].copy_(X1[t])
        batch.slots[1].copy_(X2[t])
        batch.update()
        ref.update(X2[t].contiguous())
    with pytest.raises(pkg.TuckerError) as ei:
        a.ranks
    assert ei.value.code == 3                      # ECAPACITY latched in the first state only
    assert b.ranks == ref.ranks and b.n_d == 9
    Rb, Rr = b.reconstruct(0, 9), ref.reconstruct(0, 9)
    assert float(torch.linalg.norm(Rb - Rr) / torch.linalg.norm(Rr)) <= 1e-12
    with pytest.raises(pkg.TuckerError) as ei:      # the batch refuses once a state has reported
        batch.update()
    assert ei.value.code == 7
    batch.close()
    for x in (a, b, ref):
        x.close()


def test_launch_plan_changes_no_result(pkg):
    """A small launch plan (a few CTAs per pass) gives the same state as the default plan."""
    import torch

    s = LowRankStream((40, 28, 12), (3, 3, 2, 3), 14, 1e-4, seed=8)
    Xg = to_device(s.tensor(0, 14).astype(np.float32).astype(np.float64), torch.float32)
    a = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=20)
    b = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=20)
    pkg.tucker_set_launch_plan(b.h, grid_proj=3, grid_tc=1, grid_isvd=2, grid_cv=5)
    assert pkg.tucker_get_launch_plan(b.h) == dict(grid_proj=3, grid_tc=1, grid_isvd=2, grid_cv=5)
    with pytest.raises(pkg.TuckerError):
        pkg.tucker_set_launch_plan(b.h, grid_isvd=100000)
    for t in range(6, 14):
        a.update(Xg[t].contiguous())
        b.update(Xg[t].contiguous())
    assert a.ranks == b.ranks
    Ra, Rb = a.reconstruct(0, 14).double(), b.reconstruct(0, 14).double()
    assert float(torch.linalg.norm(Ra - Rb) / torch.linalg.norm(Ra)) <= 1e-6
    a.close()
    b.close()


def test_stream_update_batched_equals_single_updates(pkg):
    """tucker_stream_update_batched (each state's slice by pointer, one graph launch per call,
    the graph cached per list of states) gives the same states as one tucker_stream_update per
    state; the slice buffers change from call to call."""
    import torch

    n_init, T = 5, 12
    entries = []
    for s, tau, prec, dt in _small_streams()[:3]:
        X = s.tensor(0, T).astype(np.float32).astype(np.float64)
        Xg = to_device(X, torch.float32)
        a = pkg.TuckerStream(Xg[:n_init].contiguous(), tau, precision="mixed", steps_cap=T + 4)
        b = pkg.TuckerStream(Xg[:n_init].contiguous(), tau, precision="mixed", steps_cap=T + 4)
        entries.append((a, b, Xg))
    st = torch.cuda.current_stream().cuda_stream
    for t in range(n_init, T):
        ys = [e[2][t].clone() for e in entries]          # fresh buffers every step
        pkg.tucker_stream_update_batched([e[0].h for e in entries], [y.data_ptr() for y in ys], st)
        for e in entries:
            e[1].update(e[2][t].contiguous())
        torch.cuda.synchronize()
    for a, b, _ in entries:
        assert a.ranks == b.ranks
        Ra, Rb = a.reconstruct(0, T).double(), b.reconstruct(0, T).double()
        assert float(torch.linalg.norm(Ra - Rb) / torch.linalg.norm(Rb)) <= 1e-12
        assert a.error_norm() == b.error_norm()
    with pytest.raises(pkg.TuckerError):
        pkg.tucker_stream_update_batched([entries[0][0].h, entries[0][0].h],
                                         [entries[0][2][0].data_ptr()] * 2, st)
    for a, b, _ in entries:
        a.close()
        b.close()
