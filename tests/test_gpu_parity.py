"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars (written here, derived in the design doc):
  FP64 form  -- identical ranks every step; reconstruction, subspaces and aligned core within
                1e-9 relative; error bookkeeping within 1e-8 relative.
  mixed form -- identical ranks except at decisions within DELTA_DEC (relative) of eps^2;
                reconstruction within 1e-5 relative of the oracle's.
"""

import math

import numpy as np
import pytest

import oracle as O
from tests.parity import aligned_core_diff, decision_margins, subspace_sin, to_device
from workloads import CONFIG1, BlobField, LowRankStream, config1_tensor

pytestmark = pytest.mark.gpu

DELTA_DEC = 1e-3
TOL = {"fp64": 1e-9, "mixed": 1e-5}


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


def _run(pkg, X, n_init, tau, precision, dtype, steps=None, check_every=True, caps=None,
         core_cap=0):
    """Stream X (n_1 x ... x n_{d-1} x T, FP64) through both; return per-step records."""
    import torch

    tdt = torch.float32 if dtype == "f32" else torch.float64
    T = X.shape[-1] if steps is None else steps
    # both sides see exactly the same values: round to the slice type first
    Xs = X.astype(np.float32).astype(np.float64) if dtype == "f32" else X
    st = O.init_stream(Xs[..., :n_init].copy(order="F"), tau)
    Xg = to_device(Xs[..., :T].copy(order="F"), tdt)
    ts = pkg.TuckerStream(Xg[:n_init].contiguous(), tau, precision=precision,
                          steps_cap=T + 4, rank_cap=caps, core_cap=core_cap)
    recs = []
    assert ts.ranks == st.ranks, ("init", ts.ranks, st.ranks)
    diverged = False
    for t in range(n_init, T):
        O.stream_update(st, Xs[..., t].copy(order="F"))
        ts.update(Xg[t].contiguous())
        lg = st.log[-1]
        margin = decision_margins(lg)
        rec = dict(t=t, ranks_o=st.ranks, ranks_g=ts.ranks if check_every else None, margin=margin)
        recs.append(rec)
        if check_every and rec["ranks_g"] != rec["ranks_o"]:
            assert margin < DELTA_DEC or precision == "fp64" and margin < 1e-9, \
                f"rank mismatch at t={t}: gpu {rec['ranks_g']} oracle {rec['ranks_o']} margin {margin}"
            diverged = True
            break
    return st, ts, Xs[..., :T], recs, diverged


def _compare_final(pkg, st, ts, Xs, precision):
    import torch

    tol = TOL[precision]
    nd = ts.n_d
    Xh_o = O.reconstruct(st.C, st.Us)
    Xh_g = pkg.paper_order(ts.reconstruct(0, nd)).cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(Xh_g - Xh_o) / np.linalg.norm(Xh_o)
    # the reconstruction is returned in the slice type: FP32 output adds ~6e-8 relative rounding
    rtol = max(tol, 2e-7) if ts.dtype == torch.float32 else tol
    assert rel < rtol, f"reconstruction rel diff {rel}"
    # error guarantee on the GPU's own reconstruction
    true = np.linalg.norm(Xs - Xh_g) / np.linalg.norm(Xs)
    assert true <= st.tau * (1 + 1e-6), true
    eb, dn = ts.error_norm()
    assert abs(dn - math.sqrt(st.data_norm2)) <= 1e-6 * dn
    # the bookkeeping bounds the true error up to the Gram route's absolute resolution
    # (eigenvalues of A A^T carry errors ~ u ||A||^2 per truncation)
    true_abs = np.linalg.norm(Xs - Xh_g)
    slack = 64 * 2.2e-16 * dn ** 2 * Xs.shape[-1] * (1e6 if precision == "mixed" else 1.0)
    assert eb ** 2 >= true_abs ** 2 * (1 - 1e-4) - slack, (eb, true_abs)
    # factors and aligned core
    C_g = ts.core().cpu().numpy()
    Us_g = [ts.factor(k).cpu().numpy() for k in range(ts.d)]
    for k in range(ts.d):
        assert Us_g[k].shape == st.Us[k].shape
        s = subspace_sin(st.Us[k], Us_g[k])
        assert s < max(tol, 1e-8) * 100, (k, s)
        np.testing.assert_allclose(Us_g[k].T @ Us_g[k], np.eye(Us_g[k].shape[1]), atol=1e-6 if precision == "mixed" else 1e-9)
    cd = aligned_core_diff(st.C, st.Us, C_g, Us_g)
    assert cd < 100 * tol, cd
    return rel


def test_config1_fp64_exact_parity(pkg):
    """Plain FP64 form on the exact-rank workload (24x20x16 slices, ranks (4,4,3,6), tau 1e-3)."""
    s = config1_tensor()
    X = s.tensor(0, CONFIG1["steps"])
    st, ts, Xs, recs, div = _run(pkg, X, CONFIG1["n_init"], CONFIG1["tau"], "fp64", "f64")
    assert not div
    for r in recs:
        assert r["ranks_g"] == (4, 4, 3, 6)
    _compare_final(pkg, st, ts, Xs, "fp64")
    eb, _ = ts.error_norm()
    assert abs(eb ** 2 - st.err2) <= 1e-8 * st.err2
    info = ts.step_info()
    assert abs(info["eps"] - st.log[-1]["eps"]) <= 1e-12 * info["eps"]
    ts.close()


def test_config1_mixed_parity(pkg):
    """Mixed form, FP32 slices, same workload: identical ranks, reconstruction within 1e-5."""
    s = config1_tensor()
    X = s.tensor(0, CONFIG1["steps"])
    st, ts, Xs, recs, div = _run(pkg, X, CONFIG1["n_init"], CONFIG1["tau"], "mixed", "f32")
    assert not div
    _compare_final(pkg, st, ts, Xs, "mixed")
    ts.close()


def _growth_stream(seed=11, n=(37, 29, 11), T=16):
    rng = np.random.default_rng(seed)
    A = [np.linalg.qr(rng.standard_normal((m, 5)))[0] for m in n]
    X = np.zeros(n + (T,), order="F")
    for t in range(T):
        r_use = 2 if t < 6 else (4 if t < 10 else 5)
        G = rng.standard_normal((r_use,) * 3)
        X[..., t] = O.reconstruct(G, [a[:, :r_use] for a in A])
    X += 1e-6 * rng.standard_normal(X.shape)
    return X


@pytest.mark.parametrize("precision,dtype,n", [("fp64", "f64", (37, 29, 11)),
                                                ("fp64", "f32", (37, 29, 11)),
                                                ("mixed", "f32", (37, 29, 11)),
                                                ("mixed", "f32", (40, 28, 12))])
def test_rank_growth_ragged(pkg, precision, dtype, n):
    """Spatial ranks grow (2 -> 4 -> 5): ragged sizes (37 x 29 x 11: not multiples of any tile,
    SIMT mode-1 path) and 40 x 28 x 12 (tensor-core mode-1 pass, residual Gram on tcgen05)."""
    X = _growth_stream(n=n)
    st, ts, Xs, recs, div = _run(pkg, X, 6, 1e-3, precision, dtype)
    assert not div
    assert st.ranks[:3] == (5, 5, 5)
    _compare_final(pkg, st, ts, Xs, precision)
    ts.close()


def test_blob_field_mixed_small(pkg):
    """Advected-blob workload (4 spatial modes incl. variables) at a reduced grid, tau = 1e-4."""
    bf = BlobField(grid=(40, 36, 24), nvar=5, nblobs=12, noise=1e-5, seed=3)
    T = 26
    X = np.stack([bf.slice(t).astype(np.float64) for t in range(T)], axis=-1)
    X = np.asfortranarray(X)
    st, ts, Xs, recs, div = _run(pkg, X, 8, 1e-4, "mixed", "f32")
    if not div:
        _compare_final(pkg, st, ts, Xs, "mixed")
    ts.close()


def test_blob_field_fp64_small(pkg):
    bf = BlobField(grid=(40, 36, 24), nvar=5, nblobs=12, noise=1e-5, seed=3)
    T = 20
    X = np.asfortranarray(np.stack([bf.slice(t).astype(np.float64) for t in range(T)], axis=-1))
    st, ts, Xs, recs, div = _run(pkg, X, 8, 1e-4, "fp64", "f32")
    assert not div
    _compare_final(pkg, st, ts, Xs, "fp64")
    ts.close()


def test_matrix_stream_d2(pkg):
    """d = 2: column-basis growth + incremental SVD of a matrix stream."""
    rng = np.random.default_rng(12)
    n, T, r = 50, 40, 6
    A = rng.standard_normal((n, r)) @ rng.standard_normal((r, T)) + 1e-7 * rng.standard_normal((n, T))
    X = np.asfortranarray(A)
    st, ts, Xs, recs, div = _run(pkg, X, 3, 1e-5, "fp64", "f64")
    assert not div and ts.ranks == st.ranks
    _compare_final(pkg, st, ts, Xs, "fp64")
    ts.close()


def test_zero_slice_and_in_span_slice(pkg):
    import torch

    s = LowRankStream((16, 12, 10), (3, 3, 2, 4), 10, 1e-4, seed=5)
    X = s.tensor(0, 10)
    Xz = X.copy(order="F")
    Xz[..., 7] = 0.0
    Xz[..., 8] = 0.5 * X[..., 2] - 0.25 * X[..., 4]
    st, ts, Xs, recs, div = _run(pkg, Xz, 6, 1e-3, "fp64", "f64", steps=10)
    assert not div
    _compare_final(pkg, st, ts, Xs, "fp64")
    ts.close()


def test_capacity_and_bad_input_errors(pkg):
    import torch

    s = LowRankStream((16, 12, 10), (3, 3, 2, 4), 10, 1e-4, seed=5)
    X = s.tensor(0, 10)
    Xg = to_device(X, torch.float64)
    # a spatial rank cap below the initial rank: the initial ST-HOSVD reports ECAPACITY
    with pytest.raises(pkg.TuckerError) as ei:
        pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="fp64", rank_cap=[2, 0, 0, 0])
    assert ei.value.code == 3
    # steps capacity: the update after the last row is latched and reported
    ts = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="fp64", steps_cap=7)
    ts.update(Xg[6].contiguous())
    ts.update(Xg[7].contiguous())
    with pytest.raises(pkg.TuckerError) as ei:
        ts.ranks
    assert ei.value.code == 3
    with pytest.raises(pkg.TuckerError) as ei:
        ts.update(Xg[8].contiguous())
    assert ei.value.code == 7
    ts.close()
    # non-finite slice -> ENUMERIC latched
    ts = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="fp64", steps_cap=16)
    bad = Xg[6].clone()
    bad[0, 0, 0] = float("nan")
    ts.update(bad)
    with pytest.raises(pkg.TuckerError) as ei:
        ts.error_norm()
    assert ei.value.code == 4
    ts.close()
    # argument errors are synchronous
    with pytest.raises(pkg.TuckerError) as ei:
        pkg.TuckerStream(Xg[:6].contiguous(), -1.0, precision="fp64")
    assert ei.value.code == 1
    with pytest.raises(pkg.TuckerError) as ei:
        pkg.TuckerStream(torch.zeros_like(Xg[:6]).contiguous(), 1e-3, precision="fp64")
    assert ei.value.code == 1


@pytest.mark.parametrize("precision,dtype", [("fp64", "f64"), ("mixed", "f32")])
def test_eigensolver_at_the_shared_memory_limit(pkg, precision, dtype):
    """n_1 = 136: the FP64 eigensolver's matrix and vectors (200 KB) fill shared memory together
    with its static arrays; every eigensolve of this stream runs at that size."""
    rng = np.random.default_rng(17)
    n, T = (136, 10, 8), 12
    A = [np.linalg.qr(rng.standard_normal((m, 4)))[0] for m in n]
    X = np.zeros(n + (T,), order="F")
    for t in range(T):
        r_use = 2 if t < 6 else 4
        G = rng.standard_normal((r_use,) * 3)
        X[..., t] = O.reconstruct(G, [a[:, :r_use] for a in A])
    X += 1e-6 * rng.standard_normal(X.shape)
    st, ts, Xs, recs, div = _run(pkg, X, 6, 1e-3, precision, dtype)
    assert not div
    assert st.ranks[0] == 4
    _compare_final(pkg, st, ts, Xs, precision)
    ts.close()


def test_graph_form_equals_launch_sequence(pkg):
    """The captured-graph update (conditional growth bodies) and the launch-by-launch update
    (phase profiling on) give the same state on a stream whose spatial ranks grow."""
    import torch

    X = _growth_stream(n=(40, 28, 12))
    Xg = to_device(X.astype(np.float32).astype(np.float64), torch.float32)
    a = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=24)
    b = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=24)
    pkg.tucker_profile_enable(b.h, 1)
    for t in range(6, X.shape[-1]):
        a.update(Xg[t].contiguous())
        b.update(Xg[t].contiguous())
        assert a.ranks == b.ranks, t
    assert pkg.tucker_graph_kernels(a.h) > 0 and pkg.tucker_graph_kernels(b.h) == 0
    assert a.ranks[:3] == (5, 5, 5)
    Ra, Rb = a.reconstruct(0, a.n_d).double(), b.reconstruct(0, b.n_d).double()
    assert float(torch.linalg.norm(Ra - Rb) / torch.linalg.norm(Rb)) <= 1e-12
    assert a.error_norm() == b.error_norm()
    a.close()
    b.close()


@pytest.mark.slow
def test_full_size_blob_stream_as_benchmarked(pkg):
    """The benchmark's workload at full size and in its launch configuration: advected blobs
    192 x 192 x 96 x 12 FP32 (170 MB slices), tau = 1e-4, n_init = 10, mixed form, the graph form
    of the update, the bench's capacities. Ranks are compared every step (flips allowed only at
    decisions within DELTA_DEC of eps^2); the reconstructions of sampled slices (first initial
    slice, last update) against the FP64 oracle within 1e-5 relative; the running error bound
    stays within tau."""
    import torch

    bf = BlobField(grid=(192, 192, 96), nvar=12, nblobs=40, noise=1e-5, seed=2)
    T = 14
    dev = torch.device("cuda")
    gs = [bf.slice_torch(t, dev) for t in range(T)]                      # (12, 96, 192, 192)
    xs = [g.cpu().numpy().T.astype(np.float64) for g in gs]              # paper order, FP64
    st = O.init_stream(np.asfortranarray(np.stack(xs[:10], axis=-1)), 1e-4)
    ts = pkg.TuckerStream(torch.stack(gs[:10]).contiguous(), 1e-4, precision="mixed",
                          rank_cap=[0, 0, 0, 0, 24], steps_cap=T + 4, core_cap=4 << 20)
    assert ts.ranks == st.ranks
    ok = True
    for t in range(10, T):
        O.stream_update(st, xs[t])
        ts.update(gs[t])
        if ts.ranks != st.ranks:
            assert decision_margins(st.log[-1]) < DELTA_DEC, (t, ts.ranks, st.ranks)
            ok = False
            break
    assert pkg.tucker_graph_kernels(ts.h) > 0
    if ok:
        for t in (0, T - 1):
            g = pkg.paper_order(ts.reconstruct(t, t + 1)[0]).cpu().numpy().astype(np.float64)
            o = O.reconstruct_slices(st, t, t + 1)[..., 0]
            rel = np.linalg.norm(g - o) / np.linalg.norm(o)
            assert rel < 1e-5, (t, rel)
    eb, dn = ts.error_norm()
    assert eb <= 1e-4 * dn * (1 + 1e-6)
    ts.close()


def test_async_error_norm_read(pkg):
    """tucker_error_norm_async copies (err^2, ||X||^2) into pinned host memory in stream order."""
    import torch

    s = LowRankStream((16, 12, 10), (3, 3, 2, 4), 12, 1e-4, seed=5)
    Xg = to_device(s.tensor(0, 12), torch.float64)
    ts = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="fp64", steps_cap=16)
    out = torch.zeros((6, 2), dtype=torch.float64).pin_memory()
    st = torch.cuda.current_stream()
    for i, t in enumerate(range(6, 12)):
        ts.update(Xg[t].contiguous())
        pkg.tucker_error_norm_async(ts.h, out[i].data_ptr(), st.cuda_stream)
    torch.cuda.synchronize()
    eb, dn = ts.error_norm()
    assert abs(float(out[5, 0]) - eb * eb) <= 1e-14 * max(eb * eb, 1e-300)
    assert abs(float(out[5, 1]) - dn * dn) <= 1e-14 * dn * dn
    assert all(float(out[i + 1, 1]) > float(out[i, 1]) for i in range(5))   # data norm grows
    ts.close()


def test_update_from_host_equals_device_update(pkg):
    """tucker_stream_update_host (slices in pinned host memory, copied on the library's copy
    stream into alternating staging buffers) gives the same state as updates from device slices."""
    import torch

    X = _growth_stream(n=(40, 28, 12))
    Xg = to_device(X.astype(np.float32).astype(np.float64), torch.float32)
    a = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=24)
    b = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=24)
    host = [Xg[t].cpu().pin_memory() for t in range(6, X.shape[-1])]
    for i, t in enumerate(range(6, X.shape[-1])):
        a.update(Xg[t].contiguous())
        b.update_host(host[i])
    assert a.ranks == b.ranks
    assert a.ranks[:3] == (5, 5, 5)
    assert a.error_norm() == b.error_norm()
    Ra, Rb = a.reconstruct(0, a.n_d), b.reconstruct(0, b.n_d)
    assert torch.equal(Ra, Rb)
    with pytest.raises(ValueError):
        b.update_host(Xg[6])          # a device tensor is not a host slice
    a.close()
    b.close()
