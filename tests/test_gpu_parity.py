"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars (each derived from the arithmetic of the form it checks):
  FP64 form  -- identical ranks every step; reconstruction, subspaces and aligned core within
                1e-9 relative; error bookkeeping within 1e-8 relative.
  mixed form -- identical ranks at every step; a decision whose oracle statistic lies within
                DELTA_DEC (relative) of eps^2 is replayed (tucker_replay_next forces the oracle's
                branch or cut), every other decision must come out the same. Reconstruction
                within 1e-5 relative of the oracle's (the bar of the method's accuracy target);
                subspace sines and the aligned core within the bars below, about ten times the
                largest values measured on these streams; the running bound covers the true
                error up to the relative error RHO of the mixed-precision discarded energies.
"""

import math

import numpy as np
import pytest

import oracle as O
from tests.parity import (aligned_core_diff, oracle_tails, replay_for, subspace_sin,
                          to_device)
from workloads import CONFIG1, BlobField, LowRankStream, config1_tensor

pytestmark = pytest.mark.gpu

# relative distance of a near-cutoff decision from eps^2: in the mixed form the statistics near
# eps^2 deviate from the oracle's by up to ~5e-3 eps^2 (||E_k||^2 at n_k = 384; 2e-3 at 256,
# 6e-4 at 96) and ~1.7e-2 eps^2 (q^2 of Alg. 3 after two 384-wide modes: the FP32 errors of the
# projections accumulate in d); the FP64 form's agree with the oracle's to ~2e-9 eps^2, the
# oracle's own accuracy (its augmented factors are not re-orthogonalised, reading R6)
DELTA_DEC = {"mixed": 3e-2, "fp64": 1e-8}
# deviation of a statistic near eps^2, relative to eps^2 (the same measurements)
RHO = {"mixed": 3e-2, "fp64": 1e-8}
# Alg. 3's q^2 = ||(I - V V^T) d||^2 is sensitive to the FP32 errors of d at first order: an
# error c u ||d|| of the projected slice moves q^2 by up to 2 q c u ||d||, i.e. a fraction
# 2 c u sqrt(d) / tau of eps^2 (c ~ 50 after a 384-wide tensor-core mode: up to ~0.13 at
# tau = 1e-4; measured up to 7e-2); the squared-error bound takes it at that size
DELTA_Q = {"mixed": 1.5e-1, "fp64": 1e-8}
# residual formation error of the arithmetic, in units of its unit roundoff times ||Y||: an FP32
# residual E = Y - U P carries up to about 50 u ||Y|| at n_k = 384 (the same measurement), so a
# discarded ||E_k||^2 is off by at most 2 ||E_k|| C u ||Y|| + (C u ||Y||)^2
RES_C = 64.0
UNIT = {"mixed": 2.0 ** -24, "fp64": 2.0 ** -53}
TOL = {"fp64": 1e-9, "mixed": 1e-5}
# largest principal-angle sine over the factors and aligned-core difference: about ten times the
# largest values measured on these streams (sines 9e-7 FP64 / 3.5e-4 mixed, both from the weakest
# directions of U_d, whose singular values sit near the numerical cut; cores 4e-11 / 5e-7)
SIN_BAR = {"fp64": 1e-5, "mixed": 3e-3}
CORE_BAR = {"fp64": 1e-9, "mixed": 1e-5}


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


def _run(pkg, X, n_init, tau, precision, dtype, steps=None, caps=None, core_cap=0,
         check_tails=True):
    """Stream X (n_1 x ... x n_{d-1} x T, FP64) through both, the oracle first at every step;
    near-cutoff decisions are replayed into the library. Returns (oracle state, library state,
    the slices as both saw them, per-step records)."""
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
    for t in range(n_init, T):
        O.stream_update(st, Xs[..., t].copy(order="F"))
        lg = st.log[-1]
        rp = replay_for(lg, DELTA_DEC[precision], DELTA_Q[precision])
        if rp is not None:
            ts.replay_next(*rp)
        ts.update(Xg[t].contiguous())
        g = ts.step_log(t - n_init, 1)[0]
        assert g["ranks"] == st.ranks, f"t={t}: gpu {g['ranks']} oracle {st.ranks} (replay {rp})"
        assert g["replayed"] == (rp is not None)
        if check_tails:
            _check_step(lg, g, precision, st.data_norm2)
        recs.append(dict(t=t, ranks=st.ranks, replay=rp, log=g,
                         slack=_step_slack(lg, len(lg["modes"]) + 1, precision, st.data_norm2)))
    return st, ts, Xs[..., :T], recs


STATS = {"e2": 0.0, "tail": 0.0, "q2": 0.0}   # largest deviations seen, relative to eps^2


def _step_slack(lg, d, precision, data2):
    """Largest difference between the library's and the oracle's squared error added by one
    update: each of the d - 1 spatial residuals and the incremental SVD's residual (norms below
    eps) may be off by 2 eps C u ||Y|| + (C u ||Y||)^2, each tail by RHO eps^2, and the energy
    that the exact compact SVD of Alg. 3 drops as numerically zero (reading R4: eigenvalues of
    S'S'^T below m u lambda_1) is itself rounding noise, at most m u_fp64 S_1^2 <= m u ||X||^2
    on either side (both solve it in FP64)."""
    eps = lg["eps"]
    cy = RES_C * UNIT[precision] * math.sqrt(lg["y2"])
    m = lg["ranks"][-1] + 1
    # a grown mode's tail is also limited by its Gram's resolution, C u trace(G) = C u ||E_k||^2
    gram = sum(RES_C * UNIT[precision] * md.e_norm2 for md in lg["modes"] if md.grew)
    return ((d - 1) * (2.0 * eps * cy + cy * cy) + RHO[precision] * d * eps * eps
            + DELTA_Q[precision] * eps * eps + 2.0 * m * 2.0 ** -53 * data2 + gram)


def _oracle_step_discarded(lg):
    """The oracle's squared error added by one update (its bookkeeping, Prop. 1, Prop. 2)."""
    info = lg["isvd"]
    return sum(m.discarded for m in lg["modes"]) + (0.0 if info.augmented else info.q ** 2) + info.dropped


def _check_step(lg, g, precision, data2):
    """Per-step statistics against the oracle's, relative to eps^2: ||E_k||^2 of every mode, the
    tails of Alg. 1 at and one below the cut of a grown mode (differences trace(G) - top
    eigenvalues, so they carry the trace's relative error times trace / tail as well), q^2 of
    Alg. 3."""
    eps2 = lg["eps"] ** 2
    rho = RHO[precision]
    # far from eps^2 a statistic only needs the relative accuracy of its arithmetic (FP32 products
    # accumulated over up to a few hundred terms in the mixed form)
    rel = 1e-5 if precision == "mixed" else 1e-9
    if eps2 > 0.0:   # (a zero slice has eps = 0)
        for k, m in enumerate(lg["modes"]):
            STATS["e2"] = max(STATS["e2"], abs(g["e_norm2"][k] - m.e_norm2) / eps2)
            if m.grew and g["grew"][k] and g["r_add"][k] == m.r_add:
                t = oracle_tails(m)
                STATS["tail"] = max(STATS["tail"], abs(g["tail_cut"][k] - t[m.r_add]) / eps2)
        STATS["q2"] = max(STATS["q2"], abs(g["q"] ** 2 - lg["isvd"].q ** 2) / eps2)
    # ||Y||^2: FP64 sums of the slice in the FP64 form; FP32 partial sums over 32 elements
    # accumulated in FP64 in the mixed form
    assert abs(g["eps"] - lg["eps"]) <= (1e-12 if precision == "fp64" else 1e-6) * lg["eps"]
    for k, m in enumerate(lg["modes"]):
        assert abs(g["e_norm2"][k] - m.e_norm2) <= rho * eps2 + rel * m.e_norm2, (k, g["e_norm2"][k], m.e_norm2)
        if m.grew and g["grew"][k] and g["r_add"][k] == m.r_add:
            t = oracle_tails(m)
            slack = rho * eps2 + 10 * rel * m.e_norm2
            assert abs(g["tail_cut"][k] - t[m.r_add]) <= slack, (k, g["tail_cut"][k], t[m.r_add])
            assert abs(g["tail_prev"][k] - t[m.r_add - 1]) <= slack, (k, g["tail_prev"][k], t[m.r_add - 1])
    assert abs(g["q"] ** 2 - lg["isvd"].q ** 2) <= DELTA_Q[precision] * eps2 + rel * lg["isvd"].q ** 2
    # the update's contribution to the running bound
    d = len(lg["modes"]) + 1
    do = _oracle_step_discarded(lg)
    assert abs(g["discarded"] - do) <= _step_slack(lg, d, precision, data2) + 1e-9 * do, (g["discarded"], do)


def _compare_final(pkg, st, ts, Xs, precision, report="", recs=None):
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
    # the running bound covers the true error: the oracle's bound covers its own reconstruction
    # (Prop. 1, Prop. 2, App. D; pinned on the CPU), the library's squared bound differs from the
    # oracle's by at most the summed per-update slack (checked step by step in _check_step; the
    # initial ST-HOSVD's part is FP64 on both sides), and the library's reconstruction differs
    # from the oracle's by the measured d_rec
    true_abs = np.linalg.norm(Xs - Xh_g)
    d_rec = np.linalg.norm(Xh_g - Xh_o)
    sigma = sum(r["slack"] for r in recs) if recs else 0.0
    assert abs(eb ** 2 - st.err2) <= sigma + 1e-9 * st.err2, (eb ** 2, st.err2, sigma)
    assert eb ** 2 >= max(true_abs - d_rec, 0.0) ** 2 - sigma - 1e-9 * st.err2, (eb, true_abs, d_rec, sigma)
    # factors and aligned core
    C_g = ts.core().cpu().numpy()
    Us_g = [ts.factor(k).cpu().numpy() for k in range(ts.d)]
    sines = []
    for k in range(ts.d):
        assert Us_g[k].shape == st.Us[k].shape
        sines.append(subspace_sin(st.Us[k], Us_g[k]))
        np.testing.assert_allclose(Us_g[k].T @ Us_g[k], np.eye(Us_g[k].shape[1]), atol=1e-6 if precision == "mixed" else 1e-9)
    cd = aligned_core_diff(st.C, st.Us, C_g, Us_g)
    print(f"PARITY {report} {precision}: recon {rel:.2e} sines {max(sines):.2e} core {cd:.2e} "
          f"bound/true {eb / max(true_abs, 1e-300):.4f} stats/eps2 e2 {STATS['e2']:.2e} "
          f"tail {STATS['tail']:.2e} q2 {STATS['q2']:.2e}")
    for key in STATS:
        STATS[key] = 0.0
    assert max(sines) < SIN_BAR[precision], sines
    assert cd < CORE_BAR[precision], cd
    return rel


def test_config1_fp64_exact_parity(pkg):
    """Plain FP64 form on the exact-rank workload (24x20x16 slices, ranks (4,4,3,6), tau 1e-3)."""
    s = config1_tensor()
    X = s.tensor(0, CONFIG1["steps"])
    st, ts, Xs, recs = _run(pkg, X, CONFIG1["n_init"], CONFIG1["tau"], "fp64", "f64")
    for r in recs:
        assert r["ranks"] == (4, 4, 3, 6)
    _compare_final(pkg, st, ts, Xs, "fp64", "config1", recs)
    eb, _ = ts.error_norm()
    assert abs(eb ** 2 - st.err2) <= 1e-8 * st.err2
    info = ts.step_info()
    assert abs(info["eps"] - st.log[-1]["eps"]) <= 1e-12 * info["eps"]
    ts.close()


def test_config1_mixed_parity(pkg):
    """Mixed form, FP32 slices, same workload: identical ranks, reconstruction within 1e-5."""
    s = config1_tensor()
    X = s.tensor(0, CONFIG1["steps"])
    st, ts, Xs, recs = _run(pkg, X, CONFIG1["n_init"], CONFIG1["tau"], "mixed", "f32")
    _compare_final(pkg, st, ts, Xs, "mixed", "config1", recs)
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
    st, ts, Xs, recs = _run(pkg, X, 6, 1e-3, precision, dtype)
    assert st.ranks[:3] == (5, 5, 5)
    _compare_final(pkg, st, ts, Xs, precision, f"growth{n}", recs)
    ts.close()


def test_blob_field_mixed_small(pkg):
    """Advected-blob workload (4 spatial modes incl. variables) at a reduced grid, tau = 1e-4."""
    bf = BlobField(grid=(40, 36, 24), nvar=5, nblobs=12, noise=1e-5, seed=3)
    T = 26
    X = np.stack([bf.slice(t).astype(np.float64) for t in range(T)], axis=-1)
    X = np.asfortranarray(X)
    st, ts, Xs, recs = _run(pkg, X, 8, 1e-4, "mixed", "f32")
    _compare_final(pkg, st, ts, Xs, "mixed", "blob40", recs)
    ts.close()


def test_blob_field_fp64_small(pkg):
    bf = BlobField(grid=(40, 36, 24), nvar=5, nblobs=12, noise=1e-5, seed=3)
    T = 20
    X = np.asfortranarray(np.stack([bf.slice(t).astype(np.float64) for t in range(T)], axis=-1))
    st, ts, Xs, recs = _run(pkg, X, 8, 1e-4, "fp64", "f32")
    _compare_final(pkg, st, ts, Xs, "fp64", "blob40", recs)
    ts.close()


def test_matrix_stream_d2(pkg):
    """d = 2: column-basis growth + incremental SVD of a matrix stream."""
    rng = np.random.default_rng(12)
    n, T, r = 50, 40, 6
    A = rng.standard_normal((n, r)) @ rng.standard_normal((r, T)) + 1e-7 * rng.standard_normal((n, T))
    X = np.asfortranarray(A)
    st, ts, Xs, recs = _run(pkg, X, 3, 1e-5, "fp64", "f64")
    assert ts.ranks == st.ranks
    _compare_final(pkg, st, ts, Xs, "fp64", "d2", recs)
    ts.close()


def test_zero_slice_and_in_span_slice(pkg):
    import torch

    s = LowRankStream((16, 12, 10), (3, 3, 2, 4), 10, 1e-4, seed=5)
    X = s.tensor(0, 10)
    Xz = X.copy(order="F")
    Xz[..., 7] = 0.0
    Xz[..., 8] = 0.5 * X[..., 2] - 0.25 * X[..., 4]
    st, ts, Xs, recs = _run(pkg, Xz, 6, 1e-3, "fp64", "f64", steps=10)
    _compare_final(pkg, st, ts, Xs, "fp64", "zero", recs)
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
    st, ts, Xs, recs = _run(pkg, X, 6, 1e-3, precision, dtype)
    assert st.ranks[0] == 4
    _compare_final(pkg, st, ts, Xs, precision, "n136", recs)
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


def _blob_lockstep(pkg, bf, T, n_init, tau, caps=None, core_cap=0, samples=()):
    """An advected-blob stream generated on the device (the benchmark's recipe), through the
    oracle and the library in lockstep with near-cutoff decisions replayed; the sampled slices'
    reconstructions against the oracle's. Returns the per-step records and the max rel diff."""
    import torch

    dev = torch.device("cuda")
    gs = [bf.slice_torch(t, dev) for t in range(T)]                      # row-major, FP32
    xs = [g.cpu().numpy().T.astype(np.float64) for g in gs]              # paper order, FP64
    st = O.init_stream(np.asfortranarray(np.stack(xs[:n_init], axis=-1)), tau)
    ts = pkg.TuckerStream(torch.stack(gs[:n_init]).contiguous(), tau, precision="mixed",
                          rank_cap=caps, steps_cap=T + 4, core_cap=core_cap)
    assert ts.ranks == st.ranks
    recs = []
    for t in range(n_init, T):
        O.stream_update(st, xs[t])
        lg = st.log[-1]
        rp = replay_for(lg, DELTA_DEC["mixed"], DELTA_Q["mixed"])
        if rp is not None:
            ts.replay_next(*rp)
        ts.update(gs[t])
        g = ts.step_log(t - n_init, 1)[0]
        assert g["ranks"] == st.ranks, (t, g["ranks"], st.ranks, rp)
        _check_step(lg, g, "mixed", st.data_norm2)
        recs.append(dict(t=t, log=g, replay=rp))
    worst = 0.0
    for t in samples:
        g = pkg.paper_order(ts.reconstruct(t, t + 1)[0]).cpu().numpy().astype(np.float64)
        o = O.reconstruct_slices(st, t, t + 1)[..., 0]
        worst = max(worst, np.linalg.norm(g - o) / np.linalg.norm(o))
    eb, dn = ts.error_norm()
    assert eb <= tau * dn * (1 + 1e-6)
    return st, ts, recs, worst


def test_full_size_stream_as_benchmarked(pkg):
    """The benchmark's default workload at full size and in its launch configuration: advected
    blobs 384 x 384 x 256 x 4 FP32 (604 MB slices, 80 blobs), tau = 1e-4, n_init = 10, mixed
    form, the graph form of the update, the bench's capacities. Every step's ranks and
    statistics against the oracle's (near-cutoff decisions replayed); the reconstructions of
    sampled slices (an initial slice, the last update) within 1e-5 relative of the oracle's."""
    T = 14
    bf = BlobField(grid=(384, 384, 256), nvar=4, nblobs=80, noise=1e-5, seed=5)
    st, ts, recs, worst = _blob_lockstep(pkg, bf, T, 10, 1e-4, caps=[0, 0, 0, 0, 24],
                                         core_cap=4 << 20, samples=(0, T - 1))
    assert pkg.tucker_graph_kernels(ts.h) > 0
    assert worst < 1e-5, worst
    print(f"PARITY full-size 384x384x256x4 mixed: recon {worst:.2e} replays "
          f"{sum(r['replay'] is not None for r in recs)}")
    ts.close()


@pytest.mark.parametrize("grid", [(256, 224, 16), (384, 40, 16), (64, 384, 16)])
def test_rank_growth_above_192(pkg, grid):
    """Spatial growth at n_k > 192 (beyond the register tridiagonalization): 256 x 224 (the
    tensor-core Gram of two row blocks, the subspace eigensolver reading G from global memory),
    384 x 40 and 64 x 384 (the blocked residual product and the three-row-block Gram). The
    subspace eigensolver must take every grown cut at these sizes (no fallback), with the tails
    at and below the cut within RHO eps^2 of the oracle's."""
    bf = BlobField(grid=grid, nvar=2, nblobs=20, noise=1e-5, seed=11)
    st, ts, recs, worst = _blob_lockstep(pkg, bf, 22, 10, 1e-4, samples=(0, 21))
    big = [k for k, n in enumerate(grid) if n > 192]
    grown = [(r["t"], k) for r in recs for k in big if r["log"]["grew"][k]]
    assert grown, "no growth in a mode above 192"
    for r in recs:
        for k in range(len(grid)):
            if r["log"]["grew"][k] and grid[k] >= 48:
                assert r["log"]["eig_path"][k] == 1, (r["t"], k, r["log"]["eig_path"])
    assert worst < 1e-5, worst
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
