"""Orthogonality of the streaming factor over long streams (Sec. 3.1's remark on the incremental
SVD's U' U'' products) and its restoration (tucker_restore_orthogonality: the polar factor of
U_d), against the oracle on the same slices."""

import math

import numpy as np
import pytest

import oracle as O
from tests.parity import replay_for, to_device
from workloads import LowRankStream, SineWave

pytestmark = pytest.mark.gpu

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


def _sine(pkg, prec, T):
    import torch

    sw = SineWave(n=(40, 40), steps_each=T // 2, freqs_a=(5, 5, 5), freqs_b=(5, 5, 7), noise=1e-3)
    X = np.stack([sw.slice(t) for t in range(T)], axis=-1)
    dt = "f64" if prec == "fp64" else "f32"
    Xs = X if dt == "f64" else X.astype(np.float32).astype(np.float64)
    Xg = to_device(Xs, torch.float64 if dt == "f64" else torch.float32)
    n_init = 40
    ts = pkg.TuckerStream(Xg[:n_init].contiguous(), 1e-2, precision=prec, steps_cap=T + 4)
    st = O.init_stream(Xs[..., :n_init].copy(order="F"), 1e-2)
    return ts, st, Xs, Xg, n_init


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_streaming_factor_stays_orthonormal_over_a_long_stream(pkg, prec):
    """||U_d^T U_d - I||_F stays at rounding level as n_d grows: measured at n_d = 100..640 on a
    rank-bump sine stream, in lockstep with the oracle (near-cutoff decisions replayed). The
    bar: 64 u_fp64 per update (U_d is FP64 in both forms; each update multiplies it by an
    orthogonal (r_d + 1) x r~_d matrix whose columns are orthonormal to ~r_d u)."""
    T = 640
    ts, st, Xs, Xg, n_init = _sine(pkg, prec, T)
    seen = []
    for t in range(n_init, T):
        O.stream_update(st, Xs[..., t].copy(order="F"))
        rp = replay_for(st.log[-1], DELTA_DEC[prec], DELTA_Q[prec])
        if rp is not None:
            ts.replay_next(*rp)
        ts.update(Xg[t])
        if (t + 1) % 120 == 0:
            assert ts.ranks == st.ranks
            eg = ts.orthogonality_error()[-1]
            eo = O.orthogonality_error(st.Us[-1])
            seen.append((t + 1, eg, eo))
    print("n_d, ||U_d^T U_d - I||_F library, oracle:", seen)
    for nd, eg, eo in seen:
        assert eg <= 64 * 2.0 ** -53 * nd, (nd, eg)
    # spatial factors change only at growth, where they are re-orthogonalised in FP64
    assert max(ts.orthogonality_error()[:-1]) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_restoration_keeps_the_state_and_the_stream_follows_the_oracle(pkg, prec):
    import torch

    s = LowRankStream((40, 28, 12), (4, 3, 3, 5), 60, 1e-4, seed=13)
    X = s.tensor(0, 60)
    dt = "f64" if prec == "fp64" else "f32"
    Xs = X if dt == "f64" else X.astype(np.float32).astype(np.float64)
    Xg = to_device(Xs, torch.float64 if dt == "f64" else torch.float32)
    ts = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision=prec, steps_cap=64)
    st = O.init_stream(Xs[..., :6].copy(order="F"), 1e-3)
    for t in range(6, 40):
        O.stream_update(st, Xs[..., t].copy(order="F"))
        rp = replay_for(st.log[-1], DELTA_DEC[prec], DELTA_Q[prec])
        if rp is not None:
            ts.replay_next(*rp)
        ts.update(Xg[t])
    C0 = ts.core().cpu().numpy()
    S0, V0 = (x.cpu().numpy() for x in ts.sv())
    Ud0 = ts.factor(ts.d - 1).cpu().numpy()
    b0, xn = ts.error_norm()
    change = ts.restore_orthogonality()
    Ud1 = ts.factor(ts.d - 1).cpu().numpy()
    b1, _ = ts.error_norm()
    assert ts.orthogonality_error()[-1] <= 1e-13
    # the polar factor the oracle computes by SVD from the same U_d
    W, _, Zt = np.linalg.svd(Ud0, full_matrices=False)
    np.testing.assert_allclose(Ud1, W @ Zt, atol=1e-13)
    # the change is what the bound took on, and it is tiny for a factor at rounding level
    dch = np.linalg.norm((Ud1 - Ud0) * S0[None, :])
    assert change == pytest.approx(dch, rel=1e-6, abs=1e-18 * xn)
    assert b1 == pytest.approx(b0 + change, rel=1e-14, abs=1e-300)
    assert change <= 1e-10 * xn
    # C, S, V untouched
    assert np.array_equal(ts.core().cpu().numpy(), C0)
    S1, V1 = (x.cpu().numpy() for x in ts.sv())
    assert np.array_equal(S1, S0) and np.array_equal(V1, V0)
    # streaming goes on with the oracle
    O.restore_orthogonality(st)
    for t in range(40, 60):
        O.stream_update(st, Xs[..., t].copy(order="F"))
        rp = replay_for(st.log[-1], DELTA_DEC[prec], DELTA_Q[prec])
        if rp is not None:
            ts.replay_next(*rp)
        ts.update(Xg[t])
        assert ts.ranks == st.ranks
    Xh = pkg.paper_order(ts.reconstruct(0, 60)).cpu().numpy()
    ref = O.reconstruct(st.C, st.Us)
    bar = 1e-9 if prec == "fp64" else 1e-5
    assert np.linalg.norm(Xh - ref) <= bar * np.linalg.norm(ref)
    assert np.linalg.norm(Xs - Xh) <= ts.error_norm()[0] * (1 + 1e-6)
