"""Block update on the GPU (tucker_stream_update_block: B slices at once, the Conclusions'
future work) against the oracle's block_update on the same slices: ranks after every block,
the step log (one record per slice, the block's decisions in the first), the bookkeeping, the
reconstruction, and the bound against the true error."""

import math

import numpy as np
import pytest

import oracle as O
from tests.parity import replay_for, to_device
from workloads import LowRankStream

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-5}
BOOK = {"fp64": 1e-8, "mixed": 3e-2}


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


def _block_replay(lg, delta):
    """The oracle's decisions of a block that lie within delta (relative) of their cutoffs: the
    spatial modes' against eps^2, the first row's Alg. 3 branch against eps_row^2 (the replay hook
    reaches the first row only), as tucker_replay_next's (grow, augment); None otherwise."""
    grow, _ = replay_for(dict(eps=lg["eps"], modes=lg["modes"], isvd=_NoQ), delta) or (None, -1)
    r0 = lg["rows"][0]
    e2 = lg["eps_row"] ** 2
    aug = int(r0.augmented) if abs(r0.q ** 2 - e2) < delta * e2 else -1
    if grow is None and aug < 0:
        return None
    return (grow if grow is not None else [-1] * len(lg["modes"])), aug


class _NoQ:
    q = math.inf
    augmented = False


def _run(pkg, prec, B, n, ranks, noise, tau, T, seed, n_init=6):
    import torch

    s = LowRankStream(n, ranks, T, noise, seed=seed)
    X = s.tensor(0, T)
    dt = "f64" if prec == "fp64" else "f32"
    Xs = X if dt == "f64" else X.astype(np.float32).astype(np.float64)
    Xg = to_device(Xs, torch.float64 if dt == "f64" else torch.float32)
    ts = pkg.TuckerStream(Xg[:n_init].contiguous(), tau, precision=prec, steps_cap=T + 4,
                          block_cap=B)
    st = O.init_stream(Xs[..., :n_init].copy(order="F"), tau)
    assert ts.ranks == st.ranks
    for t0 in range(n_init, T, B):
        t1 = min(t0 + B, T)
        O.block_update(st, Xs[..., t0:t1].copy(order="F"))
        lg = st.log[-1]
        rp = _block_replay(lg, 3e-2 if prec == "mixed" else 1e-8)
        # the later rows' branches must be clear of eps_row (no replay reaches them)
        for row in lg["rows"][1:]:
            assert abs(row.q ** 2 - lg["eps_row"] ** 2) > 0.15 * lg["eps_row"] ** 2, t0
        if rp is not None:
            ts.replay_next(*rp)
        ts.update_block(Xg[t0:t1].contiguous())
        assert ts.ranks == st.ranks, (t0, ts.ranks, st.ranks)
    return ts, st, Xs


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("B", [3, 4])
def test_block_update_follows_the_oracle(pkg, prec, B):
    # three initial slices: the streaming rank grows to 6 inside blocks (rows after the first too)
    ts, st, Xs = _run(pkg, prec, B, (40, 28, 12), (4, 3, 3, 6), 1e-4, 1e-3, 34, seed=21, n_init=3)
    T = Xs.shape[-1]
    Xh = pkg.paper_order(ts.reconstruct(0, T)).cpu().numpy()
    ref = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(Xh - ref) <= TOL[prec] * np.linalg.norm(ref)
    eb, xn = ts.error_norm()
    assert xn ** 2 == pytest.approx(st.data_norm2, rel=1e-6 if prec == "mixed" else 1e-12)
    assert eb ** 2 == pytest.approx(st.err2, rel=BOOK[prec], abs=1e-12 * st.data_norm2)
    assert np.linalg.norm(Xs - Xh) <= eb * (1 + 1e-5)
    # one record per slice; n_d counts slices
    log = ts.step_log()
    assert len(log) == T - 3 and log[-1]["n_d"] == T
    for i, rec in enumerate(log):
        first = (i % B == 0)
        if not first:
            assert rec["y_norm2"] == 0.0 and not any(rec["grew"])
    assert sum(r["augmented"] for r in log) == sum(r.augmented for lg in st.log if lg["kind"] == "block"
               for r in lg["rows"])


def test_block_update_with_rank_growth_fp64(pkg):
    """Noise above tau: the spatial ranks grow inside blocks and both branches of Alg. 3 occur;
    the FP64 form follows the oracle (decisions within 1e-8 of their cutoffs replayed)."""
    ts, st, Xs = _run(pkg, "fp64", 4, (24, 20, 16), (4, 4, 3, 6), 3e-3, 2e-3, 42, seed=9)
    grew = sum(sum(m.grew for m in lg["modes"]) for lg in st.log if lg["kind"] == "block")
    assert grew > 0
    T = Xs.shape[-1]
    Xh = pkg.paper_order(ts.reconstruct(0, T)).cpu().numpy()
    ref = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(Xh - ref) <= 1e-9 * np.linalg.norm(ref)
    eb, _ = ts.error_norm()
    assert eb ** 2 == pytest.approx(st.err2, rel=1e-8)
    assert np.linalg.norm(Xs - Xh) <= eb * (1 + 1e-9)


def test_block_of_one_is_the_single_update_and_caps_are_checked(pkg):
    import torch

    s = LowRankStream((40, 28, 12), (4, 3, 3, 6), 20, 1e-4, seed=22)
    X = s.tensor(0, 20).astype(np.float32).astype(np.float64)
    Xg = to_device(X, torch.float32)
    a = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=24, block_cap=2)
    b = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision="mixed", steps_cap=24)
    for t in range(6, 14):
        a.update_block(Xg[t:t + 1].contiguous())
        b.update(Xg[t])
    assert a.ranks == b.ranks
    ra = pkg.paper_order(a.reconstruct(0, 14)).cpu().numpy()
    rb = pkg.paper_order(b.reconstruct(0, 14)).cpu().numpy()
    assert np.linalg.norm(ra - rb) <= 1e-6 * np.linalg.norm(rb)
    with pytest.raises(pkg.TuckerError):
        a.update_block(Xg[14:17].contiguous())        # 3 slices above block_cap = 2
    a.update_block(Xg[14:16].contiguous())            # the state is still usable
    assert a.step_log()[-1]["n_d"] == 16
