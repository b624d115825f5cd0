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


def test_block_graph_form_equals_launch_sequence(pkg):
    """The captured block graph (one per block size, the rows unrolled, conditional growth
    bodies) and the launch-by-launch block (phase profiling on) give the same state on a stream
    whose spatial ranks grow; blocks of two sizes alternate."""
    import torch

    s = LowRankStream((40, 28, 12), (4, 3, 3, 6), 40, 3e-3, seed=23)
    X = s.tensor(0, 40).astype(np.float32).astype(np.float64)
    Xg = to_device(X, torch.float32)
    a = pkg.TuckerStream(Xg[:4].contiguous(), 2e-3, precision="mixed", steps_cap=44, block_cap=4)
    b = pkg.TuckerStream(Xg[:4].contiguous(), 2e-3, precision="mixed", steps_cap=44, block_cap=4)
    pkg.tucker_profile_enable(b.h, 1)
    t = 4
    sizes = [4, 3]
    i = 0
    while t < 40:
        B = min(sizes[i % 2], 40 - t)
        a.update_block(Xg[t:t + B].contiguous())
        b.update_block(Xg[t:t + B].contiguous())
        assert a.ranks == b.ranks, t
        t += B
        i += 1
    assert pkg.tucker_block_graph_kernels(a.h, 4) > 0 and pkg.tucker_block_graph_kernels(a.h, 3) > 0
    assert pkg.tucker_block_graph_kernels(b.h, 4) == 0
    assert any(any(r["grew"]) for r in a.step_log())
    Ra, Rb = a.reconstruct(0, a.n_d).double(), b.reconstruct(0, b.n_d).double()
    assert float(torch.linalg.norm(Ra - Rb) / torch.linalg.norm(Rb)) <= 1e-12
    assert a.error_norm() == b.error_norm()
    a.close()
    b.close()


def test_block_update_on_the_fp16_pass_at_n1_384(pkg):
    """Blocks of 4 advected-blob slices of 384 x 96 x 16 x 2 (mode-1 fibers of 384: the FP16
    tensor-core pass over the block's 4 x 96 x 16 x 2 fibers) against the oracle's block update
    on the same slices, in lockstep with near-cutoff decisions replayed."""
    import torch
    from workloads import BlobField

    bf = BlobField(grid=(384, 96, 16), nvar=2, nblobs=12, noise=1e-5, seed=5)
    dev = torch.device("cuda")
    T, n_init, B, tau = 18, 6, 4, 1e-3
    gs = [bf.slice_torch(t, dev) for t in range(T)]
    xs = [g.cpu().numpy().T.astype(np.float64) for g in gs]
    X = np.stack(xs, axis=-1)
    st = O.init_stream(np.asfortranarray(X[..., :n_init]), tau)
    ts = pkg.TuckerStream(torch.stack(gs[:n_init]).contiguous(), tau, precision="mixed",
                          steps_cap=T + 4, block_cap=B)
    assert ts.ranks == st.ranks
    for t0 in range(n_init, T, B):
        t1 = min(t0 + B, T)
        O.block_update(st, np.asfortranarray(X[..., t0:t1]))
        lg = st.log[-1]
        for row in lg["rows"][1:]:
            assert abs(row.q ** 2 - lg["eps_row"] ** 2) > 0.15 * lg["eps_row"] ** 2, t0
        rp = _block_replay(lg, 3e-2)
        if rp is not None:
            ts.replay_next(*rp)
        ts.update_block(torch.stack(gs[t0:t1]).contiguous())
        assert ts.ranks == st.ranks, (t0, ts.ranks, st.ranks)
    Xh = pkg.paper_order(ts.reconstruct(0, T)).cpu().numpy()
    ref = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(Xh - ref) <= 1e-5 * np.linalg.norm(ref)
    eb, _ = ts.error_norm()
    assert np.linalg.norm(X - Xh) <= eb * (1 + 1e-5)
    assert eb <= tau * np.linalg.norm(X) * (1 + 1e-6)
