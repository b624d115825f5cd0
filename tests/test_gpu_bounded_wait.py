"""The bounded waits of the tensor-core pass: a wait that runs out (its producer withholds the
loads through the test hook tucker_test_stall_next, so the awaited barrier never completes) gives
up after its time limit, the kernel latches TUCKER_ETIMEOUT and ends, the next synchronizing call
reports it, the state refuses further work, and the CUDA context stays usable: a new state on
the same device streams and matches the oracle. No fault, trap or unbounded wait is involved."""

import time

import numpy as np
import pytest

import oracle as O
from tests.parity import to_device
from workloads import LowRankStream

pytestmark = pytest.mark.gpu

ETIMEOUT, ESTATE = 5, 7


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


def _stream(pkg, seed):
    import torch

    s = LowRankStream((40, 28, 12), (4, 3, 3, 4), 16, 1e-4, seed=seed)
    Xs = s.tensor(0, 16).astype(np.float32).astype(np.float64)
    Xg = to_device(Xs, torch.float32)
    ts = pkg.TuckerStream(Xg[:5].contiguous(), 1e-3, precision="mixed", steps_cap=20)
    return ts, Xs, Xg


@pytest.mark.parametrize("graph", [True, False])
def test_a_wait_that_runs_out_latches_etimeout_and_the_context_stays_usable(pkg, graph):
    ts, Xs, Xg = _stream(pkg, 31)
    if not graph:
        pkg.tucker_profile_enable(ts.h, 1)   # launch by launch
    for t in range(5, 8):
        ts.update(Xg[t])
    before = ts.ranks
    pkg.tucker_test_stall_next(ts.h)
    t0 = time.time()
    ts.update(Xg[8])
    with pytest.raises(pkg.TuckerError) as e:
        ts.ranks                                     # synchronizes
    waited = time.time() - t0
    assert e.value.code == ETIMEOUT
    assert 0.5 < waited < 30.0, waited               # the wait gave up after its limit
    with pytest.raises(pkg.TuckerError) as e2:
        ts.update(Xg[9])
    assert e2.value.code in (ETIMEOUT, ESTATE)
    ts.close()
    # the context is usable: a fresh state streams and follows the oracle
    ts2, Xs2, Xg2 = _stream(pkg, 32)
    st = O.init_stream(Xs2[..., :5].copy(order="F"), 1e-3)
    for t in range(5, 16):
        O.stream_update(st, Xs2[..., t].copy(order="F"))
        ts2.update(Xg2[t])
    assert ts2.ranks == st.ranks
    Xh = pkg.paper_order(ts2.reconstruct(0, 16)).cpu().numpy()
    ref = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(Xh - ref) <= 1e-5 * np.linalg.norm(ref)
    assert before is not None
    ts2.close()
