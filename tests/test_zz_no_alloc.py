"""tucker_reconstruct_noalloc (through the C ABI) against tucker_reconstruct.

The allocation-free entry point serves callers that cannot allocate device memory when they
reconstruct: a process whose device memory another allocator has already reserved in full, a
device without stream-ordered memory pools, or a latency-critical loop that must not pay for an
allocation. It keeps its temporaries in one fixed device array that every call shares, so these
tests run it twice in a row on different slice ranges. The second call then works on what the
first call left in the array. They also check that a request above the array's size is refused
before any device work.

This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

from tests.parity import to_device
from workloads import LowRankStream

pytestmark = pytest.mark.gpu

# the parity tests' bars: FP64 output within 1e-9 relative, FP32 output within 2e-7
TOL = {"f64": 1e-9, "f32": 2e-7}


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


def _noalloc(pkg, ts, t0, t1):
    import torch

    out = torch.full((t1 - t0,) + tuple(reversed(ts.n)), float("nan"), dtype=ts.dtype, device="cuda")
    pkg.tucker_reconstruct_noalloc(ts.h, t0, t1, out.data_ptr(), ts._sp())
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision,dtype", [("fp64", "f64"), ("mixed", "f32")])
def test_noalloc_matches_reconstruct_on_two_calls(pkg, precision, dtype):
    import torch

    tdt = torch.float64 if dtype == "f64" else torch.float32
    s = LowRankStream((16, 12, 10), (3, 3, 2, 4), 14, 1e-4, seed=5)
    X = s.tensor(0, 14)
    Xg = to_device(X, tdt)
    ts = pkg.TuckerStream(Xg[:6].contiguous(), 1e-3, precision=precision, steps_cap=32)
    for t in range(6, 14):
        ts.update(Xg[t].contiguous())
    # the second call covers a shorter range than the first, so the array holds stale values
    for t0, t1 in [(0, 14), (3, 9)]:
        ref = ts.reconstruct(t0, t1)
        out = _noalloc(pkg, ts, t0, t1)
        assert torch.isfinite(out).all()
        rel = (torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double())).item()
        assert rel <= TOL[dtype], (t0, t1, rel)
    ts.close()


def test_noalloc_refuses_ranges_above_the_scratch_size(pkg):
    import torch

    # 256 x 256 x 16 FP64 slices: the partial expansion C x_4 U_4 x_1 U_1 x_2 U_2 holds
    # 256 * 256 * r_3 * T values, 1 MiB per slice at r_3 = 2, so 10 slices need 10 MiB per
    # temporary, above half of the 16 MiB array; 4 slices fit.
    s = LowRankStream((256, 256, 16), (3, 3, 2, 3), 10, 1e-6, seed=9)
    X = s.tensor(0, 10)
    Xg = to_device(X, torch.float64)
    ts = pkg.TuckerStream(Xg.contiguous(), 1e-3, precision="fp64", steps_cap=16,
                          rank_cap=[8, 8, 4, 8])
    assert ts.ranks[2] == 2
    half = pkg.NOALLOC_SCRATCH_BYTES // 2
    assert 256 * 256 * 2 * 10 * 8 > half >= 256 * 256 * 2 * 4 * 8
    out = torch.full((10,) + tuple(reversed(ts.n)), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TuckerError) as ei:
        pkg.tucker_reconstruct_noalloc(ts.h, 0, 10, out.data_ptr(), ts._sp())
    assert ei.value.code == 1 and "scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())          # refused before any device work
    # a range that fits still works on the same state, twice in a row
    for t0, t1 in [(0, 4), (6, 10)]:
        ref = ts.reconstruct(t0, t1)
        out = _noalloc(pkg, ts, t0, t1)
        rel = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        assert rel <= TOL["f64"], (t0, t1, rel)
    ts.close()
