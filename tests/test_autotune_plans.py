"""Host logic of the batched form's launch-shape tuner (paper_2308_16395_gb300/autotune.py): every
plan it can produce lies inside the ranges tucker_set_launch_plan accepts (projection grid
1..4096, tensor-core grid 1..SM count, ISVD grid 1..304, core/V grid 1..65535), a whole share is
the library's default launch shape, and the shares follow the streams' slice sizes."""

import pytest

from paper_2308_16395_gb300 import autotune

NSM = 152
ISVD_MAX = 304   # the ISVD row passes' grid (one wave at two blocks per SM)


def _in_range(p, nsm):
    return (1 <= p["grid_proj"] <= 4096 and 1 <= p["grid_tc"] <= nsm
            and 1 <= p["grid_isvd"] <= ISVD_MAX and 1 <= p["grid_cv"] <= 65535)


@pytest.mark.parametrize("share", [0.0, 1e-9, 1e-4, 0.003, 0.01, 0.2, 0.5, 0.999, 1.0, 3.0, 64.0])
def test_every_plan_is_accepted_by_the_library(share):
    for nsm in (1, 76, NSM):
        assert _in_range(autotune.plan_for(share, nsm), nsm)


def test_whole_share_is_the_default_shape_and_shares_are_monotone():
    full = autotune.plan_for(1.0, NSM)
    assert full == dict(grid_proj=2 * NSM, grid_tc=NSM, grid_isvd=min(2 * NSM, ISVD_MAX),
                        grid_cv=4 * NSM)
    prev = None
    for share in [1e-6, 1e-3, 0.01, 0.05, 0.1, 0.3, 0.6, 1.0]:
        p = autotune.plan_for(share, NSM)
        if prev is not None:
            assert all(p[k] >= prev[k] for k in p)
        prev = p


class _FakeStream:
    def __init__(self, n, h):
        self.n, self.h = n, h


def test_apply_plans_shares_follow_slice_sizes(monkeypatch):
    seen = {}
    monkeypatch.setattr(autotune, "tucker_set_launch_plan",
                        lambda h, **p: seen.__setitem__(h, dict(p)))
    streams = [_FakeStream((32, 32, 32), 1), _FakeStream((64, 64, 64), 2),
               _FakeStream((160, 160, 160), 3)]
    for c in autotune.CANDIDATES:
        plans = autotune.apply_plans(streams, c, NSM)
        assert [seen[s.h] for s in streams] == plans
        assert all(_in_range(p, NSM) for p in plans)
        # a larger slice never gets a smaller launch
        for a, b in zip(plans, plans[1:]):
            assert all(b[k] >= a[k] for k in a)
    # with c large enough every stream reaches the whole default shape
    plans = autotune.apply_plans(streams, 1e6, NSM)
    assert all(p == autotune.plan_for(1.0, NSM) for p in plans)
