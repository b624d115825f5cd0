"""Launch-shape autotuner for streams updated concurrently (the batched form).

A launch plan (``tucker_set_launch_plan``) sets how many CTAs each grid-stride pass of a state's
update uses; the defaults fill the whole GPU, which is right for one stream and wrong for 64
concurrent ones. Stream i of a batch gets the share f_i = min(1, c * N_i / sum_j N_j) of the
default CTA counts (N_i: elements per slice). The tuner times the batched graph for each
candidate c on the stream's own next time steps (warm-up steps of the caller) and keeps the
fastest. Results do not depend on the plan, only the time does.
"""

from __future__ import annotations

import torch

from . import TuckerBatch, tucker_set_launch_plan

CANDIDATES = (1.0, 2.0, 4.0, 8.0, 16.0, 64.0)


def plan_for(share: float, nsm: int) -> dict:
    """CTA counts for a share in (0, 1] of the default whole-GPU launch shape."""
    share = min(max(share, 1e-6), 1.0)

    def g(full, cap=None):
        v = max(1, int(round(full * share)))
        return min(v, cap) if cap else v

    return dict(grid_proj=g(2 * nsm), grid_tc=g(nsm), grid_isvd=g(2 * nsm, cap=304), grid_cv=g(4 * nsm))


def apply_plans(streams, c: float, nsm: int) -> list[dict]:
    sizes = [_elems(s) for s in streams]
    tot = float(sum(sizes))
    plans = [plan_for(c * n / tot, nsm) for n in sizes]
    for s, p in zip(streams, plans):
        tucker_set_launch_plan(s.h, **p)
    return plans


def _elems(s) -> int:
    n = 1
    for v in s.n:
        n *= int(v)
    return n


def tune_batch(streams, feed, steps_per_candidate: int = 2, candidates=CANDIDATES, nsm=None):
    """Pick the share multiplier c for a batch of TuckerStreams by timing.

    ``feed(batch)`` writes the next time step's slices into ``batch.slots`` (it is called once per
    tuning step; the streams advance by one update each time). Returns (best_c, timings in ms per
    step for each candidate); the best plans are left applied to the streams.
    """
    if nsm is None:
        nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    stream = torch.cuda.current_stream()
    times = {}
    for c in candidates:
        apply_plans(streams, c, nsm)
        batch = TuckerBatch(streams)
        ms = []
        for i in range(steps_per_candidate):
            feed(batch)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.update()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        batch.close()
        times[c] = min(ms)
    best = min(times, key=times.get)
    apply_plans(streams, best, nsm)
    return best, times
