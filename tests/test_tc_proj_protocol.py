"""Model check of the barrier protocol of the tensor-core projection pass (k_tc_proj, residual
form): TMA producer, TF32 splitters, MMA issuer, P epilogue and residual epilogue over a ring of
stages, two P buffers in tensor memory and one residual buffer.

Each role is a coroutine issuing the waits and arrivals the kernel issues, in the same order;
tensor-core work completes in issue order (one pipe); durations are random. An mbarrier wait
names a phase by its parity, so a wait for phase k is only sound if the barrier has not already
completed phase k + 1 when the wait starts (it would then see the parity as pending and wait
for ever). The check: every role finishes, and no wait ever starts on a barrier two phases
ahead. A planted bug (MMA2 not waiting for the residual epilogue to release the residual buffer)
must be caught, so the check is not vacuous.
"""

import heapq
import random


class _Bar:
    def __init__(self, name):
        self.name, self.done = name, 0


def _simulate(ntiles, nchunks, stages, rng, plant_bug=False):
    clock = [0.0]
    events, seq = [], [0]

    def at(delay, fn):
        seq[0] += 1
        heapq.heappush(events, (clock[0] + delay, seq[0], fn))

    full = [_Bar("full%d" % s) for s in range(stages)]
    conv = [_Bar("conv%d" % s) for s in range(stages)]
    empty = [_Bar("empty%d" % s) for s in range(stages)]
    d1full = [_Bar("d1full%d" % b) for b in range(2)]
    pready = [_Bar("pready%d" % b) for b in range(2)]
    mma2done = [_Bar("mma2done%d" % b) for b in range(2)]
    d2full, d2free = _Bar("d2full"), _Bar("d2free")
    errors = []
    pipe_free = [0.0]

    def tensor(duration, on_done):
        start = max(pipe_free[0], clock[0])
        pipe_free[0] = start + duration
        seq[0] += 1
        heapq.heappush(events, (pipe_free[0], seq[0], on_done))

    def done(bar):
        return lambda: setattr(bar, "done", bar.done + 1)

    def wait(bar, phase):
        if bar.done > phase + 1:
            errors.append("%s: wait for phase %d after %d completions" % (bar.name, phase, bar.done))
        return ("wait", bar, phase)

    def producer():
        q = 0
        for _ in range(ntiles):
            for _ in range(nchunks):
                s = q % stages
                if q >= stages:
                    yield wait(empty[s], q // stages - 1)
                at(rng.uniform(0.3, 0.9), done(full[s]))     # TMA copy lands
                q += 1

    def splitters():
        q = 0
        for _ in range(ntiles):
            for _ in range(nchunks):
                s = q % stages
                yield wait(full[s], q // stages)
                yield ("delay", rng.uniform(0.2, 0.45))
                conv[s].done += 1
                q += 1

    def issuer():
        def mma2(jt):
            yield wait(pready[jt & 1], jt >> 1)
            if jt >= 1 and not plant_bug:
                yield wait(d2free, jt - 1)

            def fin(jt=jt):
                d2full.done += 1
                mma2done[jt & 1].done += 1
            tensor(rng.uniform(0.5, 0.9), fin)

        q, pend = 0, -1
        for it in range(ntiles):
            b = it & 1
            if it >= 2:
                yield wait(mma2done[b], (it >> 1) - 1)
            for _ in range(nchunks):
                s = q % stages
                yield wait(conv[s], q // stages)
                tensor(rng.uniform(0.05, 0.3), done(empty[s]))
                q += 1
                if pend >= 0 and pready[pend & 1].done > (pend >> 1):
                    yield from mma2(pend)
                    pend = -1
            tensor(0.0, done(d1full[b]))
            if pend >= 0:
                yield from mma2(pend)
            pend = it
        if pend >= 0:
            yield from mma2(pend)

    def epilogue_p():
        for it in range(ntiles):
            yield wait(d1full[it & 1], it >> 1)
            yield ("delay", rng.uniform(0.5, 1.5))
            pready[it & 1].done += 1

    def epilogue_residual():
        for it in range(ntiles):
            yield wait(d2full, it)
            yield ("delay", rng.uniform(0.5, 4.5))
            d2free.done += 1

    roles = [producer(), splitters(), issuer(), epilogue_p(), epilogue_residual()]
    pending, finished = {}, set()

    def run(i):
        while True:
            try:
                cmd = next(roles[i])
            except StopIteration:
                finished.add(i)
                return
            if cmd[0] == "delay":
                at(cmd[1], lambda i=i: run(i))
                return
            _, bar, phase = cmd
            if bar.done > phase:
                continue
            pending[i] = (bar, phase)
            return

    for i in range(len(roles)):
        run(i)
    while True:
        woke = True
        while woke:
            woke = False
            for i, (bar, phase) in list(pending.items()):
                if bar.done > phase:
                    del pending[i]
                    run(i)
                    woke = True
        if not events:
            break
        clock[0], _, fn = heapq.heappop(events)
        fn()
    return errors, len(finished) == len(roles)


def test_projection_pass_protocol_has_no_deadlock_or_phase_aliasing():
    rng = random.Random(7)
    for _ in range(600):
        ntiles, nchunks = rng.randint(1, 14), rng.randint(1, 8)
        errors, all_done = _simulate(ntiles, nchunks, 2, rng)
        assert not errors, (ntiles, nchunks, errors[:3])
        assert all_done, (ntiles, nchunks)


def test_the_check_catches_a_missing_buffer_release_wait():
    rng = random.Random(7)
    caught = 0
    for _ in range(200):
        errors, _ = _simulate(rng.randint(3, 14), rng.randint(1, 8), 2, rng, plant_bug=True)
        caught += bool(errors)
    assert caught > 0


def _simulate_blocked(ntiles, nchunks, nblocks, stages, rng, plant_bug=False):
    """The blocked form (n_k > 256): MMA2 in nblocks column blocks per tile, two residual
    buffers, the U_k rows of one block in a single shared buffer that the residual epilogue
    refills (a TMA load) once the block before has completed. Besides the phase check, a refill
    that lands before the MMA2 reading the buffer's previous block has completed is an error.
    The planted bug issues the refill before waiting for that MMA2."""
    clock = [0.0]
    events, seq = [], [0]

    def at(delay, fn):
        seq[0] += 1
        heapq.heappush(events, (clock[0] + delay, seq[0], fn))

    full = [_Bar("full%d" % s) for s in range(stages)]
    conv = [_Bar("conv%d" % s) for s in range(stages)]
    empty = [_Bar("empty%d" % s) for s in range(stages)]
    d1full = [_Bar("d1full%d" % b) for b in range(2)]
    pready = [_Bar("pready%d" % b) for b in range(2)]
    mma2done = [_Bar("mma2done%d" % b) for b in range(2)]
    d2full = [_Bar("d2full%d" % b) for b in range(2)]
    d2free = [_Bar("d2free%d" % b) for b in range(2)]
    bload = _Bar("bload")
    errors = []
    pipe_free = [0.0]

    def tensor(duration, on_done):
        start = max(pipe_free[0], clock[0])
        pipe_free[0] = start + duration
        seq[0] += 1
        heapq.heappush(events, (pipe_free[0], seq[0], on_done))

    def done(bar):
        return lambda: setattr(bar, "done", bar.done + 1)

    def wait(bar, phase):
        if bar.done > phase + 1:
            errors.append("%s: wait for phase %d after %d completions" % (bar.name, phase, bar.done))
        return ("wait", bar, phase)

    def producer():
        q = 0
        for _ in range(ntiles):
            for _ in range(nchunks):
                s = q % stages
                if q >= stages:
                    yield wait(empty[s], q // stages - 1)
                at(rng.uniform(0.3, 0.9), done(full[s]))
                q += 1

    def splitters():
        q = 0
        for _ in range(ntiles):
            for _ in range(nchunks):
                s = q % stages
                yield wait(full[s], q // stages)
                yield ("delay", rng.uniform(0.2, 0.45))
                conv[s].done += 1
                q += 1

    def issuer():
        st = {"g2": 0, "tile": -1, "nb": 0}

        def ready():
            g2, tile, nb = st["g2"], st["tile"], st["nb"]
            if nb == 0 and pready[tile & 1].done <= (tile >> 1):
                return False
            if bload.done <= g2:
                return False
            if g2 >= 2 and d2free[g2 & 1].done <= (g2 >> 1) - 1:
                return False
            return True

        def issue():
            g2, tile, nb = st["g2"], st["tile"], st["nb"]
            last = nb + 1 == nblocks

            def fin(g2=g2, tile=tile, last=last):
                d2full[g2 & 1].done += 1
                if last:
                    mma2done[tile & 1].done += 1
            tensor(rng.uniform(0.1, 0.4), fin)
            st["g2"] += 1
            if last:
                st["tile"], st["nb"] = -1, 0
            else:
                st["nb"] += 1

        def blocking():
            g2, tile, nb = st["g2"], st["tile"], st["nb"]
            if nb == 0:
                yield wait(pready[tile & 1], tile >> 1)
            yield wait(bload, g2)
            if g2 >= 2:
                yield wait(d2free[g2 & 1], (g2 >> 1) - 1)
            issue()

        q = 0
        for it in range(ntiles):
            b = it & 1
            if it >= 2:
                yield wait(mma2done[b], (it >> 1) - 1)
            for _ in range(nchunks):
                s = q % stages
                yield wait(conv[s], q // stages)
                tensor(rng.uniform(0.05, 0.3), done(empty[s]))
                q += 1
                while st["tile"] >= 0 and ready():
                    issue()
            tensor(0.0, done(d1full[b]))
            while st["tile"] >= 0:
                yield from blocking()
            st["tile"], st["nb"] = it, 0
        while st["tile"] >= 0:
            yield from blocking()

    def epilogue_p():
        for it in range(ntiles):
            yield wait(d1full[it & 1], it >> 1)
            yield ("delay", rng.uniform(0.5, 1.5))
            pready[it & 1].done += 1

    def land(gg):
        # B2 block gg lands in the buffer: the MMA2 of block gg - 1 must have finished reading it
        def fn():
            if gg >= 1 and d2full[(gg - 1) & 1].done <= (gg - 1) >> 1:
                errors.append("B2 block %d overwrote block %d in use" % (gg, gg - 1))
            bload.done += 1
        return fn

    def epilogue_residual():
        nblk = ntiles * nblocks
        at(rng.uniform(0.2, 0.6), land(0))          # B2 block 0
        g = 0
        for _ in range(ntiles):
            for _ in range(nblocks):
                if plant_bug and g + 1 < nblk:
                    at(rng.uniform(0.0, 0.2), land(g + 1))
                yield wait(d2full[g & 1], g >> 1)
                if g + 1 < nblk and not plant_bug:
                    at(rng.uniform(0.2, 0.6), land(g + 1))   # B2 block g + 1 into the freed buffer
                yield ("delay", rng.uniform(0.3, 1.5))
                d2free[g & 1].done += 1
                g += 1

    roles = [producer(), splitters(), issuer(), epilogue_p(), epilogue_residual()]
    pending, finished = {}, set()

    def run(i):
        while True:
            try:
                cmd = next(roles[i])
            except StopIteration:
                finished.add(i)
                return
            if cmd[0] == "delay":
                at(cmd[1], lambda i=i: run(i))
                return
            _, bar, phase = cmd
            if bar.done > phase:
                continue
            pending[i] = (bar, phase)
            return

    for i in range(len(roles)):
        run(i)
    while True:
        woke = True
        while woke:
            woke = False
            for i, (bar, phase) in list(pending.items()):
                if bar.done > phase:
                    del pending[i]
                    run(i)
                    woke = True
        if not events:
            break
        clock[0], _, fn = heapq.heappop(events)
        fn()
    return errors, len(finished) == len(roles)


def test_blocked_residual_protocol_has_no_deadlock_or_phase_aliasing():
    rng = random.Random(11)
    for _ in range(600):
        ntiles, nchunks, nb = rng.randint(1, 12), rng.randint(1, 16), rng.randint(3, 4)
        errors, all_done = _simulate_blocked(ntiles, nchunks, nb, 2, rng)
        assert not errors, (ntiles, nchunks, nb, errors[:3])
        assert all_done, (ntiles, nchunks, nb)


def test_blocked_check_catches_a_refill_before_the_block_completed():
    rng = random.Random(11)
    caught = 0
    for _ in range(200):
        errors, _ = _simulate_blocked(rng.randint(3, 12), rng.randint(1, 16), 3, 2, rng, plant_bug=True)
        caught += bool(errors)
    assert caught > 0
