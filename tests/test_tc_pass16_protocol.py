"""Model check of the barrier protocol of the FP16 tensor-core pass (k_tc_pass16, residual form):
TMA producer, splitters (per chunk: the FP16 parts to shared memory, then the previous tile's E
at the tensor-memory columns the chunk overwrites, then the chunk's FP32 values into them), MMA
issuer, epilogue (P into the staging tile and MMA2's A operand), P writers (the staged P out,
handed over and back through two barriers), over a ring of stages
that carries a tile's input chunks and then (residual form) the blocks of U_k's rows that MMA2
reads, one tile of the input in tensor memory released block by block, and one pair of P
accumulators over which the epilogue writes MMA2's A operand. The splitters' conversion barrier
of a stage completes for input chunks only, so the issuer tracks its parity per stage.

Each role is a coroutine issuing the waits and arrivals the kernel issues, in the same order;
tensor-core work runs in issue order on one pipe; durations are random. Two kinds of check:
no wait starts on a barrier that has already completed the phase after the one it names (its
parity would read as pending for ever), every role finishes; and no data hazard: a stage is
refilled only after its MMAs ran, a tensor-memory block is overwritten by the next tile only
after the epilogue read its E, MMA2 reads a block only once the tile's chunks are stored and
reads the A operand of its own tile, the P accumulators are overwritten only after the
epilogue read them and after the MMA2 that read the A operand stored over them. Planted bugs
(a missing wait) must be caught.
"""

import heapq
import random

import pytest


class _Bar:
    def __init__(self, name):
        self.name, self.done = name, 0


def _simulate(ntiles, nchunks, stages, rng, resid=True, bug=None):
    nblk = (nchunks + 1) // 2          # 128-column blocks, two 64-column chunks each
    clock = [0.0]
    events, seq = [], [0]
    errors = []

    def at(delay, fn):
        seq[0] += 1
        heapq.heappush(events, (clock[0] + delay, seq[0], fn))

    per_tile = nchunks + (nblk if resid else 0)    # ring items per tile
    full = [_Bar("full%d" % s) for s in range(stages)]
    conv = [_Bar("conv%d" % s) for s in range(stages)]
    empty = [_Bar("empty%d" % s) for s in range(stages)]
    d1full, pready, xst = _Bar("d1full"), _Bar("pready"), _Bar("xst")
    efull = [_Bar("efull%d" % b) for b in range(nblk)]
    pstaged, pfree = _Bar("pstaged"), _Bar("pfree")
    pst_tile, pst_out = [-1], [-1]      # tile in the staging tile; last tile written out
    pipe_free = [0.0]
    # data state
    stage_chunk = [None] * stages        # ring item q whose data the stage holds
    stage_used = [True] * stages         # its MMAs have run
    blk_stored = [[-1] * 2 for _ in range(nblk)]   # tile whose chunk (2 b + j) is in TMEM
    chunk_read = [-1] * nchunks         # last tile whose E the splitters read at chunk c's columns
    efull_tile = [-1] * nblk            # last tile whose MMA2 wrote block b
    pacc_tile, pacc_read = [-1], [-1]
    p16_tile, mma2_done_tile = [-1], [-1]

    def tensor(duration, start_fn, on_done):
        start = max(pipe_free[0], clock[0])
        pipe_free[0] = start + duration
        seq[0] += 1
        heapq.heappush(events, (start, seq[0], start_fn))
        seq[0] += 1
        heapq.heappush(events, (pipe_free[0], seq[0], on_done))

    def wait(bar, phase):
        if bar.done > phase + 1:
            errors.append("%s: wait for phase %d after %d completions" % (bar.name, phase, bar.done))
        return ("wait", bar, phase)

    def producer():
        q = 0
        for _ in range(ntiles):
            for _ in range(per_tile):
                s = q % stages
                if q >= stages:
                    yield wait(empty[s], q // stages - 1)

                def land(s=s, q=q):
                    if not stage_used[s]:
                        errors.append("stage %d refilled before its MMAs ran" % s)
                    stage_chunk[s], stage_used[s] = q, False
                    full[s].done += 1
                at(rng.uniform(0.3, 1.2), land)
                q += 1

    def read_e(it, c):
        # E of tile it at chunk c's columns: its block's MMA2 must have written it
        if efull_tile[c // 2] < it:
            errors.append("E of tile %d at chunk %d read before MMA2 wrote it" % (it, c))
        chunk_read[c] = it

    def splitters():
        q = 0
        for it in range(ntiles):
            for c in range(nchunks):
                s = q % stages
                yield wait(full[s], q // stages)
                yield ("delay", rng.uniform(0.1, 0.4))
                conv[s].done += 1            # FP16 parts in shared memory: MMA1 may run
                if resid:
                    b = c // 2
                    if it > 0:
                        if bug != "no_efull_wait":
                            yield wait(efull[b], it - 1)
                        yield ("delay", rng.uniform(0.02, 0.2))
                        read_e(it - 1, c)
                    # the store into tensor memory, now and then late
                    yield ("delay", rng.uniform(2.0, 6.0) if rng.random() < 0.1 else rng.uniform(0.02, 0.1))
                    if it > 0 and chunk_read[c] < it - 1:
                        errors.append("tile %d overwrote chunk %d's columns before E of tile %d was read" % (it, c, it - 1))
                    blk_stored[b][c % 2] = it
                    if c == nchunks - 1:
                        xst.done += 1
                q += 1
            q += per_tile - nchunks             # the U_k-row items go to the issuer
        if resid and ntiles > 0:
            # E of the last tile
            for c in range(nchunks):
                if bug != "no_efull_wait":
                    yield wait(efull[c // 2], ntiles - 1)
                yield ("delay", rng.uniform(0.02, 0.2))
                read_e(ntiles - 1, c)

    def issuer():
        q = 0
        xuse = [0] * stages                 # input chunks converted in each stage so far
        for it in range(ntiles):
            if not resid and it > 0 and bug != "no_pacc_wait":
                yield wait(pready, it - 1)
            for c in range(nchunks):
                s = q % stages
                if bug == "conv_by_item":
                    yield wait(conv[s], q // stages)
                else:
                    yield wait(conv[s], xuse[s])
                xuse[s] += 1

                def start(s=s, q=q, it=it, c=c):
                    if stage_chunk[s] != q:
                        errors.append("MMA1 read stage %d without chunk %d" % (s, q))
                    if c == 0:
                        if pacc_read[0] < it - 1:
                            errors.append("MMA1 of tile %d overwrote P before it was read" % it)
                        if resid and mma2_done_tile[0] < it - 1:
                            errors.append("MMA1 of tile %d overwrote the A operand of tile %d" % (it, it - 1))
                        pacc_tile[0] = it

                def fin(s=s):
                    stage_used[s] = True
                    empty[s].done += 1
                tensor(rng.uniform(0.05, 0.3), start, fin)
                q += 1
            tensor(0.0, lambda: None, lambda: setattr(d1full, "done", d1full.done + 1))
            if resid:
                yield wait(pready, it)
                if bug != "no_xst_wait":
                    yield wait(xst, it)
                for b in range(nblk):
                    s = q % stages
                    if bug != "no_u_wait":
                        yield wait(full[s], q // stages)

                    def start2(b=b, it=it, s=s, q=q):
                        if blk_stored[b][0] != it or (2 * b + 1 < nchunks and blk_stored[b][1] != it):
                            errors.append("MMA2 of tile %d read TMEM block %d before it was stored" % (it, b))
                        if p16_tile[0] != it:
                            errors.append("MMA2 of tile %d read the A operand of tile %s" % (it, p16_tile[0]))
                        if stage_chunk[s] != q:
                            errors.append("MMA2 read stage %d without U rows item %d" % (s, q))

                    def fin2(b=b, it=it, s=s):
                        efull_tile[b] = it
                        efull[b].done += 1
                        stage_used[s] = True
                        empty[s].done += 1
                        if b == nblk - 1:
                            mma2_done_tile[0] = it
                    tensor(rng.uniform(0.1, 0.5), start2, fin2)
                    q += 1

    def epilogue():
        for it in range(ntiles):
            yield wait(d1full, it)
            if it > 0 and bug != "no_pfree_wait":
                yield wait(pfree, it - 1)
            yield ("delay", rng.uniform(0.2, 0.8))
            if pacc_tile[0] != it:
                errors.append("epilogue read P of tile %s for tile %d" % (pacc_tile[0], it))
            if pst_out[0] < it - 1:
                errors.append("P of tile %d staged before tile %d was written out" % (it, it - 1))
            pst_tile[0] = it
            pacc_read[0] = it
            if resid:
                if mma2_done_tile[0] < it - 1:
                    errors.append("A operand of tile %d written while MMA2 of tile %d reads it" % (it, it - 1))
                p16_tile[0] = it
            pready.done += 1
            pstaged.done += 1

    def writers():
        for it in range(ntiles):
            if bug != "no_pstaged_wait":
                yield wait(pstaged, it)
            # the staged P out, now and then slowly
            yield ("delay", rng.uniform(3.0, 8.0) if rng.random() < 0.1 else rng.uniform(0.3, 2.0))
            if pst_tile[0] != it:
                errors.append("tile %d's P written out from a staging tile holding tile %s" % (it, pst_tile[0]))
            pst_out[0] = it
            pfree.done += 1

    roles = [producer(), splitters(), issuer(), epilogue(), writers()]
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


@pytest.mark.parametrize("resid,stages", [(True, 4), (True, 2), (True, 3), (False, 4)])
def test_fp16_pass_protocol_has_no_deadlock_aliasing_or_hazard(resid, stages):
    rng = random.Random(11)
    for _ in range(500):
        ntiles, nchunks = rng.randint(1, 12), rng.randint(1, 6)
        errors, all_done = _simulate(ntiles, nchunks, stages, rng, resid=resid)
        assert not errors, (ntiles, nchunks, errors[:3])
        assert all_done, (ntiles, nchunks)


# (the wait on the P read-out before a tile's MMA1 exists in the projection form only: in the
# residual form that MMA1 follows, on the same in-order pipe, the previous tile's MMA2, which
# waited for the read-out)
# (nor is the MMA issuer's wait for the stored tile (xst) one whose absence shows here: the
# splitters store a tile's chunks before epi-1 can run on it, and MMA2 also waits for epi-1)
@pytest.mark.parametrize("bug,resid", [("no_pacc_wait", False), ("no_efull_wait", True),
                                       ("no_u_wait", True), ("conv_by_item", True),
                                       ("no_pfree_wait", True), ("no_pstaged_wait", True),
                                       ("no_pfree_wait", False), ("no_pstaged_wait", False)])
def test_the_check_catches_a_missing_wait(bug, resid):
    rng = random.Random(5)
    caught = 0
    for _ in range(300):
        errors, done = _simulate(rng.randint(2, 12), rng.randint(1, 6), 4, rng,
                                 resid=resid, bug=bug)
        caught += bool(errors) or not done
    assert caught > 0
