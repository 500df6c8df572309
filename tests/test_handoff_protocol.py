"""A model of the tile hand-offs of the warp chain (rs_chain.cuh) and of the
split column stream (rs_stream.cuh), run on the CPU under random schedules.

Each warp is a sequence of barrier waits and actions written as the kernels
order them: TMA stages filled by a producer (full), read by every compute
warp (consumed), and rings of RING tiles between warps (ready, free), every
wait on a parity derived from the tile index as the kernels derive it.  An
mbarrier is modelled by its arrival count and completed phases: a wait on
parity p succeeds once the phase of that parity has completed, i.e. while
the current phase's parity differs from p.  The checks: every schedule
finishes (no deadlock), a warp reads a ring slot or a stage only when it
holds the tile it expects, and nothing is overwritten before all of its
readers are done with it."""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count = count
        self.arrived = 0
        self.phase = 0          # completed phases

    def arrive(self):
        self.arrived += 1
        assert self.arrived <= self.count
        if self.arrived == self.count:
            self.arrived = 0
            self.phase += 1

    def test(self, parity):
        return (self.phase & 1) != parity


def run(warps, rng, pending_copies, max_steps=2_000_000):
    """Step the warps (generators yielding barriers to wait on, with their
    parities) in random order until all finish; TMA copies land at random
    later steps."""
    live = {i: (w, None) for i, w in enumerate(warps)}
    for i in list(live):
        live[i] = (live[i][0], next(live[i][0], StopIteration))
    steps = 0
    while live:
        steps += 1
        assert steps < max_steps, "no progress: deadlock"
        if pending_copies and rng.random() < 0.3:
            k = rng.randrange(len(pending_copies))
            pending_copies.pop(k)()
        ready = [i for i, (g, w) in live.items() if w is StopIteration or w[0].test(w[1])]
        if not ready:
            assert pending_copies, "every warp waits and no copy is in flight: deadlock"
            continue
        i = rng.choice(ready)
        g, w = live[i]
        if w is StopIteration:
            del live[i]
            continue
        live[i] = (g, next(g, StopIteration))
    assert not pending_copies


def chain_model(NW, RING, S, ntiles, rng):
    """The warp chain: NW compute warps, one producer."""
    full = [Barrier(1) for _ in range(S)]
    consumed = [Barrier(NW) for _ in range(S)]
    ready = [[Barrier(1) for _ in range(RING)] for _ in range(NW - 1)]
    freed = [[Barrier(1) for _ in range(RING)] for _ in range(NW - 1)]
    stage = [None] * S                       # tile held by each stage
    stage_readers = [set() for _ in range(S)]
    ring = [[None] * RING for _ in range(NW - 1)]
    ring_read = [[True] * RING for _ in range(NW - 1)]
    copies = []

    def land(s, t):
        def f():
            stage[s] = t
            stage_readers[s] = set()
            full[s].arrive()
        return f

    for t in range(min(S, ntiles)):
        copies.append(land(t, t))

    def compute(w):
        for t in range(ntiles):
            s, q, use = t % S, t % RING, t // RING
            yield (full[s], (t // S) & 1)
            if w > 0:
                yield (ready[w - 1][q], use & 1)
            if w < NW - 1 and t >= RING:
                yield (freed[w][q], (use - 1) & 1)
            assert stage[s] == t, "stage read before its tile landed"
            stage_readers[s].add(w)
            if w > 0:
                assert ring[w - 1][q] == t, "ring slot read before its tile was written"
                ring_read[w - 1][q] = True
            if w < NW - 1:
                assert ring_read[w][q], "ring slot overwritten before it was read"
                ring[w][q] = t
                ring_read[w][q] = False
                ready[w][q].arrive()
            if w > 0:
                freed[w - 1][q].arrive()
            consumed[s].arrive()

    def producer():
        for t in range(ntiles - S):
            s = t % S
            yield (consumed[s], (t // S) & 1)
            assert stage_readers[s] == set(range(NW)), "stage refilled before every warp read it"
            copies.append(land(s, t + S))

    run([compute(w) for w in range(NW)] + [producer()], rng, copies)


def split_model(KR, S, ntiles, rng):
    """The split column stream: 2 KR compute warps (warp 2p the chain of
    sequence p, warp 2p + 1 its finished columns), one producer.  Ring g is
    written by warp g and read by warp g + 1, and an odd ring (a sequence's
    finished columns) also by warp g + 2."""
    NW = 2 * KR
    RING = 4 if KR == 1 else 2
    NR = NW - 1
    readers = {g: [g + 1] + ([g + 2] if g % 2 == 1 and g + 2 <= NW - 1 else []) for g in range(NR)}
    full = [Barrier(1) for _ in range(S)]
    consumed = [Barrier(NW) for _ in range(S)]
    ready = [[Barrier(1) for _ in range(RING)] for _ in range(NR)]
    freed = [[Barrier(len(readers[g])) for _ in range(RING)] for g in range(NR)]
    stage = [None] * S
    stage_readers = [set() for _ in range(S)]
    ring = [[None] * RING for _ in range(NR)]
    ring_readers = [[set(readers[g]) for _ in range(RING)] for g in range(NR)]
    copies = []

    def land(s, t):
        def f():
            stage[s] = t
            stage_readers[s] = set()
            full[s].arrive()
        return f

    for t in range(min(S, ntiles)):
        copies.append(land(t, t))

    def compute(W):
        chain, seq = W % 2 == 0, W // 2
        writes, reads_prev, reads_in = W < NW - 1, W > 0, (not chain) and seq > 0
        for t in range(ntiles):
            s, q, use = t % S, t % RING, t // RING
            yield (full[s], (t // S) & 1)
            if reads_prev:
                yield (ready[W - 1][q], use & 1)
            if reads_in:
                yield (ready[W - 2][q], use & 1)
            if writes and t >= RING:
                yield (freed[W][q], (use - 1) & 1)
            assert stage[s] == t
            stage_readers[s].add(W)
            for g in ([W - 1] if reads_prev else []) + ([W - 2] if reads_in else []):
                assert ring[g][q] == t, "ring slot read before its tile was written"
                ring_readers[g][q].add(W)
            if writes:
                assert ring_readers[W][q] == set(readers[W]), "ring slot overwritten before all its readers"
                ring[W][q] = t
                ring_readers[W][q] = set()
                ready[W][q].arrive()
            if reads_prev:
                freed[W - 1][q].arrive()
            if reads_in:
                freed[W - 2][q].arrive()
            consumed[s].arrive()

    def producer():
        for t in range(ntiles - S):
            s = t % S
            yield (consumed[s], (t // S) & 1)
            assert stage_readers[s] == set(range(NW))
            copies.append(land(s, t + S))

    run([compute(W) for W in range(NW)] + [producer()], rng, copies)


@pytest.mark.parametrize("NW,RING,S,ntiles", [(8, 2, 11, 40), (2, 2, 5, 17), (4, 2, 7, 3), (8, 2, 11, 11),
                                              (8, 3, 11, 29), (3, 2, 6, 25)])
def test_chain_handoffs(NW, RING, S, ntiles):
    for seed in range(6):
        chain_model(NW, RING, S, ntiles, random.Random(seed))


@pytest.mark.parametrize("KR,ntiles", [(1, 30), (2, 27), (3, 21), (4, 19), (4, 5), (1, 3)])
def test_split_stream_handoffs(KR, ntiles):
    for seed in range(6):
        split_model(KR, 8, ntiles, random.Random(100 + seed))


def test_model_catches_a_wrong_parity():
    """A planted mistake: the producer waiting on the wrong parity refills
    a stage before every warp has read it (or waits forever); the model must
    notice."""
    def bad_chain(NW, RING, S, ntiles, rng):
        full = [Barrier(1) for _ in range(S)]
        consumed = [Barrier(NW) for _ in range(S)]
        stage = [None] * S
        readers = [set() for _ in range(S)]
        copies = []

        def land(s, t):
            def f():
                stage[s] = t
                readers[s] = set()
                full[s].arrive()
            return f

        for t in range(min(S, ntiles)):
            copies.append(land(t, t))

        def compute(w):
            for t in range(ntiles):
                s = t % S
                yield (full[s], (t // S) & 1)
                assert stage[s] == t
                readers[s].add(w)
                consumed[s].arrive()

        def producer():
            for t in range(ntiles - S):
                s = t % S
                yield (consumed[s], ((t // S) + 1) & 1)      # wrong parity
                assert readers[s] == set(range(NW)), "stage refilled before every warp read it"
                copies.append(land(s, t + S))

        run([compute(w) for w in range(NW)] + [producer()], rng, copies)

    with pytest.raises(AssertionError):
        bad_chain(4, 2, 5, 20, random.Random(1))
