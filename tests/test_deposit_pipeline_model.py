"""A model of the deposit kernel's hand-over protocol (csrc/particles.cu,
deposit_core), checked on random interleavings of its warps.

The kernel has no block barrier inside its stage loop. Stage k (a row
segment and a species) sits in staging buffer k % 2, filled by bulk copies
whose completion an mbarrier counts; the warp that finishes a stage last
refills that buffer with stage k + 2. A unit's field tiles alternate between
two copies: at the start of unit u every warp waits until all warps are done
with unit u - 1 (the 'free' barrier of copy (u + 1) % 2), stores its share of
unit u + 1's tiles into that copy and arrives on its 'full' barrier, then
waits for the 'full' phase of unit u. Waits use the mbarrier parity rule: a
wait for phase m returns once the barrier has left phase m, so it needs the
barrier never to run two phases ahead of a waiter.

The model runs the same sequence of arrivals and parity waits for 8 warps in
random orders, with copies landing at random times, and checks that no warp
reads a buffer or tile before its data is there, that nothing is overwritten
while a warp still reads it, and that the run ends (no deadlock). Two planted
protocol mistakes must be caught.
"""
import random

import pytest

NW, NB = 8, 2


class Barrier:
    """mbarrier: an arrival count and a transaction count per phase."""

    def __init__(self, count):
        self.count, self.pending, self.phase, self.tx = count, count, 0, 0

    def expect_tx(self, n):
        self.tx += n

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        self._advance()

    def complete_tx(self, n):
        self.tx -= n
        assert self.tx >= 0
        self._advance()

    def _advance(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        # the phase with this parity has completed once the current one differs
        return (self.phase & 1) != parity


class Hazard(AssertionError):
    pass


def run(myunits, nsp, seed, free_parity=None, refill_at=NW):
    rnd = random.Random(seed)
    nst = myunits * nsp
    mbar = [Barrier(1) for _ in range(NB)]
    tfull = [Barrier(NW) for _ in range(2)]   # one arrival per warp stands for its 32 threads
    tfree = [Barrier(NW) for _ in range(2)]
    sdone = [0] * NB
    buf_stage, buf_landed = [None] * NB, [False] * NB
    tile_unit = [None, None]
    readers_buf = [set() for _ in range(NB)]
    readers_tile = [set(), set()]
    inflight = []

    def issue(k):
        b = k % NB
        if readers_buf[b]:
            raise Hazard(f"buffer {b} refilled with stage {k} while in use")
        buf_stage[b], buf_landed[b] = k, False
        mbar[b].expect_tx(1)
        mbar[b].arrive()
        inflight.append((b, k))

    def load(u, w):
        x = u & 1
        if readers_tile[x]:
            raise Hazard(f"tile copy {x} overwritten with unit {u} while in use")
        if w == 0:
            tile_unit[x] = u
        tfull[x].arrive()

    for k in range(min(NB, nst)):
        issue(k)

    def warp(w):
        load(0, w)
        yield
        for k in range(nst):
            b = k % NB
            u, s = divmod(k, nsp)
            if s == 0:
                if u + 1 < myunits:
                    if u >= 1:
                        par = ((u - 1) >> 1) & 1 if free_parity is None else free_parity(u)
                        while not tfree[(u + 1) & 1].done(par):
                            yield "wait"
                    load(u + 1, w)
                    yield
                while not tfull[u & 1].done((u >> 1) & 1):
                    yield "wait"
                if tile_unit[u & 1] != u:
                    raise Hazard(f"unit {u} read tile copy holding unit {tile_unit[u & 1]}")
                readers_tile[u & 1].add(w)
            while not mbar[b].done((k // NB) & 1):
                yield "wait"
            if buf_stage[b] != k or not buf_landed[b]:
                raise Hazard(f"stage {k} read before its copy landed")
            readers_buf[b].add(w)
            yield
            readers_buf[b].discard(w)
            sdone[b] += 1
            if sdone[b] == refill_at:
                sdone[b] = 0
                if k + NB < nst:
                    issue(k + NB)
            if s == nsp - 1:
                readers_tile[u & 1].discard(w)
                tfree[u & 1].arrive()
            yield

    gens = [warp(w) for w in range(NW)]
    alive, stuck = set(range(NW)), 0
    while alive:
        if inflight and rnd.random() < 0.3:
            b, k = inflight.pop(0)
            buf_landed[b] = True
            mbar[b].complete_tx(1)
        w = rnd.choice(sorted(alive))
        try:
            r = next(gens[w])
            stuck = stuck + 1 if r == "wait" else 0
        except StopIteration:
            alive.discard(w)
            stuck = 0
        if stuck > 20000 and not inflight:
            raise Hazard("deadlock")
    assert not inflight


@pytest.mark.parametrize("nsp", [1, 2, 3])
@pytest.mark.parametrize("myunits", [1, 2, 3, 5, 8])
def test_protocol_has_no_hazard_or_deadlock(myunits, nsp):
    for seed in range(30):
        run(myunits, nsp, seed)


def test_planted_protocol_mistakes_are_caught():
    # waiting for the free phase of unit u instead of u - 1
    with pytest.raises(Hazard):
        for seed in range(30):
            run(5, 2, seed, free_parity=lambda u: (u >> 1) & 1)
    # refilling a buffer when the second-to-last warp is done
    with pytest.raises(Hazard):
        for seed in range(30):
            run(5, 2, seed, refill_at=NW - 1)
