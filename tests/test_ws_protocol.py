"""A model of the slot hand-over of the warp-specialised 3D closure kernel
(ws3_kernel in csrc/lbmhd3.cu), checked under random schedules on the CPU.

Producer warps write plane index K (unit-local k = 0 .. n + 1) into slot
K mod F and arrive on full[K mod B]; consumer warps, for row j of a unit
starting at index Kb, wait on full[(Kb + j + 2) mod B] with the phase parity
of that index, read slots Kb + j .. Kb + j + 2 and hand back slot Kb + j on
empty[(Kb + j) mod F] (and the unit's last two slots after its last row);
a producer waits on empty[K mod F] for the hand-back of K - F before it
writes.  Barriers follow the mbarrier rules: a phase completes when its
count of arrivals is reached, and a parity wait passes when the phase of
that parity has completed, i.e. the current phase's parity differs.

The model checks that every read sees the plane it expects, that no phase
of a barrier collects arrivals meant for two different planes, and that the
schedule never deadlocks -- for the kernel's ring lengths (F = B = 4), and
that the same checks catch a barrier ring shorter than the slot ring.  A
second model follows the failure path: every wait gives up after a bounded
number of polls, sets the CTA's abort flag and the status, and every warp
checks the flag once per plane; with the producers' announcements dropped
(the host-requested fault) every warp must still finish."""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0
        self.tags = set()  # planes whose arrivals the current phase collected

    def arrive(self, tag):
        self.tags.add(tag)
        if len(self.tags) > 1:
            raise AssertionError(f"one phase collected arrivals for planes {sorted(self.tags)}")
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count
            self.tags = set()

    def passed(self, parity):
        return (self.phase & 1) != parity


def producer(units, F, B, slots, full, empty):
    K = 0
    for n in units:
        for k in range(n + 2):
            if K >= F:
                b, par = empty[K % F], ((K // F) - 1) & 1
                while not b.passed(par):
                    yield "wait"
            slots[K % F].append(K)  # this warp's part of plane K
            yield "write"
            full[K % B].arrive(K)
            K += 1
            yield "arrive"


def consumer(units, F, B, P, slots, full, empty):
    Kb = 0
    for n in units:
        for j in range(n):
            Kf = Kb + j + 2
            b, par = full[Kf % B], (Kf // B) & 1
            while not b.passed(par):
                yield "wait"
            for K in (Kb + j, Kb + j + 1, Kf):
                got = slots[K % F][-P:]
                if len(got) < P or any(t != K for t in got):
                    raise AssertionError(f"row {Kb + j} read slot {K % F} holding {got}, not plane {K}")
            yield "read"
            empty[(Kb + j) % F].arrive(Kb + j)
            yield "arrive"
        empty[(Kb + n) % F].arrive(Kb + n)
        empty[(Kb + n + 1) % F].arrive(Kb + n + 1)
        Kb += n + 2
        yield "unit"


def run(units, F, B, P, C, seed):
    """One random schedule; warps run at skewed speeds.  Returns normally or
    raises AssertionError (a wrong read, mixed phase or deadlock)."""
    rng = random.Random(seed)
    slots = [[] for _ in range(F)]
    full = [Barrier(P) for _ in range(B)]
    empty = [Barrier(C) for _ in range(F)]
    warps = [producer(units, F, B, slots, full, empty) for _ in range(P)]
    warps += [consumer(units, F, B, P, slots, full, empty) for _ in range(C)]
    speed = [rng.choice((1, 1, 2, 8)) for _ in warps]
    live = list(range(len(warps)))
    stalled = 0
    while live:
        w = rng.choices(live, weights=[speed[i] for i in live])[0]
        try:
            step = next(warps[w])
        except StopIteration:
            live.remove(w)
            stalled = 0
            continue
        stalled = stalled + 1 if step == "wait" else 0
        if stalled > 20000:
            raise AssertionError("deadlock: every live warp waits")


UNITS = [[1, 3, 2, 5, 1, 1, 4], [2, 2, 2], [6, 1, 7, 1, 2], [1] * 9]


@pytest.mark.parametrize("units", UNITS)
def test_kernel_rings_hand_over_correctly(units):
    """F = B = 4, as in the kernel: every schedule reads the right planes."""
    for seed in range(60):
        run(units, F=4, B=4, P=3, C=2, seed=seed)


def test_longer_barrier_ring_is_also_safe():
    for units in UNITS:
        for seed in range(30):
            run(units, F=4, B=6, P=3, C=2, seed=seed)
            run(units, F=6, B=6, P=3, C=2, seed=seed)


def test_barrier_ring_shorter_than_slot_ring_is_caught():
    """B < F lets a producer warp arrive for plane K while another producer
    has not yet arrived for K - B on the same barrier: the model must find
    that (a mixed phase, a wrong read or a deadlock) in some schedule."""
    found = 0
    for units in UNITS:
        for seed in range(200):
            try:
                run(units, F=6, B=4, P=3, C=2, seed=seed)
            except AssertionError:
                found += 1
    assert found > 0


def producer_bounded(units, F, B, full, empty, ctl, drop, limit):
    K = 0
    for n in units:
        for k in range(n + 2):
            if ctl["abort"]:
                return
            if K >= F:
                b, par, polls = empty[K % F], ((K // F) - 1) & 1, 0
                while not b.passed(par):
                    polls += 1
                    if polls > limit:
                        ctl["abort"] = ctl["status"] = True
                        return
                    yield "wait"
            if not drop:
                full[K % B].arrive(K)
            K += 1
            yield "arrive"


def consumer_bounded(units, F, B, full, empty, ctl, limit):
    Kb = 0
    for n in units:
        for j in range(n):
            if ctl["abort"]:
                return
            Kf = Kb + j + 2
            b, par, polls = full[Kf % B], (Kf // B) & 1, 0
            while not b.passed(par):
                polls += 1
                if polls > limit:
                    ctl["abort"] = ctl["status"] = True
                    return
                yield "wait"
            empty[(Kb + j) % F].arrive(Kb + j)
            yield "arrive"
        empty[(Kb + n) % F].arrive(Kb + n)
        empty[(Kb + n + 1) % F].arrive(Kb + n + 1)
        Kb += n + 2


@pytest.mark.parametrize("drop", [False, True])
def test_bounded_waits_end_every_warp(drop):
    """With every announcement made, the run ends with no abort; with them
    dropped, the waits expire, the status is set, and every warp returns
    (a bounded number of scheduling steps)."""
    for units in UNITS:
        for seed in range(20):
            rng = random.Random(seed)
            P, C, F, B = 3, 2, 4, 4
            full = [Barrier(P) for _ in range(B)]
            empty = [Barrier(C) for _ in range(F)]
            ctl = {"abort": False, "status": False}
            warps = [producer_bounded(units, F, B, full, empty, ctl, drop, 500) for _ in range(P)]
            warps += [consumer_bounded(units, F, B, full, empty, ctl, 500) for _ in range(C)]
            live, steps = list(range(len(warps))), 0
            while live:
                w = rng.choice(live)
                try:
                    next(warps[w])
                except StopIteration:
                    live.remove(w)
                steps += 1
                assert steps < 10 ** 6, "a warp never returned"
            assert ctl["status"] == drop
