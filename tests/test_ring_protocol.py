"""The bulk-copy ring of the persistent ratio kernel (ratio_dots_persist_kernel),
checked on the CPU as a model of its mbarriers.

Warp 8 loads, item after item, the walker's two vectors into one of two vector
buffers; consumer warp w takes rows w, w + 8, ... of every item and streams
their segments through SPW ring slots of its own: its lane 0 issues the bulk
copies SPW segments ahead of the reads, across item boundaries, and refills a
slot right after the warp has read it. An mbarrier wait names the parity of the
phase it waits for, so it is answered by ANY completed phase of that parity: a
wait for fill n of a slot while fill n - 1 is still unread would be answered by
fill n - 2. In the kernel a slot's fills are issued and read by one warp, in
order, so that cannot happen; with one ring shared by all warps in stream order
it can (an item whose row count is not a multiple of eight shifts the rows
against the slots).

The model runs the vector loader, the eight warps and the copies in flight
under random interleavings and asserts, at every successful wait, that the
awaited fill (or vector load) is the one that completed, and that the schedule
never stalls with nothing in flight."""
import random

import pytest

NW = 8


def _run(items, nseg, seed, per_warp=True, spw=4, tns=16):
    rnd = random.Random(seed)
    F, E = {}, {}                   # completed phases of each slot's full / empty barrier
    VF, VE, varr = [0, 0], [0, 0], [0, 0]
    held = {}                       # the fill that a slot holds
    vheld = [None, None]
    pending = []                    # copies in flight
    shared = {"g": 0}               # stream position of the shared-ring variant

    def passes(done, n):
        # try_wait.parity(n & 1): true when the latest phase of that parity is complete
        return (done & 1) != (n & 1)

    def vector_loader():
        nv = 0
        for nrows in items:
            if nrows == 0:
                continue
            buf = nv & 1
            if nv >= 2:
                while not passes(VE[buf], (nv >> 1) - 1):
                    yield "wait"
                assert VE[buf] >= nv >> 1, "vector buffer refilled before it was released"
            pending.append(("v", buf, nv))
            nv += 1
            yield "go"

    def stream(warp):
        # this warp's segments over all items, in the kernel's order
        for it, nrows in enumerate(items):
            for r in range(warp, nrows, 8):
                for sg in range(nseg):
                    yield it, r, sg

    def warp_agent(warp):
        if per_warp:
            todo = list(stream(warp))
            issued = 0

            def issue():
                nonlocal issued
                if issued < len(todo):
                    s = (warp, issued % spw)
                    pending.append(("s", s, (warp, issued)))
                    issued += 1
            for _ in range(spw):
                issue()
        c, nv, g0 = 0, 0, 0
        for it, nrows in enumerate(items):
            if nrows == 0:
                continue
            buf = nv & 1
            while not passes(VF[buf], nv >> 1):
                yield "wait"
            assert vheld[buf] == nv, "vector wait answered by an older load"
            for r in range(warp, nrows, 8):
                for sg in range(nseg):
                    if per_warp:
                        s, m, tag = (warp, c % spw), c // spw, (warp, c)
                    else:
                        gg = g0 + r * nseg + sg
                        s, m, tag = gg % tns, gg // tns, ("g", gg)
                    while not passes(F.get(s, 0), m):
                        yield "wait"
                    assert held.get(s) == tag, "slot wait answered by an older fill"
                    yield "go"
                    c += 1
                    if per_warp:
                        issue()
                    else:
                        E[s] = E.get(s, 0) + 1
            g0 += nrows * nseg
            varr[buf] += 1
            if varr[buf] == NW:
                varr[buf] = 0
                VE[buf] += 1
            nv += 1
            yield "go"

    def shared_producer():
        # the variant: one producer lane fills a shared ring in stream order
        for nrows in items:
            for r in range(nrows):
                for _ in range(nseg):
                    n = shared["g"]
                    shared["g"] += 1
                    s, m = n % tns, n // tns
                    if m >= 1:
                        while not passes(E.get(s, 0), m - 1):
                            yield "wait"
                    pending.append(("s", s, ("g", n)))
                    yield "go"

    agents = [vector_loader()] + [warp_agent(w) for w in range(NW)]
    if not per_warp:
        agents.append(shared_producer())
    alive = list(range(len(agents)))
    idle = 0
    while alive or pending:
        moved = False
        if pending and rnd.random() < 0.5:
            # a slot's copies complete in issue order (its next fill is issued
            # only after the previous one was read)
            kind = pending.pop(rnd.randrange(len(pending)))
            if kind[0] == "s":
                held[kind[1]] = kind[2]
                F[kind[1]] = F.get(kind[1], 0) + 1
            else:
                vheld[kind[1]] = kind[2]
                VF[kind[1]] += 1
            moved = True
        order = alive[:]
        rnd.shuffle(order)
        for a in order:
            try:
                step = next(agents[a])
            except StopIteration:
                alive.remove(a)
                moved = True
                continue
            if step == "go":
                moved = True
                break
        idle = 0 if (moved or pending) else idle + 1
        assert idle < 1000, "stalled with nothing in flight"


def _cases(n):
    rnd = random.Random(7)
    for seed in range(n):
        items = [rnd.choice([0, 1, 5, 8, 17, 32]) for _ in range(rnd.randint(1, 6))]
        yield items, rnd.choice([1, 2, 3]), seed


def test_per_warp_slots_never_alias_or_stall():
    for items, nseg, seed in _cases(300):
        for spw in (1, 2, 4):
            _run(items, nseg, seed, spw=spw)


def test_one_shared_ring_in_stream_order_aliases():
    """The design the kernel avoids: a wait answered by an older fill."""
    with pytest.raises(AssertionError, match="older fill"):
        for items, nseg, seed in _cases(300):
            _run(items, nseg, seed, per_warp=False)
