"""The exchange of partial dot products in the persistent sweep kernel, checked
on the CPU as a model of its slots and tags.

Each ratio CTA writes, per proposal p (counted from the launch's start; queue
length k), its 2k + 1 partials of Eq. 3's ratio into buffer p & 1, each as one
64-bit word whose tag is 1 + p mod 3 (the slots are cleared to tag 0 before
every launch), and it also tags the next four slots of that buffer. A reader
of proposal p polls slots [0, 2k + 1) of the buffer until each carries p's
tag. The protocol is sound when no slot that a reader polls can hold an older
word with p's tag: then the only word with that tag is p's own. Walkers follow
one another inside a launch behind the flush barriers, and a flush empties the
queue when k reaches K.

The model replays the writes in proposal order and checks, at each read, the
proposal that last wrote every polled slot."""
import numpy as np
import pytest

EXTRA = 4          # slots tagged beyond a proposal's own 2k + 1


def tag(p):
    return 1 + p % 3


def replay(walkers, K, extra=EXTRA, by_electron=False):
    """walkers: per walker of the launch, its accept decisions (one per
    proposal). Returns the list of (p, slot, last writer) for every polled
    slot whose current word carries p's tag without being p's own. With
    by_electron the buffer is chosen by the walker's own proposal index j
    instead of p."""
    nj = 2 * K + 1
    last = np.full((2, nj), -1, dtype=np.int64)     # proposal that last wrote each slot
    wtag = np.zeros((2, nj), dtype=np.int64)        # its tag (0: cleared)
    bad = []
    p = 0
    for acc in walkers:
        k = 0
        for j, a in enumerate(acc):
            b = (j if by_electron else p) & 1
            njk = 2 * k + 1
            # readers that poll before the writers' stores land see the old words
            for s in range(njk):
                if wtag[b, s] == tag(p) and last[b, s] != p:
                    bad.append((p, s, int(last[b, s])))
            hi = min(nj, njk + extra)
            last[b, :hi] = p
            wtag[b, :hi] = tag(p)
            if a:
                k += 1
            if k == K or j == len(acc) - 1:
                k = 0                                # flush (queue full, or end of sweep)
            p += 1
    return bad


def _walkers(rng, n_walkers, N, p_acc):
    return [rng.random(N) < p_acc for _ in range(n_walkers)]


@pytest.mark.parametrize("K", [1, 2, 4, 16, 32, 64])
@pytest.mark.parametrize("N", [1, 2, 3, 7, 64, 129])
@pytest.mark.parametrize("p_acc", [0.0, 0.3, 0.95, 1.0])
def test_no_stale_word_carries_the_awaited_tag(K, N, p_acc):
    rng = np.random.default_rng(1000 * K + N)
    for n_walkers in (1, 3):
        assert replay(_walkers(rng, n_walkers, N, p_acc), K) == []


def test_every_acceptance_pattern_of_short_walkers():
    # exhaustive over all accept patterns of up to 10 proposals, two walkers
    # behind each other in one launch
    for K in (2, 3, 4, 8):
        for N in range(1, 11):
            for bits in range(1 << N):
                acc = [(bits >> i) & 1 == 1 for i in range(N)]
                assert replay([acc, acc[::-1]], K) == [], (K, N, bits)


def test_the_extra_slots_are_needed():
    # without the slots tagged ahead, a queue that grows by one per proposal
    # meets a word from six proposals back with the same tag
    K = 32
    acc = [True] * 64
    assert replay([acc], K, extra=0) != []
    assert replay([acc], K, extra=3) != []
    assert replay([acc], K, extra=EXTRA) == []


def test_buffers_by_electron_index_would_not_do():
    # choosing the buffer by the walker's own proposal index j: after a walker
    # of odd length, the next walker's second proposal polls a buffer last
    # written three proposals earlier, whose tag is its own
    assert replay([[False] * 3] * 3, 1, by_electron=True) != []
    assert replay([[False] * 3] * 3, 1) == []


def test_two_tags_would_not_do():
    # with tags 1 + p mod 2 a buffer's word from two proposals back carries
    # the tag of the proposal that polls it
    K, N = 8, 20
    nj = 2 * K + 1
    last = np.full((2, nj), -1)
    hits = 0
    for p in range(N):
        b = p & 1
        if p >= 2 and 1 + (last[b, 0] % 2) == 1 + (p % 2):
            hits += 1
        last[b, :] = p
    assert hits > 0
