"""Checks of the seeded input generator (Philox4x32-10 + Box-Muller).

The generator is not part of the method; these tests pin its published
properties: a bijection on counters for a fixed key, uniform 53-bit output,
N(0,1) Gaussians, and the counter layout that both sides of the parity tests
rely on. Bit equality with cuRAND's own Philox4x32-10 is checked on the GPU
(tests/test_gpu_philox.py).
"""
import numpy as np
import pytest
from scipy import stats

from paper_1708_00744_b300 import inputs


def test_philox_is_injective_on_counters():
    n = 200_000
    c = np.arange(n, dtype=np.uint64)
    x = inputs.philox4x32_10(c, 0, 0, 0, seed=12345)
    packed = {(int(a), int(b), int(cc), int(d)) for a, b, cc, d in zip(*[w[:50000] for w in x])}
    assert len(packed) == 50000
    lo = (x[0].astype(np.uint64) << np.uint64(32)) | x[1].astype(np.uint64)
    assert np.unique(lo).size == n


def test_philox_depends_on_every_counter_word_and_key_word():
    base = [np.uint64(5), np.uint64(6), np.uint64(7), np.uint64(8)]
    ref = np.array(inputs.philox4x32_10(*base, seed=(9 << 32) | 10))
    for w in range(4):
        c = list(base)
        c[w] = c[w] ^ np.uint64(1)
        out = np.array(inputs.philox4x32_10(*c, seed=(9 << 32) | 10))
        # avalanche: about half of the 128 output bits flip
        flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(ref.ravel(), out.ravel()))
        assert 30 < flips < 98
    for s in ((8 << 32) | 10, (9 << 32) | 11):
        out = np.array(inputs.philox4x32_10(*base, seed=s))
        flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(ref.ravel(), out.ravel()))
        assert 30 < flips < 98


def test_uniform_mapping_is_exact():
    assert inputs.uniform_from_words(0, 0) == 0.0
    assert inputs.uniform_from_words(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert inputs.uniform_from_words(0x80000000, 0) == 0.5


def test_uniform_distribution():
    u = np.concatenate([inputs.metropolis_uniforms(seed, s, 4096) for seed in range(3) for s in range(4)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)


def test_gaussian_distribution():
    a = inputs.initial_matrix(0, 300).ravel()
    assert stats.kstest(a, "norm").pvalue > 1e-4
    assert abs(a.mean()) < 5 / np.sqrt(a.size)
    assert abs(a.var() - 1.0) < 5 * np.sqrt(2.0 / a.size)


def test_counter_layout_streams_are_distinct_and_reproducible():
    n = 33                                                  # odd: last block uses one of two
    a1 = inputs.initial_matrix(7, n)
    a2 = inputs.initial_matrix(7, n)
    assert np.array_equal(a1, a2) and a1.shape == (n, n)
    g0 = inputs.proposal_gaussians(7, 0, n)
    g1 = inputs.proposal_gaussians(7, 1, n)
    assert not np.array_equal(g0, g1) and not np.array_equal(g0, a1)
    # row j of the proposal Gaussians does not depend on which other rows are drawn
    assert np.array_equal(inputs.proposal_gaussians(7, 0, n, electrons=[5])[0], g0[5])
    # walker seeds differ
    assert not np.array_equal(inputs.initial_matrix(inputs.walker_seed(1000, 1), 8),
                              inputs.initial_matrix(inputs.walker_seed(1000, 2), 8))


@pytest.mark.parametrize("seed", [0, 1, 2**32 + 3])
def test_box_muller_pairs_from_one_output(seed):
    x = inputs.philox4x32_10(np.uint64(3), np.uint64(0), np.uint64(inputs.TAG_MATRIX), np.uint64(1), seed)
    z0, z1 = inputs.gaussian_pairs(*x)
    row = inputs.initial_matrix(seed, 8)[3]
    assert row[2] == z0 and row[3] == z1
