"""Seeded synthetic inputs for the delayed-update move loop.

This module is the ONLY code shared between the CUDA path's tests and the CPU
oracle. It draws random numbers and nothing else: it holds none of the
method's arithmetic (no determinants, ratios, inverses or updates).

Generator: Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror
and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written here
from its published definition (two 32x32->64 multiplies per round with the
multipliers 0xD2511F53 and 0xCD9E8D57, Weyl key increments 0x9E3779B9 and
0xBB67AE85, 10 rounds). The CUDA kernels carry their own implementation of
the same published definition; the two agree bit for bit on the integer
outputs.

Counter layout (our definition; the paper draws no random numbers of its own):
  key      = (seed & 0xffffffff, seed >> 32), walker seed = base seed + walker
  counter  = (a, b, tag, word3) with
    tag 0: Metropolis uniform of electron j in sweep s   -> (j, s, 0, 0)
    tag 1: proposal Gaussians of electron j in sweep s   -> (j, s, 1, blk)
    tag 2: initial Slater matrix, row i                  -> (i, 0, 2, blk)
  uniform  u = (((x0 << 32) | x1) >> 11) * 2^-53, in [0, 1) and exact in fp64
  Gaussian pair from one output: u1 from (x0, x1), u2 from (x2, x3),
           rho = sqrt(-2 log(1 - u1)),  (rho cos(2 pi u2), rho sin(2 pi u2))
           (Box-Muller, Ann. Math. Stat. 29, 1958); block blk gives entries
           2 blk and 2 blk + 1 of the row.

Workload shapes follow the paper's solid-state sizes (N from hundreds to
thousands, Sec. III): A_ij ~ N(0, 1), proposal v = a_j + sigma * g with
g ~ N(0, 1)^N (sigma = 0.1 gives DMC-like, sigma = 1.0 VMC-like acceptance).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x32_10", "uniform_from_words", "gaussian_pairs",
    "metropolis_uniforms", "proposal_gaussians", "initial_matrix",
    "walker_seed", "serving_trace", "SERVING_SIZES", "TAG_UNIFORM", "TAG_PROPOSAL",
    "TAG_MATRIX",
]

TAG_UNIFORM = 0
TAG_PROPOSAL = 1
TAG_MATRIX = 2

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, seed: int):
    """Philox4x32-10 outputs for counters (c0, c1, c2, c3) under `seed`.

    The counter words are broadcast against each other; the result is four
    uint32 arrays (x0, x1, x2, x3).
    """
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    shape = np.broadcast(np.asarray(c0), np.asarray(c1), np.asarray(c2), np.asarray(c3)).shape
    x0 = np.broadcast_to(np.asarray(c0, dtype=np.uint64), shape).copy() & _MASK
    x1 = np.broadcast_to(np.asarray(c1, dtype=np.uint64), shape).copy() & _MASK
    x2 = np.broadcast_to(np.asarray(c2, dtype=np.uint64), shape).copy() & _MASK
    x3 = np.broadcast_to(np.asarray(c3, dtype=np.uint64), shape).copy() & _MASK
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64(seed >> 32)
    for _ in range(10):
        p0 = _M0 * x0
        p1 = _M1 * x2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        x0, x1, x2, x3 = (hi1 ^ x1 ^ k0), lo1, (hi0 ^ x3 ^ k1), lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def uniform_from_words(hi, lo):
    """53-bit uniform in [0, 1) from two 32-bit words (exact in fp64)."""
    bits = (np.asarray(hi, dtype=np.uint64) << _S32) | np.asarray(lo, dtype=np.uint64)
    return (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian_pairs(x0, x1, x2, x3):
    """Box-Muller pair from one Philox output."""
    u1 = uniform_from_words(x0, x1)
    u2 = uniform_from_words(x2, x3)
    rho = np.sqrt(-2.0 * np.log(1.0 - u1))
    ang = 2.0 * np.pi * u2
    return rho * np.cos(ang), rho * np.sin(ang)


def _gaussian_rows(seed: int, rows, a_word1: int, tag: int, n: int, row_is_word0=True):
    rows = np.asarray(rows, dtype=np.uint64)
    nblk = (n + 1) // 2
    blk = np.arange(nblk, dtype=np.uint64)[None, :]
    r = rows[:, None]
    x = philox4x32_10(r, np.uint64(a_word1), np.uint64(tag), blk, seed)
    z0, z1 = gaussian_pairs(*x)
    out = np.empty((rows.shape[0], 2 * nblk), dtype=np.float64)
    out[:, 0::2] = z0
    out[:, 1::2] = z1
    return out[:, :n]


def metropolis_uniforms(seed: int, sweep: int, n: int) -> np.ndarray:
    """u[j] for electrons j = 0..n-1 of one sweep (counter (j, sweep, 0, 0))."""
    j = np.arange(n, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(j, np.uint64(sweep), np.uint64(TAG_UNIFORM), np.uint64(0), seed)
    return uniform_from_words(x0, x1)


def proposal_gaussians(seed: int, sweep: int, n: int, electrons=None) -> np.ndarray:
    """g rows for one sweep: row j is the N(0,1)^n draw for electron j."""
    if electrons is None:
        electrons = np.arange(n)
    return _gaussian_rows(seed, electrons, sweep, TAG_PROPOSAL, n)


def initial_matrix(seed: int, n: int) -> np.ndarray:
    """Initial Slater matrix, A_ij ~ N(0, 1); row i holds electron i's orbitals."""
    return _gaussian_rows(seed, np.arange(n), 0, TAG_MATRIX, n)


def walker_seed(base_seed: int, walker: int) -> int:
    return (int(base_seed) + int(walker)) & 0xFFFFFFFFFFFFFFFF


# Electron counts of the serving workload: a geometric set, drawn uniformly
# (log-uniform in N), spanning the paper's sizes (hundreds to thousands).
SERVING_SIZES = (128, 256, 512, 1024, 2048, 4096)


def serving_trace(seed: int, rate_hz: float, duration_s: float, sizes=SERVING_SIZES,
                  nsweeps: int = 20, max_requests: int | None = None):
    """Poisson stream of walker requests: exponential inter-arrival times of
    mean 1/rate_hz over [0, duration_s), N uniform over `sizes`, and request i
    carries walker key walker_seed(10**6 * (seed + 1), i). Uses numpy's PCG64
    generator seeded with `seed` (the arrival process is an input, not a step
    of the method)."""
    rng = np.random.default_rng(seed)
    out, t, i = [], 0.0, 0
    base = 10**6 * (int(seed) + 1)
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s or (max_requests is not None and i >= max_requests):
            return out
        out.append(dict(id=i, seed=walker_seed(base, i), N=int(rng.choice(sizes)),
                        nsweeps=int(nsweeps), arrival_s=float(t)))
        i += 1
