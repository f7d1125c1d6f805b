"""Shared helpers of the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import inputs

torch = pytest.importorskip("torch")

# Tolerances of the fp64 path. The bar is 1e-10 on every metric. Where a walk
# goes through ill-conditioned matrices, two correct fp64 implementations of a
# running inverse disagree by more than that (the forward error of a linear
# solve grows with kappa(A); Higham, Accuracy and Stability of Numerical
# Algorithms, Sec. 7). The tolerance of each metric is therefore
#     max(1e-10, 10 x the disagreement of the oracle's own two fp64 readings)
# on the same walk and decisions: the Sherman-Morrison reading (Eq. 1-2) and
# the delayed reading (Eq. 3-4) started from the inverse computed the other
# way round (the LU of A instead of A'), or for a direct calculation the LU
# of A and of its transpose. The starting inverse of an ill-conditioned
# matrix differs between two correct fp64 computations by about u kappa(A),
# and the ratios of the whole walk inherit that difference. A GPU error ten times larger than the oracle's own spread
# fails. Errors: ratios |r - r_ref| / max(1, |r_ref|) (relative for
# |r| >= 1, absolute below, where a determinant ratio is a cancelling sum);
# A^{-1} norm-wise relative; log|det| absolute over max(1, |log|det||).
RTOL_RATIO = 1e-10
RTOL_INV = 1e-10
RTOL_LOGDET = 1e-10
NEAR_TIE = 1e-10
U64 = 2.0 ** -53
SPREAD_MARGIN = 10.0


# The device forms each ratio's dot products in fp64 within a CTA and sums the
# CTAs' partial sums as double-fp32 pairs (48 significant bits), so its
# rounding of proposal j's ratio is bounded by about 2^-47 times the size of
# Eq. 1's terms, terms_j = 1 + sum_i |(A^{-1})_ij u_i| (Higham, Sec. 3.1: the
# error of a dot product scales with the sum of |terms|). Where that sum is
# large (an ill-conditioned ratio: terms of 1e5 cancelling to O(1)), any other
# summation order misses the oracle's by far more than the oracle's two readings
# (which sum that dot in the same order) miss each other; the ratio bar of
# proposal j is therefore max(the bar above, EXCHANGE_MARGIN 2^-47 terms_j /
# max(1, |r_j|)).
EXCHANGE_EPS = 2.0 ** -47
EXCHANGE_MARGIN = 10.0


class Tol(dict):
    """Per-metric fp64 tolerances: keys ratio, inverse, logdet; with the
    oracle's ratios and terms attached, a ratio check takes the device's
    ratios and holds each to its own bound."""

    ref_ratios = None
    terms = None

    def ratio_bounds(self):
        r = np.asarray(self.ref_ratios)
        return np.maximum(self["ratio"], EXCHANGE_MARGIN * EXCHANGE_EPS * np.asarray(self.terms)
                          / np.maximum(1.0, np.abs(r)))

    def check(self, label, ratio=None, inverse=None, logdet=None):
        got = dict(ratio=ratio, inverse=inverse, logdet=logdet)
        text = []
        if isinstance(ratio, np.ndarray) and ratio.size > 1:
            assert self.ref_ratios is not None, "elementwise ratio check needs the oracle's ratios"
            ref = np.asarray(self.ref_ratios).reshape(ratio.shape)
            err = np.abs(ratio - ref) / np.maximum(1.0, np.abs(ref))
            bnd = self.ratio_bounds().reshape(ratio.shape)
            worst = int(np.argmax(err / bnd))
            text.append("ratio %.1e (tol %.1e; worst against its bound %.1e / %.1e)"
                        % (err.max(), self["ratio"], err.flat[worst], bnd.flat[worst]))
            assert np.all(err < bnd), (label, "ratio", err.flat[worst], bnd.flat[worst], worst)
            got["ratio"] = None
        text += ["%s %.1e (tol %.1e)" % (k, v, self[k]) for k, v in got.items() if v is not None]
        print("%s: " % label + " ".join(text))
        for k, v in got.items():
            if v is not None:
                assert v < self[k], (label, k, v, self[k])


def spread_tol(ref, alt):
    """max(1e-10, SPREAD_MARGIN x |alt - ref|) per metric, from two oracle
    readings of the same walk (dicts with ratios / Ainv / logabs; a missing
    key leaves that metric at the flat bar); the reference's ratios and
    terms ride along for per-proposal ratio bounds."""
    t = Tol(ratio=RTOL_RATIO, inverse=RTOL_INV, logdet=RTOL_LOGDET)
    if "ratios" in ref and "ratios" in alt:
        t["ratio"] = max(t["ratio"], SPREAD_MARGIN * rel_ratio_err(alt["ratios"], ref["ratios"]))
    if "Ainv" in ref and "Ainv" in alt:
        t["inverse"] = max(t["inverse"], SPREAD_MARGIN * rel_norm_err(alt["Ainv"], ref["Ainv"]))
    if "logabs" in ref and "logabs" in alt:
        t["logdet"] = max(t["logdet"], SPREAD_MARGIN * logdet_err(alt["logabs"], ref["logabs"]))
    if "ratios" in ref and "terms" in ref:
        t.ref_ratios, t.terms = ref["ratios"], ref["terms"]
    return t


def oracle_walk(A0, G, U, sigma, K_alt=16, override=None):
    """The oracle's Sherman-Morrison trajectory (the reference), its delayed
    reading with queue length K_alt replaying the same decisions, and the
    per-metric tolerance from their spread. Returns (ref, tol)."""
    ref = oracle.sweeps(oracle.SM, A0, G, U, sigma, override=override)
    alt = oracle.sweeps(oracle.DELAYED + oracle.ALT_INIT, A0, G, U, sigma, K=K_alt,
                        override=ref["accepted"].astype(np.int8))
    return ref, spread_tol(ref, alt)


def oracle_moves_walk(A0, elec, vrows, decisions, K, flush_after=None, K_alt=None):
    """Explicit moves through the oracle: the reading the library follows
    (delayed with K, Sherman-Morrison for K = 1), the other reading, and the
    tolerance from their spread. Returns (ref, tol)."""
    main = oracle.DELAYED if K > 1 else oracle.SM
    ref = oracle.moves(main, A0, elec, vrows, decisions, K=K, flush_after=flush_after)
    if main == oracle.DELAYED:
        alt = oracle.moves(oracle.SM + oracle.ALT_INIT, A0, elec, vrows, decisions)
    else:
        alt = oracle.moves(oracle.DELAYED + oracle.ALT_INIT, A0, elec, vrows, decisions, K=K_alt or 16,
                           flush_after=flush_after)
    return ref, spread_tol(ref, alt)


def direct_tol(A):
    """Tolerance of a direct calculation (the recompute): A^{-1} and log|det A|
    by the oracle's LU of A against the LU of A' (other pivots, other
    rounding). Returns (inverse in the library layout, (sign, logabs), tol)."""
    inv = oracle.inverse_colmajor(A)
    inv_t = np.ascontiguousarray(oracle.inverse(np.ascontiguousarray(A.T)))   # (A')^{-1} = (A^{-1})'
    s, l = oracle.slogdet(A)
    _, lt = oracle.slogdet(np.ascontiguousarray(A.T))
    tol = spread_tol(dict(Ainv=inv, logabs=l), dict(Ainv=inv_t, logabs=lt))
    return inv, (s, l), tol


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def device_draws(base_seed, nwalkers, N, sweeps):
    """The Gaussians and uniforms of the given sweeps exactly as the library
    draws them on the device (walker w's key base_seed + w):
    G [nwalkers][len(sweeps)][N][N], U [nwalkers][len(sweeps)][N]. The oracle
    is given these, so that a comparison measures the update arithmetic and
    not the last-bit difference between the device's Box-Muller (its own log
    and sincos) and numpy's, which an ill-conditioned walk amplifies; the
    uniforms are checked to equal the input generator's bit for bit."""
    from paper_1708_00744_b300.qmcdu import qmcdu_proposal_draws
    sweeps = list(sweeps)
    g = torch.empty(nwalkers, N, N, dtype=torch.float64, device="cuda")
    u = torch.empty(nwalkers, N, dtype=torch.float64, device="cuda")
    G = np.zeros((nwalkers, len(sweeps), N, N))
    U = np.zeros((nwalkers, len(sweeps), N))
    for t, s in enumerate(sweeps):
        qmcdu_proposal_draws(N, nwalkers, base_seed, s, g, u)
        G[:, t] = g.cpu().numpy()
        U[:, t] = u.cpu().numpy()
    for w in range(nwalkers):
        for t, s in enumerate(sweeps):
            assert np.array_equal(U[w, t], inputs.metropolis_uniforms(inputs.walker_seed(base_seed, w), s, N))
    return G, U


def device_gaussians(key, N, sweeps):
    """One walker's draws of the given sweeps under Philox key `key`:
    G [len(sweeps)][N][N], U [len(sweeps)][N] (see device_draws)."""
    G, U = device_draws(key, 1, N, sweeps)
    return G[0], U[0]


def walker_inputs(base_seed, batch, N, nsweeps):
    """Initial matrices (the input generator's) and the device's draws of
    sweeps 0..nsweeps-1 (per walker lists of [nsweeps][N][N] and [nsweeps][N])."""
    A = np.stack([inputs.initial_matrix(inputs.walker_seed(base_seed, b), N) for b in range(batch)])
    if not nsweeps:
        return A, [None] * batch, [None] * batch
    G, U = device_draws(base_seed, batch, N, range(nsweeps))
    return A, [G[b] for b in range(batch)], [U[b] for b in range(batch)]


def tie_override(ref_ratios, U):
    """Replay the oracle's decision only where it was a near tie."""
    p = np.minimum(1.0, ref_ratios ** 2)
    ties = np.abs(p - U) < NEAR_TIE
    ov = np.full(U.shape, -1, dtype=np.int8)
    ov[ties] = (U[ties] < p[ties]).astype(np.int8)
    return ov, int(ties.sum())


def rel_ratio_err(x, ref):
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0))) if x.size else 0.0


def rel_norm_err(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def logdet_err(x, ref):
    return abs(x - ref) / max(1.0, abs(ref))
