"""Shared helpers of the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import pytest

from paper_1708_00744_b300 import inputs

torch = pytest.importorskip("torch")

# Tolerances of the fp64 path. The bar is 1e-10; it presumes a well
# conditioned walker (N u kappa <= 1e-10). Two fp64 implementations of a
# running inverse differ by the forward error of a linear solve, about
# N u kappa_1(A) (Higham, Accuracy and Stability of Numerical Algorithms,
# Sec. 7), so the tolerance is max(1e-10, N u kappa_1(A)) for the walker's
# matrix. Errors: ratios |r - r_ref| / max(1, |r_ref|) (relative for |r| >= 1,
# absolute below, where a determinant ratio is a cancelling sum); A^{-1}
# norm-wise relative; log|det| absolute over max(1, |log|det||).
RTOL_RATIO = 1e-10
RTOL_INV = 1e-10
RTOL_LOGDET = 1e-10
NEAR_TIE = 1e-10
U64 = 2.0 ** -53


def fp64_tol(*mats):
    """max(1e-10, N u kappa_1) over the given matrices."""
    t = 1e-10
    for m in mats:
        m = np.asarray(m)
        t = max(t, m.shape[-1] * U64 * np.linalg.cond(m, 1))
    return t


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def walker_inputs(base_seed, batch, N, nsweeps):
    A = np.stack([inputs.initial_matrix(inputs.walker_seed(base_seed, b), N) for b in range(batch)])
    G = [np.stack([inputs.proposal_gaussians(inputs.walker_seed(base_seed, b), s, N)
                   for s in range(nsweeps)]).reshape(nsweeps, N, N) if nsweeps else None
         for b in range(batch)]
    U = [np.stack([inputs.metropolis_uniforms(inputs.walker_seed(base_seed, b), s, N)
                   for s in range(nsweeps)]).reshape(nsweeps, N) if nsweeps else None
         for b in range(batch)]
    return A, G, U


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
