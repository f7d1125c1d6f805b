"""qmcdu_ratio_noalloc: the ratio entry point for callers that cannot
allocate device memory (because cudaMalloc may synchronise the device, or
because another allocator owns the device's memory). It must give what the
handle's qmcdu_ratio gives for the same walker and queue, call after call,
and what the oracle gives, while using only the library's fixed scratch array:
the device's free memory is the same before and after a run of calls.

Collected last (file name) so that a run stopping at the first failure has
already run every other test; it also passes when run alone in a fresh
process, where its first call performs the per-device set-up."""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import inputs
from paper_1708_00744_b300.qmcdu import Walkers, load, qmcdu_ratio_noalloc

from gpu_common import need_gpu, torch

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the fp64 bar of the parity tests, on |r - r_ref| / max(1, |r_ref|)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _err(got, ref):
    return abs(got - ref) / max(1.0, abs(ref))


def _queue(A0, Ainv_cm, queued, vq):
    """The caller-held queue in the change form: P rows = columns idx_m of
    A^{-1}, V rows = the changes u_m = v_m - a_idx_m, Kinv = (I + V P')^{-1}."""
    P = Ainv_cm[queued]
    V = vq - A0[queued]
    Kinv = np.linalg.inv(np.eye(len(queued)) + V @ P.T) if len(queued) else np.zeros((0, 0))
    return P, V, Kinv


def _noalloc(N, k, a, u, P, V, Kinv):
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    args = (_cuda(P), _cuda(V), _cuda(Kinv)) if k else (None, None, None)
    qmcdu_ratio_noalloc(N, k, _cuda(a), _cuda(u), *args, out)
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("N,K,k", [(300, 16, 7), (1000, 64, 40), (64, 8, 0)])
def test_noalloc_ratio_matches_handle_ratio_twice(N, K, k):
    need_gpu()
    rng = np.random.default_rng(N + K)
    A0 = inputs.initial_matrix(11, N)
    W = Walkers(N, K, "fp64", 1)
    W.set_matrix(A0[None])
    Ainv0 = np.zeros((1, N, N))
    W.get_inverse(Ainv0)                  # row c = column c of A^{-1} (no queue yet)
    Ainv0 = Ainv0[0]
    # queue k accepted moves of distinct electrons through the handle
    idx = rng.choice(N, size=k + 2, replace=False)
    queued, props = idx[:k], idx[k:]
    vq = np.stack([A0[j] + 0.2 * rng.standard_normal(N) for j in queued]) if k else np.zeros((0, N))
    r_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for j, vrow in zip(queued, vq):
        W.ratio(np.array([j]), _cuda(vrow[None]), r_dev)
        W.accept(np.ones(1, dtype=np.uint8))
    P, V, Kinv = _queue(A0, Ainv0, queued, vq)
    for j in props:                       # two calls in a row, different proposals
        v = A0[j] + 0.2 * rng.standard_normal(N)
        W.ratio(np.array([j]), _cuda(v[None]), r_dev)      # the handle's entry point
        W.accept(np.zeros(1, dtype=np.uint8))              # reject: the queue stays as it is
        got, ref = _noalloc(N, k, Ainv0[j], v - A0[j], P, V, Kinv), r_dev.item()
        assert _err(got, ref) < TOL, (j, got, ref)
    W.close()


@pytest.mark.parametrize("N,K,k", [(80, 8, 0), (300, 256, 255)])
def test_noalloc_ratio_matches_oracle(N, K, k):
    """k = 0 (null queue pointers) and a queue one short of the 256 limit,
    against oracle.moves (the delayed reading: look-ahead determinants of
    Eq. 3) with the queued moves accepted and the proposals rejected."""
    need_gpu()
    rng = np.random.default_rng(3 * N + k)
    A0 = inputs.initial_matrix(21, N)
    Ainv0 = oracle.inverse_colmajor(A0)
    idx = rng.choice(N, size=k + 2, replace=False)
    queued, props = idx[:k], idx[k:]
    vq = np.stack([A0[j] + 0.1 * rng.standard_normal(N) for j in queued]) if k else np.zeros((0, N))
    P, V, Kinv = _queue(A0, Ainv0, queued, vq)
    for j in props:
        v = A0[j] + 0.1 * rng.standard_normal(N)
        ref = oracle.moves(oracle.DELAYED, A0, np.concatenate([queued, [j]]), np.vstack([vq, v]),
                           np.concatenate([np.ones(k, np.uint8), [0]]), K=K)["ratios"][-1]
        got = _noalloc(N, k, Ainv0[j], v - A0[j], P, V, Kinv)
        assert _err(got, ref) < TOL, (N, k, j, got, ref)


def test_noalloc_at_its_limits_n8192_k256():
    """N = 8192 and k = 256 fill the 32 x 513 partial sums and the shared
    buffers. A0 = diag(d) has the closed-form inverse diag(1/d); the reference
    ratio is the generalised determinant lemma (Eq. 3) taken directly: the
    ratio of det(I + [V; u] D^{-1} [E, e_j]) over det(I + V D^{-1} E), two
    small determinants by LU, a different route from the kernel's Schur
    complement through Kinv."""
    need_gpu()
    N, k = 8192, 256
    rng = np.random.default_rng(8192)
    d = rng.uniform(0.5, 2.0, N)
    Ainv_cm_rows = lambda rows: np.stack([np.eye(1, N, r)[0] / d[r] for r in rows])
    idx = rng.choice(N, size=k + 2, replace=False)
    queued, props = idx[:k], idx[k:]
    V = 0.3 * rng.standard_normal((k, N))          # changes of the queued rows
    P = Ainv_cm_rows(queued)                       # columns idx_m of D^{-1}
    Kinv = np.linalg.inv(np.eye(k) + V @ P.T)
    for j in props:
        u = 0.3 * rng.standard_normal(N)
        cols = np.concatenate([queued, [j]])
        S = np.eye(k + 1) + np.vstack([V, u])[:, cols] / d[cols][None, :]
        s1, l1 = np.linalg.slogdet(S)
        s0, l0 = np.linalg.slogdet(S[:k, :k])
        ref = s1 * s0 * np.exp(l1 - l0)
        got = _noalloc(N, k, np.eye(1, N, j)[0] / d[j], u, P, V, Kinv)
        assert _err(got, ref) < TOL, (j, got, ref)


def test_noalloc_allocates_nothing():
    """After the first call on the device (module load and the scratch
    address look-up, which may allocate), further calls leave the device's
    free memory unchanged."""
    need_gpu()
    N, k = 512, 32
    rng = np.random.default_rng(5)
    a, u = _cuda(rng.standard_normal(N)), _cuda(rng.standard_normal(N))
    P, V = _cuda(rng.standard_normal((k, N))), _cuda(rng.standard_normal((k, N)))
    Kinv = _cuda(np.eye(k))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    qmcdu_ratio_noalloc(N, k, a, u, P, V, Kinv, out, stream=stream)   # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    vals = []
    for _ in range(20):
        qmcdu_ratio_noalloc(N, k, a, u, P, V, Kinv, out, stream=stream)
        torch.cuda.synchronize()
        vals.append(out.item())
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert len(set(vals)) == 1            # the shared scratch is reset by every call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Checked in the C entry point itself, before any launch."""
    need_gpu()
    lib = load()
    p = torch.zeros(16, dtype=torch.float64, device="cuda").data_ptr()
    assert lib.qmcdu_ratio_noalloc(8193, 0, p, p, None, None, None, p, None) == 1
    assert b"8192" in lib.qmcdu_last_error(None)
    assert lib.qmcdu_ratio_noalloc(4, 5, p, p, p, p, p, p, None) == 1
    assert lib.qmcdu_ratio_noalloc(64, 300, p, p, p, p, p, p, None) == 1
