"""qmcdu_ratio_noalloc: the ratio entry point for callers that cannot
allocate device memory (because cudaMalloc may synchronise the device, or
because another allocator owns the device's memory). It must give what the
handle's qmcdu_ratio gives for the same walker and queue, call after call,
while using only the library's fixed scratch array.

Collected last (file name) so that a run stopping at the first failure has
already run every other test; it also passes when run alone in a fresh
process, where its first call performs the per-device set-up."""
import numpy as np
import pytest

from paper_1708_00744_b300 import inputs
from paper_1708_00744_b300.qmcdu import Walkers, load, qmcdu_ratio_noalloc

from gpu_common import need_gpu, torch

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the fp64 bar of the parity tests, on |r - r_ref| / max(1, |r_ref|)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("N,K", [(300, 16), (1000, 64)])
def test_noalloc_ratio_matches_handle_ratio_twice(N, K):
    need_gpu()
    rng = np.random.default_rng(N + K)
    A0 = inputs.initial_matrix(11, N)
    W = Walkers(N, K, "fp64", 1)
    W.set_matrix(A0[None])
    Ainv0 = np.zeros((1, N, N))
    W.get_inverse(Ainv0)                  # row c = column c of A^{-1} (no queue yet)
    Ainv0 = Ainv0[0]
    # queue k accepted moves of distinct electrons through the handle
    k = min(K - 1, 7)
    idx = rng.choice(N, size=k + 2, replace=False)
    queued, props = idx[:k], idx[k:]
    vq = np.stack([A0[j] + 0.2 * rng.standard_normal(N) for j in queued])
    r_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for j, vrow in zip(queued, vq):
        W.ratio(np.array([j]), _cuda(vrow[None]), r_dev)
        W.accept(np.ones(1, dtype=np.uint8))
    P = Ainv0[queued]                     # rows: columns idx_m of A^{-1} at the last flush
    Kinv = np.linalg.inv(vq @ P.T)        # (V P')^{-1}
    P_d, V_d, K_d = _cuda(P), _cuda(vq), _cuda(Kinv)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for j in props:                       # two calls in a row, different proposals
        v = A0[j] + 0.2 * rng.standard_normal(N)
        v_d = _cuda(v[None])
        W.ratio(np.array([j]), v_d, r_dev)            # the handle's entry point
        W.accept(np.zeros(1, dtype=np.uint8))         # reject: the queue stays as it is
        qmcdu_ratio_noalloc(N, k, _cuda(Ainv0[j]), v_d, P_d, V_d, K_d, out)
        torch.cuda.synchronize()
        ref, got = r_dev.item(), out.item()
        assert abs(got - ref) / max(1.0, abs(ref)) < TOL, (j, got, ref)
    W.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Checked in the C entry point itself, before any launch."""
    need_gpu()
    lib = load()
    p = torch.zeros(16, dtype=torch.float64, device="cuda").data_ptr()
    assert lib.qmcdu_ratio_noalloc(8193, 0, p, p, None, None, None, p, None) == 1
    assert b"8192" in lib.qmcdu_last_error(None)
    assert lib.qmcdu_ratio_noalloc(4, 5, p, p, p, p, p, p, None) == 1
    assert lib.qmcdu_ratio_noalloc(64, 300, p, p, p, p, p, p, None) == 1
