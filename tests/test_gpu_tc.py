"""The tensor-core contraction of the fp32 flush (split-bf16 x3 on tcgen05)
against an fp64 product: C = alpha A B' + beta C, ragged sizes, both layouts
of B. Error bound: each operand is represented to 2^-16 relative (hi + lo of
bf16) and the dropped lo*lo term is ~2^-16 of the product, so
|C - C_ref| <= 4 * 2^-16 * (|A| |B|')_ij + fp32 accumulation."""
import numpy as np
import pytest

from paper_1708_00744_b300.qmcdu import qmcdu_gemm_bf16x3

from gpu_common import need_gpu, torch

pytestmark = pytest.mark.gpu


def _check(M, N, K, b_trans=False, alpha=1.0, beta=0.0, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N) if b_trans else (N, K)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    Bn = B.T if b_trans else B
    ref = alpha * (A.astype(np.float64) @ Bn.astype(np.float64).T) + beta * C0.astype(np.float64)
    scale = np.abs(A.astype(np.float64)) @ np.abs(Bn.astype(np.float64)).T
    Ad, Bd, Cd = (torch.from_numpy(x).cuda() for x in (A, B, C0))
    qmcdu_gemm_bf16x3(Ad, Bd, Cd, alpha=alpha, beta=beta, b_trans=b_trans)
    torch.cuda.synchronize()
    C = Cd.cpu().numpy().astype(np.float64)
    err = np.abs(C - ref)
    bound = 4 * 2.0 ** -16 * abs(alpha) * scale + 2.0 ** -22 * (np.abs(ref) + 1)
    assert np.all(err <= bound), float(np.max(err / bound))
    return float(np.max(err / np.maximum(scale, 1e-30)))


@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (130, 72, 50), (256, 256, 512), (1, 1, 1),
                                   (300, 200, 1000), (128, 16, 2048), (513, 257, 64)])
def test_gemm_bf16x3_matches_fp64(M, N, K):
    need_gpu()
    rel = _check(M, N, K, seed=M + N + K)
    # a single bf16 product would be ~2^-9 off: the hi*lo terms are in
    assert rel < 2.0 ** -13


@pytest.mark.parametrize("M,N,K", [(200, 300, 64), (128, 256, 16)])
def test_gemm_bf16x3_transposed_b_and_beta(M, N, K):
    need_gpu()
    _check(M, N, K, b_trans=True, alpha=-1.0, beta=1.0, seed=7)


def test_gemm_bf16x3_empty_k():
    need_gpu()
    _check(64, 48, 0, alpha=1.0, beta=0.5)
