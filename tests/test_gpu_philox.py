"""Philox4x32-10: the library's device generator, the numpy input generator
and cuRAND's implementation agree bit for bit (Salmon et al., SC'11)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1708_00744_b300 import inputs
from paper_1708_00744_b300.qmcdu import qmcdu_philox4x32_10

from gpu_common import need_gpu, torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _counters(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, 2**32, size=(4, n), dtype=np.uint64)
    c[:, :4] = [[0, 0xFFFFFFFF, 1, 7], [0, 0xFFFFFFFF, 0, 3], [0, 0xFFFFFFFF, 0, 2], [0, 0xFFFFFFFF, 0, 5]]
    return c


def test_library_philox_matches_numpy_generator():
    need_gpu()
    n = 1 << 20
    c = _counters(n, 3)
    seed = (0x12345678 << 32) | 0x9ABCDEF0
    dev = [torch.from_numpy(c[w].astype(np.uint32).view(np.int32)).cuda() for w in range(4)]
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    qmcdu_philox4x32_10(*dev, seed, out)
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    ref = np.stack(inputs.philox4x32_10(c[0], c[1], c[2], c[3], seed), axis=1)
    assert np.array_equal(got, ref)


def test_library_philox_matches_curand():
    need_gpu()
    src = os.path.join(HERE, "philox_curand_ref.cu")
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "libphilox_ref.so")
        subprocess.check_call(["nvcc", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-Xcompiler", "-fPIC", "-shared", "-o", so, src])
        lib = ctypes.CDLL(so)
        n = 1 << 16
        c = _counters(n, 5)
        seed = 0xDEADBEEF00C0FFEE
        ctr = torch.from_numpy(np.ascontiguousarray(c.T.astype(np.uint32)).view(np.int32)).cuda()
        ref = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
        assert lib.curand_philox_ref(ctypes.c_void_p(ctr.data_ptr()), ctypes.c_uint(seed & 0xFFFFFFFF),
                                     ctypes.c_uint(seed >> 32), ctypes.c_void_p(ref.data_ptr()),
                                     ctypes.c_int(n)) == 0
        dev = [torch.from_numpy(c[w].astype(np.uint32).view(np.int32)).cuda() for w in range(4)]
        out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
        qmcdu_philox4x32_10(*dev, seed, out)
        assert torch.equal(out.view(n, 4), ref)
        npref = np.stack(inputs.philox4x32_10(c[0], c[1], c[2], c[3], seed), axis=1)
        assert np.array_equal(ref.cpu().numpy().view(np.uint32), npref)


@pytest.mark.parametrize("N,nw,seed,sweep", [(7, 3, 5, 0), (512, 2, 1000, 3), (2048, 1, 0, 1)])
def test_sweep_draws_match_the_input_generator(N, nw, seed, sweep):
    """qmcdu_proposal_draws (the sweep's own draw kernel): uniforms bit for bit
    (53 bits of two Philox words), Gaussians to rounding (Box-Muller with the
    device's log, sqrt and sincos against numpy's)."""
    need_gpu()
    from paper_1708_00744_b300.qmcdu import qmcdu_proposal_draws
    g = torch.zeros(nw, N, N, dtype=torch.float64, device="cuda")
    u = torch.zeros(nw, N, dtype=torch.float64, device="cuda")
    qmcdu_proposal_draws(N, nw, seed, sweep, g, u)
    torch.cuda.synchronize()
    for w in range(nw):
        key = inputs.walker_seed(seed, w)
        assert np.array_equal(u[w].cpu().numpy(), inputs.metropolis_uniforms(key, sweep, N))
        ref = inputs.proposal_gaussians(key, sweep, N)
        assert np.max(np.abs(g[w].cpu().numpy() - ref)) <= 4e-15 * np.max(np.abs(ref))
