"""Multideterminant walkers (qmcdu_md_*): the delayed update combined with the
table method, Psi = sum_I c_I det(A_I) with single and double excitations,
against the oracle's reading of the same method (the table with the
reference inverse under the delayed update) within the spread of its second
reading (the table with Sherman-Morrison updates); the oracle's pins tie
both to the definition (every det(A_I))."""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import inputs
from paper_1708_00744_b300.qmcdu import MultiDetWalkers, QmcduError, Walkers

from gpu_common import logdet_err, need_gpu, rel_ratio_err, spread_tol, torch

pytestmark = pytest.mark.gpu


def _expansion(rng, N, nv, nsingle, ndouble):
    exc = [(-1, -1, -1, -1)]
    for _ in range(nsingle):
        exc.append((int(rng.integers(N)), int(rng.integers(nv)), -1, -1))
    for _ in range(ndouble):
        o = rng.choice(N, 2, replace=False)
        a = rng.choice(nv, 2, replace=False)
        exc.append((int(o[0]), int(a[0]), int(o[1]), int(a[1])))
    coef = 0.3 * rng.standard_normal(len(exc))
    coef[0] = 1.0
    return np.array(exc, dtype=np.int32), coef


@pytest.mark.parametrize("N,K,nv,sigma,nsweeps", [(128, 8, 12, 0.3, 2), (96, 1, 6, 0.5, 1), (200, 32, 16, 0.2, 1),
                                                   (256, 32, 16, 0.2, 1)])
def test_multideterminant_walk_matches_oracle(N, K, nv, sigma, nsweeps):
    need_gpu()
    rng = np.random.default_rng(N + K + nv)
    A0 = inputs.initial_matrix(600 + N, N)
    B0 = rng.standard_normal((N, nv))
    exc, coef = _expansion(rng, N, nv, 14, 10)
    G = rng.standard_normal((nsweeps, N, N))
    H = rng.standard_normal((nsweeps, N, nv))
    U = rng.random((nsweeps, N))
    # the reading the library follows (the table with the reference inverse
    # under the delayed update, queue length K) and the table with
    # Sherman-Morrison updates replaying its decisions: near a singular
    # reference determinant (the N = 200 walk starts at kappa_1 = 6e6) the
    # two differ by far more than 1e-10, as the single-determinant readings do
    ref = oracle.md_sweeps(oracle.MD_TABLE_DELAYED, A0, B0, G, H, U, sigma, exc, coef, K=K)
    alt = oracle.md_sweeps(oracle.MD_TABLE, A0, B0, G, H, U, sigma, exc, coef,
                           override=ref["accepted"].astype(np.int8))
    tol = spread_tol(ref, alt)
    assert 0.2 < ref["accepted"].mean() < 0.98
    W = Walkers(N, K, "fp64", 1)
    W.set_matrix(A0[None])
    md = MultiDetWalkers(W, nv, exc, coef)
    md.set_virtuals(B0[None])
    cur_A, cur_B = A0.copy(), B0.copy()
    v_d = torch.zeros(1, N, dtype=torch.float64, device="cuda")
    w_d = torch.zeros(1, nv, dtype=torch.float64, device="cuda")
    R_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    r_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    R = np.zeros((nsweeps, N))
    for s in range(nsweeps):
        for j in range(N):
            v = cur_A[j] + sigma * G[s, j]
            w = cur_B[j] + sigma * H[s, j]
            v_d.copy_(torch.from_numpy(v[None]))
            w_d.copy_(torch.from_numpy(w[None]))
            md.ratio(np.array([j]), v_d, w_d, R_d, r_d)
            R[s, j] = R_d.item()
            a = bool(ref["accepted"][s, j])           # the oracle's decision (near ties checked below)
            md.accept(np.array([a], dtype=np.uint8))
            if a:
                cur_A[j], cur_B[j] = v, w
    la = np.zeros(1)
    sg = np.zeros(1, dtype=np.int32)
    md.logpsi(la, sg)
    md.close()
    W.close()
    # decisions from the device's ratios: the oracle's except within the
    # ratio error of a tie
    e = rel_ratio_err(R, ref["ratios"])
    p, pg = np.minimum(1.0, ref["ratios"] ** 2), np.minimum(1.0, R ** 2)
    far = np.abs(p - U) > 2 * e + 1e-12
    assert np.array_equal((U < pg)[far], ref["accepted"][far])
    label = "multideterminant N=%d K=%d nv=%d ndet=%d" % (N, K, nv, len(coef))
    tol.check(label, ratio=e, logdet=logdet_err(la[0], ref["logabs"]))
    assert sg[0] == ref["sign"]


def test_multideterminant_errors():
    need_gpu()
    W = Walkers(16, 4, "fp64", 1)
    W.set_matrix(np.eye(16)[None])
    with pytest.raises(QmcduError) as e:
        MultiDetWalkers(W, 4, [(0, 4, -1, -1)], [1.0])          # virtual index out of range
    assert e.value.status == 1
    md = MultiDetWalkers(W, 4, [(-1, -1, -1, -1), (0, 1, -1, -1)], [1.0, 0.5])
    v = torch.zeros(1, 16, dtype=torch.float64, device="cuda")
    w = torch.zeros(1, 4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(QmcduError) as e:
        md.ratio(np.array([0]), v, w, out)                      # before set_virtuals
    assert e.value.status == 2
    with pytest.raises(QmcduError) as e:
        md.accept(np.array([1], dtype=np.uint8))                # no pending ratio
    assert e.value.status == 2
    md.close()
    W.close()
    W32 = Walkers(16, 4, "fp32", 1)
    with pytest.raises(QmcduError) as e:
        MultiDetWalkers(W32, 4, [(-1, -1, -1, -1)], [1.0])      # fp64 handles only
    assert e.value.status == 1
    W32.close()
