"""Parity of the CUDA path with the CPU oracle (fp64), through the C ABI.

Every case runs the same seeded inputs through libqmcdu and through the oracle
and compares element by element: accept decisions exactly (near ties, where
|min(1, r^2) - u| < 1e-10, replay the oracle's decision and are counted),
ratios, A^{-1} and log|det A| within the fp64 tolerances of tests/gpu_common.py.
Sizes span one and several 256-element chunks with ragged tails.
"""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import inputs
from paper_1708_00744_b300.qmcdu import QmcduError, Walkers

from gpu_common import (RTOL_LOGDET, RTOL_RATIO, device_gaussians, direct_tol, logdet_err, need_gpu,
                        oracle_moves_walk, oracle_walk, rel_norm_err, rel_ratio_err, tie_override,
                        torch, walker_inputs)

pytestmark = pytest.mark.gpu


def run_sweeps(N, K, sigma, batch, nsweeps, base_seed, precision="fp64", override=None):
    W = Walkers(N, K, precision, batch)
    A, G, U = walker_inputs(base_seed, batch, N, nsweeps)
    W.set_matrix(A)
    acc = np.zeros((nsweeps, batch, N), dtype=np.uint8)
    rat = np.zeros((nsweeps, batch, N))
    ties = np.zeros((nsweeps, batch), dtype=np.int64)
    for s in range(nsweeps):
        ov = None if override is None else np.ascontiguousarray(override[s])
        W.sweep(base_seed, s, sigma, override=ov, accepted_out=acc[s], ratios_out=rat[s],
                near_ties_out=ties[s])
    Af = np.zeros((batch, N, N))
    Ai = np.zeros((batch, N, N))
    la = np.zeros(batch)
    sg = np.zeros(batch, dtype=np.int32)
    W.get_matrix(Af)
    W.get_inverse(Ai)
    W.logdet(la, sg)
    W.close()
    return dict(A0=A, G=G, U=U, acc=acc, rat=rat, ties=ties, A=Af, Ainv=Ai, logabs=la, sign=sg)


@pytest.mark.parametrize("N,K,sigma", [(1, 1, 0.5), (2, 2, 1.0), (3, 2, 0.1), (7, 3, 1.0),
                                       (64, 1, 0.1), (64, 8, 0.1), (65, 16, 1.0), (200, 1, 1.0),
                                       (257, 32, 0.1), (511, 64, 1.0), (300, 256, 0.1)])
def test_sweeps_match_oracle(N, K, sigma):
    need_gpu()
    batch, nsweeps, base = 2, 2, 100 + N
    A, G, U = walker_inputs(base, batch, N, nsweeps)
    walks = [oracle_walk(A[b], G[b], U[b], sigma, K_alt=max(2, K)) for b in range(batch)]
    refs = [w[0] for w in walks]
    override = np.full((nsweeps, batch, N), -1, dtype=np.int8)
    nties = 0
    for b in range(batch):
        ov, t = tie_override(refs[b]["ratios"], U[b])
        override[:, b, :] = ov
        nties += t
    out = run_sweeps(N, K, sigma, batch, nsweeps, base, override=override if nties else None)
    for b, (ref, tol) in enumerate(walks):
        assert np.array_equal(out["acc"][:, b, :].astype(bool), ref["accepted"]), (b, nties)
        tol.check("N=%d K=%d sigma=%g walker %d" % (N, K, sigma, b),
                  ratio=out["rat"][:, b, :],
                  inverse=rel_norm_err(out["Ainv"][b], ref["Ainv"]),
                  logdet=logdet_err(out["logabs"][b], ref["logabs"]))
        # the oracle is given the device's draws and both sides form
        # v = fl(a_j + fl(sigma g)): the rows are identical
        assert np.array_equal(out["A"][b], ref["A"])
        assert out["sign"][b] == ref["sign"]
    assert out["ties"].sum() == nties


def test_sweep_n64_matches_golden_fixture():
    """One sweep of the 64-electron walker from seed 0 (tests/golden)."""
    import json
    import os
    need_gpu()
    doc = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sweep_n64_seed0.json")))
    for case in doc["cases"]:
        out = run_sweeps(case["n"], case["K"], case["sigma"], 1, case["nsweeps"], case["seed"])
        got = "".join("1" if x else "0" for x in out["acc"][0, 0])
        assert got == case["accepted"][0]
        assert rel_ratio_err(out["rat"][0, 0], np.array(case["ratios"][0])) < RTOL_RATIO
        assert logdet_err(out["logabs"][0], case["final_logabs"]) < RTOL_LOGDET


# (700, 100): queues past 32 moves (several row units and k x k parts per walker)
# and fp64 rows of two bulk-copy segments, the second ragged (ld = 704)
@pytest.mark.parametrize("N,K,precision", [(5, 1, "fp64"), (5, 3, "fp64"), (64, 8, "fp64"),
                                           (130, 1, "fp64"), (130, 7, "fp64"), (300, 32, "fp64"),
                                           (700, 100, "fp64"), (600, 80, "fp32")])
def test_per_call_moves_match_oracle(N, K, precision):
    """qmcdu_ratio / qmcdu_accept with caller-made rows, repeated electrons
    (which force a flush) and explicit flushes. fp32 walkers are held to the
    mixed-precision bound 8 N u_w kappa_1 (u_w = 2^-24) of the walk's
    worst-conditioned matrix."""
    need_gpu()
    rng = np.random.default_rng(N * 10 + K)
    batch, nmoves = 3, 3 * N // 2 + 5
    step = 0.3
    if N > 500:
        batch, nmoves = 2, N + 5
    if precision == "fp32":
        # forced accepts of arbitrary rows drive kappa up; a short, gentle walk
        # keeps the fp32 bound meaningful
        nmoves, step = N // 4 + 5, 0.05
    A0 = np.stack([inputs.initial_matrix(7 + b, N) for b in range(batch)])
    cur = A0.copy()
    W = Walkers(N, K, precision, batch)
    W.set_matrix(A0)
    elec = rng.integers(0, N, size=(nmoves, batch))
    vrows = np.zeros((nmoves, batch, N))
    masks = (rng.random((nmoves, batch)) < 0.75).astype(np.uint8)
    flush_after = rng.random(nmoves) < 0.05
    ratios = np.zeros((nmoves, batch))
    kappa = np.array([np.linalg.cond(A0[b], 1) for b in range(batch)])
    v_dev = torch.zeros(batch, N, dtype=torch.float64, device="cuda")
    r_dev = torch.zeros(batch, dtype=torch.float64, device="cuda")
    for m in range(nmoves):
        for b in range(batch):
            vrows[m, b] = cur[b, elec[m, b]] + step * rng.standard_normal(N)
        v_dev.copy_(torch.from_numpy(vrows[m]))
        W.ratio(elec[m], v_dev, r_dev)
        ratios[m] = r_dev.cpu().numpy()
        W.accept(masks[m])
        for b in range(batch):
            if masks[m, b]:
                cur[b, elec[m, b]] = vrows[m, b]
                kappa[b] = max(kappa[b], np.linalg.cond(cur[b], 1))
        if flush_after[m]:
            W.flush()
    Af = np.zeros((batch, N, N))
    Ai = np.zeros((batch, N, N))
    la = np.zeros(batch)
    sg = np.zeros(batch, dtype=np.int32)
    W.get_matrix(Af)
    W.get_inverse(Ai)
    W.logdet(la, sg)
    W.close()
    for b in range(batch):
        ref, tol = oracle_moves_walk(A0[b], elec[:, b], vrows[:, b], masks[:, b], K,
                                     flush_after=flush_after.astype(np.uint8))
        if precision == "fp32":
            bound = 8 * N * 2.0 ** -24 * kappa[b]
            tol = type(tol)(ratio=bound, inverse=bound, logdet=bound)
        tol.check("N=%d K=%d walker %d" % (N, K, b),
                  ratio=ratios[:, b] if precision == "fp64" else rel_ratio_err(ratios[:, b], ref["ratios"]),
                  inverse=rel_norm_err(Ai[b], ref["Ainv"]), logdet=logdet_err(la[b], ref["logabs"]))
        if precision == "fp64":
            assert np.array_equal(Af[b], ref["A"])     # rows stored as given
        assert sg[b] == ref["sign"]


@pytest.mark.parametrize("N,batch,fp64_flush", [(1, 3, 0), (7, 2, 0), (64, 4, 0), (100, 1, 0), (513, 2, 0),
                                                (100, 1, 1), (513, 2, 1), (2048, 1, 0)])
def test_recompute_matches_oracle_lu(N, batch, fp64_flush):
    """Sec. III's direct calculation: A^{-1} and log|det A| from A alone. The
    rank-nb updates of fp64 handles run on the tensor cores as the flush's
    emulated-fp64 contraction (fp64_flush = 1: on the fp64 units)."""
    need_gpu()
    A = np.stack([inputs.initial_matrix(50 + b, N) for b in range(batch)])
    W = Walkers(N, 4 if N >= 4 else 1, "fp64", batch)
    W.set_option("fp64_flush", fp64_flush)
    W.set_matrix(A)
    Ai = np.zeros((batch, N, N))
    la = np.zeros(batch)
    sg = np.zeros(batch, dtype=np.int32)
    W.get_inverse(Ai)
    W.logdet(la, sg)
    W.sweep(50, 0, 0.1)
    drift = np.zeros((batch, 2))
    W.recompute(drift)
    W.close()
    for b in range(batch):
        inv, (s, l), tol = direct_tol(A[b])
        assert sg[b] == s
        tol.check("recompute N=%d walker %d" % (N, b), inverse=rel_norm_err(Ai[b], inv),
                  logdet=logdet_err(la[b], l))
        # the drift after the sweep: the running values against the LU of the
        # final matrix, held to the spread of the oracle's readings of that sweep
        seed = inputs.walker_seed(50, b)
        G, U = device_gaussians(seed, N, [0])
        wref, wtol = oracle_walk(A[b], G, U, 0.1)
        wtol.check("drift N=%d walker %d" % (N, b), inverse=drift[b, 1],
                   logdet=drift[b, 0] / max(1.0, abs(wref["logabs"])))


def test_recompute_special_matrices():
    """Closed forms: permutation (sign = parity, log|det| = 0), diagonal."""
    need_gpu()
    N = 37
    rng = np.random.default_rng(1)
    perm = rng.permutation(N)
    Pm = np.zeros((N, N))
    Pm[np.arange(N), perm] = 1.0
    inv_count = sum(1 for i in range(N) for j in range(i + 1, N) if perm[i] > perm[j])
    d = rng.uniform(0.5, 2.0, N) * rng.choice([-1.0, 1.0], N)
    A = np.stack([Pm, np.diag(d)])
    W = Walkers(N, 1, "fp64", 2)
    W.set_matrix(A)
    Ai = np.zeros((2, N, N))
    la = np.zeros(2)
    sg = np.zeros(2, dtype=np.int32)
    W.get_inverse(Ai)
    W.logdet(la, sg)
    W.close()
    assert sg[0] == (-1 if inv_count % 2 else 1) and la[0] == 0.0
    assert np.array_equal(Ai[0], Pm)                 # colmajor(P^{-1}) = (P^T)^T = P
    assert sg[1] == int(np.prod(np.sign(d))) and abs(la[1] - np.sum(np.log(np.abs(d)))) < 1e-13
    assert np.allclose(np.diag(Ai[1]), 1.0 / d, rtol=1e-15, atol=0)


def test_forced_accept_matches_oracle_forced_mode():
    """100% acceptance, the paper's test condition (Sec. III)."""
    need_gpu()
    N, K, batch = 96, 16, 1
    A, G, U = walker_inputs(9, batch, N, 1)
    ov = np.ones((1, batch, N), dtype=np.int8)
    ref, tol = oracle_walk(A[0], G[0], U[0], 0.1, override=ov[:, 0])
    out = run_sweeps(N, K, 0.1, batch, 1, 9, override=ov)
    assert out["acc"].all()
    tol.check("forced accept", ratio=out["rat"][:, 0],
              inverse=rel_norm_err(out["Ainv"][0], ref["Ainv"]))


def test_error_paths():
    need_gpu()
    N = 8
    W = Walkers(N, 4, "fp64", 1)
    W.set_matrix(np.eye(N)[None])
    with pytest.raises(QmcduError) as e:
        W.accept(np.ones(1, dtype=np.uint8))         # no pending ratio
    assert e.value.status == 2
    v = torch.zeros(1, N, dtype=torch.float64, device="cuda")
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(QmcduError) as e:
        W.ratio(np.array([N]), v, r)                  # electron out of range
    assert e.value.status == 1
    W.ratio(np.array([3]), v, r)                      # v = 0: r = 0
    assert r.item() == 0.0
    W.accept(np.ones(1, dtype=np.uint8))              # accepting r = 0 is singular
    with pytest.raises(QmcduError) as e:
        W.sync()
    assert e.value.status == 3
    W.set_matrix(np.eye(N)[None])                     # reload clears the latch
    W.sync()
    with pytest.raises(QmcduError) as e:
        W.set_matrix(np.zeros((1, N, N)))             # singular matrix
        W.sync()
    assert e.value.status == 3
    W.close()


_N2048 = {}


def _walk_n2048(A, G, U, sigma):
    key = sigma
    if key not in _N2048:
        _N2048[key] = oracle_walk(A[0], G[0], U[0], sigma, K_alt=32)
    return _N2048[key]


@pytest.mark.parametrize("K", [1, 64])
def test_full_size_sweep_n2048(K):
    """The benchmark's walker (N = 2048, sigma = 0.1, fp64): one full sweep
    compared with the oracle's Sherman-Morrison trajectory."""
    need_gpu()
    N, sigma, base = 2048, 0.1, 0
    A, G, U = walker_inputs(base, 1, N, 1)
    ref, tol = _walk_n2048(A, G, U, sigma)
    ov, nties = tie_override(ref["ratios"], U[0])
    out = run_sweeps(N, K, sigma, 1, 1, base, override=ov[:, None, :] if nties else None)
    assert np.array_equal(out["acc"][:, 0].astype(bool), ref["accepted"])
    tol.check("N=2048 K=%d ties %d" % (K, nties), ratio=out["rat"][:, 0],
              inverse=rel_norm_err(out["Ainv"][0], ref["Ainv"]),
              logdet=logdet_err(out["logabs"][0], ref["logabs"]))


@pytest.mark.parametrize("fp64_flush", [0, 1])
def test_recompute_of_a_badly_scaled_matrix(fp64_flush):
    """A = D1 G D2 with rows and columns scaled over 2^-30 .. 2^30: the
    recompute equilibrates A by powers of two before the elimination, so that
    the tensor-core update (fp64_flush = 0) and the fp64 units agree with the
    oracle's LU within the LU-of-A against LU-of-A' spread."""
    need_gpu()
    N = 300
    rng = np.random.default_rng(5)
    d1, d2 = 2.0 ** rng.uniform(-30, 30, N), 2.0 ** rng.uniform(-30, 30, N)
    A = d1[:, None] * inputs.initial_matrix(77, N) * d2[None, :]
    W = Walkers(N, 16, "fp64", 1)
    W.set_option("fp64_flush", fp64_flush)
    W.set_matrix(A[None])
    Ai = np.zeros((1, N, N))
    la = np.zeros(1)
    sg = np.zeros(1, dtype=np.int32)
    W.get_inverse(Ai)
    W.logdet(la, sg)
    W.close()
    inv, (s, l), tol = direct_tol(A)
    assert sg[0] == s
    # column by column, relative to each column's largest entry (the scalings
    # make a norm-wise check blind to the small columns), against the same
    # measure of the oracle's two LUs (of A and of A')
    inv_t = np.ascontiguousarray(oracle.inverse(np.ascontiguousarray(A.T)))

    def colerr(x, ref):
        return float(np.max(np.max(np.abs(x - ref), axis=1) / np.max(np.abs(ref), axis=1)))

    bar = max(1e-10, 10.0 * colerr(inv_t, inv))
    err = colerr(Ai[0], inv)
    print("recompute of D1 G D2 (fp64_flush %d): column-wise %.1e (tol %.1e), logdet %.1e (tol %.1e)"
          % (fp64_flush, err, bar, logdet_err(la[0], l), tol["logdet"]))
    assert err < bar
    assert logdet_err(la[0], l) < tol["logdet"]
