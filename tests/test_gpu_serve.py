"""Walker subsets and the serving loop on the GPU: qmcdu_load_walkers draws
the same matrices as the input generator; qmcdu_sweep_walkers advances listed
walkers, each with its own key and sweep number, along the oracle's
trajectory; qmcdu_recompute_walkers leaves the other walkers alone; a request
served by qmcdu_server_* follows the oracle's trajectory, and its results are
bit-identical alone and in a mix of walkers of other sizes that join and
leave around it."""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import inputs
from paper_1708_00744_b300.qmcdu import Server, Walkers

from gpu_common import (device_gaussians, direct_tol, logdet_err, need_gpu, oracle_walk, rel_norm_err,
                        rel_ratio_err, spread_tol, torch)

pytestmark = pytest.mark.gpu


def _oracle_run(seed, N, nsweeps, sigma, K):
    A0 = inputs.initial_matrix(seed, N)
    G, U = device_gaussians(seed, N, range(nsweeps))
    ref = oracle.sweeps(oracle.DELAYED, A0, G, U, sigma, K=K)
    alt = oracle.sweeps(oracle.SM + oracle.ALT_INIT, A0, G, U, sigma, override=ref["accepted"].astype(np.int8))
    return A0, U, ref, spread_tol(ref, alt)


def _tie_free(ref, U):
    p = np.minimum(1.0, ref["ratios"] ** 2)
    return int((np.abs(p - U) < 1e-10).sum()) == 0


def test_load_walkers_draws_the_initial_matrices():
    need_gpu()
    N, seeds = 77, [5, 900, 2**40 + 3]
    W = Walkers(N, 8, "fp64", 4)
    W.load_walkers(1, 3, seeds=seeds)
    A = np.zeros((4, N, N))
    W.get_matrix(A)
    la = np.zeros(4)
    sg = np.zeros(4, dtype=np.int32)
    W.logdet(la, sg)
    W.close()
    for t, s in enumerate(seeds):
        ref = inputs.initial_matrix(s, N)
        # Box-Muller through the device's log/sincos vs numpy's: rounding only
        assert np.max(np.abs(A[1 + t] - ref)) <= 1e-14 * np.max(np.abs(ref))
        _, (rs, rl), tol = direct_tol(ref)
        assert sg[1 + t] == rs
        tol.check("initial matrix %d" % t, logdet=logdet_err(la[1 + t], rl))
    assert not A[0].any()                     # walker 0 untouched


@pytest.mark.parametrize("N,K", [(96, 8), (200, 32)])
def test_sweep_walkers_follow_the_oracle(N, K):
    """Walkers 3 and 0 of a handle of four, with their own keys and sweep
    numbers, in two listed sweeps; walkers 1 and 2 are never touched."""
    need_gpu()
    sigma = 0.3
    seeds = {3: 4242, 0: 77}
    W = Walkers(N, K, "fp64", 4)
    W.load_walkers(0, 1, seeds=[seeds[0]])
    W.load_walkers(3, 1, seeds=[seeds[3]])
    Ab = np.zeros((4, N, N))
    W.get_matrix(Ab)
    la0 = np.zeros(4)
    sg0 = np.zeros(4, dtype=np.int32)
    W.logdet(la0, sg0)
    acc = np.zeros((2, 2, N), dtype=np.uint8)
    rat = np.zeros((2, 2, N))
    ties = np.zeros((2, 2), dtype=np.int64)
    for s in range(2):
        # walker 3 runs its sweeps 0 and 1; walker 0 its sweeps 5 and 6
        W.sweep_walkers([3, 0], [seeds[3], seeds[0]], [s, 5 + s], sigma,
                        accepted_out=acc[s], ratios_out=rat[s], near_ties_out=ties[s])
    Af = np.zeros((4, N, N))
    W.get_matrix(Af)
    Ai = np.zeros((4, N, N))
    W.get_inverse(Ai)
    la = np.zeros(4)
    sg = np.zeros(4, dtype=np.int32)
    W.logdet(la, sg)
    W.close()
    assert np.array_equal(Af[1:3], Ab[1:3]) and np.array_equal(la[1:3], la0[1:3])
    for t, (w, first) in enumerate(((3, 0), (0, 5))):
        seed = seeds[w]
        A0 = inputs.initial_matrix(seed, N)
        G, U = device_gaussians(seed, N, [first, first + 1])
        ref = oracle.sweeps(oracle.DELAYED, A0, G, U, sigma, K=K)
        alt = oracle.sweeps(oracle.SM + oracle.ALT_INIT, A0, G, U, sigma, override=ref["accepted"].astype(np.int8))
        tol = spread_tol(ref, alt)
        assert _tie_free(ref, U)
        assert np.array_equal(acc[:, t].astype(bool), ref["accepted"])
        tol.check("walker %d" % w, ratio=rat[:, t],
                  inverse=rel_norm_err(Ai[w], ref["Ainv"]), logdet=logdet_err(la[w], ref["logabs"]))
        assert sg[w] == ref["sign"]
        assert ties[:, t].sum() == 0


def test_recompute_walkers_leaves_the_others_alone():
    need_gpu()
    N, K = 128, 16
    W = Walkers(N, K, "fp64", 5)
    W.load_walkers(0, 5, seeds=[10, 11, 12, 13, 14])
    for s in range(2):
        W.sweep_walkers([0, 1, 2, 3, 4], [10, 11, 12, 13, 14], [s] * 5, 0.2)
    Ai0 = np.zeros((5, N, N))
    W.get_inverse(Ai0)
    drift = np.zeros((2, 2))
    W.recompute_walkers(2, 2, drift)
    Ai1 = np.zeros((5, N, N))
    W.get_inverse(Ai1)
    A = np.zeros((5, N, N))
    W.get_matrix(A)
    la = np.zeros(5)
    sg = np.zeros(5, dtype=np.int32)
    W.logdet(la, sg)
    W.close()
    for w in (0, 1, 4):
        assert np.array_equal(Ai1[w], Ai0[w])
    for t, w in enumerate((2, 3)):
        seed = 10 + w
        G, U = device_gaussians(seed, N, range(2))
        wref, wtol = oracle_walk(inputs.initial_matrix(seed, N), G, U, 0.2, K_alt=K)
        wtol.check("drift walker %d" % w, inverse=drift[t, 1],
                   logdet=drift[t, 0] / max(1.0, abs(wref["logabs"])))
        inv, (rs, rl), tol = direct_tol(A[w])
        assert sg[w] == rs
        tol.check("recompute walker %d" % w, logdet=logdet_err(la[w], rl),
                  inverse=rel_norm_err(Ai1[w], inv))


def test_sweep_walkers_rejects_bad_lists():
    need_gpu()
    from paper_1708_00744_b300.qmcdu import QmcduError
    W = Walkers(32, 4, "fp64", 3)
    W.load_walkers(0, 3, seeds=[1, 2, 3])
    for walkers, sweeps in (([0, 0], [0, 0]), ([3], [0]), ([1], [-1])):
        with pytest.raises(QmcduError) as e:
            W.sweep_walkers(walkers, [1] * len(walkers), sweeps, 0.1)
        assert e.value.status == 1
    with pytest.raises(QmcduError):
        W.load_walkers(2, 2, seeds=[1, 2])
    W.close()


def _classes(precision):
    # group shape per class from the server's default rule (N / 128 CTAs, at least 1)
    return [dict(N=64, slots=3), dict(N=128, slots=2), dict(N=256, slots=2)]


def test_served_request_follows_the_oracle():
    need_gpu()
    sigma, nsweeps = 0.3, 3
    reqs = [dict(id=i, seed=3000 + i, N=(64, 128, 256)[i % 3], nsweeps=nsweeps,
                 arrival_s=0.0005 * i) for i in range(6)]
    srv = Server(_classes("fp64"), precision="fp64", sigma=sigma, recompute_every=2,
                 keep_traces=True, hbm_budget=4 * 10**9)
    srv.submit(reqs)
    srv.run()
    res = {r["id"]: r for r in srv.results()}
    assert len(res) == len(reqs)
    for q in reqs:
        r = res[q["id"]]
        assert r["status"] == 0 and r["recomputes"] == 2
        acc, rat = srv.trace(q["id"], nsweeps, q["N"])
        K = min(q["N"], 32)
        A0, U, ref, tol = _oracle_run(q["seed"], q["N"], nsweeps, sigma, K)
        assert _tie_free(ref, U)
        assert np.array_equal(acc.astype(bool), ref["accepted"])
        assert r["accepted"] == int(ref["accepted"].sum())
        assert r["sign"] == ref["sign"]
        tol.check("request %d" % q["id"], ratio=rat,
                  logdet=logdet_err(r["logabs"], ref["logabs"]))
        tol.check("request %d drift" % q["id"], inverse=r["drift_inverse"],
                  logdet=r["drift_logdet"] / max(1.0, abs(ref["logabs"])))
    srv.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_served_results_are_identical_alone_and_in_the_mix(precision):
    need_gpu()
    sigma, nsweeps = 0.2, 4
    rng = np.random.default_rng(17)
    reqs = [dict(id=i, seed=7000 + i, N=int(rng.choice([64, 128, 256])), nsweeps=nsweeps,
                 arrival_s=0.0004 * i) for i in range(14)]
    kw = dict(precision=precision, sigma=sigma, recompute_every=3, keep_traces=True,
              hbm_budget=4 * 10**9)
    srv = Server(_classes(precision), **kw)
    srv.submit(reqs)
    srv.run()
    mix = {r["id"]: r for r in srv.results()}
    st = srv.stats()
    traces = {q["id"]: srv.trace(q["id"], nsweeps, q["N"]) for q in reqs}
    srv.close()
    assert st["finished"] == len(reqs)
    assert st["mixed_walker_sweeps"] > 0          # walkers did join running pools
    for q in reqs[:6]:
        alone = Server(_classes(precision), **kw)
        alone.submit([dict(q, arrival_s=0.0)])
        alone.run()
        r = alone.results()[0]
        acc, rat = alone.trace(q["id"], nsweeps, q["N"])
        alone.close()
        m = mix[q["id"]]
        assert np.array_equal(acc, traces[q["id"]][0])
        assert np.array_equal(rat, traces[q["id"]][1])
        assert r["logabs"] == m["logabs"] and r["sign"] == m["sign"]
        assert r["accepted"] == m["accepted"]


def test_server_under_a_tight_budget_evicts_and_finishes():
    need_gpu()
    from paper_1708_00744_b300.qmcdu import qmcdu_footprint
    classes = [dict(N=128, slots=2), dict(N=256, slots=2)]
    b256 = qmcdu_footprint(256, 32, "fp32", 2) + 2 * 256 + 48
    b128 = qmcdu_footprint(128, 32, "fp32", 2) + 2 * 128 + 48
    budget = b256 + b128 // 2
    reqs = [dict(id=i, seed=i, N=(128, 256)[(i // 3) % 2], nsweeps=2, arrival_s=0.002 * i)
            for i in range(12)]
    srv = Server(classes, precision="fp32", hbm_budget=budget)
    srv.submit(reqs)
    srv.run()
    st = srv.stats()
    assert st["finished"] == len(reqs) and st["failed"] == 0
    assert st["peak_bytes"] <= budget and st["pools_destroyed"] > 0
    srv.close()


def test_spin_resolved_walkers_are_two_independent_determinants():
    """Two determinants per walker (N_up, N_down): each spin's sweep follows
    the oracle's trajectory for its own matrix and draws, and the walker's
    log|det| and sign are the sum and the product."""
    need_gpu()
    from paper_1708_00744_b300.spin import SpinWalkers
    n_up, n_down, K, sigma, nsweeps = 96, 80, 16, 0.3, 2
    seeds = [11, 12]
    S = SpinWalkers(n_up, n_down, K, "fp64", batch=2)
    S.load(seeds)
    acc_u = np.zeros((nsweeps, 2, n_up), dtype=np.uint8)
    acc_d = np.zeros((nsweeps, 2, n_down), dtype=np.uint8)
    rat_u = np.zeros((nsweeps, 2, n_up))
    rat_d = np.zeros((nsweeps, 2, n_down))
    for s in range(nsweeps):
        S.sweep(seeds, s, sigma, acc_u[s], acc_d[s], rat_u[s], rat_d[s])
    la, sg = S.logdet()
    S.close()
    for b, seed in enumerate(seeds):
        tot, sign = 0.0, 1
        for n, key, acc, rat in ((n_up, seed, acc_u, rat_u), (n_down, seed + (1 << 40), acc_d, rat_d)):
            A0, U, ref, tol = _oracle_run(key, n, nsweeps, sigma, K)
            assert _tie_free(ref, U)
            assert np.array_equal(acc[:, b].astype(bool), ref["accepted"])
            tol.check("spin N=%d walker %d" % (n, b), ratio=rat[:, b])
            tot += ref["logabs"]
            sign *= ref["sign"]
        assert sg[b] == sign and logdet_err(la[b], tot) < 1e-9
