"""Batched walkers (a step of S sweeps + recompute through qmcdu_step, CUDA
graph replay, walker groups of uneven N, the autotuner) against eager calls
and against each walker run alone."""
import json
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import autotune
from paper_1708_00744_b300.batch import SizeClass, WalkerGroup
from paper_1708_00744_b300.qmcdu import QmcduError, Walkers

from gpu_common import (Tol, direct_tol, logdet_err, need_gpu, oracle_walk, rel_norm_err,
                        rel_ratio_err, tie_override, torch, walker_inputs)

pytestmark = pytest.mark.gpu


def _eager_sweeps(N, K, batch, base, sigma, first, nsweeps, precision="fp64"):
    W = Walkers(N, K, precision, batch)
    A, _, _ = walker_inputs(base, batch, N, 0)
    W.set_matrix(A)
    acc = np.zeros((nsweeps, batch, N), dtype=np.uint8)
    rat = np.zeros((nsweeps, batch, N))
    for s in range(nsweeps):
        W.sweep(base, first + s, sigma, accepted_out=acc[s], ratios_out=rat[s])
    Ai = np.zeros((batch, N, N))
    W.get_inverse(Ai)
    W.close()
    return acc, rat, Ai


def test_step_graph_replay_equals_eager_sweeps():
    need_gpu()
    N, K, batch, base, sigma = 200, 16, 3, 41, 0.3
    stream = torch.cuda.Stream()
    W = Walkers(N, K, "fp64", batch, stream=stream)
    A, _, _ = walker_inputs(base, batch, N, 0)
    W.set_matrix(A)
    accs, rats = [], []
    for first in (0, 2, 4):          # first call captures, the others replay the graph
        acc = np.zeros((2, batch, N), dtype=np.uint8)
        rat = np.zeros((2, batch, N))
        W.step(base, first, 2, sigma, recompute=False, use_graph=True)
        W.step_results(2, acc, rat)
        accs.append(acc)
        rats.append(rat)
    Ai = np.zeros((batch, N, N))
    W.get_inverse(Ai)
    W.close()
    e_acc, e_rat, e_Ai = _eager_sweeps(N, K, batch, base, sigma, 0, 6)
    assert np.array_equal(np.concatenate(accs), e_acc)
    assert np.array_equal(np.concatenate(rats), e_rat)      # same kernels, same order: identical
    assert np.array_equal(Ai, e_Ai)


def test_step_with_recompute_reports_drift():
    need_gpu()
    N, K, batch = 150, 8, 2
    stream = torch.cuda.Stream()
    W = Walkers(N, K, "fp64", batch, stream=stream)
    A, _, _ = walker_inputs(3, batch, N, 0)
    W.set_matrix(A)
    drift = np.zeros((batch, 2))
    acc = np.zeros((3, batch, N), dtype=np.uint8)
    W.step(3, 0, 3, 0.1, recompute=True, use_graph=True, accepted_out=acc, drift_out=drift)
    W.step(3, 3, 3, 0.1, recompute=True, use_graph=True, drift_out=drift)
    Af = np.zeros((batch, N, N))
    W.get_matrix(Af)
    la = np.zeros(batch)
    sg = np.zeros(batch, dtype=np.int32)
    W.logdet(la, sg)
    W.close()
    assert acc.sum() > 0
    _, G, U = walker_inputs(3, batch, N, 6)
    for b in range(batch):
        _, (s, l), tol = direct_tol(Af[b])
        assert sg[b] == s
        tol.check("recomputed log-det walker %d" % b, logdet=logdet_err(la[b], l))
        # the drift of the second step (sweeps 3..5) within the spread of the
        # oracle's two readings over all six sweeps
        wref, wtol = oracle_walk(A[b], G[b], U[b], 0.1, K_alt=K)
        wtol.check("drift walker %d" % b, inverse=drift[b, 1],
                   logdet=drift[b, 0] / max(1.0, abs(wref["logabs"])))


def test_graph_needs_a_stream():
    need_gpu()
    W = Walkers(32, 4, "fp64", 1)
    W.set_matrix(np.eye(32)[None])
    with pytest.raises(QmcduError) as e:
        W.step(0, 0, 1, 0.1, use_graph=True)
    assert e.value.status == 1
    W.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_uneven_walkers_in_one_group_match_each_alone(use_graph):
    """Each walker's results are the same alone and in the mix (to rounding:
    the group shape changes the order of the partial sums)."""
    need_gpu()
    sigma, nsweeps = 0.2, 2
    classes = [SizeClass(96, 16, 20, base_seed=500), SizeClass(160, 32, 4, base_seed=900)]
    for c in classes:
        c.load()
    grp = WalkerGroup(classes)
    grp.step(0, nsweeps, sigma, recompute=False, use_graph=use_graph)
    steps = 1
    if use_graph:
        grp.step(nsweeps, nsweeps, sigma, recompute=False, use_graph=True)   # graph replay
        steps = 2
    grp.synchronize()
    total = steps * nsweeps
    for c in classes:
        acc, rat = c.results(nsweeps)          # the last step's sweeps
        W = Walkers(c.N, c.K, "fp64", c.batch)
        W.set_matrix(c.initial_matrices())
        e_acc = np.zeros((total, c.batch, c.N), dtype=np.uint8)
        e_rat = np.zeros((total, c.batch, c.N))
        for s in range(total):
            W.sweep(c.base_seed, s, sigma, accepted_out=e_acc[s], ratios_out=e_rat[s])
        W.close()
        assert np.array_equal(acc, e_acc[total - nsweeps:])
        # the same fp64 sums in another order: the flat bar
        Tol(ratio=1e-10, inverse=1e-10, logdet=1e-10).check(
            "group vs alone N=%d" % c.N, ratio=rel_ratio_err(rat, e_rat[total - nsweeps:]))
    grp.close()
    for c in classes:
        c.close()


def test_autotuner_picks_a_measured_candidate():
    need_gpu()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "table.json")
        best = autotune.tune(256, batch=2, precision="fp64", sigma=0.1, Ks=(8, 32),
                             ratio_ctas=(0, 4), sweeps=1, table_path=path)
        assert best["K"] in (8, 32) and best["ratio_ctas"] in (0, 4)
        assert best["value"] == max(r["value"] for r in best["candidates"])
        assert len(best["candidates"]) == 4
        table = json.load(open(path))
        entry = autotune.lookup(path, 256, 2, "fp64", best["bucket"])
        assert entry == table[autotune.table_key(256, 2, "fp64", best["bucket"])]
        assert entry["K"] == best["K"]


def test_group_at_batched_workload_shapes_matches_oracle():
    """The batched workload's two size classes in one walker group: walkers
    of N = 512 and N = 1536, fp64, K = 64, sigma = 0.1, stepped together by
    qmcdu_group_step (the first step captures the CUDA graph, the second
    replays it). Sampled walkers of each class against the oracle, element by
    element, over both sweeps."""
    need_gpu()
    sigma, K = 0.1, 64
    classes = [SizeClass(512, K, 8, base_seed=1000), SizeClass(1536, K, 2, base_seed=2000)]
    for c in classes:
        c.load()
    grp = WalkerGroup(classes)
    per_step = []
    for first in (0, 1):
        grp.step(first, 1, sigma, recompute=False, use_graph=True)
        grp.synchronize()
        per_step.append([c.results(1) for c in classes])
    grp.close()
    for ci, (c, sample) in enumerate(zip(classes, ((0, 7), (1,)))):
        Ai = np.zeros((c.batch, c.N, c.N))
        la = np.zeros(c.batch)
        sg = np.zeros(c.batch, dtype=np.int32)
        c.walkers.get_inverse(Ai)
        c.walkers.logdet(la, sg)
        A, G, U = walker_inputs(c.base_seed, c.batch, c.N, 2)
        for b in sample:
            ref, tol = oracle_walk(A[b], G[b], U[b], sigma, K_alt=K)
            assert tie_override(ref["ratios"], U[b])[1] == 0      # the group decides every move
            acc = np.concatenate([per_step[s][ci][0][:, b] for s in (0, 1)])
            rat = np.concatenate([per_step[s][ci][1][:, b] for s in (0, 1)])
            assert np.array_equal(acc.astype(bool), ref["accepted"])
            tol.check("group N=%d walker %d" % (c.N, b), ratio=rat,
                      inverse=rel_norm_err(Ai[b], ref["Ainv"]), logdet=logdet_err(la[b], ref["logabs"]))
            assert sg[b] == ref["sign"]
    for c in classes:
        c.close()


@pytest.mark.parametrize("precision,R", [("fp32", 2), ("bf16x3", 20)])
def test_group_at_mixed_workload_shapes_matches_oracle(precision, R):
    """The mixed workload's two size classes in one walker group at full size:
    64 walkers of N = 2048 and 8 of N = 4096, K = 64, sigma = 0.1, one sweep
    through qmcdu_group_step (captured as a CUDA graph). One sampled walker of
    each class against the fp64 oracle (Sherman-Morrison, its own decisions),
    within the fitted mixed-precision bound of tests/test_gpu_mixed.py (the
    split-bf16 bound is that of its in-sweep tensor-core flush). The device
    decides every move: a decision may differ from the oracle's only within
    twice the walk's ratio error of a tie, and the walks part there, so the
    comparison stops at the first such decision (A^{-1} and log|det| are
    compared only if there is none)."""
    need_gpu()
    from test_gpu_mixed import bounds
    from gpu_common import device_gaussians
    from paper_1708_00744_b300 import inputs
    sigma, K = 0.1, 64
    classes = [SizeClass(2048, K, 64, precision, base_seed=3000), SizeClass(4096, K, 8, precision, base_seed=4000)]
    for c in classes:
        c.load()
    grp = WalkerGroup(classes)
    grp.step(0, 1, sigma, recompute=False, use_graph=True)
    grp.synchronize()
    res = [c.results(1) for c in classes]
    oracle.set_threads(0)
    for c, (acc_all, rat_all), b in zip(classes, res, (37, 5)):
        key = inputs.walker_seed(c.base_seed, b)
        A = inputs.initial_matrix(key, c.N)
        G, U = device_gaussians(key, c.N, [0])
        ref = oracle.sweeps(oracle.SM, A, G, U, sigma)
        acc, rat = acc_all[0, b].astype(bool), rat_all[0, b]
        kappa = max(np.linalg.cond(A, 1), np.linalg.cond(ref["A"], 1))
        bnd = bounds(precision, sigma, R, kappa)
        p = np.minimum(1.0, ref["ratios"][0] ** 2)
        diff = np.nonzero(acc != ref["accepted"][0])[0]
        upto = int(diff[0]) if len(diff) else c.N
        e = rel_ratio_err(rat[:upto + 1], ref["ratios"][0][:upto + 1])
        for j in diff[:1]:
            assert abs(p[j] - U[0, j]) < 2 * e, ("decision far from a tie differs", c.N, b, int(j))
        line = "%s group N=%d walker %d: kappa_1 %.1e | ratio %.1e (bound %.1e) over %d of %d proposals" % (
            precision, c.N, b, kappa, e, bnd[0], upto + 1 if len(diff) else c.N, c.N)
        assert e < bnd[0], line
        if not len(diff):
            Ai = torch.zeros(c.batch, c.N, c.N, dtype=torch.float64, device="cuda")
            c.walkers.get_inverse(Ai)
            inv_b = Ai[b].cpu().numpy()
            del Ai
            la = np.zeros(c.batch)
            sg = np.zeros(c.batch, dtype=np.int32)
            c.walkers.logdet(la, sg)
            ei, el = rel_norm_err(inv_b, ref["Ainv"]), logdet_err(la[b], ref["logabs"])
            line += " | inverse %.1e (%.1e) logdet %.1e (%.1e)" % (ei, bnd[1], el, bnd[2])
            assert ei < bnd[1] and el < bnd[2], line
            assert sg[b] == ref["sign"]
        print(line)
    grp.close()
    for c in classes:
        c.close()
