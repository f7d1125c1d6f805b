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

from gpu_common import fp64_tol, need_gpu, rel_norm_err, rel_ratio_err, torch, walker_inputs

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
    for b in range(batch):
        s, l = oracle.slogdet(Af[b])
        tol = fp64_tol(A[b], Af[b])
        assert sg[b] == s and abs(la[b] - l) < tol * max(1, abs(l))
        assert drift[b, 0] < tol and drift[b, 1] < tol


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
        tol = max(fp64_tol(m) for m in c.initial_matrices())
        assert np.array_equal(acc, e_acc[total - nsweeps:])
        assert rel_ratio_err(rat, e_rat[total - nsweeps:]) < tol
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
