"""Cluster mode of the persistent sweep: the 16 ratio CTAs of an fp64 walker
form one thread-block cluster and exchange the partial dot products of every
proposal through distributed shared memory. Checked against the oracle and
against the global-memory exchange on the same seeded walkers."""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300.qmcdu import Walkers

from gpu_common import (Tol, logdet_err, need_gpu, oracle_walk, rel_norm_err, rel_ratio_err,
                        tie_override, walker_inputs)

pytestmark = pytest.mark.gpu


def run(N, K, base, sigma, nsweeps, cluster, override=None, batch=1, fp64_flush=0):
    W = Walkers(N, K, "fp64", batch)
    W.set_option("cluster", cluster)
    W.set_option("fp64_flush", fp64_flush)
    A, _, _ = walker_inputs(base, batch, N, 0)
    W.set_matrix(A)
    acc = np.zeros((nsweeps, batch, N), dtype=np.uint8)
    rat = np.zeros((nsweeps, batch, N))
    for s in range(nsweeps):
        W.sweep(base, s, sigma, override=None if override is None else override[s],
                accepted_out=acc[s], ratios_out=rat[s])
    Ai = np.zeros((batch, N, N))
    la = np.zeros(batch)
    sg = np.zeros(batch, dtype=np.int32)
    W.get_inverse(Ai)
    W.logdet(la, sg)
    shape = W.sweep_shape()
    W.close()
    return dict(acc=acc, rat=rat, Ainv=Ai, logabs=la, sign=sg, shape=shape)


@pytest.mark.parametrize("N,K,fp64_flush", [(1024, 32, 0), (1100, 16, 0), (1024, 24, 1)])
def test_cluster_mode_matches_oracle(N, K, fp64_flush):
    need_gpu()
    base, sigma, nsweeps = 8100 + N, 0.3, 2
    A, G, U = walker_inputs(base, 1, N, nsweeps)
    ref, tol = oracle_walk(A[0], G[0], U[0], sigma, K_alt=K)
    ov, nties = tie_override(ref["ratios"], U[0])
    out = run(N, K, base, sigma, nsweeps, 2, override=ov[:, None, :] if nties else None,
              fp64_flush=fp64_flush)
    assert out["shape"]["ratio_ctas"] == 16 and out["shape"]["flush_ctas"] % 16 == 0
    assert np.array_equal(out["acc"][:, 0].astype(bool), ref["accepted"])
    tol.check("cluster N %d K %d shape %s" % (N, K, out["shape"]),
              ratio=out["rat"][:, 0],
              inverse=rel_norm_err(out["Ainv"][0], ref["Ainv"]),
              logdet=logdet_err(out["logabs"][0], ref["logabs"]))
    assert out["sign"][0] == ref["sign"]


def test_cluster_and_global_exchange_agree():
    need_gpu()
    N, K, base, sigma, nsweeps = 2048, 32, 9300, 0.1, 2
    a = run(N, K, base, sigma, nsweeps, 1)
    b = run(N, K, base, sigma, nsweeps, 2)
    assert a["shape"]["ratio_ctas"] != 16 or a["shape"]["flush_ctas"] % 16 != 0
    assert b["shape"]["ratio_ctas"] == 16
    assert np.array_equal(a["acc"], b["acc"])
    # two orders of the same fp64 sums: the flat bar, each ratio widened by
    # the size of its terms (the oracle's) as against the oracle
    A, G, U = walker_inputs(base, 1, N, nsweeps)
    ref = oracle.sweeps(oracle.SM, A[0], G[0], U[0], sigma)
    t = Tol(ratio=1e-10, inverse=1e-10, logdet=1e-10)
    t.ref_ratios, t.terms = a["rat"][:, 0], ref["terms"]
    t.check("cluster vs global", ratio=b["rat"][:, 0], inverse=rel_norm_err(b["Ainv"], a["Ainv"]))


def test_two_walkers_two_clusters_groups():
    need_gpu()
    N, K, batch, base, sigma = 1024, 16, 2, 5150, 0.3
    A, G, U = walker_inputs(base, batch, N, 1)
    out = run(N, K, base, sigma, 1, 2, batch=batch)
    assert out["shape"]["ratio_ctas"] == 16 and out["shape"]["groups"] == 2
    for b in range(batch):
        ref, tol = oracle_walk(A[b], G[b], U[b], sigma, K_alt=K)
        assert np.array_equal(out["acc"][:, b].astype(bool), ref["accepted"])
        tol.check("two clusters walker %d" % b, ratio=out["rat"][:, b],
                  inverse=rel_norm_err(out["Ainv"][b], ref["Ainv"]))
