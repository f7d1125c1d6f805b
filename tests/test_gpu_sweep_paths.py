"""The persistent sweep kernel against the oracle and against the
host-driven per-proposal kernels, over CTA-group shapes, batches larger than
the SM count, and the bounded device waits."""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300.qmcdu import QmcduError, Walkers

from gpu_common import (logdet_err, need_gpu, oracle_walk, rel_norm_err, rel_ratio_err, tie_override,
                        walker_inputs)

pytestmark = pytest.mark.gpu


def sweep_once(N, K, batch, base, sigma, precision="fp64", options=(), nsweeps=1, override=None):
    W = Walkers(N, K, precision, batch)
    for name, val in options:
        W.set_option(name, val)
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


@pytest.mark.parametrize("N,K,ratio_ctas,flush_ctas", [
    (257, 32, 1, 1), (257, 32, 3, 3), (257, 32, 3, 20), (257, 32, 9, 0),
    (64, 8, 2, 7), (1000, 64, 0, 0), (1000, 64, 32, 0), (129, 1, 4, 0)])
def test_group_shapes_match_oracle(N, K, ratio_ctas, flush_ctas):
    need_gpu()
    base, sigma, nsweeps = 300 + N, 0.3, 2
    A, G, U = walker_inputs(base, 1, N, nsweeps)
    ref, tol = oracle_walk(A[0], G[0], U[0], sigma, K_alt=max(2, K))
    ov, nties = tie_override(ref["ratios"], U[0])
    out = sweep_once(N, K, 1, base, sigma, nsweeps=nsweeps,
                     options=(("ratio_ctas", ratio_ctas), ("flush_ctas", flush_ctas)),
                     override=ov[:, None, :] if nties else None)
    assert np.array_equal(out["acc"][:, 0].astype(bool), ref["accepted"])
    tol.check("shape %s" % out["shape"], ratio=out["rat"][:, 0],
              inverse=rel_norm_err(out["Ainv"][0], ref["Ainv"]),
              logdet=logdet_err(out["logabs"][0], ref["logabs"]))
    if ratio_ctas:
        assert out["shape"]["ratio_ctas"] <= max(1, ratio_ctas)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_equals_host_driven(precision):
    need_gpu()
    N, K, batch, base, sigma = 300, 16, 3, 77, 0.5
    a = sweep_once(N, K, batch, base, sigma, precision, nsweeps=2)
    b = sweep_once(N, K, batch, base, sigma, precision, options=(("sweep_persistent", 0),), nsweeps=2)
    assert np.array_equal(a["acc"], b["acc"])
    tol = 1e-10 if precision == "fp64" else 1e-3
    assert rel_ratio_err(a["rat"], b["rat"]) < tol
    for w in range(batch):
        assert rel_norm_err(a["Ainv"][w], b["Ainv"][w]) < tol


@pytest.mark.parametrize("N", [40, 41])
def test_batch_larger_than_sm_count(N):
    """One CTA per walker, several walkers per CTA group when needed; with odd
    N a walker's last proposal and the next walker's first land on the same
    partial-sum buffer parity of the electron index, which the exchange must
    not depend on."""
    need_gpu()
    K, batch, base, sigma = 8, 400, 5, 0.4
    out = sweep_once(N, K, batch, base, sigma)
    assert out["shape"]["flush_ctas"] == 1 and out["shape"]["ratio_ctas"] == 1
    A, G, U = walker_inputs(base, batch, N, 1)
    for w in (0, 1, 147, 148, 299, 399):
        ref, tol = oracle_walk(A[w], G[w], U[w], sigma, K_alt=K)
        assert np.array_equal(out["acc"][0, w].astype(bool), ref["accepted"][0])
        tol.check("walker %d" % w, ratio=out["rat"][0, w],
                  inverse=rel_norm_err(out["Ainv"][w], ref["Ainv"]))


def test_wait_budget_expires_cleanly():
    """A wait that nothing releases ends with ERR_TIMEOUT; the context stays
    usable and a reload recovers the handle."""
    need_gpu()
    N, K = 128, 8
    A, _, _ = walker_inputs(1, 1, N, 0)
    W = Walkers(N, K, "fp64", 1)
    W.set_matrix(A)
    W.set_option("wait_budget_ns", 50_000_000)
    W.set_option("test_stall", 1)
    with pytest.raises(QmcduError) as e:
        W.sweep(1, 0, 0.1)
        W.sync()
    assert e.value.status == 6
    W.set_option("wait_budget_ns", 0)
    W.set_matrix(A)
    acc = np.zeros((1, N), dtype=np.uint8)
    W.sweep(1, 0, 0.1, accepted_out=acc)
    W.sync()
    assert acc.sum() > 0
    W.close()


@pytest.mark.parametrize("N,K,sigma,fp64_flush", [(1000, 32, 1.0, 0), (700, 64, 1.0, 0), (300, 16, 0.3, 1),
                                                  (130, 1, 1.0, 0)])
def test_fixed_slots_match_oracle(N, K, sigma, fp64_flush):
    """Sec. II's fixed slots (QMCDU_OPT_FIXED_SLOT): rejected proposals take
    queue slots as zero changes, the queue is flushed every K proposals.
    Against the oracle's fixed-slot reading (same decisions, ratios, inverse
    and log-det), with sigma = 1 for many rejections; the emulated-fp64 flush
    (K = 32), the fp64 units (K = 64, and fp64_flush = 1), K = 1."""
    need_gpu()
    base, nsweeps = 6100 + N, 2
    A, G, U = walker_inputs(base, 1, N, nsweeps)
    ref = oracle.sweeps(oracle.DELAYED_SLOT, A[0], G[0], U[0], sigma, K=K)
    alt = oracle.sweeps(oracle.SM + oracle.ALT_INIT, A[0], G[0], U[0], sigma,
                        override=ref["accepted"].astype(np.int8))
    from gpu_common import spread_tol
    tol = spread_tol(ref, alt)
    ov, nties = tie_override(ref["ratios"], U[0])
    out = sweep_once(N, K, 1, base, sigma, nsweeps=nsweeps,
                     options=(("fixed_slot", 1), ("fp64_flush", fp64_flush)),
                     override=ov[:, None, :] if nties else None)
    assert 0.3 < ref["accepted"].mean() < 0.95
    assert np.array_equal(out["acc"][:, 0].astype(bool), ref["accepted"])
    tol.check("fixed slots N=%d K=%d shape %s" % (N, K, out["shape"]),
              ratio=out["rat"][:, 0],
              inverse=rel_norm_err(out["Ainv"][0], ref["Ainv"]),
              logdet=logdet_err(out["logabs"][0], ref["logabs"]))
    assert out["sign"][0] == ref["sign"]


def test_fixed_slots_need_the_persistent_sweep():
    need_gpu()
    W = Walkers(64, 8, "fp64", 1)
    W.set_matrix(np.eye(64)[None])
    W.set_option("fixed_slot", 1)
    W.set_option("sweep_persistent", 0)
    with pytest.raises(QmcduError) as e:
        W.sweep(1, 0, 0.1)
    assert e.value.status == 2
    W.close()
