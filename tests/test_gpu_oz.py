"""The emulated-fp64 flush of the persistent sweep (fp64 operands cut into
8-bit slices, tensor-core products accumulated exactly, integer
recombination) against the oracle, and against the sweep whose flush uses the
fp64 arithmetic units only, on the same seeded walkers."""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300.qmcdu import Walkers

from gpu_common import (Tol, logdet_err, need_gpu, oracle_walk, rel_norm_err, rel_ratio_err,
                        tie_override, walker_inputs)

pytestmark = pytest.mark.gpu

OZ_KIND = 2000


def run(N, K, base, sigma, nsweeps, fp64_flush, options=(), override=None, batch=1):
    W = Walkers(N, K, "fp64", batch)
    W.set_option("fp64_flush", fp64_flush)
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


# ragged sizes (column tiles of 128 and 64, row chunks of 256 and 128 with a
# tail), K at and below 32, groups of 3 CTAs up to the whole GPU
@pytest.mark.parametrize("N,K,ratio_ctas,flush_ctas", [
    (64, 8, 2, 7), (300, 32, 0, 0), (257, 32, 3, 3), (520, 16, 4, 40), (777, 24, 0, 0),
    (1000, 32, 32, 0)])
def test_emulated_flush_matches_oracle(N, K, ratio_ctas, flush_ctas):
    need_gpu()
    base, sigma, nsweeps = 700 + N, 0.3, 2
    A, G, U = walker_inputs(base, 1, N, nsweeps)
    ref, tol = oracle_walk(A[0], G[0], U[0], sigma, K_alt=K)
    ov, nties = tie_override(ref["ratios"], U[0])
    out = run(N, K, base, sigma, nsweeps, 2,
              options=(("ratio_ctas", ratio_ctas), ("flush_ctas", flush_ctas)),
              override=ov[:, None, :] if nties else None)
    assert out["shape"]["col_tile"] == OZ_KIND
    assert np.array_equal(out["acc"][:, 0].astype(bool), ref["accepted"])
    tol.check("emulated N %d K %d shape %s" % (N, K, out["shape"]),
              ratio=out["rat"][:, 0],
              inverse=rel_norm_err(out["Ainv"][0], ref["Ainv"]),
              logdet=logdet_err(out["logabs"][0], ref["logabs"]))
    assert out["sign"][0] == ref["sign"]


def test_emulated_and_fp64_flush_agree():
    """Same walker, flush on the fp64 units vs emulated: same decisions, and
    results that differ by far less than the fp64 tolerance."""
    need_gpu()
    N, K, base, sigma, nsweeps = 1536, 32, 9100, 0.1, 3
    a = run(N, K, base, sigma, nsweeps, 1)
    b = run(N, K, base, sigma, nsweeps, 2)
    assert a["shape"]["col_tile"] != OZ_KIND and b["shape"]["col_tile"] == OZ_KIND
    assert np.array_equal(a["acc"], b["acc"])
    # the emulation is accurate to fp64 arithmetic: the flat bar between them,
    # each ratio widened by the size of its terms (the oracle's)
    A, G, U = walker_inputs(base, 1, N, nsweeps)
    ref = oracle.sweeps(oracle.SM, A[0], G[0], U[0], sigma)
    t = Tol(ratio=1e-10, inverse=1e-10, logdet=1e-10)
    t.ref_ratios, t.terms = a["rat"][:, 0], ref["terms"]
    t.check("fp64 units vs emulated", ratio=b["rat"][:, 0], inverse=rel_norm_err(b["Ainv"], a["Ainv"]),
            logdet=logdet_err(b["logabs"][0], a["logabs"][0]))


def test_emulated_flush_batch_of_walkers():
    """Several walkers, each on its own group of CTAs, against the oracle."""
    need_gpu()
    N, K, batch, base, sigma = 384, 16, 3, 4242, 0.3
    A, G, U = walker_inputs(base, batch, N, 1)
    out = run(N, K, base, sigma, 1, 0, batch=batch)
    assert out["shape"]["col_tile"] == OZ_KIND and out["shape"]["groups"] >= 2
    for b in range(batch):
        ref, tol = oracle_walk(A[b], G[b], U[b], sigma, K_alt=K)
        assert np.array_equal(out["acc"][:, b].astype(bool), ref["accepted"])
        tol.check("emulated batch walker %d" % b, ratio=out["rat"][:, b],
                  inverse=rel_norm_err(out["Ainv"][b], ref["Ainv"]))
