"""The benchmarked configuration against the oracle at full size, and the
emulated-fp64 flush on walkers whose inverse spans many binades.

* The headline walker (N = 2048, fp64, K = 32, the emulated-fp64 tensor-core
  flush, the autotuner's ratio-CTA count) through qmcdu_step: two sweeps and
  the fp64 recompute, replayed from a captured CUDA graph, element by element
  against the oracle's delayed reading (Eq. 3-4, K = 32).
* A well-conditioned N = 2048 walker (A = I + 0.05 G / sqrt(N), proposals
  small enough that kappa_1 stays below 20 over the walk) held to the flat
  1e-10 bar on ratios, A^{-1} and log|det A|.
* Dynamic range: A = D1 G D2 with D1, D2 diagonal and log-uniform over
  2^(-20) .. 2^20, so that the columns of A^{-1} and the rows of the queue
  span about 40 binades. The emulated flush cuts its operands into 8-bit
  slices relative to a shared power of two; an element far below the shared
  maximum keeps few bits, so this is where such a scheme loses accuracy.
"""
import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import autotune, inputs
from paper_1708_00744_b300.qmcdu import Walkers

from gpu_common import (Tol, device_gaussians, logdet_err, need_gpu, oracle_moves_walk, oracle_walk,
                        rel_norm_err, rel_ratio_err, spread_tol, tie_override, torch, walker_inputs)

pytestmark = pytest.mark.gpu

OZ_KIND = 2000          # sweep_shape()["col_tile"] of the emulated-fp64 flush


def _sweep_walker(W, N, base, sigma, nsweeps, override=None):
    acc = np.zeros((nsweeps, 1, N), dtype=np.uint8)
    rat = np.zeros((nsweeps, 1, N))
    for s in range(nsweeps):
        W.sweep(base, s, sigma, override=None if override is None else override[s],
                accepted_out=acc[s], ratios_out=rat[s])
    Ai = np.zeros((1, N, N))
    la = np.zeros(1)
    sg = np.zeros(1, dtype=np.int32)
    W.get_inverse(Ai)
    W.logdet(la, sg)
    return acc[:, 0], rat[:, 0], Ai[0], la[0], sg[0]


def test_headline_step_n2048_k32_matches_oracle():
    """qmcdu_step as the benchmark runs it (graph replay, recompute at the
    end) against oracle.sweeps(DELAYED, K = 32) on the same seeded walker."""
    need_gpu()
    N, K, sigma, base, nsw = 2048, 32, 0.1, 0, 2
    A, G, U = walker_inputs(base, 1, N, nsw)
    ref = oracle.sweeps(oracle.DELAYED, A[0], G[0], U[0], sigma, K=K)
    alt = oracle.sweeps(oracle.SM + oracle.ALT_INIT, A[0], G[0], U[0], sigma,
                        override=ref["accepted"].astype(np.int8))
    tol = spread_tol(ref, alt)
    # no near tie on this walk: qmcdu_step decides every move itself
    assert ref["near_ties"] == 0 and tie_override(ref["ratios"], U[0])[1] == 0
    tuned = autotune.tune(N, batch=1, precision="fp64", sigma=sigma, Ks=[K], sweeps=1,
                          seed=base + 12345)
    stream = torch.cuda.Stream()
    W = Walkers(N, K, "fp64", 1, stream=stream)
    W.set_option("ratio_ctas", tuned["ratio_ctas"])
    W.set_matrix(A)
    drift = np.zeros((1, 2))
    W.step(base, 0, nsw, sigma, recompute=True, use_graph=True, drift_out=drift)
    acc = np.zeros((nsw, 1, N), dtype=np.uint8)
    rat = np.zeros((nsw, 1, N))
    ties = np.zeros((nsw, 1), dtype=np.int64)
    W.step_results(nsw, acc, rat, ties)
    shape = W.sweep_shape()
    Ai = np.zeros((1, N, N))
    Af = np.zeros((1, N, N))
    la = np.zeros(1)
    sg = np.zeros(1, dtype=np.int32)
    W.get_inverse(Ai)            # after the recompute: A^{-1} by Gauss-Jordan from A
    W.get_matrix(Af)
    W.logdet(la, sg)
    W.close()
    assert shape["col_tile"] == OZ_KIND, shape
    assert np.array_equal(acc[:, 0].astype(bool), ref["accepted"])
    assert ties.sum() == 0
    assert np.array_equal(Af[0], ref["A"])
    assert sg[0] == ref["sign"]
    tol.check("headline N=2048 K=32 (ratio_ctas %d, acceptance %.3f)"
              % (tuned["ratio_ctas"], ref["accepted"].mean()),
              ratio=rat[:, 0],
              inverse=rel_norm_err(Ai[0], ref["Ainv"]),
              logdet=logdet_err(la[0], ref["logabs"]))
    # the running values just before the recompute, against the recomputed ones
    tol.check("headline drift", inverse=drift[0, 1],
              logdet=drift[0, 0] / max(1.0, abs(ref["logabs"])))


@pytest.mark.parametrize("K", [32, 1])
def test_well_conditioned_n2048_flat_bar(K):
    """kappa_1 < 20 along the whole walk (8.4 at the start, 18.7 at the end):
    ratios, the running A^{-1} and log|det| within the flat 1e-10 (no
    spread widening)."""
    need_gpu()
    N, base, nsw = 2048, 31, 2
    G0 = inputs.initial_matrix(base, N)
    A0 = np.eye(N) + 0.05 * G0 / np.sqrt(N)
    sigma = 0.05 / np.sqrt(N)            # |sigma g| ~ 0.05: a row moves by 5% of its norm
    G, U = device_gaussians(base, N, range(nsw))
    ref = oracle.sweeps(oracle.SM, A0, G, U, sigma)
    kappa = max(np.linalg.cond(A0, 1), np.linalg.cond(ref["A"], 1))
    assert kappa < 50, kappa
    ov, nties = tie_override(ref["ratios"], U)
    W = Walkers(N, K, "fp64", 1)
    W.set_matrix(A0[None])
    acc, rat, Ai, la, sg = _sweep_walker(W, N, base, sigma, nsw,
                                         override=ov[:, None, :] if nties else None)
    shape = W.sweep_shape()
    W.close()
    if K == 32:
        assert shape["col_tile"] == OZ_KIND, shape
    assert np.array_equal(acc.astype(bool), ref["accepted"])
    flat = Tol(ratio=1e-10, inverse=1e-10, logdet=1e-10)
    flat.check("well-conditioned N=2048 K=%d kappa_1 %.2f acceptance %.3f"
               % (K, kappa, ref["accepted"].mean()),
               ratio=rel_ratio_err(rat, ref["ratios"]), inverse=rel_norm_err(Ai, ref["Ainv"]),
               logdet=logdet_err(la, ref["logabs"]))
    assert sg == ref["sign"]


def _log_uniform(rng, n, span=20.0):
    return 2.0 ** rng.uniform(-span, span, n)


def _against_units_and_oracle(label, emu, units, ref, tol):
    """The emulated flush against the fp64-unit flush on the same inputs, and
    against the oracle within the oracle's own spread or ten times the fp64
    units' error, whichever is larger. Two correct fp64 flushes of these long,
    increasingly ill-conditioned walks differ by about as much as the oracle's
    two readings do, so the first comparison takes the oracle's spread too
    (each ratio widened by the size of its terms)."""
    t = Tol(ratio=tol["ratio"], inverse=tol["inverse"], logdet=tol["logdet"])
    t.ref_ratios, t.terms = units["rat"], ref["terms"]
    t.check(label + ": emulated vs fp64 units", ratio=emu["rat"], inverse=rel_norm_err(emu["Ainv"], units["Ainv"]),
            logdet=logdet_err(emu["logabs"], units["logabs"]))
    eu = dict(ratio=rel_ratio_err(units["rat"], ref["ratios"]), inverse=rel_norm_err(units["Ainv"], ref["Ainv"]),
              logdet=logdet_err(units["logabs"], ref["logabs"]))
    t2 = Tol({k: max(tol[k], 10.0 * eu[k]) for k in ("ratio", "inverse", "logdet")})
    t2.check(label + ": emulated vs oracle (fp64 units %s)" % ", ".join("%s %.1e" % kv for kv in eu.items()),
             ratio=rel_ratio_err(emu["rat"], ref["ratios"]), inverse=rel_norm_err(emu["Ainv"], ref["Ainv"]),
             logdet=logdet_err(emu["logabs"], ref["logabs"]))


@pytest.mark.parametrize("N,K", [(1024, 32), (1000, 24)])
def test_emulated_flush_dynamic_range_sweep(N, K):
    """A = G D2 (orbital scales over 2^-20 .. 2^20): A^{-1}'s columns and the
    queued rows span ~40 binades. Proposals v = a_j + sigma g with sigma =
    0.1 * 2^-20, so that the smallest orbitals move by O(1) relative to their
    scale and the largest barely. The persistent sweep with the emulated
    flush against the same sweep with the fp64 units and against the oracle."""
    need_gpu()
    base, nsw = 5100 + N, 2
    rng = np.random.default_rng(N + K)
    d2 = _log_uniform(rng, N)
    A0 = inputs.initial_matrix(base, N) * d2[None, :]
    sigma = 0.1 * 2.0 ** -20
    G, U = device_gaussians(base, N, range(nsw))
    ref, tol = oracle_walk(A0, G, U, sigma, K_alt=K)
    ov, nties = tie_override(ref["ratios"], U)
    out = {}
    for flush in (1, 0):           # the fp64 units; the default, emulated
        W = Walkers(N, K, "fp64", 1)
        W.set_option("fp64_flush", flush)
        W.set_matrix(A0[None])
        acc, rat, Ai, la, sg = _sweep_walker(W, N, base, sigma, nsw,
                                             override=ov[:, None, :] if nties else None)
        shape = W.sweep_shape()
        W.close()
        assert (shape["col_tile"] == OZ_KIND) == (flush == 0), shape
        assert np.array_equal(acc.astype(bool), ref["accepted"])
        assert sg == ref["sign"]
        out[flush] = dict(rat=rat, Ainv=Ai, logabs=la)
    inv = ref["Ainv"]
    colspan = np.log2(np.abs(inv).max(axis=1) / np.maximum(np.abs(inv).min(axis=1), 1e-300))
    print("A^{-1} columns span %.0f binades (median), acceptance %.3f"
          % (np.median(colspan), ref["accepted"].mean()))
    _against_units_and_oracle("dynamic range sweep N=%d K=%d" % (N, K), out[0], out[1], ref, tol)


@pytest.mark.parametrize("N,K", [(1024, 32), (1100, 17)])
def test_emulated_flush_dynamic_range_per_call(N, K):
    """A = D1 G D2 through qmcdu_ratio / qmcdu_accept / qmcdu_flush (the
    per-call emulated flush, oz_flush_kernel): electron scales D1 and orbital
    scales D2 both over 2^-20 .. 2^20, proposals v = a_j + 0.1 D1_j (g o d2)
    (a move of a few per cent of the row, orbital by orbital)."""
    need_gpu()
    rng = np.random.default_rng(7 * N + K)
    d1, d2 = _log_uniform(rng, N), _log_uniform(rng, N)
    A0 = d1[:, None] * inputs.initial_matrix(3 + N, N) * d2[None, :]
    nmoves = N + K // 2
    elec = rng.integers(0, N, nmoves).astype(np.int32)   # repeats flush the queue first
    masks = (rng.random(nmoves) < 0.8).astype(np.uint8)
    cur = A0.copy()
    vrows = np.zeros((nmoves, N))
    for m in range(nmoves):
        j = elec[m]
        vrows[m] = cur[j] + 0.1 * d1[j] * rng.standard_normal(N) * d2
        if masks[m]:
            cur[j] = vrows[m]
    out = {}
    for flush in (1, 0):           # the fp64 units; the default, emulated
        W = Walkers(N, K, "fp64", 1)
        W.set_option("fp64_flush", flush)
        W.set_matrix(A0[None])
        v_dev = torch.zeros(1, N, dtype=torch.float64, device="cuda")
        r_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
        ratios = np.zeros(nmoves)
        for m in range(nmoves):
            v_dev.copy_(torch.from_numpy(vrows[m][None]))
            W.ratio(elec[m:m + 1], v_dev, r_dev)
            ratios[m] = r_dev.item()
            W.accept(masks[m:m + 1])
        Ai = np.zeros((1, N, N))
        la = np.zeros(1)
        sg = np.zeros(1, dtype=np.int32)
        W.get_inverse(Ai)
        W.logdet(la, sg)
        W.close()
        out[flush] = dict(rat=ratios, Ainv=Ai[0], logabs=la[0], sign=sg[0])
    ref, tol = oracle_moves_walk(A0, elec, vrows, masks, K)
    assert out[0]["sign"] == ref["sign"]
    _against_units_and_oracle("dynamic range per call N=%d K=%d" % (N, K), out[0], out[1], ref, tol)
