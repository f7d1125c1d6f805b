"""Autotuner: the delay K and the persistent sweep's ratio-CTA count per
(N, batch, precision, acceptance).

The paper picks K per architecture and problem size by hand and notes that an
autotuner could choose it (Sec. II-III). Here each candidate (K, ratio CTAs)
runs short timed sweeps of the walker's own kind on the device (CUDA events on
the handle's stream); the fastest in accepted-move updates per second wins.
Results can be kept in a JSON table keyed by N, batch, precision and the
measured acceptance bucket.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import inputs
from .qmcdu import Walkers


def acceptance_bucket(acc: float) -> str:
    """DMC-like (>= 0.9), VMC-like (0.3 .. 0.9) or low (< 0.3) acceptance."""
    return "high" if acc >= 0.9 else ("mid" if acc >= 0.3 else "low")


def table_key(N, batch, precision, bucket):
    return "%d:%d:%s:%s" % (N, batch, precision, bucket)


def default_candidates(N, precision):
    Ks = [K for K in (16, 32, 64, 128) if K <= N]
    chunk_targets = (32, 64) if precision == "fp64" else (64, 128)
    ratio = sorted({0} | {max(1, N // c) for c in chunk_targets})
    return Ks or [1], ratio


def _time_config(N, K, batch, precision, sigma, ratio_ctas, sweeps, seed, stream):
    import torch
    A = np.stack([inputs.initial_matrix(inputs.walker_seed(seed, b), N) for b in range(batch)])
    W = Walkers(N, K, precision, batch, stream=stream)
    try:
        W.set_option("ratio_ctas", ratio_ctas)
        W.set_matrix(A)
        W.sweep(seed, 0, sigma)                        # warm-up
        acc = torch.zeros(sweeps, batch, N, dtype=torch.uint8, device="cuda")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s = stream if stream is not None else torch.cuda.current_stream()
        e0.record(s)
        for i in range(sweeps):
            W.sweep(seed, 1 + i, sigma, accepted_out=acc[i])
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        accepted = int(acc.sum().item())
    finally:
        W.close()
    return accepted / (ms * 1e-3), accepted / float(sweeps * batch * N), ms / sweeps


def tune(N, batch=1, precision="fp64", sigma=0.1, Ks=None, ratio_ctas=None, sweeps=1, seed=0,
         table_path=None, stream=None, verbose=False):
    """Time every candidate and return the fastest:
    dict(K, ratio_ctas, value (updates/s), acceptance, bucket, candidates)."""
    dK, dR = default_candidates(N, precision)
    Ks = list(Ks) if Ks is not None else dK
    ratio_ctas = list(ratio_ctas) if ratio_ctas is not None else dR
    results = []
    for K in Ks:
        for rc in ratio_ctas:
            value, acc, ms = _time_config(N, K, batch, precision, sigma, rc, sweeps, seed, stream)
            results.append({"K": K, "ratio_ctas": rc, "value": value, "acceptance": acc,
                            "ms_per_sweep": ms})
            if verbose:
                print("autotune N=%d batch=%d %s K=%d ratio_ctas=%d: %.0f updates/s, %.2f ms/sweep"
                      % (N, batch, precision, K, rc, value, ms))
    best = max(results, key=lambda r: r["value"])
    out = dict(best)
    out["bucket"] = acceptance_bucket(best["acceptance"])
    out["candidates"] = results
    if table_path:
        table = {}
        if os.path.exists(table_path):
            with open(table_path) as f:
                table = json.load(f)
        table[table_key(N, batch, precision, out["bucket"])] = {
            "K": best["K"], "ratio_ctas": best["ratio_ctas"], "value": best["value"]}
        with open(table_path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return out


def lookup(table_path, N, batch, precision, bucket):
    """A tuned entry from a table written by tune(), or None."""
    if not table_path or not os.path.exists(table_path):
        return None
    with open(table_path) as f:
        return json.load(f).get(table_key(N, batch, precision, bucket))


def default_K(N, precision="fp64"):
    """The K the tuner settles on without timing (host only): min(32, N). At
    fp64 the emulated tensor-core flush takes queues of at most 32 (its 16
    accumulator blocks of K columns fill tensor memory) and K = 32 was the
    fastest measured point at every N from 512 to 4096, at both acceptances
    and in fp32 too (the K sweep of the benchmark). Used where a K must be
    known before any GPU work, e.g. by a CPU run that reports the same
    configuration as the device run."""
    return max(1, min(32, int(N)))
