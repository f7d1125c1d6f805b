#!/usr/bin/env python
"""Benchmark of the delayed Slater-determinant update on one B300.

Metric: accepted-move updates per second (the paper's Monte Carlo column
updates per second over complete sweeps, Sec. III), whole job.

Workloads (--workload):
  single  (default) one walker of N = 2048 electrons in fp64, A_ij ~ N(0,1),
          proposal v = a_j + 0.1 g (DMC-like acceptance), K tuned by the
          autotuner (untimed, before the measurement). A step is ten full
          Metropolis sweeps followed by the fp64 recompute of A^{-1} and
          log|det A| (qmcdu_step). The same walker with K = 1
          (Sherman-Morrison) on the same GPU gives the speedup.
  uneven  256 walkers of N = 512 and 64 of N = 1536, fp64, sigma = 0.1, K = 64,
          both size classes stepped together (qmcdu_group_step); a step is one
          sweep of every walker.
  mixed   64 walkers of N = 2048 and 8 of N = 4096 with A^{-1}, panels and the
          flush in fp32 (k x k algebra, ratios, log-det in fp64), sigma = 0.1,
          K = 64; a step is one sweep of every walker.
Inputs are synthetic (seeded Philox draws). L2 is flushed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own independent walkers (weak scaling);
the slowest rank's time counts and rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# ALU peaks of one B300 (148 SMs at the 2032 MHz maximum SM clock): 2 FP64 FMA
# per SM per clock (a DFMA loop measures 1.127 TFLOP/s at the clock it ran at),
# 128 FP32 FMA per SM per clock.
SMS, SM_MHZ = 148, 2032.0
FP64_PEAK_TFLOPS = SMS * 2 * 2 * SM_MHZ * 1e6 / 1e12      # 1.203
OZ_FLUSH_KIND = 2000      # sweep_shape()["col_tile"] of the emulated-fp64 tensor-core flush
OZ_PRODUCTS = 28          # fp16 slice products per emulated fp64 product (slice pairs j + l <= 6)
FP32_PEAK_TFLOPS = SMS * 128 * 2 * SM_MHZ * 1e6 / 1e12    # 77.0
HBM_PEAK_FALLBACK_GBS = 6400.0

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the sweep kernel,
# from one ncu capture; keyed by the sha256 of kernels_sweep.cu at capture time
# and the workload (a stale key gives null).
#   single: one sweep of one N = 2048 fp64 walker, K = 32, emulated flush: the
#   mean of two launches, 102.0 MB read + 78.0 MB written (the working set stays
#   in L2); command in profiles/sweep_kernel_fp64_emulated_n2048_k32.md.
NCU_TRAFFIC = {"33173a30f5baa151:single": (102.494208e6 + 78.629376e6 + 101.690624e6 + 76.275712e6) / 2}

WORKLOADS = {
    "single": [dict(N=2048, batch=1)],
    "uneven": [dict(N=512, batch=256), dict(N=1536, batch=64)],
    "mixed": [dict(N=2048, batch=64), dict(N=4096, batch=8)],
    # serving: Poisson arrivals, N uniform over the size set; slots per pool
    "ksweep": [dict(N=2048, batch=1)],
    "kernels": [dict(N=512, batch=128)],
    "serve": [dict(N=128, batch=16), dict(N=256, batch=16), dict(N=512, batch=16),
              dict(N=1024, batch=8), dict(N=2048, batch=8), dict(N=4096, batch=8)],
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="single", choices=sorted(WORKLOADS))
    p.add_argument("--N", type=int, default=None, help="override N (single workload)")
    p.add_argument("--K", default="auto", help="delay K, or 'auto' (autotuner)")
    p.add_argument("--sigma", type=float, default=0.1)
    p.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16x3"])
    p.add_argument("--sweeps-per-step", type=int, default=None)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--k1-steps", type=int, default=1, help="steps of the K=1 comparison")
    p.add_argument("--cpu-moves", type=int, default=-1,
                   help="proposals in the CPU-oracle sample (default: sized for ~15 s)")
    p.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    p.add_argument("--window", type=float, default=20.0, help="serve: seconds of arrivals timed")
    p.add_argument("--budget-gb", type=float, default=150.0, help="serve: HBM budget (GB)")
    p.add_argument("--reps", type=int, default=5, help="ksweep: timed sweeps per point (median)")
    p.add_argument("--ksweep-N", default="512,1024,2048,4096", help="ksweep: electron counts")
    p.add_argument("--kernels-batch", type=int, default=512, help="kernels: walkers of the ratio run")
    a = p.parse_args()
    a.classes = [dict(c) for c in WORKLOADS[a.workload]]
    if a.N is not None and a.workload == "single":
        a.classes[0]["N"] = a.N
    if a.precision is None:
        a.precision = "fp32" if a.workload in ("mixed", "serve") else "fp64"
    if a.sweeps_per_step is None:
        a.sweeps_per_step = 10 if a.workload == "single" else 1
    a.N = a.classes[0]["N"]
    return a


def workload_name(a):
    if a.workload == "ksweep":
        return ("one %s walker, N in {%s}, K in {1, 16, 32, 64, 128, 256}, sigma 0.1 and 1.0 "
                "and forced acceptance; median of %d single sweeps per point"
                % (a.precision, a.ksweep_N, a.reps))
    if a.workload == "kernels":
        return "kernel microbenchmarks: batched ratio, split-bf16 GEMM, fp64 recompute"
    if a.workload == "serve":
        return ("serving: Poisson arrivals at %g/s for %g s, N uniform over {%s}, %s + fp64 "
                "recompute every 10 sweeps, sigma=%g, 20 sweeps per request, %g GB budget"
                % (a.rate, a.window, ", ".join(str(c["N"]) for c in a.classes), a.precision,
                   a.sigma, a.budget_gb))
    cls = " + ".join("%d x N=%d" % (c["batch"], c["N"]) for c in a.classes)
    rec = " + fp64 recompute" if a.workload == "single" else ""
    return "%s walkers, %s, K=%s, sigma=%g, %d sweep(s)%s per step" % (
        cls, a.precision, a.K, a.sigma, a.sweeps_per_step, rec)


def config(a, world):
    def k_of(c):
        k = c.get("K", a.K)
        return int(k) if str(k).isdigit() else k
    return {"workload": workload_name(a), "name": a.workload,
            "classes": [{"N": c["N"], "batch": c["batch"], "K": k_of(c)} for c in a.classes],
            "precision": a.precision, "sigma": a.sigma, "sweeps_per_step": a.sweeps_per_step,
            "recompute_every_sweeps": a.sweeps_per_step if a.workload == "single" else None,
            "l2": "flushed between timed steps (256 MB write)", "parallelism": "walkers x %d" % world}


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_sample(a, max_moves, K, threads=1):
    """The fp64 CPU oracle (delayed look-ahead + Woodbury with the same K; K = 1:
    Sherman-Morrison) on the first `max_moves` proposals of sweep 0 of one
    walker, on `threads` OpenMP threads (0: all cores). The oracle times its
    update work itself, after its setup (an O(N^3) LU inverse of the starting
    matrix), so that the figure is the update throughput. Returns (accepted,
    seconds of update work, threads used)."""
    import oracle
    from paper_1708_00744_b300 import inputs
    A = inputs.initial_matrix(a.seed, a.N)
    G = inputs.proposal_gaussians(a.seed, 0, a.N)[None]
    U = inputs.metropolis_uniforms(a.seed, 0, a.N)[None]
    method = oracle.SM if K == 1 else oracle.DELAYED
    oracle.build()
    used = oracle.set_threads(threads)
    out = oracle.sweeps(method, A, G, U, a.sigma, K=K, max_moves=max_moves)
    dt = oracle.last_update_seconds()
    acc = int(out["accepted"][0, :max_moves].sum())
    return acc, dt, used


def host_cpu():
    """CPU model and logical core count of this host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def cpu_sample_size(a, K, seconds=15.0):
    if a.cpu_moves > 0:
        return min(a.cpu_moves, a.N)
    # about 4 N^2 flops per accepted move at ~1 GFLOP/s, plus the look-ahead
    per_move = 4.0 * a.N * a.N / 1.0e9 + 2.0 * a.N * (2 * K + 1) / 1.0e9
    return int(max(16, min(a.N, seconds / per_move)))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def source_hash(name):
    with open(os.path.join(ROOT, "paper_1708_00744_b300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ------------------------------------------------------------------ GPU arm
def run_ours(a, rank, world, local_rank):
    import torch
    from paper_1708_00744_b300 import autotune, inputs
    from paper_1708_00744_b300.qmcdu import Walkers, qmcdu_group_create, qmcdu_group_destroy, \
        qmcdu_group_step

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    nsw = a.sweeps_per_step
    recompute = a.workload == "single"
    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # ---- K (and the ratio-CTA count) from the autotuner, untimed
    tuned = None
    for c in a.classes:
        if a.K == "auto" and a.workload == "single":
            t = autotune.tune(c["N"], batch=c["batch"], precision=a.precision, sigma=a.sigma,
                              sweeps=1, seed=a.seed + 12345)
            c["K"], c["ratio_ctas"] = t["K"], t["ratio_ctas"]
            tuned = {"K": t["K"], "ratio_ctas": t["ratio_ctas"],
                     "candidates": [{k: r[k] for k in ("K", "ratio_ctas", "ms_per_sweep")}
                                    for r in t["candidates"]]}
        else:
            c["K"] = 64 if a.K == "auto" else int(a.K)
            c.setdefault("ratio_ctas", 0)
    if a.K == "auto" and len({c["K"] for c in a.classes}) == 1:
        a.K = str(a.classes[0]["K"])          # the configuration names the K that ran
    barrier()

    # ---- handles: one per size class, each on its own stream
    hs = []
    for i, c in enumerate(a.classes):
        st = torch.cuda.Stream()
        base = a.seed + 100000 * i + rank * c["batch"]
        A0 = torch.from_numpy(np.stack([inputs.initial_matrix(inputs.walker_seed(base, b), c["N"])
                                        for b in range(c["batch"])])).pin_memory()
        W = Walkers(c["N"], c["K"], a.precision, c["batch"], stream=st)
        W.set_option("ratio_ctas", c.get("ratio_ctas", 0))
        W.set_matrix(A0)
        drift = torch.zeros(c["batch"], 2, dtype=torch.float64, device=dev)
        hs.append(dict(W=W, stream=st, base=base, A0=A0, cls=c, drift=drift))
    s0 = hs[0]["stream"]
    group = qmcdu_group_create([h["W"].h for h in hs]) if len(hs) > 1 else None
    nprop = sum(c["N"] * c["batch"] for c in a.classes) * nsw

    def step(handles, sweep0, use_graph):
        if len(handles) == 1 or group is None:
            for h in handles:
                h["W"].step(h["base"], sweep0, nsw, a.sigma, recompute=recompute,
                            use_graph=use_graph,
                            drift_out=h.get("drift") if recompute else None)
        else:
            qmcdu_group_step(group, [h["base"] for h in handles], sweep0, nsw, a.sigma, recompute,
                             use_graph)

    def accepted_in_step(handles):
        tot = 0
        for h in handles:
            c = h["cls"]
            acc = np.zeros((nsw, c["batch"], c["N"]), dtype=np.uint8)
            h["W"].step_results(nsw, acc)
            tot += int(acc.sum())
        return tot

    last = {}     # the drift of the last timed run

    def timed(handles, nsteps, nwarm, sweep0, use_graph, profile=False):
        stream = handles[0]["stream"]
        sweep = sweep0
        for _ in range(nwarm):
            step(handles, sweep, use_graph)
            sweep += nsw
        barrier()
        if profile:
            for h in handles:
                h["W"].profile_enable(True)
        ms, accepted = [], 0
        drift_max = np.zeros(2)
        for _ in range(nsteps):
            flush_buf.zero_()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            step(handles, sweep, use_graph)
            sweep += nsw
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            accepted += accepted_in_step(handles)
            if recompute:
                for h in handles:
                    if "drift" in h:
                        drift_max = np.maximum(drift_max, h["drift"].cpu().numpy().max(axis=0))
        prof = None
        if profile:
            prof = [dict(h["W"].profile_read(), sweep_times_ms=h["W"].profile_sweep_times().tolist())
                    for h in handles]
            for h in handles:
                h["W"].profile_enable(False)
        last["drift"] = drift_max if recompute else None
        return ms, accepted, prof, sweep

    clocks = ClockSampler(local_rank)
    clocks.start()
    ms, accepted, prof, sweep_next = timed(hs, a.steps, a.warmup, 0, use_graph=False, profile=True)
    drift = last["drift"]
    flush_kinds = [h["W"].sweep_shape()["col_tile"] for h in hs]
    clk = clocks.stop()
    # the same steps replayed from the captured CUDA graph
    msg, accg, _, sweep_next = timed(hs, a.steps, 1, sweep_next, use_graph=True)

    # end to end through the public API with host buffers: upload A from pinned
    # host memory, run the step (graph replay), read accept masks and log-dets back.
    e2e_s, e2e_acc = [], 0
    h2d = sum(c["batch"] * c["N"] * c["N"] * 8 for c in a.classes)
    d2h = sum(nsw * c["batch"] * c["N"] + c["batch"] * 12 for c in a.classes)
    for it in range(a.warmup + a.steps):
        barrier()
        t0 = time.perf_counter()
        for h in hs:
            h["W"].set_matrix(h["A0"])
        step(hs, 0, True)
        got = 0
        for h in hs:
            c = h["cls"]
            acc = np.zeros((nsw, c["batch"], c["N"]), dtype=np.uint8)
            la = np.zeros(c["batch"])
            sg = np.zeros(c["batch"], dtype=np.int32)
            h["W"].step_results(nsw, acc)
            h["W"].logdet(la, sg)
            got += int(acc.sum())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if it >= a.warmup:
            e2e_s.append(dt)
            e2e_acc += got
    if group is not None:
        qmcdu_group_destroy(group)
    for h in hs:
        h["W"].close()

    # K = 1 (Sherman-Morrison) on the same GPU, same walker (single workload)
    k1 = None
    if a.workload == "single" and a.k1_steps > 0:
        c = a.classes[0]
        W1 = Walkers(c["N"], 1, a.precision, c["batch"], stream=s0)
        W1.set_matrix(hs[0]["A0"])
        h1 = [dict(W=W1, stream=s0, base=hs[0]["base"], cls=dict(c, K=1))]
        # eager launches: the profile's per-launch events are recorded there
        ms1, acc1, prof1, _ = timed(h1, a.k1_steps, 1, 0, use_graph=False, profile=True)
        W1.close()
        k1 = (ms1, acc1, prof1[0])

    # end-of-run reduction over ranks (the only collective): sums of counts,
    # max of times
    from paper_1708_00744_b300.shard import reduce_counters
    red = reduce_counters({"total_ms": sum(ms), "accepted": accepted, "graph_ms": sum(msg),
                           "graph_accepted": accg, "e2e_s": sum(e2e_s), "e2e_acc": e2e_acc,
                           "k1_ms": sum(k1[0]) if k1 else 0.0,
                           "k1_accepted": k1[1] if k1 else 0})
    res = dict(ms=ms, total_ms=red["total_ms"], accepted=red["accepted"], prof=prof, clocks=clk,
               graph_ms=red["graph_ms"], graph_accepted=red["graph_accepted"],
               e2e_s=red["e2e_s"], e2e_acc=red["e2e_acc"], h2d=h2d, d2h=d2h,
               nprop=nprop, tuned=tuned, k1=None, flush_kinds=flush_kinds, drift=drift)
    if k1 is not None:
        res["k1"] = dict(ms=red["k1_ms"], accepted=red["k1_accepted"], prof=k1[2])
    return res


# ------------------------------------------------------------------ K sweep
def run_ksweep(a):
    """Updates/s of one fp64 walker against K (the paper's Fig. 1 axes), with
    sigma 0.1 (DMC-like), sigma 1.0 (VMC-like) and forced acceptance (the
    paper's test condition): per point the median of --reps single sweeps timed
    with CUDA events, L2 flushed before each."""
    import torch
    from paper_1708_00744_b300 import inputs
    from paper_1708_00744_b300.qmcdu import Walkers
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rows = []
    for N in [int(x) for x in a.ksweep_N.split(",")]:
        A0 = inputs.initial_matrix(a.seed, N)[None]
        acc = torch.zeros(1, N, dtype=torch.uint8, device="cuda")
        ones = torch.ones(1, N, dtype=torch.int8, device="cuda")
        for mode in ("sigma=0.1", "sigma=1.0", "forced"):
            sigma = 1.0 if mode == "sigma=1.0" else 0.1
            for K in (1, 16, 32, 64, 128, 256):
                if K > N:
                    continue
                W = Walkers(N, K, a.precision, 1, stream=st)
                W.set_matrix(A0)
                ov = ones if mode == "forced" else None
                W.sweep(a.seed, 0, sigma, override=ov, accepted_out=acc)     # warm-up
                ms, got = [], []
                for r in range(a.reps):
                    flush_buf.zero_()
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    W.sweep(a.seed, 1 + r, sigma, override=ov, accepted_out=acc)
                    e1.record(st)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                    got.append(int(acc.sum().item()))
                W.close()
                order = np.argsort(ms)
                med = order[len(ms) // 2]
                rows.append({"N": N, "mode": mode, "K": K, "ms_per_sweep": ms[med],
                             "updates_per_s": got[med] / (ms[med] * 1e-3),
                             "proposals_per_s": N / (ms[med] * 1e-3),
                             "acceptance": got[med] / N,
                             "ms_spread": [min(ms), max(ms)]})
    # speedup over K = 1 per (N, mode)
    for r in rows:
        k1 = [x for x in rows if x["N"] == r["N"] and x["mode"] == r["mode"] and x["K"] == 1]
        r["vs_k1"] = r["updates_per_s"] / k1[0]["updates_per_s"] if k1 else None
    return rows


# ------------------------------------------------------------------ kernels
def run_kernels(a):
    """Microbenchmarks of single kernels, timed with CUDA events: the batched
    per-call ratio (Eq. 3 through a queue of k = 128 moves; HBM-bound), the
    per-call fp64 flush (Eq. 4) emulated on the tensor cores and on the fp64
    units, the split-bf16 x3 tensor-core GEMM, and the fp64 recompute."""
    import torch
    from paper_1708_00744_b300 import inputs
    from paper_1708_00744_b300.qmcdu import Walkers, qmcdu_gemm_bf16x3
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {}

    def timed(fn, reps, stream, flush=True):
        ms = []
        for _ in range(reps):
            if flush:
                flush_buf.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    # ratio: walkers of N = 512 with 128 queued moves; each ratio reads
    # A^{-1}[:, j], the proposal and the 2 x 128 queue rows of every walker.
    # fp64 does one FMA per 8 bytes read, above B300's fp64 ridge (1.2 TFLOP/s
    # over 6.5 TB/s = 0.19 flop/B): ALU-bound. fp32 halves the bytes and has
    # 64x the ALU rate: HBM-bound.
    N, K, B, k = 512, 256, a.kernels_batch, 128
    for prec in ("fp64", "fp32"):
        es = 8 if prec == "fp64" else 4
        W = Walkers(N, K, prec, B, stream=st)
        W.load_walkers(0, B, seeds=[a.seed + b for b in range(B)])
        r = torch.zeros(B, dtype=torch.float64, device="cuda")
        ones = np.ones(B, dtype=np.uint8)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(a.seed)
        torch.cuda.synchronize()
        for m in range(k):
            # a fresh random row per move (a repeated row would make A singular),
            # drawn on the handle's stream so that the ratio kernel reads it after
            with torch.cuda.stream(st):
                v = torch.randn(B, N, dtype=torch.float64, device="cuda", generator=gen)
            W.ratio(np.full(B, m, dtype=np.int32), v, r)
            W.accept(ones)
        with torch.cuda.stream(st):
            v = torch.randn(B, N, dtype=torch.float64, device="cuda", generator=gen)
        elec = np.full(B, N - 1, dtype=np.int32)
        W.ratio(elec, v, r)
        ms = timed(lambda: W.ratio(elec, v, r), 20, st)
        W.sync()
        W.close()
        bytes_per = (2 * k + 1) * N * es * B + k * k * 8 * B   # rows, column, Kinv
        flops = 2.0 * ((2 * k + 1) * N + 2 * k * k) * B
        out["ratio_" + prec] = {"walkers": B, "N": N, "k": k, "ms": ms,
                                "algorithmic_bytes": bytes_per,
                                "GB_per_s": bytes_per / (ms * 1e-3) / 1e9,
                                "TFLOP_per_s": flops / (ms * 1e-3) / 1e12,
                                "note": "one qmcdu_ratio call (three kernels) with its host "
                                        "argument copy"}
    # flush of Eq. 4 through the per-call API: one fp64 walker of N = 2048,
    # K = 32, with k = 31 accepted moves queued (refilled, untimed, before each
    # call); the contraction emulated on the tensor cores vs the fp64 units
    Nf, Kf = 2048, 32
    A0h = np.asarray(inputs.initial_matrix(inputs.walker_seed(a.seed + 11, 0), Nf))
    A0 = torch.from_numpy(A0h).cuda()
    for mode, name in ((2, "flush_fp64_emulated"), (1, "flush_fp64_units")):
        W = Walkers(Nf, Kf, "fp64", 1, stream=st)
        W.set_option("fp64_flush", mode)
        W.set_matrix(A0h[None])
        r = torch.zeros(1, dtype=torch.float64, device="cuda")
        gen = torch.Generator(device="cuda")
        gen.manual_seed(a.seed + 1)
        ms_l = []
        for rep in range(6):
            for m in range(Kf - 1):     # K accepts would flush inside the last accept
                j = m + Kf * rep          # distinct electrons, each row still the initial one
                with torch.cuda.stream(st):
                    # a proposal close to the current row keeps the ratio O(1)
                    v = A0[j:j + 1] + 0.05 * torch.randn(1, Nf, dtype=torch.float64, device="cuda",
                                                         generator=gen)
                W.ratio(np.array([j], dtype=np.int32), v, r)
                W.accept(np.ones(1, dtype=np.uint8))
            flush_buf.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            W.flush()
            e1.record(st)
            e1.synchronize()
            if rep > 0:
                ms_l.append(e0.elapsed_time(e1))
        W.sync()
        W.close()
        ms = float(np.median(ms_l))
        fl = 4.0 * Nf * Nf * (Kf - 1)
        out[name] = {"N": Nf, "k": Kf - 1, "ms": ms, "fp64_equivalent_TFLOP_per_s": fl / (ms * 1e-3) / 1e12,
                     "note": "one qmcdu_flush call: W = P Kinv (fp64 GEMM) and the two N x N x k "
                             "contractions"}
    # split-bf16 x3 GEMM on tcgen05: C = A B', 4096^3
    M = Nn = Kk = 4096
    Ag = torch.randn(M, Kk, device="cuda")
    Bg = torch.randn(Nn, Kk, device="cuda")
    Cg = torch.zeros(M, Nn, device="cuda")
    cur = torch.cuda.current_stream()
    qmcdu_gemm_bf16x3(Ag, Bg, Cg)
    ms = timed(lambda: qmcdu_gemm_bf16x3(Ag, Bg, Cg), 10, cur)
    fl = 2.0 * M * Nn * Kk
    out["gemm_bf16x3"] = {"M": M, "N": Nn, "K": Kk, "ms": ms,
                          "fp32_equivalent_TFLOP_per_s": fl / (ms * 1e-3) / 1e12,
                          "bf16_tensor_TFLOP_per_s": 3 * fl / (ms * 1e-3) / 1e12}
    del Ag, Bg, Cg
    # fp64 recompute (Gauss-Jordan with partial pivoting) of 8 walkers of N = 2048
    Nr, Br = 2048, 8
    W = Walkers(Nr, 32, "fp64", Br, stream=st)
    W.load_walkers(0, Br, seeds=[a.seed + 7 + b for b in range(Br)])
    W.recompute()
    ms = timed(lambda: W.recompute(), 5, st)
    W.sync()
    W.close()
    out["recompute_fp64"] = {"walkers": Br, "N": Nr, "ms": ms,
                             "TFLOP_per_s": 2.0 * Nr ** 3 * Br / (ms * 1e-3) / 1e12}
    return out


# ------------------------------------------------------------------ serving
def serve_once(a, trace, plain, until, budget):
    """One run of the library's serving loop over `trace`, stopped when the
    server clock passes `until` (< 0: when every request has finished). plain:
    the one-walker-per-launch fp64 path (one slot per pool, one walker
    resident, one pool in flight, each walker's sweep on the whole GPU)."""
    from paper_1708_00744_b300.qmcdu import Server
    if plain:
        classes = [dict(N=c["N"], slots=1, group_ctas=148) for c in a.classes]
        srv = Server(classes, precision="fp64", sigma=a.sigma, recompute_every=10,
                     hbm_budget=budget, max_walkers=1, max_inflight=1)
    else:
        classes = [dict(N=c["N"], slots=c["batch"]) for c in a.classes]
        srv = Server(classes, precision=a.precision, sigma=a.sigma, recompute_every=10,
                     hbm_budget=budget)
    srv.submit(trace)
    srv.run(until_s=until)
    st = srv.stats()
    per_class = {str(c["N"]): srv.class_stats(i) for i, c in enumerate(a.classes)}
    res = srv.results()
    srv.close()
    return st, res, per_class


def serve_summary(st, res, per_class, seconds):
    ok = [r for r in res if r["status"] == 0]
    return {"seconds": seconds, "updates_per_s": st["accepted"] / seconds,
            "proposals_per_s": st["proposals"] / seconds,
            "walker_sweeps_per_s": st["walker_sweeps"] / seconds,
            "acceptance": st["accepted"] / max(1.0, st["proposals"]),
            "sweep_latency_ms": {"p50": st["sweep_ms_p50"], "p99": st["sweep_ms_p99"]},
            "request_latency_s": {"p50": st["request_s_p50"], "p99": st["request_s_p99"]},
            "admission_wait_s": {"p50": st["wait_s_p50"], "p99": st["wait_s_p99"]},
            "requests": {"arrived": int(st["submitted"]), "finished": len(ok),
                         "failed": int(st["failed"])},
            "per_class": {n: {"walker_sweeps": int(v["walker_sweeps"]),
                              "sweep_ms_p50": v["sweep_ms_p50"], "sweep_ms_p99": v["sweep_ms_p99"],
                              "finished": int(v["finished"]), "request_s_p50": v["request_s_p50"],
                              "request_s_p99": v["request_s_p99"]}
                          for n, v in per_class.items()},
            "peak_gb_held": st["peak_bytes"] / 1e9, "pools_created": int(st["pools_created"]),
            "pools_destroyed": int(st["pools_destroyed"]), "rounds": int(st["rounds"]),
            "max_walkers_resident": int(st["max_resident"]),
            "max_pools_in_flight": int(st["max_inflight"]),
            "walker_sweeps_in_mixed_rounds": int(st["mixed_walker_sweeps"]),
            "max_drift_logdet": max([r["drift_logdet"] for r in ok] or [0.0]),
            "max_drift_inverse": max([r["drift_inverse"] for r in ok] or [0.0])}


def run_serve(a):
    import torch
    from paper_1708_00744_b300 import inputs
    torch.cuda.set_device(0)
    budget = int(a.budget_gb * 1e9)
    sizes = tuple(c["N"] for c in a.classes)
    # warm-up (untimed): one request of every class through a server of its own
    warm = [dict(id=i, seed=99 + i, N=n, nsweeps=1, arrival_s=0.0) for i, n in enumerate(sizes)]
    for plain in (False, True):
        serve_once(a, warm, plain, -1.0, budget)
    # capacity: makespan of a backlog of the same size mix, all present at t = 0
    backlog = [dict(r, arrival_s=0.0) for r in
               inputs.serving_trace(a.seed + 7, 1000.0, 1.0, sizes=sizes, nsweeps=20,
                                    max_requests=48)]
    st_c, res_c, pc_c = serve_once(a, backlog, False, -1.0, budget)
    makespan = st_c["last_round_end_s"]
    capacity = len(backlog) / makespan
    # the offered load (Poisson at --rate) for --window seconds; the loop stops there
    trace = inputs.serving_trace(a.seed, a.rate, a.window, sizes=sizes, nsweeps=20)
    clocks = ClockSampler(0)
    clocks.start()
    st, res, pc = serve_once(a, trace, False, a.window, budget)
    clk = clocks.stop()
    batched = serve_summary(st, res, pc, a.window)
    st_p, res_p, pc_p = serve_once(a, trace, True, a.window, budget)
    plain = serve_summary(st_p, res_p, pc_p, a.window)
    # below capacity: 70 % of it, every request served to the end
    low_rate = 0.7 * capacity
    trace_lo = inputs.serving_trace(a.seed + 1, low_rate, a.window, sizes=sizes, nsweeps=20)
    st_l, res_l, pc_l = serve_once(a, trace_lo, False, -1.0, budget)
    below = dict(serve_summary(st_l, res_l, pc_l, st_l["last_round_end_s"]),
                 offered_rate_per_s=low_rate)
    sat = dict(serve_summary(st_c, res_c, pc_c, makespan), requests_per_s=capacity)
    return dict(batched=batched, plain=plain, below=below, saturation=sat, clocks=clk,
                capacity_req_s=capacity, requests_in_trace=len(trace))


def roofline_for(a, res):
    """Dominant kernel: the persistent sweep kernel (one launch per sweep and
    size class). Its algorithmic work is the Eq. 4 flush, 4 N^2 flops per
    accepted move, plus the ratio dot products, 2 (2k + 2) N flops per proposal
    with k the mean queue length (about K/2 at high acceptance), and the W-panel
    append, 4 k N flops per accepted move."""
    profs = res["prof"] or []
    if not profs:
        return None
    flops, ms, launches = 0.0, 0.0, 0
    acc_frac = res["accepted"] / max(1.0, res["nprop"] * a.steps * max(1, a.gpus))
    for c, prof in zip(a.classes, profs):
        N, K = c["N"], c["K"]
        props = a.steps * a.sweeps_per_step * N * c["batch"]
        acc = props * acc_frac
        kbar = 0.0 if K == 1 else (K - 1) / 2.0
        flops += 4.0 * N * N * acc + 2.0 * (2 * kbar + 2) * N * props + 4.0 * kbar * N * acc
        ms = max(ms, prof.get("sweep_kernel_ms", 0.0))
        launches += int(prof.get("sweep_kernels", 0))
    if not launches or ms <= 0:
        return None
    nlaunch_per_class = launches / len(profs)
    achieved = flops / (ms * 1e-3) / 1e12
    key = "%s:%s" % (source_hash("kernels_sweep.cu"), a.workload)
    kinds = res.get("flush_kinds") or []
    out = {"kernel": "sweep_kernel (persistent fused sweep: Eq. 3 ratios, bordered append, Eq. 4 flush)",
           "achieved": achieved, "unit": "TFLOP/s", "traffic": NCU_TRAFFIC.get(key),
           "flops_per_launch": flops / nlaunch_per_class, "launches": launches,
           "avg_launch_ms": ms / nlaunch_per_class,
           "share_of_step": ms / res["total_ms"] if res["total_ms"] else None}
    if a.precision == "fp64" and kinds and all(k == OZ_FLUSH_KIND for k in kinds):
        # the flush's fp64 contraction runs on the tensor cores as OZ_PRODUCTS
        # fp16 slice products per fp64 product: its ceiling is the measured
        # 16-bit tensor rate / OZ_PRODUCTS
        bf16 = measured_peaks().get("bf16_tflops_sustained")
        src_ = "measured bf16 sustained (MEASURED_PEAKS.json) / %d fp16 slice products (fp16 and bf16 share the tensor rate)" % OZ_PRODUCTS
        if not bf16:
            bf16, src_ = 1400.0, "fallback bf16 sustained 1.4 PFLOP/s / %d slice products" % OZ_PRODUCTS
        peak = bf16 / OZ_PRODUCTS
        out.update(bound="tensor", peak=peak, frac=achieved / peak, peak_source=src_,
                   unit="TFLOP/s (fp64-equivalent)",
                   fp64_units_frac=achieved / FP64_PEAK_TFLOPS)
    else:
        peak = FP64_PEAK_TFLOPS if a.precision == "fp64" else FP32_PEAK_TFLOPS
        out.update(bound="alu", peak=peak, frac=achieved / peak,
                   peak_source="derived: 148 SMs x %s FMA/clk x 2 x 2032 MHz"
                               % ("2 FP64" if a.precision == "fp64" else "128 FP32"))
    return out


def k1_roofline(a, k1):
    """K = 1's sweep kernel (Sherman-Morrison, Eq. 2, on the fp64 units):
    4 N^2 flops per accepted move plus the ratio's 2 x 2 N per proposal,
    against the fp64 units' peak."""
    prof = k1.get("prof") or {}
    ms = prof.get("sweep_kernel_ms", 0.0)
    if ms <= 0:
        return None
    N = a.N
    props = a.k1_steps * a.sweeps_per_step * N * a.classes[0]["batch"]
    flops = 4.0 * N * N * k1["accepted"] + 4.0 * N * props
    achieved = flops / (ms * 1e-3) / 1e12
    return {"kernel": "sweep_kernel, K = 1", "bound": "alu", "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "peak_source": "derived: 148 SMs x 2 FP64 FMA/clk x 2 x 2032 MHz"}


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    a.gpus = world if world > 1 else a.gpus
    metric = "accepted-move updates/s"

    if a.impl == "reference":
        if rank != 0:
            return
        # the K the autotuner settles on for this workload, from its host-side
        # rule (the reference arm runs before, and without, any GPU work)
        from paper_1708_00744_b300 import autotune
        K = autotune.default_K(a.N, a.precision) if a.K == "auto" else int(a.K)
        a.K = str(K)
        # every host core (the oracle's loops over independent elements run on
        # OpenMP threads); each step a bounded sample sized from a one-core
        # estimate, so that the run ends within about a minute
        nm = cpu_sample_size(a, K, seconds=max(4.0, 120.0 / max(1, a.steps + a.warmup)))
        vals, used = [], 1
        for it in range(a.warmup + a.steps):
            acc, dt, used = cpu_oracle_sample(a, nm, K, threads=0)
            if it >= a.warmup:
                vals.append(acc / dt)
        v = float(np.median(vals))
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "updates/s",
                "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
                "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                "config": config(a, 1),
                "cpu_baseline": {"value": v, "unit": "updates/s", "cores": used, "kind": "oracle",
                                 "host": host_cpu(),
                                 "sample": "first %d proposals of sweep 0 of one N=%d walker, K=%d, "
                                           "update work timed by the oracle after its setup inverse; "
                                           "median of %d steps" % (nm, a.N, K, a.steps)},
                "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if a.workload in ("ksweep", "kernels"):
        if world > 1 and rank != 0:
            return
        clocks = ClockSampler(0)
        clocks.start()
        if a.workload == "ksweep":
            rows = run_ksweep(a)
            best = max((r for r in rows if r["N"] == 2048 and r["mode"] == "sigma=0.1"),
                       key=lambda r: r["updates_per_s"], default=None)
            extra = {"table": rows}
            value = best["updates_per_s"] if best else None
        else:
            k = run_kernels(a)
            extra = {"kernels": k}
            value = k["ratio_fp32"]["GB_per_s"]
            metric = "ratio (fp32 walkers) HBM GB/s"
        line = {"metric": metric, "value": value,
                "unit": "updates/s" if a.workload == "ksweep" else "GB/s", "n_gpus": 1,
                "steps": a.reps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(a, 1),
                "clocks": clocks.stop()}
        line.update(extra)
        print(json.dumps(line))
        return

    if a.workload == "serve":
        if world > 1 and rank != 0:
            return                     # one serving loop per GPU: run it on rank 0's
        r = run_serve(a)
        b = r["batched"]
        line = {"metric": metric, "value": b["updates_per_s"], "unit": "updates/s",
                "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": a.window * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "f32 (bf16x3 flush)"}[a.precision],
                "data": "synthetic", "config": config(a, 1),
                "serving": dict(b, offered_rate_per_s=a.rate, requests_in_trace=r["requests_in_trace"],
                                capacity_req_per_s=r["capacity_req_s"]),
                "plain_one_walker_fp64": r["plain"],
                "saturation_backlog_48": r["saturation"],
                "below_capacity": r["below"],
                "speedup_vs_plain": b["updates_per_s"] / max(1e-9, r["plain"]["updates_per_s"]),
                "roofline": None, "clocks": r["clocks"],
                "e2e": {"value": b["updates_per_s"], "unit": "updates/s",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": None,
                        "note": "requests carry keys; matrices are drawn on the device"}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(a, rank, world, local_rank)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    total_s = res["total_ms"] * 1e-3
    value = res["accepted"] / total_s
    line = {"metric": metric, "value": value, "unit": "updates/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": res["total_ms"] / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "f32 (bf16x3 flush)"}[a.precision],
            "data": "synthetic",
            "config": config(a, a.gpus)}
    line["accepted_moves"] = res["accepted"]
    line["acceptance"] = res["accepted"] / (res["nprop"] * a.steps * a.gpus)
    line["graph_replay"] = {"value": res["graph_accepted"] / (res["graph_ms"] * 1e-3),
                            "ms_per_step": res["graph_ms"] / a.steps}
    if res["tuned"]:
        line["autotune"] = res["tuned"]
    if res["k1"]:
        k1v = res["k1"]["accepted"] / (res["k1"]["ms"] * 1e-3)
        line["k1_sherman_morrison"] = {"value": k1v, "unit": "updates/s",
                                       "ms_per_step": res["k1"]["ms"] / a.k1_steps,
                                       "roofline": k1_roofline(a, res["k1"])}
        line["speedup_vs_k1"] = value / k1v
    line["roofline"] = roofline_for(a, res)
    profs0 = res["prof"] or []
    if len(profs0) == 1 and profs0[0].get("sweep_times_ms"):
        st = np.asarray(profs0[0]["sweep_times_ms"])
        line["sweep_latency_ms"] = {"p50": float(np.percentile(st, 50)), "p99": float(np.percentile(st, 99)),
                                    "sweeps": int(st.size),
                                    "what": "device time of each persistent sweep launch (CUDA events), "
                                            "one sweep of the timed walker"}
    if res.get("drift") is not None:
        line["error"] = {"drift_logdet": float(res["drift"][0]), "drift_inverse": float(res["drift"][1]),
                         "what": "largest drift over the timed steps of the running log|det A| "
                                 "(absolute) and A^{-1} (Frobenius, relative) against the fp64 "
                                 "recompute that ends each step; element-wise parity with the CPU "
                                 "oracle at this configuration: tests/test_gpu_headline.py"}
    line["e2e"] = {"value": res["e2e_acc"] / res["e2e_s"], "unit": "updates/s",
                   "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]}
    profs = res["prof"] or []
    line["gpu_launches"] = int(sum(p.get("launches", 0) for p in profs))
    if len(profs) == 1:
        prof = profs[0]
        sweep_ms = prof.get("sweep_kernel_ms", 0.0)
        rec_ms = prof.get("recompute_ms", 0.0)
        line["breakdown_ms_per_step"] = {
            "sweep kernel": sweep_ms / a.steps,
            "recompute (fp64 Gauss-Jordan)": rec_ms / a.steps,
            "proposal draws + log-det + launches": (res["total_ms"] - sweep_ms - rec_ms) / a.steps}
        nprop = a.steps * a.sweeps_per_step * a.N
        line["sweep_phases_us_per_proposal"] = {
            k[6:-3]: v * 1000.0 / nprop for k, v in prof.items()
            if k.startswith("sweep_") and k.endswith("_ms") and k != "sweep_kernel_ms"
            and isinstance(v, float)}
    line["clocks"] = res["clocks"]
    if a.gpus == 1:
        K = a.classes[0]["K"]
        nm = cpu_sample_size(a, K)
        acc, dt, _ = cpu_oracle_sample(a, nm, K, threads=1)
        nall = a.N
        acc_all, dt_all, used = cpu_oracle_sample(a, nall, K, threads=0)
        line["cpu_baseline"] = {
            "value": acc / dt, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": "first %d proposals of sweep 0 of one walker (N=%d, K=%d): %.1f s of update work "
                      "on one thread, timed by the oracle after its setup inverse" % (nm, a.N, K, dt),
            "all_cores": {"value": acc_all / dt_all, "cores": used,
                          "sample": "the whole sweep 0 (%d proposals), %.1f s" % (nall, dt_all)},
            "host": host_cpu()}
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
