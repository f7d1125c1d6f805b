#!/usr/bin/env python
"""Benchmark of the delayed Slater-determinant update on one B300.

Metric: accepted-move updates per second (the paper's Monte Carlo column
updates per second over complete sweeps, Sec. III), whole job.

Workload (default): one walker of N = 2048 electrons in fp64, A_ij ~ N(0,1),
proposal v = a_j + 0.1 g (DMC-like acceptance), delay K = 64. A step is ten
full Metropolis sweeps followed by the fp64 recompute of A^{-1} and log|det A|
(the recompute every ten sweeps of the workload). Inputs are synthetic
(seeded Philox draws). The same workload also runs with K = 1
(Sherman-Morrison on the same GPU) for the speedup.

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
FP32_PEAK_TFLOPS = SMS * 128 * 2 * SM_MHZ * 1e6 / 1e12    # 77.0
HBM_PEAK_FALLBACK_GBS = 6400.0

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the flush kernels,
# from one ncu capture; keyed by the sha256 of kernels_gemm.cu at capture time.
NCU_TRAFFIC = {}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=2048)
    p.add_argument("--K", type=int, default=64)
    p.add_argument("--batch", type=int, default=1)
    p.add_argument("--sigma", type=float, default=0.1)
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--sweeps-per-step", type=int, default=10)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--k1-steps", type=int, default=1, help="steps of the K=1 comparison")
    p.add_argument("--cpu-moves", type=int, default=-1,
                   help="proposals in the CPU-oracle sample (default: sized for ~15 s)")
    return p.parse_args()


def workload_name(a):
    return ("%d walker(s) x N=%d %s, K=%d, sigma=%g, %d sweeps + fp64 recompute per step"
            % (a.batch, a.N, a.precision, a.K, a.sigma, a.sweeps_per_step))


def config(a, world):
    return {"workload": workload_name(a), "N": a.N, "K": a.K, "walkers_per_gpu": a.batch,
            "walkers": a.batch * world, "precision": a.precision, "sigma": a.sigma,
            "sweeps_per_step": a.sweeps_per_step, "recompute_every_sweeps": a.sweeps_per_step,
            "l2": "flushed between timed steps (256 MB write)", "parallelism": "walkers x %d" % world}


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_sample(a, max_moves):
    """The fp64 CPU oracle (delayed look-ahead + Woodbury with the same K; K = 1:
    Sherman-Morrison) on the first `max_moves` proposals of sweep 0 of one
    walker. The oracle's setup (an O(N^3) LU inverse of the starting matrix) is
    timed by a zero-proposal run and subtracted, so that the figure is the update
    throughput. Returns (accepted, seconds of update work, seconds of setup)."""
    import oracle
    from paper_1708_00744_b300 import inputs
    A = inputs.initial_matrix(a.seed, a.N)
    G = inputs.proposal_gaussians(a.seed, 0, a.N)[None]
    U = inputs.metropolis_uniforms(a.seed, 0, a.N)[None]
    method = oracle.SM if a.K == 1 else oracle.DELAYED
    oracle.build()
    t0 = time.perf_counter()
    oracle.sweeps(method, A, G, U, a.sigma, K=a.K, max_moves=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    out = oracle.sweeps(method, A, G, U, a.sigma, K=a.K, max_moves=max_moves)
    dt = time.perf_counter() - t0 - t_setup
    acc = int(out["accepted"][0, :max_moves].sum())
    return acc, max(dt, 1e-9), t_setup


def cpu_sample_size(a, seconds=15.0):
    if a.cpu_moves > 0:
        return min(a.cpu_moves, a.N)
    # about 2 N^2 K flop-equivalents per K accepted proposals at ~1 GFLOP/s
    per_move = 4.0 * a.N * a.N / 1.0e9 + 2.0 * a.N * (2 * a.K + 1) / 1.0e9
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
    from paper_1708_00744_b300 import inputs
    from paper_1708_00744_b300.qmcdu import Walkers

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    dist = None
    if world > 1:
        import torch.distributed as dist
    N, B, nsw = a.N, a.batch, a.sweeps_per_step
    base = a.seed + rank * B
    A0 = np.stack([inputs.initial_matrix(inputs.walker_seed(base, b), N) for b in range(B)])
    A0_pinned = torch.from_numpy(A0).pin_memory()
    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    acc_dev = torch.zeros(nsw, B, N, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def time_steps(W, K, nsteps, nwarm, sweep0, profile=False):
        """Device-timed steps on resident state; returns (ms list, accepted, profile)."""
        sweep = sweep0
        for _ in range(nwarm):
            for s in range(nsw):
                W.sweep(base, sweep, a.sigma)
                sweep += 1
            W.recompute()
        barrier()
        if profile:
            W.profile_enable(True)
        ms, accepted = [], 0
        for _ in range(nsteps):
            flush_buf.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for s in range(nsw):
                W.sweep(base, sweep, a.sigma, accepted_out=acc_dev[s])
                sweep += 1
            W.recompute()
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            accepted += int(acc_dev.sum().item())
        prof = W.profile_read() if profile else None
        if profile:
            W.profile_enable(False)
        return ms, accepted, prof, sweep

    W = Walkers(N, a.K, a.precision, B, stream=stream)
    W.set_matrix(A0_pinned)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms, accepted, prof, sweep_next = time_steps(W, a.K, a.steps, a.warmup, 0, profile=True)
    clk = clocks.stop()

    # end to end through the public API with host buffers: upload A from pinned
    # host memory, run the step, read the accept masks and log-dets back.
    h_logabs = torch.zeros(B, dtype=torch.float64).pin_memory()
    h_sign = torch.zeros(B, dtype=torch.int32).pin_memory()
    h_acc = torch.zeros(nsw, B, N, dtype=torch.uint8).pin_memory()
    e2e_s, e2e_acc = [], 0
    for it in range(a.warmup + a.steps):
        barrier()
        t0 = time.perf_counter()
        W.set_matrix(A0_pinned)
        for s in range(nsw):
            W.sweep(base, s, a.sigma, accepted_out=acc_dev[s])
        W.recompute()
        h_acc.copy_(acc_dev, non_blocking=True)
        W.logdet(h_logabs, h_sign)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if it >= a.warmup:
            e2e_s.append(dt)
            e2e_acc += int(h_acc.sum())
    W.close()

    # K = 1 (Sherman-Morrison) on the same GPU, same workload
    k1 = None
    if a.K != 1 and a.k1_steps > 0:
        W1 = Walkers(N, 1, a.precision, B, stream=stream)
        W1.set_matrix(A0_pinned)
        ms1, acc1, _, _ = time_steps(W1, 1, a.k1_steps, 1, 0)
        W1.close()
        k1 = (ms1, acc1)

    def allmax(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def allsum(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    total_ms = allmax(sum(ms))
    total_acc = allsum(accepted)
    e2e_t = allmax(sum(e2e_s))
    e2e_total_acc = allsum(e2e_acc)
    res = dict(ms=ms, total_ms=total_ms, accepted=total_acc, prof=prof, clocks=clk,
               e2e_s=e2e_t, e2e_acc=e2e_total_acc, k1=None)
    if k1 is not None:
        res["k1"] = dict(ms=allmax(sum(k1[0])), accepted=allsum(k1[1]))
    return res


def roofline_for(a, res):
    """Dominant kernel: the persistent sweep kernel (one launch per sweep). Its
    algorithmic work is the Eq. 4 flush, 4 N^2 flops per accepted move, plus
    the ratio dot products, 2 (2k + 2) N flops per proposal with k the mean
    queue length (about K/2 at high acceptance), and the W-panel append,
    4 k N flops per accepted move."""
    prof = res["prof"] or {}
    N, K = a.N, a.K
    acc_per_gpu = res["accepted"] / max(1, a.gpus)
    prop_per_gpu = a.steps * a.sweeps_per_step * a.N * a.batch
    kbar = 0.0 if K == 1 else (K - 1) / 2.0
    flops = 4.0 * N * N * acc_per_gpu + 2.0 * (2 * kbar + 2) * N * prop_per_gpu + 4.0 * kbar * N * acc_per_gpu
    launches = prof.get("sweep_kernels", 0)
    ms = prof.get("sweep_kernel_ms", 0.0)
    if not launches or ms <= 0:
        return None
    achieved = flops / launches / (ms / launches * 1e-3) / 1e12
    peak = FP64_PEAK_TFLOPS if a.precision == "fp64" else FP32_PEAK_TFLOPS
    key = source_hash("kernels_sweep.cu")
    return {"kernel": "sweep_kernel (persistent fused sweep: Eq. 3 ratios, bordered append, Eq. 4 flush)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(key),
            "peak_source": "derived: 148 SMs x %s FMA/clk x 2 x 2032 MHz"
                           % ("2 FP64" if a.precision == "fp64" else "128 FP32"),
            "flops_per_launch": flops / launches, "launches": launches,
            "avg_launch_ms": ms / launches,
            "share_of_step": ms / res["total_ms"] if res["total_ms"] else None}


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
        nm = cpu_sample_size(a, seconds=max(2.0, 60.0 / max(1, a.steps + a.warmup)))
        vals = []
        for it in range(a.warmup + a.steps):
            acc, dt, _ = cpu_oracle_sample(a, nm)
            if it >= a.warmup:
                vals.append(acc / dt)
        v = float(np.median(vals))
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "updates/s",
                "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
                "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                "config": config(a, 1),
                "cpu_baseline": {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                                 "sample": "first %d proposals of sweep 0, one walker "
                                           "(setup inverse timed apart and excluded)" % nm},
                "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
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
            "dtype": "f64" if a.precision == "fp64" else "f32", "data": "synthetic",
            "config": config(a, a.gpus)}
    line["accepted_moves"] = res["accepted"]
    line["acceptance"] = res["accepted"] / (a.steps * a.sweeps_per_step * a.N * a.batch * a.gpus)
    if res["k1"]:
        k1v = res["k1"]["accepted"] / (res["k1"]["ms"] * 1e-3)
        line["k1_sherman_morrison"] = {"value": k1v, "unit": "updates/s",
                                       "ms_per_step": res["k1"]["ms"] / a.k1_steps}
        line["speedup_vs_k1"] = value / k1v
    line["roofline"] = roofline_for(a, res)
    line["e2e"] = {"value": res["e2e_acc"] / res["e2e_s"], "unit": "updates/s",
                   "h2d_bytes_per_step": a.batch * a.N * a.N * 8,
                   "d2h_bytes_per_step": a.sweeps_per_step * a.batch * a.N + a.batch * 12}
    prof = res["prof"] or {}
    line["gpu_launches"] = int(prof.get("launches", 0))
    sweep_ms = prof.get("sweep_kernel_ms", 0.0)
    rec_ms = prof.get("recompute_ms", 0.0)
    line["breakdown_ms_per_step"] = {
        "sweep kernel": sweep_ms / a.steps,
        "recompute (fp64 Gauss-Jordan)": rec_ms / a.steps,
        "proposal draws + log-det + launches": (res["total_ms"] - sweep_ms - rec_ms) / a.steps}
    nprop = a.steps * a.sweeps_per_step * a.N
    line["sweep_phases_us_per_proposal"] = {
        k[6:-3]: v * 1000.0 / nprop for k, v in prof.items()
        if k.startswith("sweep_") and k.endswith("_ms") and k != "sweep_kernel_ms"}
    line["clocks"] = res["clocks"]
    if a.gpus == 1:
        nm = cpu_sample_size(a)
        acc, dt, t_setup = cpu_oracle_sample(a, nm)
        line["cpu_baseline"] = {"value": acc / dt, "unit": "updates/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "first %d proposals of sweep 0 of one walker (N=%d, K=%d): "
                                          "%.1f s of updates; the %.1f s setup inverse excluded"
                                          % (nm, a.N, a.K, dt, t_setup)}
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
