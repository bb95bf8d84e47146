"""Benchmark of the GB300 tiled Cholesky library; prints ONE JSON line.

Default workload (one "step" = one full factorization A = L L^T through the
C ABI): FP64, n = 65536, squared-exponential covariance of n points uniform in
the unit square (lengthscale 0.1, nugget 1e-2, seed 1), dataflow schedule with
the priority queue, SYRK/GEMM on the tensor cores with binary64 accuracy
(exact bf16 slicing; --flags 0 selects the DFMA engine).  Metric: TFLOP/s
counting n^3/3 flops per factorization.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 65536] [--nb 128]
                  [--schedule dataflow|fork_join|fork_join_naive]
                  [--workload fp64|mixed|batched|serve] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): a single factorization does not shard,
so N ranks run N independent replicas of the same workload; value = all ranks'
flops / the slowest rank's time (weak scaling).

--impl reference times the CPU oracle (the paper's task-asynchronous tiled
algorithm over OpenMP task dependencies, plain C tile loops) on the host cores,
each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Cholesky TFLOP/s (n³/3) vs peak, FP64 vs mixed; served solves/s with p50/p99 latency"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 on GB300 runs on the CUDA cores (tcgen05 has no FP64 kind): 152 SMs x
# 2 DFMA lanes per clock per SM x 2 flop x 2.07 GHz maximum SM clock = 1.26
# TFLOP/s, the 1.25 TFLOP/s nominal figure.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--n", type=int, default=65536)
    p.add_argument("--nb", type=int, default=0)
    p.add_argument("--schedule", default="dataflow")
    p.add_argument("--workload", default="fp64", choices=["fp64", "mixed", "batched", "serve", "sweep"])
    p.add_argument("--sweep-nb", default="")
    p.add_argument("--sweep-sched", default="")
    p.add_argument("--sweep-engine", default="", help="sweep: tc (tensor-core FP64 engine), simt (DFMA engine)")
    p.add_argument("--noop", action="store_true")
    p.add_argument("--trace", action="store_true")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--tc-min-order", type=int, default=0,
                   help="batched FP64: order above which a matrix runs on the tensor cores (0 = 1024)")
    p.add_argument("--serve-requests", type=int, default=120)
    p.add_argument("--serve-rates", default="20,80,320")
    p.add_argument("--serve-nmax", type=int, default=8192)
    p.add_argument("--serve-slots", type=int, default=4)
    p.add_argument("--serve-budget-gb", type=float, default=64.0)
    p.add_argument("--precision", default="fp32")
    p.add_argument("--nugget", type=float, default=1e-2, help="SE covariance nugget (mixed workload)")
    p.add_argument("--no-fp64-compare", action="store_true",
                   help="mixed workload: skip the FP64 factor+solve time-to-solution comparison")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    # default: FP64 SYRK/GEMM on the tensor cores (CHOL_FLAG_FP64_TC = 16) with the
    # priority ready queue (CHOL_FLAG_PRIORITY = 2); --flags 0 selects the DFMA engine
    p.add_argument("--flags", type=int, default=-1)
    p.add_argument("--num-ctas", type=int, default=0)
    return p.parse_args()


# ------------------------------------------------------------------ distributed
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
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
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------ CPU oracle baseline
def cpu_oracle_sample(target_s: float = 15.0, nmax: int = 8192, nb: int = 256):
    """Time the oracle's OpenMP-task tiled factorization on all host cores on
    an SE-covariance matrix whose order is chosen for about target_s seconds."""
    import oracle
    import seeded_inputs as si
    threads = os.cpu_count() or 1
    n0 = 1024
    A = si.se_covariance(n0, seed=1, nugget=1e-2)
    t = time.perf_counter()
    oracle.potrf_tiled_tasks(A, min(nb, n0), nthreads=threads)
    dt = time.perf_counter() - t
    rate = n0 ** 3 / 3 / max(dt, 1e-6)
    n = int((target_s * rate * 3) ** (1 / 3))
    n = max(n0, min(nmax, (n // 256) * 256))
    A = si.se_covariance(n, seed=1, nugget=1e-2)
    t = time.perf_counter()
    _, info = oracle.potrf_tiled_tasks(A, nb, nthreads=threads)
    dt = time.perf_counter() - t
    return {"value": n ** 3 / 3 / dt / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"oracle task-async tiled FP64 Cholesky (OpenMP depend, plain C tile loops), SE covariance "
                      f"n={n} nb={nb}, one factorization, {dt:.1f} s on {threads} host threads",
            "seconds": dt, "n": n, "info": info}


def run_reference(args, world, rank):
    """--impl reference: the oracle timed on the host cores."""
    if rank != 0:
        return
    import oracle
    import seeded_inputs as si
    threads = os.cpu_count() or 1
    # calibrate one sample size for ~15 s per step
    n0 = 1024
    A = si.se_covariance(n0, seed=1, nugget=1e-2)
    t = time.perf_counter()
    oracle.potrf_tiled_tasks(A, 256, nthreads=threads)
    rate = n0 ** 3 / 3 / max(time.perf_counter() - t, 1e-6)
    per_step = max(5.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    n = max(n0, min(8192, (int((per_step * rate * 3) ** (1 / 3)) // 256) * 256))
    A = si.se_covariance(n, seed=1, nugget=1e-2)
    for _ in range(args.warmup):
        oracle.potrf_tiled_tasks(A, 256, nthreads=threads)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.potrf_tiled_tasks(A, 256, nthreads=threads)
        times.append(time.perf_counter() - t)
    ms = 1e3 * statistics.mean(times)
    value = n ** 3 / 3 / (ms / 1e3) / 1e12
    sample = (f"oracle task-async tiled FP64 Cholesky (OpenMP depend) on {threads} host threads, SE covariance "
              f"n={n} nb=256 per step (bounded sample of the n={args.n} workload)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"fp64 tiled Cholesky, SE covariance (l=0.1, nugget 1e-2, seed 1), sample n={n}",
                       "n": n, "nb": 256},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ FP64 workload
def run_fp64(args, world, rank, local):
    import torch

    import paper_2606_11937_gb300 as chol
    import seeded_inputs as si

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    tc = bool(args.flags & chol.CHOL_FLAG_FP64_TC)
    nb = args.nb or (128 if tc else chol.chol_default_nb(n, "fp64"))
    A0 = si.se_covariance_torch(n, seed=1, lengthscale=0.1, nugget=1e-2, device=dev).T  # column-major view
    A = torch.empty_strided((n, n), (1, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    o = chol.opts(schedule=args.schedule, nb=nb, flags=args.flags, num_ctas=args.num_ctas,
                  stream=stream.cuda_stream)
    flops = n ** 3 / 3.0

    def step():
        A.copy_(A0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, info, st = chol.chol_factor_ex(A, o)
        e1.record(stream)
        e1.synchronize()
        assert info == 0, f"info={info}"
        return e0.elapsed_time(e1), st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    times, kernel_ms, launches = [], [], 0
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms, st = step()
            times.append(ms)
            kernel_ms.append(st.device_ms)
            launches += st.launches + 2  # + repack + unpack
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t_wall
    total_ms = allreduce_max(sum(times), world)
    ms_per_step = total_ms / args.steps
    value = world * flops / (ms_per_step / 1e3) / 1e12

    achieved = flops / (statistics.mean(kernel_ms) / 1e3) / 1e12
    if tc:
        # SYRK/GEMM run as 36 exact bf16 slice products per FP64 product: the
        # tensor-core ceiling of this engine, in FP64-equivalent flop/s, is the
        # measured sustained bf16 rate / 36 (POTRF/TRSM stay on the FP64 pipe).
        bf16 = measured_peaks().get("bf16_tflops_sustained", 1675.7)
        peak = bf16 / 36.0
        # DRAM bytes (read + write) of the dataflow kernel per task, measured
        # by ncu on a small case of the same configuration (n = 12288, nb = 128,
        # dataflow + priority: 24.70 GB read + 19.98 GB written over 152 096
        # tasks = 293.7 KB per task), scaled by this launch's task count.  Per-task
        # DRAM bytes grow with n as block columns outgrow L2 (250 KB at n = 8192,
        # 294 KB at 12288, 545 KB measured at 32768 with an earlier kernel), so
        # this is a lower bound.
        same_cfg = nb == 128 and args.schedule == "dataflow" and args.flags == 18 and args.num_ctas == 0
        m = -(-n // nb)
        traffic = 293.7e3 * (m * (m + 1) * (m + 2) // 6) if same_cfg else None
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": "ncu DRAM bytes per task at n=12288 scaled by the task count "
                                                      "(lower bound)" if traffic else None,
                "kernel": "df_kernel<OzBody>" if args.schedule == "dataflow" else "fork-join kernels",
                "peak_source": f"measured sustained bf16 {bf16} TFLOP/s / 36 slice products (FP64-equivalent)",
                "fp64_pipe_peak": FP64_PEAK_TFLOPS}
    else:
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "df_kernel<SimtBody<double>>" if args.schedule == "dataflow" else "fork-join kernels",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s FP64)"}

    e2e = None
    if not args.no_e2e:
        h = torch.empty_strided((n, n), (1, n), dtype=torch.float64, pin_memory=True)
        et = []
        for i in range(max(1, min(3, args.steps)) + 1):
            h.copy_(A0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            chol.chol_factor_host(h, o)
            dt = time.perf_counter() - t
            if i > 0:
                et.append(dt)
        e2e_s = allreduce_max(statistics.median(et), world)  # median: host-side copies vary with the machine's load
        # chol_factor_host moves, per block of 512 columns from j0, rows j0 .. n-1
        moved = sum((n - j0) * min(512, n - j0) * 8 for j0 in range(0, n, 512))
        e2e = {"value": world * flops / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": moved,
               "d2h_bytes_per_step": moved, "seconds_per_call": [round(x, 4) for x in et]}
        del h

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample()
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"fp64 tiled right-looking Cholesky n={n} nb={nb} {args.schedule} schedule, "
                                       + ("SYRK/GEMM on tcgen05 with binary64 accuracy (exact bf16 slicing), "
                                          if tc else "DFMA tile kernels, ")
                                       + "SE covariance (l=0.1, nugget 1e-2, seed 1)",
                           "engine": "fp64-tensor-core (exact slicing)" if tc else "fp64-dfma",
                           "n": n, "nb": nb, "schedule": args.schedule, "flops_per_step": flops,
                           "l2": f"inputs larger than L2 ({n * n * 8 / 1e9:.1f} GB matrix)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "wall_s": wall}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.flags < 0:
        args.flags = 18 if args.workload == "fp64" else 0
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "fp64":
        run_fp64(args, world, rank, local)
    else:
        import bench_workloads
        bench_workloads.run(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
