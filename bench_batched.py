"""Batched and served workloads of bench.py.

batched: 4096 SPD systems, n_i = floor(exp(U(ln 32, ln 2048))) (seed 3),
  A_i = G_i G_i^T / n_i + I with G_i i.i.d. N(0, 1) (per-matrix seed), one
  N(0, 1) right-hand side each; one step = one chol_batch_run (a single CUDA
  graph launch: repack, one persistent factor+solve kernel, unpack).  Under N
  ranks the matrices are split into contiguous shards (no collective on the
  data path).  value = TFLOP/s counting sum n_i^3 / 3.

serve: requests arrive as a Poisson process at rate lambda: n log-uniform in
  [64, 8192], 1-32 right-hand sides, 30% repeat right-hand sides against a
  resident factor, SE-covariance (nugget 1e-2) or G G^T / n + I inputs chosen
  by seed; the server has a fixed device-memory budget.  value = completed
  solves per second; p50/p99 latency per rate.
"""
from __future__ import annotations

import json
import math
import statistics
import threading
import time

import numpy as np

import bench
import seeded_inputs as si


def shard(count: int, world: int, rank: int) -> range:
    """Contiguous shard of `count` items for `rank` of `world` (sizes differ by <= 1)."""
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def _gram_torch(n: int, seed: int, dev):
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    G = torch.randn((n, n), dtype=torch.float32, device=dev, generator=g)
    A = (G @ G.T).double() / n
    A = torch.tril(A) + torch.tril(A, -1).T
    A.diagonal().add_(1.0)
    return A  # symmetric: its row-major bytes are its column-major bytes


def run_batched(args, world, rank, local):
    import torch

    import paper_2606_11937_gb300 as chol

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.backends.cuda.matmul.allow_tf32 = False
    count = args.batch_count
    ns_all = si.batched_sizes(count, seed=3, lo=32, hi=2048)
    idx = list(shard(count, world, rank))
    ns = [int(ns_all[i]) for i in idx]
    A0 = [_gram_torch(n, 4_000_000 + i, dev).T for n, i in zip(ns, idx)]
    B0 = []
    for n, i in zip(ns, idx):
        g = torch.Generator(device=dev)
        g.manual_seed(5_000_000 + i)
        B0.append(torch.randn(n, dtype=torch.float64, device=dev, generator=g))
    As = [torch.empty_strided((n, n), (1, n), dtype=torch.float64, device=dev) for n in ns]
    Bs = [torch.empty_like(b) for b in B0]
    prec = args.precision if args.precision in ("fp64", "fp32") else "fp64"
    cap = args.nb
    flags = args.flags & (chol.CHOL_FLAG_PRIORITY | chol.CHOL_FLAG_FP64_SIMT)
    tuned = None
    if cap == 0:
        # autotune on this batch, timed on the real plan: the tile-order cap of
        # the CUDA-core bodies, the engine split (matrices above a split order
        # on the tensor-core bodies, or every matrix on the CUDA cores) and
        # the priority order of the ready queue
        # (engine split: (flags, order above which a matrix goes to the tensor cores))
        engines = ([(0, 64), (0, 128), (0, 256), (0, 512), (0, 1024), (chol.CHOL_FLAG_FP64_SIMT, 0)]
                   if prec == "fp64" else [(0, 128), (0, 256), (0, 512), (0, 1024), (0, 2048)])
        trials = []
        for c in (32, 64, 128, 256):
            for e, tmin in engines:
                for pr in (0, chol.CHOL_FLAG_PRIORITY):
                    plan = chol.chol_batch_plan(ns, chol.opts(nb=c, precision=prec, flags=e | pr, tc_min_order=tmin))
                    for a, a0 in zip(As, A0):
                        a.copy_(a0)
                    for b, b0 in zip(Bs, B0):
                        b.copy_(b0)
                    plan.run(As, Bs)
                    trials.append({"cap": c, "flags": e | pr, "tc_min_order": tmin, "ms": plan.stats().device_ms})
                    plan.close()
        best = min(trials, key=lambda t: t["ms"])
        cap, flags, tc_min = best["cap"], best["flags"], best["tc_min_order"]
        tuned = {"trials": trials, "chosen": best}
    else:
        tc_min = args.tc_min_order
    plan = chol.chol_batch_plan(ns, chol.opts(nb=cap, precision=prec, flags=flags, tc_min_order=tc_min))
    tc_part = (not (prec == "fp64" and flags & chol.CHOL_FLAG_FP64_SIMT)) and any(n > (tc_min or 1024) for n in ns)
    flops = sum(n ** 3 / 3.0 for n in ns)
    solve_flops = sum(2.0 * n * n for n in ns)

    def restore():
        for a, a0 in zip(As, A0):
            a.copy_(a0)
        for b, b0 in zip(Bs, B0):
            b.copy_(b0)
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        restore()
        info = plan.run(As, Bs)
    assert all(i == 0 for i in info)
    bench.barrier(world)
    times, kms = [], []
    with bench.ClockSampler(local) as clk:
        for _ in range(args.steps):
            restore()
            t = time.perf_counter()
            info = plan.run(As, Bs)
            times.append(1e3 * (time.perf_counter() - t))
            kms.append(plan.stats().device_ms)
    bench.barrier(world)
    st = plan.stats()
    check = _check_batch(As, Bs, A0, B0, ns, idx, prec) if rank == 0 else None
    ms = bench.allreduce_max(statistics.mean(times), world)
    total_flops = flops * world if world > 1 else flops  # shards are about equal; report the job total below
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([flops], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        total_flops = float(t.item())
    value = total_flops / (ms / 1e3) / 1e12
    achieved = flops / (statistics.mean(kms) / 1e3) / 1e12
    # ceilings: the tensor-core part (most of the flops of the batch) against
    # the exact-slicing ceiling (FP64: bf16 / 36) or the three-TF32-product
    # ceiling (FP32: bf16 x 1/2 nominal TF32 ratio / 3), from the measured bf16
    # burst rate (one graph launch of a fraction of a second); CUDA-core bodies
    # against the FP64 pipe or the FP32 FMA pipe (152 SMs x 128 lanes x 2 flop
    # x 2.07 GHz)
    bf16 = bench.measured_peaks().get("bf16_tflops", 1913.8)
    if tc_part and prec == "fp64":
        bound, peak = "tensor", bf16 / 36.0
        kernel = "df_kernel<OzBatchBody> + df_kernel<BatchBody<double>>"
    elif tc_part:
        bound, peak = "tensor", bf16 / 2 / 3
        kernel = "df_kernel<MixedBatchBody> + df_kernel<BatchBody<float>>"
    elif prec == "fp64":
        bound, peak, kernel = "alu", bench.FP64_PEAK_TFLOPS, "df_kernel<BatchBody<double>>"
    else:
        bound, peak, kernel = "alu", 152 * 128 * 2 * 2.07e9 / 1e12, "df_kernel<BatchBody<float>>"
    if rank == 0:
        line = {"metric": bench.METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
                "config": {"workload": f"batched factor+solve of {count} SPD systems, n log-uniform [32, 2048] "
                                       f"(seed 3), A_i = G_i G_i^T/n_i + I, 1 RHS each, {prec}, one graph launch",
                           "batch": count, "tile_cap": cap, "precision": prec, "flags": flags,
                           "tensor_core_part": f"matrices of order above {tc_min or 1024}" if tc_part else None,
                           "sum_n3_over_3": flops, "parallelism": f"contiguous shards x{world}",
                           "l2": "inputs larger than L2"},
                "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None, "kernel": kernel},
                "check": check,
                "solves_per_s": world * len(ns) / (ms / 1e3), "solve_flops": solve_flops, "tasks": list(st.tasks),
                "autotune": tuned, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    plan.close()


def _check_batch(As, Bs, A0, B0, ns, idx, prec, subset: int = 256, seed: int = 17):
    """Every solution's normwise backward error, recomputed from the inputs
    (torch, binary64), and the factor of a seeded subset of the matrices
    against the oracle's unblocked factorization (host cores, in parallel)."""
    import concurrent.futures as cf
    import os

    import torch

    import oracle
    berr = []
    for a0, x, b0 in zip(A0, Bs, B0):
        r = b0 - a0 @ x
        den = torch.max(torch.sum(torch.abs(a0), dim=1)) * torch.max(torch.abs(x)) + torch.max(torch.abs(b0))
        berr.append(float(torch.max(torch.abs(r)) / den))
    rng = np.random.default_rng(seed)
    pick = sorted(rng.choice(len(ns), size=min(subset, len(ns)), replace=False).tolist())
    host = [(A0[k].cpu().numpy(), np.tril(As[k].cpu().numpy())) for k in pick]

    def one(pair):
        A, L = pair
        Lref, info = oracle.potrf_unblocked(A)
        scale = np.sqrt(np.diag(A))[:, None]
        return float(np.max(np.abs(L - np.tril(Lref)) / scale)), info

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(one, host))
    tol_berr = 1e-14 if prec == "fp64" else 1e-6
    tol_fac = 1e-11 if prec == "fp64" else 1e-5
    return {"berr_max": max(berr), "berr_all_within": all(b <= tol_berr for b in berr), "berr_tol": tol_berr,
            "oracle_subset": len(pick), "oracle_scaled_err_max": max(r[0] for r in res),
            "oracle_all_within": all(r[0] <= tol_fac and r[1] == 0 for r in res), "oracle_tol": tol_fac}


def run_serve(args, world, rank, local):
    import torch

    import paper_2606_11937_gb300 as chol

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.backends.cuda.matmul.allow_tf32 = False
    r = si.rng(11 + rank)
    nreq = args.serve_requests
    prec = args.precision if args.precision in chol.PRECISIONS else "fp64"
    # request pool: inputs built before the clock starts
    lo, hi = math.log(64), math.log(args.serve_nmax)
    reqs = []
    made = []  # indices of requests that created a resident factor
    for k in range(nreq):
        if made and r.uniform() < 0.3:
            j = made[int(r.integers(len(made)))]
            n = reqs[j]["n"]
            reqs.append({"n": n, "A": None, "fid": reqs[j]["fid"], "nrhs": int(r.integers(1, 33))})
            continue
        n = int(math.floor(math.exp(r.uniform(lo, hi))))
        seed = 10_000 * (rank + 1) + k
        if seed % 2 == 0:
            A = si.se_covariance_torch(n, seed=seed, lengthscale=0.1, nugget=1e-2, device=dev)
        else:
            A = _gram_torch(n, seed, dev)
        fid = k + 1
        reqs.append({"n": n, "A": A.T, "fid": fid, "nrhs": int(r.integers(1, 33))})
        made.append(k)
    for q in reqs:
        g = torch.Generator(device=dev)
        g.manual_seed(int(r.integers(1 << 30)))
        q["B"] = torch.randn((q["nrhs"], q["n"]), dtype=torch.float64, device=dev, generator=g).T
        q["X"] = torch.empty_strided((q["n"], q["nrhs"]), (1, q["n"]), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    rates = [float(x) for x in args.serve_rates.split(",")]
    results = []
    for lam in rates:
        srv = chol.Server(int(args.serve_budget_gb * (1 << 30)), slots=args.serve_slots)
        arrivals = np.cumsum(r.exponential(1.0 / lam, size=nreq))
        tickets = [None] * nreq
        t0 = time.perf_counter()
        for k, q in enumerate(reqs):
            now = time.perf_counter() - t0
            if arrivals[k] > now:
                time.sleep(arrivals[k] - now)
            tickets[k] = srv.submit(q["B"], q["X"], A=q["A"], factor_id=q["fid"], precision=prec, n=q["n"])
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
        srv.close()
        ok = sum(1 for x in res if x["status"] == 0)
        results.append({"rate_per_s": lam, "completed": ok, "failed": len(res) - ok, "solves_per_s": st["solves_per_s"],
                        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                        "reused": sum(1 for x in res if x["reused_factor"]),
                        "mean_iters": statistics.mean(x["iters"] for x in res) if prec != "fp64" else 0})
    best = max(results, key=lambda x: x["solves_per_s"])
    if rank == 0:
        line = {"metric": bench.METRIC, "value": best["solves_per_s"], "unit": "solves/s", "n_gpus": world,
                "steps": len(rates), "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == "fp64" else prec, "data": "synthetic",
                "config": {"workload": f"served SPD solves, Poisson arrivals, n log-uniform [64, {args.serve_nmax}], "
                                       f"1-32 RHS, 30% repeat RHS on resident factors, {prec}",
                           "requests_per_rate": nreq, "slots": args.serve_slots,
                           "budget_gb": args.serve_budget_gb},
                "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "sweep": results}
        print(json.dumps(line), flush=True)
