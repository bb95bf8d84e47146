"""Further bench.py workloads (``--workload mixed|batched|serve|sweep``).

Each prints one JSON line with the keys of the default FP64 line.

* mixed: mixed-precision factorization (trailing SYRK/GEMM on tcgen05) of
  the SE covariance (n, --nugget, default 1e-2), then a solve of 16 N(0, 1)
  right-hand sides with FP64 iterative refinement to backward error 1e-14.
  value = factorization TFLOP/s (n^3/3); the line also carries the
  refinement iterations (with --flags 32, GMRES-based refinement: factor
  applications), the backward error, the time to solution and the
  plain FP64 path's time to solution (factor + solve) on the same inputs.
  A factorization that breaks down (not positive definite in the chosen
  precision) prints its info instead of a value.
* sweep: FP64 factorization time for every tile order x schedule (the
  paper's tile-size sweep, Section 4.1, on the GPU); one line per point.
"""
from __future__ import annotations

import json
import statistics
import time

import bench


def _common(args, world, value, unit, ms, config, dtype, extra):
    line = {"metric": bench.METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}
    line.update(extra)
    return line


def run_mixed(args, world, rank, local):
    import torch

    import paper_2606_11937_gb300 as chol
    import seeded_inputs as si

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    prec = args.precision
    nb = args.nb or chol.chol_default_nb(n, prec)
    A = si.se_covariance_torch(n, seed=1, lengthscale=0.1, nugget=args.nugget, device=dev).T
    g = torch.Generator(device=dev)
    g.manual_seed(2)
    B = torch.randn((16, n), dtype=torch.float64, device=dev, generator=g).T  # column-major n x 16
    stream = torch.cuda.current_stream(dev)
    o = chol.opts(precision=prec, schedule=args.schedule, nb=nb, stream=stream.cuda_stream, max_iter=50,
                  flags=args.flags)
    flops = n ** 3 / 3.0

    def step():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, h = chol.chol_mixed_factor(A, o)
        e1.record(stream)
        e1.synchronize()
        st = chol.chol_mixed_last_stats()
        return e0.elapsed_time(e1), st, h

    _, _, h = step()
    if h.info > 0:
        # the factorization is not positive definite in this precision: report it
        if rank == 0:
            print(json.dumps({"metric": bench.METRIC, "value": None, "unit": "TFLOP/s", "n_gpus": world,
                              "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                              "config": {"workload": f"mixed-precision ({prec}) tiled Cholesky n={n} nb={nb}, "
                                                     f"SE covariance (l=0.1, nugget {args.nugget:g}, seed 1)",
                                         "n": n, "nb": nb, "precision": prec, "nugget": args.nugget},
                              "status": "breakdown: non-positive pivot in this precision", "info": h.info}),
                  flush=True)
        h.close()
        return
    h.close()
    for _ in range(max(0, args.warmup - 1)):
        _, _, h = step()
        h.close()
    torch.cuda.synchronize()
    bench.barrier(world)
    times, kms = [], []
    with bench.ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms, st, h = step()
            times.append(ms)
            kms.append(st.device_ms)
            if len(times) < args.steps:
                h.close()
    torch.cuda.synchronize()
    bench.barrier(world)
    # solve with refinement using the last factor
    t = time.perf_counter()
    rc, X, iters, berr = h.solve(B, raise_on_error=False)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t
    # a second solve with the same handle: without the one-time setup of the
    # first (the slices of A for the tensor-core residual, its allocation)
    t = time.perf_counter()
    h.solve(B, raise_on_error=False)
    torch.cuda.synchronize()
    solve_again_s = time.perf_counter() - t
    Lm = None if args.no_fp64_compare else h.factor()
    h.close()
    fp64, factor_err = None, None
    if not args.no_fp64_compare:
        fp64, L64 = _fp64_time_to_solution(A, B, stream, chol, keep_factor=True)
        # the low-precision factor against the FP64 one (whose own residual
        # the FP64 parity tests bound): max_{i>=j} |L_ij - L64_ij| / sqrt(A_ii)
        factor_err = _scaled_factor_error(Lm, L64, A)
        del Lm, L64
    ms = bench.allreduce_max(statistics.mean(times), world)
    value = world * flops / (ms / 1e3) / 1e12
    achieved = flops / (statistics.mean(kms) / 1e3) / 1e12
    peaks = bench.measured_peaks()
    bf16 = peaks.get("bf16_tflops", 1873.4)
    peak = {"bf16": bf16, "fp16": bf16, "tf32": bf16 / 2, "fp32": bf16 / 2 / 3}[prec]
    if rank == 0:
        line = _common(args, world, value, "TFLOP/s", ms,
                       {"workload": f"mixed-precision ({prec} trailing update) tiled Cholesky n={n} nb={nb} "
                                    f"{args.schedule}, SE covariance (l=0.1, nugget {args.nugget:g}, seed 1), then solve "
                                    f"of 16 N(0,1) RHS with FP64 refinement to 1e-14",
                        "n": n, "nb": nb, "precision": prec, "schedule": args.schedule, "flags": args.flags,
                        "nugget": args.nugget,
                        "l2": f"inputs larger than L2 ({n * n * 8 / 1e9:.1f} GB FP64 matrix)"},
                       "f32", {"roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                            "frac": achieved / peak, "traffic": None,
                                            "kernel": "df_kernel<MixedBody> (whole schedule)",
                                            "peak_source": f"measured bf16 {bf16} TFLOP/s x nominal ratio for {prec}"},
                               "refinement": {"method": "gmres" if args.flags & chol.CHOL_FLAG_GMRES_IR else "classic",
                                              "status": rc, "iterations": iters, "berr": berr,
                                              "solve_s": solve_s, "time_to_solution_s": ms / 1e3 + solve_s,
                                              "solve_again_s": solve_again_s},
                               "fp64_reference_path": fp64,
                               "factor_error_vs_fp64": factor_err,
                               "clocks": clk.summary()})
        print(json.dumps(line), flush=True)


def _berr(A, X, B):
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    import torch
    R = B - A @ X
    an = torch.max(torch.sum(torch.abs(A), dim=1))
    num = torch.max(torch.abs(R), dim=0).values
    den = an * torch.max(torch.abs(X), dim=0).values + torch.max(torch.abs(B), dim=0).values
    return float(torch.max(num / den))


def _scaled_factor_error(L, Lref, A, blk: int = 4096) -> float:
    """max_{i>=j} |L_ij - Lref_ij| / sqrt(A_ii) over column blocks (column-major n x n tensors)."""
    import torch
    n = A.shape[0]
    scale = torch.sqrt(torch.diagonal(A)).reshape(n, 1)
    err = 0.0
    for c0 in range(0, n, blk):
        c1 = min(n, c0 + blk)
        d = torch.tril(L[:, c0:c1] - Lref[:, c0:c1], diagonal=-c0).abs() / scale
        err = max(err, float(d.max()))
    return err


def _fp64_time_to_solution(A, B, stream, chol, keep_factor: bool = False):
    """The plain FP64 path on the same inputs: chol_factor_ex (tensor-core
    engine, exact slicing) + chol_solve_ex, device time, with its backward
    error; the second of two runs is reported."""
    import torch
    n = A.shape[0]
    o = chol.opts(schedule="dataflow", nb=128, flags=chol.CHOL_FLAG_FP64_TC | chol.CHOL_FLAG_PRIORITY,
                  stream=stream.cuda_stream)
    L = torch.empty_strided((n, n), (1, n), dtype=torch.float64, device=A.device)
    out = None
    for _ in range(2):
        L.copy_(A)
        X = B.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info, _ = chol.chol_factor_ex(L, o)
        e1.record(stream)
        chol.chol_solve_ex(L, X, o)
        e2.record(stream)
        e2.synchronize()
        out = {"engine": "fp64 tensor-core (exact slicing), dataflow nb=128", "info": info,
               "factor_s": e0.elapsed_time(e1) / 1e3, "solve_s": e1.elapsed_time(e2) / 1e3,
               "time_to_solution_s": e0.elapsed_time(e2) / 1e3}
    out["berr"] = _berr(A, X, B)
    if keep_factor:
        return out, L
    del L
    return out


def run_sweep(args, world, rank, local):
    """Tile order x schedule sweep of the FP64 factorization (Section 4.1 on the GPU)."""
    import torch

    import paper_2606_11937_gb300 as chol
    import seeded_inputs as si

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    A0 = si.se_covariance_torch(n, seed=1, lengthscale=0.1, nugget=1e-2, device=dev).T
    A = torch.empty_strided((n, n), (1, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    nbs = [int(x) for x in (args.sweep_nb or "128,256,512,1024").split(",")]
    scheds = (args.sweep_sched or "dataflow,fork_join,fork_join_naive").split(",")
    engines = (args.sweep_engine or "tc").split(",")
    import ctypes
    import numpy as np
    rsz = ctypes.sizeof(chol.chol_trace_rec)
    eflags = {"tc": chol.CHOL_FLAG_FP64_TC | chol.CHOL_FLAG_PRIORITY, "simt": chol.CHOL_FLAG_FP64_SIMT}
    points = [(e, nb, sched) for e in engines for nb in nbs for sched in scheds
              if not (e == "tc" and nb % 128)]
    for engine, nb, sched in points:
        for flags in ([0, chol.CHOL_FLAG_NOOP] if args.noop else [0]):
            fl = flags | eflags[engine] | (args.flags & ~chol.CHOL_FLAG_NOOP)
            if sched != "dataflow":
                fl &= ~chol.CHOL_FLAG_PRIORITY
            m = -(-n // nb)
            ntask = m * (m + 1) * (m + 2) // 6
            trace = torch.empty(ntask * rsz, dtype=torch.uint8, device=dev) if args.trace else None
            o = chol.opts(schedule=sched, nb=nb, flags=fl, stream=stream.cuda_stream, num_ctas=args.num_ctas,
                          trace=trace, trace_capacity=ntask if args.trace else 0)
            ts = []
            for _ in range(max(1, args.steps)):
                A.copy_(A0)
                torch.cuda.synchronize()
                rc, info, st = chol.chol_factor_ex(A, o)
                ts.append(st.device_ms)
            ms = statistics.median(ts)
            tasks = sum(st.tasks)
            rec = {"workload": "sweep", "engine": engine, "n": n, "nb": nb, "schedule": sched, "noop": bool(flags),
                   "flags": fl, "ms": ms, "tflops": (n ** 3 / 3) / (ms / 1e3) / 1e12 if not flags else None,
                   "tasks": tasks, "us_per_task": 1e3 * ms / tasks, "launches": st.launches}
            if trace is not None:
                raw = trace.cpu().numpy()[: min(st.trace_records, ntask) * rsz]
                r = raw.view(np.dtype([("type", "<i4"), ("I", "<i4"), ("K", "<i4"), ("J", "<i4"),
                                       ("sm", "<i4"), ("matrix", "<i4"), ("t0", "<u8"), ("t1", "<u8")]))
                busy_ns = float(np.sum(r["t1"] - r["t0"]))
                ctas = args.num_ctas or 152 * (1 if fl & chol.CHOL_FLAG_FP64_TC else 4)
                span_ns = float(r["t1"].max() - r["t0"].min())
                dur = (r["t1"] - r["t0"]).astype(np.float64)
                by_type = {name: float(np.mean(dur[r["type"] == ty]) / 1e3) if np.any(r["type"] == ty) else None
                           for ty, name in enumerate(("potrf", "trsm", "syrk", "gemm"))}
                rec.update({"trace_busy_s": busy_ns / 1e9, "trace_span_s": span_ns / 1e9, "ctas": ctas,
                            "idle_us_per_task": (ctas * span_ns - busy_ns) / 1e3 / len(r),
                            "mean_task_us": busy_ns / 1e3 / len(r), "mean_us_by_type": by_type})
            if rank == 0:
                print(json.dumps(rec), flush=True)


def run(args, world, rank, local):
    if args.workload == "mixed":
        return run_mixed(args, world, rank, local)
    if args.workload == "sweep":
        return run_sweep(args, world, rank, local)
    if args.workload == "batched":
        import bench_batched
        return bench_batched.run_batched(args, world, rank, local)
    if args.workload == "serve":
        import bench_batched
        return bench_batched.run_serve(args, world, rank, local)
    raise ValueError(args.workload)
