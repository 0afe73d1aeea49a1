#!/usr/bin/env python3
"""Benchmark of the factor + solve hot path on one GB300 per rank.

Workload (the batched Laplace configuration): 512 x 512 cell-centre grid of [0,1]^2
(N = 262144), leaves of 16 x 16 points, eps = 1e-10, a(x) = 1 + 0.5 sin(2 pi x1) cos(2 pi x2),
4 right-hand sides ~ N(0,1) (seed 1), FP64 throughout.  One step = rs_build_tree +
rs_factor + rs_solve (4 RHS).  `value` is factor unknowns per second (N / factor time, CUDA
events on the launch stream, inputs already on the device for the solve); the solve rate
is reported beside it.  `e2e` repeats the step through host buffers (pinned), with every
host-device copy inside the timed region.  A 256 MiB buffer (larger than the 129 MB L2) is
rewritten before every timed step.

With --gpus N under torchrun every rank runs its own replica (the path has no exchange
step): the reported times are the max over ranks, `value` the sum of the ranks' work over
that time.  `--impl reference` times the CPU oracle on a bounded sample instead.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1303_5466_gb300 import workloads as W  # noqa: E402

METRIC = "factor unknowns/sec and solve RHS/sec at 1e-10 residual; serving p50/p99 latency"
WORKLOAD = "laplace_batched"
# Nominal FP64 rate of one GB300 (152 SMs x 4 FP64 flop/clk x 2.07 GHz = 1.26 TFLOP/s; 1.25 in
# NVIDIA's figures).  The roofline divides by the rate the library's FP64 probes measure in
# the same run (the better of DFMA chains and mma.sync f64), and reports this one beside it.
PEAK_FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes (read + write) per launch of the CPQR class (cpqr_kernel and cpqr_bl_kernel), from
# one ncu capture of dram__bytes_read.sum and dram__bytes_write.sum at this workload with one
# launch per level; None once a kernel has changed since that capture
CPQR_TRAFFIC_BYTES_PER_LAUNCH = 136.3e9
# FP32 FMA peak (no tensor cores): 152 SMs x 128 lanes x 2 flop x 2.07 GHz
PEAK_FP32_TFLOPS = 80.5
ORACLE_LEVELS = 3          # oracle sample: the three finest tree levels
# factor kernels and the profile classes (rs_op_profile) whose launches they are (the inverse
# classes run the symmetric sweep on the Laplace workload)
KERNEL_CLASSES = {"sweep (sweep_bl_dinv_kernel + gemm_oz_kernel)": ("inv_F", "inv_E", "inv_root"),
                  "cpqr_kernel+cpqr_bl_kernel": ("cpqr",), "gemm_oz_kernel": ("gemm_E",),
                  "id_T (idt_solve_kernel + gemm_oz_kernel)": ("id_T",)}
# the digit-slice GEMM forms each FP64 product from 36 bf16 digit products
OZ_BF16_PER_FP64 = 36


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default=WORKLOAD, choices=["laplace_batched", "laplace_n256"],
                   help="laplace_n256 is a quarter-size copy for profiling runs")
    p.add_argument("--serving-requests", type=int, default=600,
                   help="requests of the serving stream measured after the main step (0 = skip)")
    p.add_argument("--full-factor", action="store_true",
                   help="with --impl reference: time one full oracle factorization and 4-RHS solve of the "
                        "workload at all host cores and on one thread's sample level, printed as its own "
                        "JSON line (not the benchmark line)")
    p.add_argument("--residual-grid", type=int, default=0,
                   help="instead of the benchmark: the FP64 direct-sum residual (1 RHS) of an n x n grid's "
                        "operator (tree build alone), timed, as its own JSON line")
    p.add_argument("--factor-grid", type=int, default=0,
                   help="instead of the benchmark: one factorization of an n x n grid of the batched Laplace "
                        "workload (leaf 16), timed with its per-class profile, as its own JSON line")
    p.add_argument("--cpqr-variant", type=int, default=-1,
                   help="--factor-grid: the column-pivoted QR form forced on every level (opts.cpqr_variant; "
                        "-1 = the built-in choice per level)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                   help="--factor-grid: FP64 at eps 1e-10, or FP32 at eps 1e-6")
    p.add_argument("--serving-only", action="store_true",
                   help="instead of the benchmark: only the serving stream (e.g. --serving-requests 10000), "
                        "printed as its own JSON line")
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    p.add_argument("--no-autotune", action="store_true", help="skip the launch-shape autotuner before the steps")
    p.add_argument("--no-per-box", action="store_true", help="skip the one-box-per-launch comparison")
    p.add_argument("--no-ti", action="store_true", help="skip the translation-invariant comparison (a = 1)")
    p.add_argument("--large-grid", type=int, default=0,
                   help="instead of the benchmark: factor and solve an n x n grid (a = 1, translation-invariant "
                        "mode 2) and print its own JSON line")
    p.add_argument("--k-cut", type=int, default=512,
                   help="also measure the extra compression of Sec. 3 for boxes with k > K (0: skip)")
    return p.parse_args()


def _inputs(name=WORKLOAD):
    cfg = W.WORKLOADS[name]
    n, leaf, eps, nrhs = cfg["n"], cfg["leaf"], cfg["eps"], cfg["nrhs"]
    pts = W.grid_points(n)
    a = W.coeff_a_batched(n)
    F = W.rhs_normal(n, cfg["seed"], nrhs=nrhs)          # (N, nrhs)
    return n, leaf, eps, nrhs, pts, a, F


def _config(n, leaf, eps, nrhs, world, name=WORKLOAD):
    return {"workload": name + ": %dx%d grid, leaf %dx%d, eps %g, a=1+0.5sin(2pi x1)cos(2pi x2), "
                        "%d RHS ~ N(0,1) seed 1" % (n, n, leaf, leaf, eps, nrhs),
            "N": n * n, "nrhs": nrhs, "eps": eps, "parallelism": "replicas x%d" % world,
            "l2": "256 MiB buffer rewritten before every timed step"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _init_group(backend, device=None, timeout_s=900.0):
    """Process group of the replicas.  A rank that dies or never reaches a collective ends the
    others' next collective with an error after timeout_s, instead of leaving them waiting."""
    import datetime
    import torch.distributed as dist
    kw = {"timeout": datetime.timedelta(seconds=timeout_s)}
    if device is not None:
        kw["device_id"] = device
    dist.init_process_group(backend, **kw)


def _max_over_ranks(vals, world):
    """Element-wise max of per-rank values over all ranks (the slowest replica sets the time);
    the tensor lives where the process group's backend wants it (NCCL: the GPU, gloo: host)."""
    if world == 1:
        return vals
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def _replica_rate(world, units_per_rank, max_seconds):
    """Whole-job throughput of N independent replicas: all ranks' units over the slowest time."""
    return world * units_per_rank / max_seconds


def sample_share(levels=None):
    """Share of the factor flops in the `levels` (default ORACLE_LEVELS) finest levels, from the
    per-level counts that oracle/level_flops.py wrote from a full oracle factorization of this
    workload."""
    levels = ORACLE_LEVELS if levels is None else levels
    with open(os.path.join(ROOT, "oracle", "laplace_batched_level_flops.json")) as fh:
        fl = {int(k): v for k, v in json.load(fh).items()}
    d = max(fl)
    return sum(fl[l] for l in range(d - levels + 1, d + 1)) / sum(fl.values())


def oracle_sample(n, leaf, eps, a):
    """Time the CPU oracle on a bounded sample of the workload: the ORACLE_LEVELS finest levels
    (every box of them) on all host cores, and the finest level alone on one thread (every box
    of this grid's finest level, no rescaling across grids).  Each time is scaled to the whole
    factorization by the sample's share of the algorithmic flops; that assumes the top levels,
    where the oracle has only a few boxes to spread over its threads, run at the sample's rate,
    so the extrapolated CPU rate is an upper bound on what a full oracle run achieves."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    O.Factorization(n, leaf, eps, a=a, max_levels=ORACLE_LEVELS, threads=cores)
    dt = time.perf_counter() - t
    share = sample_share()
    est = dt / share
    t = time.perf_counter()
    O.Factorization(n, leaf, eps, a=a, max_levels=1, threads=1)
    dt1 = time.perf_counter() - t
    share1 = sample_share(1)
    est1 = dt1 / share1
    return {"value": n * n / est, "unit": "unknowns/s", "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": "oracle factor of the %d finest levels (all %d boxes) of the %dx%d workload: %.2f s measured on "
                      "%d threads; those levels are %.1f%% of the factor flops, so the full factor is estimated at "
                      "%.1f s (flop share, an optimistic bound for the CPU)"
                      % (ORACLE_LEVELS, sum(2 ** (2 * _depth_half(n, leaf) - i) for i in range(ORACLE_LEVELS)),
                         n, n, dt, cores, 100 * share, est),
            "sample_s": dt, "flop_share": share, "full_factor_estimate_s": est,
            "single_thread": {"value": n * n / est1, "unit": "unknowns/s", "cores": 1, "extrapolated": True,
                              "sample": "the finest level of the %dx%d workload (all %d leaves) on 1 thread: %.2f s "
                                        "measured; %.1f%% of the factor flops, scaled to the full factor (%.1f s)"
                                        % (n, n, (n // leaf) ** 2, dt1, 100 * share1, est1),
                              "sample_s": dt1, "flop_share": share1}}


def _depth_half(n, leaf):
    """log2(n / leaf): the tree has depth 2 x this, and 4^this leaves."""
    return (n // leaf).bit_length() - 1


SERVING_OPS = ((128, 16), (256, 16), (512, 16))


def serving_measure(P, torch, requests, seed=3, load=0.7, other_loads=(0.5, 0.9), slots=128):
    """Serving workload: three resident FP64 operators (128^2, 256^2, 512^2 grids, leaves 16^2,
    eps 1e-10); a seeded stream of requests, each naming an operator uniformly and carrying
    1-64 RHS ~ N(0,1), arriving as a Poisson process at `load` x the closed-loop capacity
    measured on a first burst (and the same stream again at each of `other_loads`).  Returns
    p50/p99 latency (submission to completion) and RHS/s.

    Device buffers are reused so that long streams fit: the right-hand sides of a request are
    the first nrhs of 64 fixed N(0,1) columns of its operator (inputs are only read), and its
    solution goes to one of `slots` output buffers, taken in turn once its previous request has
    completed."""
    import numpy as np
    ops, trees = [], []
    for n, leaf in SERVING_OPS:
        t = P.rs_build_tree(W.grid_points(n), leaf)
        trees.append(t)
        ops.append(P.rs_factor(t, eps=1e-10))
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, len(SERVING_OPS), requests)
    nrhs = rng.integers(1, 65, requests)
    gaps = rng.exponential(1.0, requests)          # scaled by 1/lambda below
    fin = [torch.from_numpy(rng.standard_normal((64, n * n))).cuda() for n, _ in SERVING_OPS]
    nmax = max(n * n for n, _ in SERVING_OPS)
    xout = [torch.empty((64 * nmax,), dtype=torch.float64, device="cuda") for _ in range(slots)]
    torch.cuda.synchronize()
    fl = [P.rs_op_stats(o)["flops_solve_per_rhs"] for o in ops]
    owner = [0] * slots                            # ticket whose output a slot holds (0: none)
    done = set()
    srv = P.rs_server_create(ops, 8 << 30, max_inflight=64)

    def args_of(i):
        k, r = int(kinds[i]), int(nrhs[i])
        return k, fin[k], r, xout[i % slots]

    def submit(i):
        q = i % slots
        while owner[q] and owner[q] not in done:   # the slot's previous request must be complete
            done.update(P.rs_server_poll(srv, 4096))
            if owner[q] not in done:
                time.sleep(1e-4)
        k, f, r, x = args_of(i)
        owner[q] = P.rs_server_submit(srv, k, f, r, x)

    try:
        # closed loop on the first burst: everything submitted at once
        burst = min(32, requests)
        t0 = time.perf_counter()
        for i in range(burst):
            submit(i)
        P.rs_server_drain(srv, 3600.0)
        burst_s = time.perf_counter() - t0
        done.update(P.rs_server_poll(srv, 1 << 16))
        cap = burst / burst_s                        # requests per second
        rhs = int(nrhs[burst:].sum())

        def open_loop(ld):
            # Poisson arrivals at ld x capacity; latencies of this phase only
            lam_ = ld * cap
            n0_ = P.rs_server_stats(srv)["completed"]
            t0_ = time.perf_counter()
            t_next = t0_
            for i in range(burst, requests):
                t_next += gaps[i] / lam_
                delay = t_next - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                submit(i)
            P.rs_server_drain(srv, 36000.0)
            wall_ = time.perf_counter() - t0_
            done.update(P.rs_server_poll(srv, 1 << 20))
            lat_ = P.rs_server_latencies(srv)[n0_:]
            return lam_, wall_, lat_

        lam, wall, lat = open_loop(load)
        st = P.rs_server_stats(srv)
        others = {}
        for ld in other_loads:
            lam2, wall2, lat2 = open_loop(ld)
            others["%.1f" % ld] = {"lambda_per_s": lam2, "p50_ms": float(np.percentile(lat2, 50)),
                                   "p99_ms": float(np.percentile(lat2, 99)), "rhs_per_s": rhs / wall2}
        # the same burst, one rs_solve per request in submission order (no cross-request batching)
        cs = torch.cuda.current_stream()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for i in range(burst):
            k, f, r, x = args_of(i)
            P.rs_solve(ops[k], f, r, x, cs)
        torch.cuda.synchronize()
        seq_s = time.perf_counter() - t1
        burst_rhs = int(nrhs[:burst].sum())
        burst_flops = float(sum(fl[int(kinds[i])] * int(nrhs[i]) for i in range(burst)))
        return {"requests": int(requests - burst), "burst_requests": int(burst), "load": load,
                "burst_rhs_per_s": burst_rhs / burst_s, "sequential_rhs_per_s": burst_rhs / seq_s,
                "burst_speedup_vs_sequential": seq_s / burst_s,
                "burst_tflops": burst_flops / burst_s / 1e12, "sequential_tflops": burst_flops / seq_s / 1e12,
                "lambda_per_s": lam, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "rhs_per_s": rhs / wall, "ticks": st["ticks"], "peak_inflight": st["peak_inflight"],
                "other_loads": others,
                "operators": "%s grids, leaf 16, eps 1e-10, FP64" % ", ".join("%d^2" % n for n, _ in SERVING_OPS),
                "stream": "seed 3: operator uniform, nrhs uniform 1-64, N(0,1) columns, Exp inter-arrivals"}
    finally:
        P.rs_server_free(srv)
        for o in ops:
            P.rs_free(o)
        for t in trees:
            P.rs_free_tree(t)


def mixed_measure(P, torch, n, leaf, pts, a, F, nrhs, st):
    """The same workload with the FP32 factor at eps 1e-6 and FP64-residual refinement to
    1e-10: factor time, refined solve time, solves made and the final residual."""
    import numpy as np
    o = P.rs_opts_default()
    o.precision = P.RS_MIXED_FP32
    o.refine_tol = 1e-10
    o.profile = 1
    f = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    x = torch.empty_like(f)
    tree = P.rs_build_tree(pts, leaf)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(st)
    op = P.rs_factor(tree, a=a, eps=1e-6, opts=o, stream=st)
    e1.record(st)
    P.rs_solve(op, f, nrhs, x, st)
    e2.record(st)
    e2.synchronize()
    s = P.rs_op_stats(op)
    prof = P.rs_op_profile(op)
    rel = P.rs_residual(op, x, f, nrhs, st)
    out = {"factor_ms": e0.elapsed_time(e1), "refined_solve_ms": e1.elapsed_time(e2), "eps": 1e-6,
           "factor_profile_ms": {k: v[0] for k, v in prof.items() if k != "solve"},
           "factor_profile_tflops": {k: v[1] / (v[0] * 1e-3) / 1e12 for k, v in prof.items()
                                     if k != "solve" and v[0] > 0 and v[1] > 0},
           "fp32_peak_tflops": PEAK_FP32_TFLOPS,
           "refine_solves": s["refine_iters"], "refine_fp64_direct_sums": s["refine_fp64_sums"],
           "residual": float(rel.max()), "bytes_factors": s["bytes_factors"]}
    P.rs_free(op)
    P.rs_free_tree(tree)
    return out


def mixed_1024_measure(P, torch, st):
    """The mixed-precision workload as configured: 1024 x 1024 grid (N = 1048576), leaves 16 x 16,
    a = 1, one RHS ~ U[-1, 1] (seed 2); FP32 factor at eps 1e-6 refined to 1e-10 with the FP64
    direct-sum residual, beside the FP64 factor at eps 1e-10 and its solve on the same grid.
    Times: CUDA events on the launch stream; the FP64 residual of each solution by the direct
    sum (outside the timings)."""
    import numpy as np
    cfg = W.WORKLOADS["laplace_mixed"]
    n, leaf = cfg["n"], cfg["leaf"]
    f = torch.from_numpy(W.rhs_uniform(n, cfg["seed"])[None, :].copy()).cuda()
    x = torch.empty_like(f)
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    out = {"n": n, "N": n * n, "nrhs": 1}
    try:
        for name, prec, eps in (("mixed", P.RS_MIXED_FP32, cfg["eps"]), ("fp64", P.RS_FP64, 1e-10)):
            o = P.rs_opts_default()
            o.precision = prec
            o.refine_tol = 1e-10
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            op = P.rs_factor(tree, eps=eps, opts=o, stream=st)
            e1.record(st)
            P.rs_solve(op, f, 1, x, st)
            e2.record(st)
            e2.synchronize()
            s = P.rs_op_stats(op)
            rel = float(P.rs_residual(op, x, f, 1, st)[0])
            out[name] = {"eps": eps, "factor_ms": e0.elapsed_time(e1), "solve_ms": e1.elapsed_time(e2),
                         "step_ms": e0.elapsed_time(e2), "residual_fp64": rel, "bytes_factors": s["bytes_factors"],
                         "root_m": s["root_m"]}
            if prec == P.RS_MIXED_FP32:
                out[name]["refine_solves"] = s["refine_iters"]
                out[name]["refine_fp64_direct_sums"] = s["refine_fp64_sums"]
            P.rs_free(op)
    finally:
        P.rs_free_tree(tree)
    out["step_speedup_mixed_vs_fp64"] = out["fp64"]["step_ms"] / out["mixed"]["step_ms"]
    return out


def per_box_measure(P, torch, leaf, pts, a, F, nrhs, st, eps):
    """The same FP64 step with every factor and solve kernel launched for one box at a time
    (opts.per_box): the unbatched GPU form the per-level launches are compared with."""
    import numpy as np
    o = P.rs_opts_default()
    o.per_box = 1
    f = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    x = torch.empty_like(f)
    tree = P.rs_build_tree(pts, leaf)
    torch.cuda.synchronize()
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(st)
    op = P.rs_factor(tree, a=a, eps=eps, opts=o, stream=st)
    e1.record(st)
    e1.synchronize()
    P.rs_solve(op, f, nrhs, x, st)           # captures the solve graph
    torch.cuda.synchronize()
    launches0 = P.rs_launch_count()
    s0, s1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    s0.record(st)
    P.rs_solve(op, f, nrhs, x, st)
    s1.record(st)
    s1.synchronize()
    factor_ms, solve_ms = e0.elapsed_time(e1), s0.elapsed_time(s1)
    out = {"factor_ms": factor_ms, "solve_ms": solve_ms,
           "step_ms": factor_ms + solve_ms, "solve_launches": P.rs_launch_count() - launches0,
           "residual_fp64": float(P.rs_residual(op, x, f, nrhs, st).max())}
    P.rs_free(op)
    P.rs_free_tree(tree)
    return out


def fwd_measure(P, torch, op, x_dev, f_dev, nrhs, st, reps=5):
    """rs_fwd_apply (y = A x through the HSS form of the factorization, O(N)) on the solution of
    the timed solve: its time for nrhs columns, and the paper's error measure
    |f - A (A^{-1} f)| / |f| with A applied that way (rs_solve inverts it to rounding)."""
    import numpy as np
    y = torch.empty_like(x_dev)
    P.rs_fwd_apply(op, x_dev, nrhs, y, st)
    torch.cuda.synchronize()
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(st)
    for _ in range(reps):
        P.rs_fwd_apply(op, x_dev, nrhs, y, st)
    e1.record(st)
    e1.synchronize()
    err = (torch.linalg.norm(y - f_dev, dim=1) / torch.linalg.norm(f_dev, dim=1)).max().item()
    return {"ms": e0.elapsed_time(e1) / reps, "nrhs": nrhs, "error_vs_f": err}


def ls_measure(P, torch, st):
    """The Lippmann-Schwinger test problem of Sec. 5.4 (plateau scatterer, kappa 25, 256^2) two
    ways: the iterative route (tree build of A alone, the translation-invariant Helmholtz
    inverse as right preconditioner, BiCGstab with A through its HSS form) and the direct route
    (complex64 factor at eps 1e-5 refined to 1e-10 with the complex128 direct sum).  Times,
    iterations and the true residuals."""
    import numpy as np
    from paper_1303_5466_gb300 import workloads as W
    cfg = W.WORKLOADS["helmholtz_ls_plateau"]
    n, leaf, kappa = cfg["n"], cfg["leaf"], cfg["kappa"]
    b = W.coeff_b_plateau(n)
    f = W.rhs_plane_wave(n, kappa)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    xd = torch.zeros_like(fd)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    out = {"n": n, "kappa": kappa, "scatterer": "plateau (coeff_b_plateau)"}
    oa = P.rs_opts_default(); oa.precision = P.RS_C128; oa.forward_only = 1
    om = P.rs_opts_default(); om.precision = P.RS_C128; om.translation_invariant = 2
    torch.cuda.synchronize()
    e0, e1, e2, e3 = ev(), ev(), ev(), ev()
    e0.record(st)
    A = P.rs_factor(tree, eps=cfg["eps"], opts=oa, stream=st, kappa=kappa, b=b)
    e1.record(st)
    M = P.rs_factor(tree, eps=cfg["eps"], opts=om, stream=st, kappa=kappa)
    e2.record(st)
    it, rel = P.rs_bicgstab(A, M, fd, xd, tol=1e-10, max_iter=200, stream=st)
    e3.record(st)
    e3.synchronize()
    res = float(P.rs_residual(A, xd.cpu().numpy(), f, 1)[0])
    out["iterative"] = {"tree_build_ms": e0.elapsed_time(e1), "preconditioner_factor_ms": e1.elapsed_time(e2),
                        "bicgstab_ms": e2.elapsed_time(e3), "iterations": it, "hss_residual": rel,
                        "true_residual_fp64": res}
    od = P.rs_opts_default(); od.precision = P.RS_C64_REFINED; od.refine_max_iter = 12
    e0, e1, e2 = ev(), ev(), ev()
    e0.record(st)
    D = P.rs_factor(tree, eps=1e-5, opts=od, stream=st, kappa=kappa, b=b)
    e1.record(st)
    xd2 = torch.zeros_like(fd)
    P.rs_solve(D, fd, 1, xd2, st)
    e2.record(st)
    e2.synchronize()
    st_d = P.rs_op_stats(D)
    out["direct_refined"] = {"factor_ms": e0.elapsed_time(e1), "refined_solve_ms": e1.elapsed_time(e2),
                             "refine_iters": st_d["refine_iters"], "true_residual_fp64": st_d["refine_residual"]}
    for op in (A, M, D):
        P.rs_free(op)
    P.rs_free_tree(tree)
    return out


def helmholtz_measure(P, torch, st):
    """The Lippmann-Schwinger workload as configured: 256 x 256 grid, kappa 25, b = exp(-40 |x -
    (1/2,1/2)|^2), f = exp(i kappa x1), leaves 16 x 16; complex64 factor at eps 1e-5 refined to
    1e-10 with the complex128 direct-sum residual, beside the complex128 factor at eps 1e-10 and
    its solve.  CUDA-event times on the launch stream."""
    import numpy as np
    cfg = W.WORKLOADS["helmholtz_ls"]
    n, leaf, kappa = cfg["n"], cfg["leaf"], cfg["kappa"]
    b = W.coeff_b_gaussian(n)
    f = torch.from_numpy(np.ascontiguousarray(W.rhs_plane_wave(n, kappa))).cuda()
    x = torch.zeros_like(f)
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    out = {"n": n, "kappa": kappa, "scatterer": "Gaussian exp(-40|x-c|^2)"}
    try:
        for name, prec, eps in (("c64_refined", P.RS_C64_REFINED, cfg["eps"]), ("c128", P.RS_C128, 1e-10)):
            o = P.rs_opts_default()
            o.precision = prec
            o.refine_tol = 1e-10
            o.refine_max_iter = 12
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            op = P.rs_factor(tree, eps=eps, opts=o, stream=st, kappa=kappa, b=b)
            e1.record(st)
            P.rs_solve(op, f, 1, x, st)
            e2.record(st)
            e2.synchronize()
            s = P.rs_op_stats(op)
            res = float(P.rs_residual(op, x, f, 1, st)[0])
            out[name] = {"eps": eps, "factor_ms": e0.elapsed_time(e1), "solve_ms": e1.elapsed_time(e2),
                         "step_ms": e0.elapsed_time(e2), "residual_c128": res, "bytes_factors": s["bytes_factors"]}
            if prec == P.RS_C64_REFINED:
                out[name]["refine_solves"] = s["refine_iters"]
            P.rs_free(op)
    finally:
        P.rs_free_tree(tree)
    out["step_speedup_c64_refined_vs_c128"] = out["c128"]["step_ms"] / out["c64_refined"]["step_ms"]
    return out


def ti_measure(P, torch, leaf, pts, F, nrhs, st, eps):
    """The translation-invariant modes (Sec. 5: one set of matrix blocks per level) on the same
    grid with a = 1, against the per-box-result factorization of that operator: factor and
    solve time, stored bytes, root size and the FP64 direct-sum residual for each mode."""
    import numpy as np
    f = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    x = torch.empty_like(f)
    tree = P.rs_build_tree(pts, leaf)
    out = {"a": "1 (constant)"}
    for mode in (0, 1, 2):
        o = P.rs_opts_default()
        o.translation_invariant = mode
        torch.cuda.synchronize()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(st)
        op = P.rs_factor(tree, eps=eps, opts=o, stream=st)
        e1.record(st)
        e1.synchronize()
        P.rs_solve(op, f, nrhs, x, st)
        torch.cuda.synchronize()
        s0, s1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        s0.record(st)
        P.rs_solve(op, f, nrhs, x, st)
        s1.record(st)
        s1.synchronize()
        stt = P.rs_op_stats(op)
        out["mode%d" % mode] = {"factor_ms": e0.elapsed_time(e1), "solve_ms": s0.elapsed_time(s1),
                                "bytes_factors": stt["bytes_factors"], "root_m": stt["root_m"],
                                "flops_factor": stt["flops_factor"],
                                "residual_fp64": float(P.rs_residual(op, x, f, nrhs, st).max())}
        P.rs_free(op)
    P.rs_free_tree(tree)
    for mode in (1, 2):
        out["mode%d" % mode]["factor_speedup_vs_per_box"] = out["mode0"]["factor_ms"] / out["mode%d" % mode]["factor_ms"]
    return out


def compressed_measure(P, torch, n, leaf, pts, a, F, nrhs, st, eps, k_cut, x_dense, reps=5):
    """The same workload with the extra compression of Sec. 3 (boxes with k > k_cut): factor
    time (compression included), solve time, stored bytes against the dense blocks they replace,
    and the change of the solution against the dense-block factor."""
    import numpy as np
    o = P.rs_opts_default()
    o.k_cut, o.hss_leaf, o.hss_eps, o.profile = k_cut, 64, 1e-12, 1
    f = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    x = torch.empty_like(f)
    tree = P.rs_build_tree(pts, leaf)
    torch.cuda.synchronize()
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(st)
    op = P.rs_factor(tree, a=a, eps=eps, opts=o, stream=st)
    e1.record(st)
    e1.synchronize()
    factor_ms = e0.elapsed_time(e1)
    P.rs_solve(op, f, nrhs, x, st)      # warm-up (workspace)
    torch.cuda.synchronize()
    t = 0.0
    for _ in range(reps):
        s0, s1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        s0.record(st)
        P.rs_solve(op, f, nrhs, x, st)
        s1.record(st)
        s1.synchronize()
        t += s0.elapsed_time(s1)
    s = P.rs_op_stats(op)
    sol = P.rs_op_profile(op)["solve"]
    xd = torch.from_numpy(np.ascontiguousarray(x_dense.T)).cuda()
    change = float(torch.linalg.norm(x - xd) / torch.linalg.norm(xd))
    rel = P.rs_residual(op, x, f, nrhs, st)
    out = {"k_cut": k_cut, "hss_leaf": 64, "hss_eps": 1e-12, "factor_ms": factor_ms, "compress_ms": s["ms_compress"],
           "solve_ms": t / reps, "compressed_boxes": s["compressed_boxes"],
           "bytes_compressed": s["bytes_compressed"], "bytes_dense_replaced": s["bytes_dense_replaced"],
           "bytes_factors": s["bytes_factors"], "bytes_solve": s["bytes_solve"],
           "flops_solve_per_rhs": s["flops_solve_per_rhs"],
           "solve_achieved_tflops": sol[1] / (sol[0] * 1e-3) / 1e12 if sol[0] else None,
           "change_vs_dense": change, "residual_fp64": float(rel.max())}
    P.rs_free(op)
    P.rs_free_tree(tree)
    return out


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        _init_group("nccl", torch.device("cuda", local))
    import paper_1303_5466_gb300 as P
    from paper_1303_5466_gb300 import build as B
    B.build()
    n, leaf, eps, nrhs, pts, a, F = _inputs(args.workload)
    N = n * n
    st = torch.cuda.current_stream()
    f_dev = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()       # N x nrhs column-major
    x_dev = torch.empty_like(f_dev)
    opts = P.rs_opts_default()
    opts.profile = 1
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    # the FP64 pipe's measured rate: the roofline peak of every FP64 kernel below
    probe = {"dfma_tflops": P.rs_fp64_probe(P.RS_PROBE_DFMA, st), "dmma_tflops": P.rs_fp64_probe(P.RS_PROBE_DMMA, st),
             "bf16_mma_tflops": P.rs_fp64_probe(P.RS_PROBE_BF16_MMA, st)}
    peak64 = max(probe["dfma_tflops"], probe["dmma_tflops"])

    def step():
        tree = P.rs_build_tree(pts, leaf)
        op = P.rs_factor(tree, a=a, eps=eps, opts=opts, stream=st)
        return tree, op

    # launch shapes picked by the library's autotuner on this workload (one-time cost, outside
    # the timed region; the table it fills applies to every factorization below)
    tune = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        tree = P.rs_build_tree(pts, leaf)
        tune = P.rs_autotune(tree, a=a, eps=eps, stream=st)
        P.rs_free_tree(tree)
        tune["seconds"] = time.perf_counter() - t0

    for _ in range(args.warmup):
        tree, op = step()
        P.rs_solve(op, f_dev, nrhs, x_dev, st)
        torch.cuda.synchronize()
        P.rs_free(op)
        P.rs_free_tree(tree)
    if world > 1:
        torch.distributed.barrier()
    tf = ts = 0.0
    prof = {}
    launches0 = P.rs_launch_count()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            tree, op = step()
            e1.record(st)
            P.rs_solve(op, f_dev, nrhs, x_dev, st)
            e2.record(st)
            e2.synchronize()
            tf += e0.elapsed_time(e1)
            ts += e1.elapsed_time(e2)
            for k, v in P.rs_op_profile(op).items():
                p = prof.setdefault(k, [0.0, 0.0, 0.0, 0])
                for i in range(4):
                    p[i] += v[i]
            last_stats = P.rs_op_stats(op)
            by_level = {c: [round(P.rs_op_profile_level(op, c, l), 2) for l in range(last_stats["depth"], -1, -1)]
                        for c in ("cpqr", "inv_F", "inv_E")}
            # residual check of the timed solve on sampled rows (outside the timing)
            x_last = x_dev.cpu().numpy().T.copy()
            P.rs_free(op)
            P.rs_free_tree(tree)
    launches = P.rs_launch_count() - launches0
    torch.cuda.synchronize()
    tf, ts = _max_over_ranks([tf, ts], world)
    K = args.steps
    factor_ms, solve_ms = tf / K, ts / K
    # end to end through host buffers (pinned): H2D of the inputs and D2H of x in the timing
    pin_f = torch.from_numpy(np.asfortranarray(F)).pin_memory().numpy()
    pin_x = torch.empty(F.shape[::-1], dtype=torch.float64).pin_memory().numpy().T
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        tree, op = step()
        P.rs_solve(op, pin_f, nrhs, pin_x, None)
        P.rs_free(op)
        P.rs_free_tree(tree)
    e2e_s = _max_over_ranks([time.perf_counter() - t0], world)[0] / K
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    # dominant factor kernel: largest summed event time over the classes it serves
    kern = {k: [sum(prof[c][i] for c in cls) for i in range(4)] for k, cls in KERNEL_CLASSES.items()}
    dom = max(kern, key=lambda k: kern[k][0])
    ms, work, _, nl = kern[dom]
    achieved = work / (ms * 1e-3) / 1e12
    sol = prof["solve"]
    rows = np.random.default_rng(5).choice(N, 64, replace=False)
    from oracle import oracle as O
    O.build()
    r = O.matvec_rows(n, x_last, rows, a=a) - F[rows]
    res = float(np.linalg.norm(r) / np.linalg.norm(F[rows]))
    out = {
        "metric": METRIC, "value": _replica_rate(world, N, factor_ms * 1e-3), "unit": "unknowns/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": factor_ms + solve_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(n, leaf, eps, nrhs, world, args.workload),
        "factor_ms": factor_ms, "solve_ms": solve_ms,
        "solve_rhs_per_s": world * nrhs / (solve_ms * 1e-3),
        "sampled_residual": res,
        "flops_factor": last_stats["flops_factor"], "bytes_factors": last_stats["bytes_factors"],
        "root_m": last_stats["root_m"],
        "host_wall_ms": {"id_phase": last_stats["ms_tree"], "inverse_phase": last_stats["ms_inverse"]},
        "roofline": {"kernel": dom, "classes": list(KERNEL_CLASSES[dom]), "bound": "alu", "achieved": achieved, "peak": peak64,
                     "unit": "TFLOP/s", "frac": achieved / peak64,
                     "peak_nominal": PEAK_FP64_NOMINAL_TFLOPS, "frac_of_nominal": achieved / PEAK_FP64_NOMINAL_TFLOPS,
                     "traffic": CPQR_TRAFFIC_BYTES_PER_LAUNCH if dom.startswith("cpqr") else None,
                     "traffic_note": "ncu DRAM read+write bytes per launch at this workload, one launch per "
                                     "level (no autotuner batching)",
                     "launches": nl, "avg_launch_ms": ms / max(nl, 1),
                     "peak_note": "of measured: the better of the library's FP64 probes in this run (DFMA chains "
                                  "%.3f, mma.sync f64 %.3f TFLOP/s); nominal 152 SMs x 4 flop/clk x 2.07 GHz"
                                  % (probe["dfma_tflops"], probe["dmma_tflops"])},
        "fp64_probe": probe,
        "roofline_solve": {"kernel": "solve matvec", "bound": "alu",
                           "achieved": sol[1] / (sol[0] * 1e-3) / 1e12 if sol[0] else None,
                           "peak": peak64, "unit": "TFLOP/s",
                           "frac": (sol[1] / (sol[0] * 1e-3) / 1e12) / peak64 if sol[0] else None,
                           "achieved_gbs": sol[2] / (sol[0] * 1e-3) / 1e9 if sol[0] else None},
        "profile_ms_per_step": {k: v[0] / K for k, v in prof.items()},
        "profile_ms_by_level": {"levels": "finest .. root (root: inv_F holds the root inverse)", **by_level},
        "profile_tflops": {k: v[1] / (v[0] * 1e-3) / 1e12 for k, v in prof.items() if v[0] > 0 and v[1] > 0},
        "roofline_by_kernel": {k: {"achieved_tflops": kern[k][1] / (kern[k][0] * 1e-3) / 1e12,
                                   "frac_fp64": kern[k][1] / (kern[k][0] * 1e-3) / 1e12 / peak64,
                                   "ms_per_step": kern[k][0] / K,
                                   **({"bf16_tflops": OZ_BF16_PER_FP64 * kern[k][1] / (kern[k][0] * 1e-3) / 1e12,
                                       "frac_bf16_mma": OZ_BF16_PER_FP64 * kern[k][1] / (kern[k][0] * 1e-3) / 1e12
                                       / probe["bf16_mma_tflops"],
                                       "note": "FP64 products from exact bf16 digit products on mma.sync; "
                                               "frac_fp64 above 1 is the gain over the FP64 pipe"}
                                      if k == "gemm_oz_kernel" else {})}
                               for k in kern if kern[k][0] > 0},
        "e2e": {"value": world * N / e2e_s, "unit": "unknowns/s",
                "step": "rs_build_tree + rs_factor + 4-RHS rs_solve from pinned host buffers, copies timed",
                "h2d_bytes_per_step": N * 2 * 8 + N * 8 + N * nrhs * 8, "d2h_bytes_per_step": N * nrhs * 8},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "autotune": tune,
    }
    # FP64 residual of the timed solve (direct sum over all pairs), and the forward apply
    # through the factorization's HSS form beside it
    tree, op = step()
    P.rs_solve(op, f_dev, nrhs, x_dev, st)
    torch.cuda.synchronize()
    r0, r1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    r0.record(st)
    out["residual_fp64"] = float(P.rs_residual(op, x_dev, f_dev, nrhs, st).max())
    r1.record(st)
    r1.synchronize()
    out["forward_apply"] = fwd_measure(P, torch, op, x_dev, f_dev, nrhs, st)
    out["forward_apply"]["direct_sum_residual_ms"] = r0.elapsed_time(r1)
    P.rs_free(op)
    P.rs_free_tree(tree)
    if args.k_cut > 0:
        out["compressed"] = compressed_measure(P, torch, n, leaf, pts, a, F, nrhs, st, eps, args.k_cut,
                                               x_dev.cpu().numpy().T.copy())
        out["compressed"]["dense_solve_ms"] = solve_ms
        out["compressed"]["dense_bytes_factors"] = last_stats["bytes_factors"]
    if not args.no_ti:
        out["translation_invariant"] = ti_measure(P, torch, leaf, pts, F, nrhs, st, eps)
        out["lippmann_schwinger"] = ls_measure(P, torch, st)
        out["helmholtz_gaussian"] = helmholtz_measure(P, torch, st)
    if not args.no_per_box:
        out["per_box_fp64"] = per_box_measure(P, torch, leaf, pts, a, F, nrhs, st, eps)
        out["per_box_fp64"]["batched_step_speedup"] = out["per_box_fp64"]["step_ms"] / (factor_ms + solve_ms)
    if not args.no_mixed:
        mx = mixed_measure(P, torch, n, leaf, pts, a, F, nrhs, st)
        mx["step_speedup_vs_fp64"] = (factor_ms + solve_ms) / (mx["factor_ms"] + mx["refined_solve_ms"])
        if "per_box_fp64" in out:
            mx["step_speedup_vs_per_box_fp64"] = out["per_box_fp64"]["step_ms"] / (mx["factor_ms"] + mx["refined_solve_ms"])
        out["mixed"] = mx
        out["mixed_1024"] = mixed_1024_measure(P, torch, st)
    if args.serving_requests > 0:
        out["serving"] = serving_measure(P, torch, args.serving_requests)
    if not args.no_cpu_baseline and args.workload == WORKLOAD:
        out["cpu_baseline"] = oracle_sample(n, leaf, eps, a)
    print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference_full(args):
    """--impl reference --full-factor: the oracle's whole factorization (every level, the root)
    and its 4-RHS solve of the batched Laplace workload on all host cores, timed once; the
    measured counterpart of the arm's extrapolated figure."""
    n, leaf, eps, nrhs, pts, a, F = _inputs()
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    S = O.Factorization(n, leaf, eps, a=a, threads=cores)
    t1 = time.perf_counter()
    S.solve(F)
    t2 = time.perf_counter()
    print(json.dumps({"oracle_full": {"workload": _config(n, leaf, eps, nrhs, 1)["workload"], "cores": cores,
                                      "factor_s": t1 - t0, "solve_4rhs_s": t2 - t1,
                                      "factor_unknowns_per_s": n * n / (t1 - t0)}}))


def run_reference(args):
    """The oracle arm: every step (warm-up and timed) factors the ORACLE_LEVELS finest levels of
    the workload (every box of them) with the oracle on all host cores, a bounded sample of the
    whole factorization.  `ms_per_step` is that measured sample time.  `value` scales the mean
    sample time to the full factor by the sample's share of the algorithmic flops (stated in
    `extrapolation`), an optimistic bound for the CPU: the oracle spreads a level over its boxes,
    and the top levels have only 2-8 of them."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    n, leaf, eps, nrhs, pts, a, F = _inputs()
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        S = O.Factorization(n, leaf, eps, a=a, max_levels=ORACLE_LEVELS, threads=cores)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
        del S
    dt = sum(times) / len(times)
    share = sample_share()
    est = dt / share
    v = n * n / est
    boxes = sum(2 ** (2 * _depth_half(n, leaf) - i) for i in range(ORACLE_LEVELS))
    sample = ("each step: oracle factor of the %d finest levels (all %d boxes) of the %dx%d workload on %d threads, "
              "%.2f s measured on average" % (ORACLE_LEVELS, boxes, n, n, cores, dt))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(n, leaf, eps, nrhs, world),
           "extrapolation": {"sample_ms_per_step": dt * 1e3, "flop_share": share,
                             "extrapolated_ms_full_factor": est * 1e3,
                             "rule": "value = N / (sample time / flop share of the sampled levels)"},
           "cpu_baseline": {"value": v, "unit": "unknowns/s", "cores": cores, "kind": "oracle", "sample": sample,
                            "extrapolated": True},
           "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_large_grid(args):
    """--large-grid n: one factorization and solve of an n x n grid with a = 1 in the
    translation-invariant mode 2 (FP64, leaf 16, eps 1e-10), with the residual on 32 sampled
    rows computed entry by entry by the oracle.  Prints one JSON line (not the benchmark line)."""
    import numpy as np
    import torch
    import paper_1303_5466_gb300 as P
    from paper_1303_5466_gb300 import workloads as W
    from oracle import oracle as O
    n = args.large_grid
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream()
    o = P.rs_opts_default()
    o.translation_invariant = 2
    o.profile = 1
    tree = P.rs_build_tree(W.grid_points(n), 16)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    op = P.rs_factor(tree, eps=1e-10, opts=o, stream=st)
    e1.record(st)
    e1.synchronize()
    factor_ms = e0.elapsed_time(e1)
    f = torch.from_numpy(W.rhs_uniform(n, 2)[None, :].copy()).cuda()
    x = torch.empty_like(f)
    P.rs_solve(op, f, 1, x, st)
    torch.cuda.synchronize()
    e0.record(st)
    P.rs_solve(op, f, 1, x, st)
    e1.record(st)
    e1.synchronize()
    solve_ms = e0.elapsed_time(e1)
    s = P.rs_op_stats(op)
    rows = np.random.default_rng(0).choice(n * n, 32, replace=False)
    xs = x.cpu().numpy()[0]
    fr = f.cpu().numpy()[0][rows]
    res = float(np.linalg.norm(np.ravel(O.matvec_rows(n, xs, rows)) - fr) / np.linalg.norm(fr))
    print(json.dumps({"large_grid": {"n": n, "N": n * n, "factor_ms": factor_ms, "solve_ms": solve_ms,
                                     "unknowns_per_s": n * n / (factor_ms * 1e-3), "root_m": s["root_m"],
                                     "bytes_factors": s["bytes_factors"], "flops_factor": s["flops_factor"],
                                     "sampled_residual": res, "residual_rows": 32,
                                     "profile_ms": {k: v[0] for k, v in P.rs_op_profile(op).items()}}}))
    P.rs_free(op)
    P.rs_free_tree(tree)


def run_residual_grid(args):
    """--residual-grid n: the FP64 direct-sum residual of one right-hand side on an n x n grid
    (the refinement's residual kernel), on an operator built by the tree build alone
    (opts.forward_only), timed with CUDA events; prints one JSON line (not the benchmark line)."""
    import torch
    import paper_1303_5466_gb300 as P
    from paper_1303_5466_gb300 import build as B
    B.build()
    n = args.residual_grid
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream()
    tree = P.rs_build_tree(W.grid_points(n), 16)
    o = P.rs_opts_default()
    o.forward_only = 1
    op = P.rs_factor(tree, eps=1e-10, opts=o, stream=st)
    f = torch.from_numpy(W.rhs_uniform(n, 2)[None, :].copy()).cuda()
    x = torch.from_numpy(W.rhs_uniform(n, 3)[None, :].copy()).cuda()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    rel = float(P.rs_residual(op, x, f, 1, st)[0])
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"residual_grid": {"n": n, "nrhs": 1, "ms": ms, "pair_terms": float(n) ** 4,
                                        "tflops": 2.0 * float(n) ** 4 / (ms * 1e-3) / 1e12, "rel": rel}}))
    P.rs_free(op)
    P.rs_free_tree(tree)


def run_factor_grid(args):
    """--factor-grid n: one factorization of the n x n batched Laplace workload (leaf 16,
    a = 1 + 0.5 sin(2 pi x1) cos(2 pi x2)) in FP64 at eps 1e-10 or FP32 at eps 1e-6, timed, with
    its per-class profile and the CPQR time of every level (finest first), the CPQR form given by
    --cpqr-variant; prints one JSON line (not the benchmark line)."""
    import torch
    import paper_1303_5466_gb300 as P
    from paper_1303_5466_gb300 import build as B
    B.build()
    n = args.factor_grid
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream()
    tree = P.rs_build_tree(W.grid_points(n), 16)
    o = P.rs_opts_default()
    o.profile = 1
    o.cpqr_variant = args.cpqr_variant
    eps = 1e-10
    if args.precision == "fp32":
        o.precision = P.RS_MIXED_FP32
        eps = 1e-6
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    op = P.rs_factor(tree, a=W.coeff_a_batched(n), eps=eps, opts=o, stream=st)
    e1.record(st)
    e1.synchronize()
    prof = P.rs_op_profile(op)
    depth = P.rs_op_stats(op)["depth"]
    print(json.dumps({"factor_grid": {"n": n, "precision": args.precision, "eps": eps, "cpqr_variant": args.cpqr_variant,
                                      "factor_ms": e0.elapsed_time(e1),
                                      "cpqr_ms_by_level": [P.rs_op_profile_level(op, "cpqr", l) for l in range(depth, 0, -1)],
                                      "profile_ms": {k: v[0] for k, v in prof.items()},
                                      "profile_tflops": {k: v[1] / (v[0] * 1e-3) / 1e12 for k, v in prof.items()
                                                         if v[0] > 0 and v[1] > 0}}}))
    P.rs_free(op)
    P.rs_free_tree(tree)


def run_serving_only(args):
    """--serving-only: the serving stream alone (three resident operators, Poisson arrivals at
    0.5, 0.7 and 0.9 x the measured capacity); prints one JSON line (not the benchmark line)."""
    import torch
    import paper_1303_5466_gb300 as P
    from paper_1303_5466_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    out = serving_measure(P, torch, args.serving_requests)
    out["wall_s"] = time.perf_counter() - t0
    print(json.dumps({"serving": out}))


def main():
    args = _args()
    if args.impl == "reference" and args.full_factor:
        run_reference_full(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.large_grid:
        run_large_grid(args)
    elif args.serving_only:
        run_serving_only(args)
    elif args.residual_grid:
        run_residual_grid(args)
    elif args.factor_grid:
        run_factor_grid(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
