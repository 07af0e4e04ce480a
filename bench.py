#!/usr/bin/env python
"""Benchmark of the sketch-preconditioned IPM on one GB300 (or N replicas).

One step = one LP solved to tolerance by Algorithm 2 (every step of the hot path: residuals
and p, sketch A D W, factor, PCG, FP64 residual and correction, fused update) on the dense
Gaussian LP with m = 1000, n = 200,000 and A in FP32 (the single-GPU configuration the
headline metric is quoted on; A is 800 MB, larger than L2, so no flush is needed).

Prints one JSON line (rank 0).  ``value`` is LPs/s over all ranks with A resident in HBM;
``e2e`` is the same metric through the C ABI from host buffers (A, b, c copied in and x, y, s
copied out inside the timed region); ``roofline`` is the CG product A D^2 A^T v measured live
with CUDA events on the library's stream; ``cpu_baseline`` times the FP64 oracle on a bounded
sample.  ``--impl reference`` runs only the oracle (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes of one CG product launch from an ncu capture of the same kernel source
# (k_cgprod.cu at the recorded hash); reported only while the kernel source is unchanged.
NCU_TRAFFIC = {"source_sha1": "7c8ddb492c5bed03423d805db0fe9600dce4135b",
               "bytes_per_launch": 803.94e6,
               "case": "dense m=1000 n=200000 FP32, ncu --metrics dram__bytes_read.sum,"
                       "dram__bytes_write.sum (profiles/k_cgprod_cg_product_dense_m1000_n200000_f32.md)"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["dense", "sparse", "scaled", "serving", "svm",
                                           "matvec"],
                    default="dense",
                    help="dense: Gaussian m x n; sparse: CSR with --nnz-per-col nonzeros per "
                         "column; scaled: dense with column scales 10^U(-3,3); serving: a "
                         "Poisson stream of mixed dense/CSR LPs through the serving loop; svm: "
                         "the l1-SVM LP on synthetic separable data with a Table 1 shape; "
                         "matvec: the CG product A D^2 A^T v alone (one step = one product)")
    ap.add_argument("--svm-shape", choices=["arcene", "dexter", "drivface", "gene_rna"],
                    default="arcene")
    ap.add_argument("--sweep", action="store_true",
                    help="svm: sweep sketch width w and relative CG tolerance (Fig. 2) instead "
                         "of timing one configuration")
    ap.add_argument("--sketch-study", action="store_true",
                    help="dense or svm: compare CountSketch (s=1), sparse sign s=2/4/8 and the "
                         "Gaussian sketch at w = 4m, and the factor routes, instead of timing "
                         "one configuration")
    ap.add_argument("--requests", type=int, default=256, help="serving: stream length")
    ap.add_argument("--rate", type=str, default="2000",
                    help="serving: arrival rates in LP/s (comma separated, one run each)")
    ap.add_argument("--max-live", type=int, default=16, help="serving: concurrent instances")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serving: admission budget")
    ap.add_argument("--plain-sample", type=int, default=0,
                    help="serving: requests solved one at a time on the plain FP64 path "
                         "(0: all of them, the same requests as the batched path)")
    ap.add_argument("--no-serving", action="store_true",
                    help="dense: leave out the serving measurement of the default line")
    ap.add_argument("--serving-requests", type=int, default=256,
                    help="dense: requests of the serving measurement in the default line")
    ap.add_argument("--serving-rates", type=str, default="16,2000",
                    help="dense: arrival rates (LP/s) of the serving measurement, one below and "
                         "one above saturation")
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--nnz-per-col", type=int, default=8)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--stream", choices=["same", "f32", "bf16", "f16"], default="same")
    ap.add_argument("--sketch-s", type=int, default=4)
    ap.add_argument("--sketch", choices=["sparse", "gaussian"], default="sparse",
                    help="sparse sign sketch with --sketch-s nonzeros per row, or Gaussian")
    ap.add_argument("--cg-batch", type=int, default=4)
    ap.add_argument("--cg-max-iter", type=int, default=None,
                    help="cap on CG iterations per solve (default: the library's, 500)")
    ap.add_argument("--study-sketches", type=str, default=None,
                    help="sketch study: comma-separated subset of s values to run (e.g. '1')")
    ap.add_argument("--no-gram-tc", action="store_true",
                    help="Gram product of the factor in double-float on the FP32 pipes instead "
                         "of the tensor cores")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed launch-shape rule for the CG product instead of the autotuner")
    ap.add_argument("--persistent", action="store_true",
                    help="run CG solves as one persistent cooperative launch each (lp_params.persistent_cg)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="host-driven CG loop instead of one CUDA graph launch per CG solve")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=20_000)
    ap.add_argument("--cpu-sample-iters", type=int, default=4)
    args = ap.parse_args()
    if args.workload == "svm":
        import synth

        pts, feats = synth.SVM_SHAPES[args.svm_shape]
        args.m, args.n = pts, 2 * feats + 2 + pts
    defaults = {"dense": (1000, 200_000), "sparse": (5000, 2_000_000), "scaled": (2000, 500_000),
                "serving": (512, 102_400), "svm": (args.m, args.n), "matvec": (1000, 200_000)}
    dm, dn = defaults[args.workload]
    args.m = args.m or dm
    args.n = args.n or dn
    return args


# --------------------------------------------------------------------------- distributed

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def shard(count: int, rank: int, world: int):
    """Requests of the serving stream this rank submits: i = rank, rank + world, ..."""
    return list(range(rank, count, world))


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- helpers

def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_sha1():
    path = os.path.join(ROOT, "paper_2003_08072_gb300", "csrc", "k_cgprod.cu")
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def metric_name(args):
    if (args.workload, args.m, args.n, args.dtype) == ("dense", 1000, 200_000, "f32"):
        return "IPM LPs/s (Algorithm 2 to tolerance, dense m=1000 n=200000 FP32 LP)"
    return f"IPM LPs/s (Algorithm 2 to tolerance, {args.workload} m={args.m} n={args.n})"


def workload_name(args):
    if args.workload == "svm":
        pts = args.m
        return (f"l1-SVM LP ({args.svm_shape} shape of Table 1: {pts} points, "
                f"{(args.n - 2 - pts) // 2} features; synthetic separable Gaussian data), "
                f"m={args.m} n={args.n} A {args.dtype.upper()}, Algorithm 2 to scaled KKT 1e-8")
    if args.workload == "sparse":
        return (f"sparse LP m={args.m} n={args.n}, {args.nnz_per_col} nonzeros per column (CSR, "
                f"FP32 values, int32 columns), feasible by construction, Algorithm 2 to scaled "
                f"KKT 1e-8")
    kind = "dense Gaussian" if args.workload == "dense" else "dense Gaussian, column scales 10^U(-3,3),"
    return (f"{kind} LP m={args.m} n={args.n} A {args.dtype.upper()} "
            f"(feasible by construction), Algorithm 2 to scaled KKT 1e-8")


def make_lp(args):
    import numpy as np

    import synth

    if args.workload == "sparse":
        return synth.sparse_lp(0, args.m, args.n, nnz_per_col=args.nnz_per_col)
    np_dt = np.float32 if args.dtype == "f32" else np.float64
    if args.workload == "svm":
        return synth.l1svm_lp(1, args.m, (args.n - 2 - args.m) // 2, dtype=np_dt)
    scale = (-3, 3) if args.workload == "scaled" else None
    return synth.dense_lp(0, args.m, args.n, dtype=np_dt, col_scale=scale)


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info

        th = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if th:
            return max(th)
    except ImportError:
        pass
    return os.cpu_count()


def sample_lp(args):
    """The instance the oracle is timed on: the workload's generator with n_s columns (the whole
    instance for the l1-SVM LPs, which are small).  Returns (lp, A as FP64, n_s)."""
    import numpy as np

    import synth

    ns = min(args.cpu_sample_n, args.n)
    np_dt = np.float32 if args.dtype == "f32" else np.float64
    if args.workload == "svm":
        lp = synth.l1svm_lp(1, args.m, (args.n - 2 - args.m) // 2, dtype=np_dt)
        return lp, lp.A.astype(np.float64), args.n
    if args.workload == "sparse":
        lp = synth.sparse_lp(0, args.m, ns, nnz_per_col=args.nnz_per_col)
        return lp, lp.to_scipy(), ns
    lp = synth.dense_lp(0, args.m, ns, dtype=np_dt,
                        col_scale=(-3, 3) if args.workload == "scaled" else None)
    return lp, lp.A.astype(np.float64), ns


def oracle_run_record(args):
    """The oracle's own end-to-end run of the full workload instance, stored by
    tests/golden/make_oracle_run.py (IPM iterations, CG products, objective), or None."""
    if args.workload not in ("dense", "scaled", "sparse") or args.sketch != "sparse":
        return None
    path = os.path.join(ROOT, "tests", "golden", f"oracle_run_{args.workload}_m{args.m}_n{args.n}"
                        f"_{args.dtype}_s{args.sketch_s}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


_FULL_LP = {}


def oracle_sample(args, iters_per_lp: float, iters_source: str):
    """Times the FP64 oracle's Algorithm 2 on the full workload instance itself (A as FP64):
    its first --cpu-sample-iters IPM iterations, each with the sketch, QR factor, PCG and
    correction at the real m and n.  LP/s = 1 / (time per iteration x IPM iterations per LP).
    The first iterations need fewer CG iterations than the later ones, so this favours the
    CPU.  Small workloads (the l1-SVM shapes) are solved to the end instead."""
    import numpy as np

    from oracle import iipm

    key = (args.workload, args.m, args.n, args.dtype, args.svm_shape)
    if key not in _FULL_LP:
        lp = make_lp(args)
        A = lp.to_scipy() if args.workload == "sparse" else np.ascontiguousarray(lp.A, dtype=np.float64)
        _FULL_LP.clear()
        _FULL_LP[key] = (lp, A)
    lp, A = _FULL_LP[key]
    whole = args.workload == "svm"
    prm = iipm.Params(ipm_max_iter=200 if whole else args.cpu_sample_iters,
                      sketch_s=args.sketch_s,
                      sketch_kind="gaussian" if args.sketch == "gaussian" else "sparse")
    t0 = time.perf_counter()
    r = iipm.ipm_solve(A, lp.b, lp.c, prm)
    dt = time.perf_counter() - t0
    if whole:
        return 1.0 / dt, (f"oracle Algorithm 2 (FP64 numpy/scipy) solving the whole instance "
                          f"({r.iters} IPM iterations, {dt:.1f} s)"), dt
    per_iter = dt / max(r.iters, 1)
    lp_s = 1.0 / (per_iter * iters_per_lp)
    sample = (f"oracle Algorithm 2 (FP64 numpy/scipy) on the full m={args.m}, n={args.n} "
              f"instance: its first {r.iters} IPM iterations ({r.cg_total} CG products, "
              f"{dt:.1f} s), time per iteration x {iters_per_lp:g} IPM iterations per LP "
              f"({iters_source})")
    return lp_s, sample, dt


# --------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import synth
    import paper_2003_08072_gb300 as pkg

    if rank == 0:
        pkg.build.build()
    barrier(world)
    pkg.load(build_if_missing=False)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lp = make_lp(args)
    prm = pkg.lp_params_default()
    prm.sketch_s = args.sketch_s
    prm.sketch_kind = 1 if args.sketch == "gaussian" else 0
    prm.cg_batch = args.cg_batch
    if args.cg_max_iter:
        prm.cg_max_iter = args.cg_max_iter
    prm.use_graphs = 0 if args.no_graphs else 1
    prm.persistent_cg = 1 if args.persistent else 0
    prm.gram_tensor_cores = 0 if args.no_gram_tc else 1
    prm.autotune = 0 if args.no_autotune else 1
    sparse = args.workload == "sparse"
    sd = (args.dtype if not sparse else "f32") if args.stream == "same" else args.stream
    prm.stream_dtype = pkg.DTYPE_CODES[sd] if not sparse else pkg.LP_F64
    a_code = pkg.LP_F32 if (args.dtype == "f32" or sparse) else pkg.LP_F64
    stream = torch.cuda.current_stream(dev)

    # ---------------- device-resident runs
    b_dev = torch.from_numpy(lp.b).to(dev)
    c_dev = torch.from_numpy(lp.c).to(dev)
    if sparse:
        keep = [torch.from_numpy(v).to(dev) for v in (lp.indptr, lp.indices, lp.values)]
        ctx = pkg.lp_create(args.m, args.n, pkg.LP_CSR, a_code, keep[2], keep[0], keep[1],
                            lp.nnz, b_dev, c_dev, prm, stream.cuda_stream)
        a_bytes = lp.values.nbytes + lp.indices.nbytes + lp.indptr.nbytes
    else:
        keep = [torch.from_numpy(lp.At).to(dev)]
        ctx = pkg.lp_create(args.m, args.n, pkg.LP_DENSE_COLMAJOR, a_code, keep[0], None, None, 0,
                            b_dev, c_dev, prm, stream.cuda_stream)
        a_bytes = lp.At.nbytes
    x = torch.empty(args.n, dtype=torch.float64, device=dev)
    y = torch.empty(args.m, dtype=torch.float64, device=dev)
    s = torch.empty(args.n, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        info = pkg.lp_ipm_solve(ctx, x, y, s)
    # the timed region runs without the library's event profiling
    pkg.lp_profile_enable(ctx, False)
    launches0 = pkg.lp_profile_read(ctx, reset=True).launches
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(pkg.lp_ipm_solve(ctx, x, y, s))
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = pkg.lp_profile_read(ctx).launches - launches0
    # one more solve, untimed, with CUDA events on the library's stream around every phase and
    # every CG product: the per-launch duration of the CG product and the phase split
    pkg.lp_profile_enable(ctx, True)
    pkg.lp_profile_read(ctx, reset=True)
    pkg.lp_ipm_solve(ctx, x, y, s)
    prof = pkg.lp_profile_read(ctx)
    pkg.lp_profile_enable(ctx, False)
    obj = float(torch.dot(c_dev, x))
    pkg.lp_destroy(ctx)
    del keep
    torch.cuda.empty_cache()
    t_max = max_over_ranks(elapsed, world)

    # ---------------- end to end from host buffers through the C ABI
    k_e2e = args.e2e_steps if args.e2e_steps is not None else args.steps
    if sparse:
        host = [torch.from_numpy(v).pin_memory() for v in (lp.indptr, lp.indices, lp.values)]
    else:
        host = [torch.from_numpy(lp.At).pin_memory()]
    b_h = torch.from_numpy(lp.b).pin_memory()
    c_h = torch.from_numpy(lp.c).pin_memory()
    xh = torch.empty(args.n, dtype=torch.float64).pin_memory()
    yh = torch.empty(args.m, dtype=torch.float64).pin_memory()
    sh = torch.empty(args.n, dtype=torch.float64).pin_memory()
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        if sparse:
            cx = pkg.lp_create(args.m, args.n, pkg.LP_CSR, a_code, host[2], host[0], host[1],
                               lp.nnz, b_h, c_h, prm, stream.cuda_stream)
        else:
            cx = pkg.lp_create(args.m, args.n, pkg.LP_DENSE_COLMAJOR, a_code, host[0], None, None,
                               0, b_h, c_h, prm, stream.cuda_stream)
        pkg.lp_ipm_solve(cx, xh, yh, sh)
        pkg.lp_destroy(cx)
    torch.cuda.synchronize(dev)
    e2e_t = max_over_ranks(time.perf_counter() - t0, world) if k_e2e else float("nan")
    h2d = a_bytes + 8 * (args.m + args.n)
    d2h = 8 * (2 * args.n + args.m)

    if rank != 0:
        return None
    peak, peak_kind = read_peaks()
    mv_avg_s = prof.matvec_ms / 1e3 / max(prof.matvec_count, 1)
    achieved = prof.matvec_bytes / mv_avg_s / 1e9 if prof.matvec_count else None
    traffic = None
    if (not sparse and args.workload == "dense" and (args.m, args.n, sd) == (1000, 200_000, "f32")
            and NCU_TRAFFIC["source_sha1"] == kernel_sha1() and NCU_TRAFFIC["bytes_per_launch"]):
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    ipm_iters = statistics.mean(i.ipm_iters for i in infos)
    cg_total = statistics.mean(i.cg_iters_total for i in infos)
    value = world * args.steps / t_max
    line = {
        "metric": metric_name(args),
        "value": value,
        "unit": "LP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": sd,
        "data": "synthetic",
        "config": {
            "workload": workload_name(args),
            "m": args.m, "n": args.n, "a_dtype": "f32" if sparse else args.dtype,
            "stream_dtype": sd,
            "sketch": (f"sparse sign s={args.sketch_s}, w=4m" if args.sketch == "sparse" else
                       "Gaussian, w=4m"), "cg_rel_tol": prm.cg_rel_tol,
            "tol": prm.tol, "sigma": prm.sigma, "gamma": prm.gamma,
            "l2": "inputs larger than L2 (A is %.0f MB)" % (a_bytes / 1e6),
            "parallelism": f"replicas x{world}",
            "cg_loop": ("persistent cooperative launch per CG solve" if args.persistent else
                        "host-driven" if args.no_graphs else "CUDA graph per CG solve"),
            "gram": ("double-float, FP32 pipes" if args.no_gram_tc else
                     "tensor cores (tcgen05, exact BF16 digit slices)"),
        },
        "roofline": {
            "kernel": ("k_csc" if sparse else "k_cgprod") + " (CG product A D^2 A^T v)",
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "peak_kind": f"{peak_kind} hbm_gbs",
            "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "traffic_source": (f"recorded constant: dram__bytes_read.sum + dram__bytes_write.sum "
                               f"per launch from one ncu capture ({NCU_TRAFFIC['case']}) of the "
                               f"same k_cgprod.cu source (sha1 {NCU_TRAFFIC['source_sha1'][:12]}); "
                               "not a counter of this run") if traffic else None,
            "bytes_per_launch": prof.matvec_bytes,
            "avg_launch_us": 1e6 * mv_avg_s,
            "launches": int(prof.matvec_count),
            "timing": "CUDA events on the library's stream around every CG product of one "
                      "profiled LP solve run after the timed steps (the timed steps run without "
                      "events)",
            "autotune": prof.as_dict()["tune"],
        },
        "e2e": {"value": (world * k_e2e / e2e_t) if k_e2e else None, "unit": "LP/s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": k_e2e},
        "gpu_launches": int(launches),
        "clocks": clk,
        "ipm_iters_per_lp": ipm_iters,
        "cg_iters_per_lp": cg_total,
        "cg_graph_solves_per_lp": statistics.mean(i.cg_graph_solves for i in infos),
        "cg_persistent_solves_per_lp": statistics.mean(i.cg_persistent_solves for i in infos),
        "objective": obj,
        "kkt": max(infos[-1].rp_rel, infos[-1].rd_rel, infos[-1].gap_rel),
        "phase_ms_per_lp": prof.as_dict()["phase_ms"],
    }
    if world == 1 and not args.no_cpu_baseline:
        rec = oracle_run_record(args)
        if rec:
            it_lp, src = rec["ipm_iters"], "the oracle's own run of this instance (tests/golden)"
        else:
            it_lp, src = ipm_iters, "the GPU solve's count, which parity tests hold within one of the oracle's"
        v, sample, secs = oracle_sample(args, it_lp, src)
        line["cpu_baseline"] = {"value": v, "unit": "LP/s", "cores": cpu_threads(),
                                "kind": "oracle", "sample": sample}
        if rec:
            line["oracle_full_run"] = {k: rec[k] for k in ("ipm_iters", "cg_total", "objective",
                                                            "kkt") if k in rec}
            line["objective_rel_diff_vs_oracle"] = abs(obj - rec["objective"]) / abs(rec["objective"])
    else:
        line["cpu_baseline"] = None
    if args.workload == "dense" and not args.no_serving and args.serving_requests > 0:
        line["serving"] = serving_section(args, rank, world, local)
    return line


def serving_section(args, rank, world, local):
    """The serving half of the metric on the C5 request generator: the serving loop (BF16
    stream, continuous batching) at one arrival rate below and one above saturation, and the
    plain one-at-a-time FP64 path on the same requests."""
    import numpy as np

    reqs, insts = serving_instances(args.serving_requests)
    rates = [float(r) for r in args.serving_rates.split(",")]
    out = serving_measure(args, rank, world, local, rates, insts, reqs)
    if rank != 0:
        return None
    runs, plain, comp = out
    best = max(runs, key=lambda r: r["value"])
    return {"metric": "serving LPs/s with p50/p99 latency, batched BF16 vs plain FP64",
            "workload": serving_workload_name(len(insts)), "unit": "LP/s",
            "value": best["value"], "runs": runs, "plain_fp64": plain,
            "speedup_vs_plain_fp64": best["value"] / plain["value"], **comp,
            "max_live": args.max_live, "budget_gb": args.budget_gb}


# --------------------------------------------------------------------------- serving

def _make_request(req):
    import synth

    kind, m, n, seed = req
    return kind, synth.serving_instance(kind, m, n, seed)


def serving_instances(count):
    """The request stream: (kind, m, n, seed) from synth.serving_requests and its instances,
    generated in a spawned process pool (before any CUDA use of the pool's workers)."""
    import multiprocessing as mp

    import synth

    reqs = synth.serving_requests(count)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        return reqs, pool.map(_make_request, reqs, chunksize=1)


def _submit(srv, pkg, kind, lp):
    if kind == "dense":
        return srv.submit(lp.m, lp.n, pkg.LP_DENSE_COLMAJOR, lp.At, lp.b, lp.c)
    return srv.submit(lp.m, lp.n, pkg.LP_CSR, lp.values, lp.b, lp.c, indptr=lp.indptr,
                      indices=lp.indices)


def plain_fp64(pkg, insts, idx):
    """The requests idx one at a time on the plain path: A in FP64, FP64 stream, one context
    per request, host buffers; returns (LP/s, {i: objective}, seconds)."""
    import numpy as np

    prm = pkg.lp_params_default()
    data = []
    for i in idx:
        kind, lp = insts[i]
        if kind == "dense":
            data.append((i, kind, lp, np.ascontiguousarray(lp.At, dtype=np.float64)))
        else:
            data.append((i, kind, lp, lp.values.astype(np.float64)))
    objs = {}
    t0 = time.perf_counter()
    for i, kind, lp, vals in data:
        x, y, s = np.empty(lp.n), np.empty(lp.m), np.empty(lp.n)
        if kind == "dense":
            ctx = pkg.lp_create(lp.m, lp.n, pkg.LP_DENSE_COLMAJOR, pkg.LP_F64, vals, None, None,
                                0, lp.b, lp.c, prm, None)
        else:
            ctx = pkg.lp_create(lp.m, lp.n, pkg.LP_CSR, pkg.LP_F64, vals, lp.indptr, lp.indices,
                                lp.nnz, lp.b, lp.c, prm, None)
        pkg.lp_ipm_solve(ctx, x, y, s)
        pkg.lp_destroy(ctx)
        objs[i] = float(lp.c @ x)
    secs = time.perf_counter() - t0
    return len(idx) / secs, objs, secs


def serving_measure(args, rank, world, local, rates, insts, reqs):
    """Serves the request stream at each arrival rate through the serving loop (batched, BF16
    stream for dense requests), then solves the same requests one at a time on the plain FP64
    path.  Returns (runs, plain, objective comparison) on rank 0."""
    import numpy as np

    import paper_2003_08072_gb300 as pkg
    import synth

    mine = shard(len(insts), rank, world)
    prm = pkg.lp_params_default()
    prm.stream_dtype = pkg.LP_BF16
    runs = []
    objs_batched, kkt_of = {}, {}
    for rate in rates:
        arrivals = synth.poisson_arrivals(len(insts), rate)
        srv = pkg.LPServer(int(args.budget_gb * 2**30), max_live=args.max_live, params=prm)
        # warm-up: one request of each kind, untimed
        for i in range(2):
            t = _submit(srv, pkg, *insts[i])
            while srv.wait_any(60_000) != t:
                pass
            srv.result(t)
        clk = ClockSampler(local)
        clk.start()
        barrier(world)
        results = {}
        done = threading.Event()

        def collect():
            while len(results) < len(mine):
                t = srv.wait_any(1000)
                if t is not None:
                    results[t] = srv.result(t)
            done.set()

        th = threading.Thread(target=collect, daemon=True)
        th.start()
        t0 = time.perf_counter()
        tickets = {}
        for i in mine:
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[_submit(srv, pkg, *insts[i])] = i
        done.wait()
        elapsed = max_over_ranks(time.perf_counter() - t0, world)
        clocks = clk.stop()
        stats = srv.stats()
        srv.close()
        lat = np.array([r["latency_s"] for r in results.values()]) * 1e3
        qd = np.array([r["queued_s"] for r in results.values()]) * 1e3
        bad = [(insts[tickets[t]][0], insts[tickets[t]][1].m, insts[tickets[t]][1].n,
                r["status"], r["error"]) for t, r in results.items() if r["status"] != 0]
        for t, r in results.items():
            i = tickets[t]
            objs_batched[i] = float(insts[i][1].c @ r["x"])
            if r["status"] == 0:
                kkt_of[i] = max(kkt_of.get(i, 0.0), r["info"].rp_rel, r["info"].rd_rel,
                                r["info"].gap_rel)
        runs.append({"rate": rate, "value": world * len(mine) / elapsed, "seconds": elapsed,
                     "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                    "p99": float(np.percentile(lat, 99)),
                                    "mean": float(lat.mean())},
                     "queued_ms": {"p50": float(np.percentile(qd, 50)),
                                   "p99": float(np.percentile(qd, 99))},
                     "failed": len(bad), "failures": bad[:4], "peak_live": stats["peak_live"],
                     "mem_peak_gb": stats["mem_peak"] / 2**30, "clocks": clocks})
    if rank != 0:
        return None
    k = len(insts) if args.plain_sample <= 0 else min(args.plain_sample, len(insts))
    plain_v, plain_objs, plain_s = plain_fp64(pkg, insts, list(range(k)))
    rel = [abs(objs_batched[i] - plain_objs[i]) / abs(plain_objs[i]) for i in plain_objs
           if i in objs_batched]
    plain = {"value": plain_v, "unit": "LP/s", "seconds": plain_s,
             "sample": (f"the same {k} requests" if k == len(insts) else f"the first {k} requests")
             + " one at a time (FP64 A, FP64 stream, one context each, host buffers)"}
    comp = {"max_rel_objective_diff_vs_plain": max(rel) if rel else None,
            "max_scaled_kkt": max(kkt_of.values()) if kkt_of else None,
            "same_requests": k == len(insts)}
    return runs, plain, comp


def run_serving(args, rank, world, local):
    import numpy as np

    reqs, insts = serving_instances(args.requests)
    import torch

    import paper_2003_08072_gb300 as pkg

    pkg.load(build_if_missing=False)
    torch.cuda.set_device(local)
    rates = [float(r) for r in args.rate.split(",")]
    out = serving_measure(args, rank, world, local, rates, insts, reqs)
    if rank != 0:
        return None
    runs, plain, comp = out
    best = max(runs, key=lambda r: r["value"])
    dense_elems = [m * n for kind, m, n, _ in reqs if kind == "dense"]
    return {
        "metric": "serving LPs/s (mixed dense FP32 / CSR 1% LP stream, Poisson arrivals)",
        "value": best["value"], "unit": "LP/s", "n_gpus": world, "steps": len(insts),
        "warmup": 2, "ms_per_step": 1e3 * best["seconds"] / len(insts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": serving_workload_name(len(insts)),
                   "mean_dense_elements": float(np.mean(dense_elems)),
                   "max_live": args.max_live, "budget_gb": args.budget_gb,
                   "stream_dtype": "bf16 (dense), f32 (CSR values)",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": best["latency_ms"], "queued_ms": best["queued_ms"],
        "runs": runs,
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": best["value"] / plain["value"],
        **comp,
        "clocks": best["clocks"],
    }


def serving_workload_name(count):
    return (f"{count} requests, m ~ U{{16..512}}, n = m U{{20..200}}, even requests dense "
            "Gaussian FP32, odd CSR at 1% density, Algorithm 2 to scaled KKT 1e-8 each")


# --------------------------------------------------------------------------- (w, tolCG) sweep

def run_sweep(args, rank, world, local):
    """Outer (IPM) and inner (CG) iterations against the sketch width w and the relative CG
    tolerance tolCG (the paper's Fig. 2 study), with the relative rule alone deciding CG's stop,
    and the condition numbers of Table 1 at the final iterate: kappa(A D^2 A^T) and the
    preconditioned kappa(Q^-1/2 A D^2 A^T Q^-1/2) from the same sketch (FP64, host)."""
    import numpy as np
    import torch

    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    if rank != 0:
        return None
    pkg.load()
    torch.cuda.set_device(local)
    lp = make_lp(args)
    A = lp.A.astype(np.float64)
    rows = []
    for wm in (2, 4, 8, 16):
        for tol in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
            prm = pkg.lp_params_default()
            prm.sketch_w = (wm * args.m + prm.sketch_s - 1) // prm.sketch_s * prm.sketch_s
            prm.cg_rel_tol = tol
            prm.cg_theory_rule = 0
            ctx = B.lp_create(args.m, args.n, B.LP_DENSE_COLMAJOR,
                              B.LP_F32 if args.dtype == "f32" else B.LP_F64, lp.At, None, None, 0,
                              lp.b, lp.c, prm, None)
            x, y, s = np.empty(args.n), np.empty(args.m), np.empty(args.n)
            t0 = time.perf_counter()
            info = B.lp_ipm_solve(ctx, x, y, s, check=False)
            secs = time.perf_counter() - t0
            row = {"w": f"{wm}m", "tolCG": tol, "status": info.status, "outer": info.ipm_iters,
                   "inner": info.cg_iters_total, "inner_per_outer": info.cg_iters_total /
                   max(info.ipm_iters, 1), "ms": 1e3 * secs,
                   "kkt": max(info.rp_rel, info.rd_rel, info.gap_rel)}
            if tol == 1e-6 and info.status == 0:
                d2 = x / s
                K = A @ (d2[:, None] * A.T)
                G = np.empty((prm.sketch_w, args.m))
                Gt = torch.empty(prm.sketch_w, args.m, dtype=torch.float64, device="cuda")
                B.lp_sketch(ctx, torch.from_numpy(np.sqrt(d2)).cuda(), info.ipm_iters - 1, Gt)
                G = Gt.cpu().numpy().T
                lam, V = np.linalg.eigh(G @ G.T)
                Qmh = (V / np.sqrt(lam)) @ V.T
                ev = np.linalg.eigvalsh(Qmh @ K @ Qmh)
                evk = np.linalg.eigvalsh(K)
                row["kappa_standard"] = float(evk[-1] / evk[0])
                row["kappa_preconditioned"] = float(ev[-1] / ev[0])
            B.lp_destroy(ctx)
            rows.append(row)
    return {"metric": "outer / inner iterations against sketch width and tolCG (Fig. 2 study)",
            "value": None, "unit": "iterations", "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic", "config": {"workload": workload_name(args)}, "sweep": rows}


# --------------------------------------------------------------------------- sketch study

def preconditioned_kappa(K, L):
    """kappa of L^T K L (the spectrum of M K for the preconditioner M = L L^T), or None when
    the result is not positive definite."""
    import numpy as np

    ev = np.linalg.eigvalsh(L.T @ K @ L)
    return float(ev[-1] / ev[0]) if ev[0] > 0 else None


def run_sketch_study(args, rank, world, local):
    """CountSketch (s = 1) against the sparse sign sketch with s = 2, 4, 8 nonzeros per row and
    the Gaussian sketch (dense A), all at w = 4m (rounded up to a multiple of s) with the default CG rules: outer and inner
    iterations and time per LP, and at the final iterate (W of the last IPM iteration):
    kappa(Q) for Q = G G^T, the preconditioned kappa with the exact Q^-1/2 (eigendecomposition,
    the paper's SVD route), with the GPU's preconditioner M (Gram product and Cholesky inverse
    in double-float) and with a host QR factor of G^T (FP64), and ||M Q - I||_2 for the last
    two.  All host arithmetic is FP64."""
    import numpy as np
    import scipy.linalg as sl
    import torch

    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    if rank != 0:
        return None
    pkg.load()
    torch.cuda.set_device(local)
    lp = make_lp(args)
    A = lp.A.astype(np.float64)
    m, n = args.m, args.n
    variants = [("CountSketch s=1", B.LP_SKETCH_SPARSE, 1), ("sparse sign s=2", B.LP_SKETCH_SPARSE, 2),
                ("sparse sign s=4", B.LP_SKETCH_SPARSE, 4), ("sparse sign s=8", B.LP_SKETCH_SPARSE, 8)]
    if 8.0 * m * m * n <= 3e11:   # the Gaussian A D W costs 2 m n w = 8 m^2 n flops per IPM iteration
        variants.append(("Gaussian", B.LP_SKETCH_GAUSSIAN, 4))
    if args.study_sketches:
        keep = {int(v) for v in args.study_sketches.split(",")}
        variants = [v for v in variants if v[1] == B.LP_SKETCH_SPARSE and v[2] in keep]
    rows = []
    for name, kind, ns in variants:
        prm = pkg.lp_params_default()
        if args.cg_max_iter:
            prm.cg_max_iter = args.cg_max_iter
        prm.sketch_kind = kind
        prm.sketch_s = ns
        prm.sketch_w = (4 * m + ns - 1) // ns * ns      # w = 4m, rounded up to a multiple of s
        ctx = B.lp_create(m, n, B.LP_DENSE_COLMAJOR, B.LP_F32 if args.dtype == "f32" else B.LP_F64,
                          lp.At, None, None, 0, lp.b, lp.c, prm, None)
        x, y, s = np.empty(n), np.empty(m), np.empty(n)
        t0 = time.perf_counter()
        info = B.lp_ipm_solve(ctx, x, y, s, check=False)
        secs = time.perf_counter() - t0
        row = {"sketch": name, "status": info.status, "outer": info.ipm_iters,
               "inner": info.cg_iters_total,
               "inner_per_outer": info.cg_iters_total / max(info.ipm_iters, 1),
               "ms": 1e3 * secs, "kkt": max(info.rp_rel, info.rd_rel, info.gap_rel),
               "obj": info.obj}
        if info.status == 0:
            w = prm.sketch_w
            d2 = x / s
            K = A @ (d2[:, None] * A.T)
            Gt = torch.empty(w, m, dtype=torch.float64, device="cuda")
            B.lp_sketch(ctx, torch.from_numpy(np.sqrt(d2)).cuda(), info.ipm_iters - 1, Gt)
            G = Gt.cpu().numpy().T
            Q = G @ G.T
            lam, V = np.linalg.eigh(Q)
            row["kappa_Q"] = float(lam[-1] / lam[0]) if lam[0] > 0 else None
            row["kappa_standard"] = float(np.linalg.cond(K))
            row["kappa_pre_exact"] = (preconditioned_kappa(K, V / np.sqrt(lam))
                                      if lam[0] > 0 else None)
            R = np.linalg.qr(G.T, mode="r")
            X = sl.solve_triangular(R, np.eye(m))
            row["kappa_pre_qr"] = preconditioned_kappa(K, X)
            row["qr_MQ_minus_I"] = float(np.linalg.norm(X @ (X.T @ Q) - np.eye(m), 2))
            Qd = torch.empty(m, m, dtype=torch.float64, device="cuda")
            Mi = torch.empty(m, m, dtype=torch.float64, device="cuda")
            try:
                B.lp_factor(ctx, Gt, Qd, Mi)
                M = Mi.cpu().numpy()
                M = 0.5 * (M + M.T)
                row["gpu_MQ_minus_I"] = float(np.linalg.norm(M @ Q - np.eye(m), 2))
                try:
                    row["kappa_pre_gpu"] = preconditioned_kappa(K, np.linalg.cholesky(M))
                except np.linalg.LinAlgError:
                    row["kappa_pre_gpu"] = None
            except pkg.LPError as e:
                row["gpu_factor"] = f"status {e.status} (the IPM's own factor shifts Q here)"
        B.lp_destroy(ctx)
        rows.append(row)
    return {"metric": "iterations and condition numbers against the sketch kind (w = 4m)",
            "value": None, "unit": "iterations", "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic", "config": {"workload": workload_name(args)}, "study": rows}


# --------------------------------------------------------------------------- reference arm

def oracle_iters_per_lp(args):
    """IPM iterations per LP for the reference arm: the oracle's own run of this instance
    (tests/golden), else the oracle solving a column sample of it to the end (a stand-in for
    workloads without a stored run)."""
    import numpy as np

    from oracle import iipm

    rec = oracle_run_record(args)
    if rec:
        return float(rec["ipm_iters"]), "the oracle's own run of this instance (tests/golden)"
    lp, A, ns = sample_lp(args)
    r = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(sketch_s=args.sketch_s))
    return float(r.iters), f"the oracle's run of the n={ns} column sample of this instance"


def run_reference(args, rank, world):
    """The FP64 oracle, as it stands, on the host cores: each step one bounded sample."""
    if rank != 0:
        return None
    iters_per_lp, src = oracle_iters_per_lp(args)
    for _ in range(args.warmup):
        oracle_sample(args, iters_per_lp, src)
    vals, secs = [], 0.0
    sample = ""
    for _ in range(args.steps):
        v, sample, dt = oracle_sample(args, iters_per_lp, src)
        vals.append(v)
        secs += dt
    value = statistics.mean(vals)
    return {
        "impl": "reference",
        "metric": metric_name(args),
        "value": value, "unit": "LP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "m": args.m, "n": args.n},
        "cpu_baseline": {"value": value, "unit": "LP/s", "cores": cpu_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "LP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_matvec(args, rank, world, local):
    """The PCG matvec alone: y = A D^2 A^T v through lp_normal_matvec on the streamed copy
    (the staged product k_cgprod plus the reduction of its partial sums), A resident in HBM
    and larger than L2.  value = algorithmic GB/s (m n b_A + 4 n + 16 m bytes per product)."""
    import numpy as np
    import torch

    import synth
    import paper_2003_08072_gb300 as pkg

    pkg.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lp = synth.dense_lp(0, args.m, args.n, dtype=np.float32)
    sd = "f32" if args.stream == "same" else args.stream
    prm = pkg.lp_params_default()
    prm.stream_dtype = pkg.DTYPE_CODES[sd]
    stream = torch.cuda.current_stream(dev)
    At = torch.from_numpy(lp.At).to(dev)
    ctx = pkg.lp_create(args.m, args.n, pkg.LP_DENSE_COLMAJOR, pkg.LP_F32, At, None, None, 0,
                        torch.from_numpy(lp.b).to(dev), torch.from_numpy(lp.c).to(dev), prm,
                        stream.cuda_stream)
    del At
    x, _, s = synth.iterate_point(1, args.m, args.n, spread=2.0)
    d2 = torch.from_numpy(x / s).to(dev)
    v = torch.from_numpy(np.random.default_rng(2).standard_normal(args.m)).to(dev)
    y = torch.empty(args.m, dtype=torch.float64, device=dev)
    code = pkg.DTYPE_CODES[sd]
    for _ in range(args.warmup):
        pkg.lp_normal_matvec(ctx, d2, v, y, None, code)
    barrier(world)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        pkg.lp_normal_matvec(ctx, d2, v, y, None, code)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    pkg.lp_destroy(ctx)
    esz = {"f32": 4, "bf16": 2, "f16": 2}[sd]
    nbytes = args.m * args.n * esz + 4 * args.n + 16 * args.m
    if rank != 0:
        return None
    peak, kind = read_peaks()
    gbs = world * args.steps * nbytes / t / 1e9
    return {"metric": f"PCG matvec HBM GB/s (A D^2 A^T v, dense m={args.m} n={args.n}, "
                      f"A streamed {sd.upper()})",
            "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": sd,
            "data": "synthetic",
            "config": {"workload": f"A D^2 A^T v, Gaussian A m={args.m} n={args.n}",
                       "l2": f"inputs larger than L2 (A is {args.m * args.n * esz / 1e6:.0f} MB)",
                       "bytes_per_product": nbytes},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak,
                         "peak_kind": f"{kind} hbm_gbs", "unit": "GB/s", "frac": gbs / peak,
                         "traffic": None}}


def main():
    args = parse_args()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "serving":
        line = run_serving(args, rank, world, local)
    elif args.workload == "matvec":
        line = run_matvec(args, rank, world, local)
    elif args.workload == "svm" and args.sweep:
        line = run_sweep(args, rank, world, local)
    elif args.sketch_study and args.workload in ("dense", "svm"):
        line = run_sketch_study(args, rank, world, local)
    else:
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
