"""Benchmark: ACR factor + solve of the n = 128 variable-coefficient workload on GB300.

Workload: -div(kappa grad u) = f, 7-point, Dirichlet, n = 128 (N = 2,097,152),
kappa = exp(g) with g a Gaussian random field (squared-exponential kernel,
length 0.1, sigma 1, seed 1); HODLR leaf 64, truncation tolerance 1e-6;
64 right-hand sides uniform on [-1, 1] (seeds 100..163) solved together.
One step = acr_factor in FP32 + FP64 iterative refinement (ACR as the
preconditioner) until every column has ||b - A x|| / ||b|| <= 1e-10.
Metric: DOF/s = N * nrhs / (factor + solve seconds) -- higher is better.

The headline steps run without per-kernel timing; a separate profiled pass of
the same step (CUDA events around every launch on the library's stream) gives
the per-kernel-class table and the roofline of the dominant class.  The FP64
comparator (plain FP64 ACR + FP64 refinement, same leaf and tolerance) is one
more step after the timed region.

``--impl reference`` times the CPU FP64 oracle (conjugate gradients on the
same operator and RHS, host cores, threaded sparse products) on bounded
samples of the same workload.  Multi-GPU: replicas only (every rank solves
its own copy; no collective on the data path); the value is the sum over
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

WORKLOAD = {
    "workload": "ACR n=128 GRF kappa (ell=0.1, sigma=1, seed 1), leaf 64, tol 1e-6, 64 uniform RHS "
                "(seeds 100..163), FP32 factorisation + FP64 refinement to rel. residual 1e-10",
    "n": 128,
    "N": 128 ** 3,
    "nrhs": 64,
    "leaf": 64,
    "tol": 1e-6,
    "rtol": 1e-10,
    "kappa_seed": 1,
    "rhs_seeds": "100..163",
    "l2": "inputs larger than L2 (factor store is tens of GB, rebuilt every step)",
    "parallelism": "replicas",
}
METRIC = "factor+solve DOF/s at n=128 (FP32 ACR + FP64 refinement to 1e-10)"


def reduce_step_time(ms, world, dist, device):
    """Replicas: every rank times its own copy; the job time is the slowest rank's."""
    if world <= 1 or dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, N, nrhs, ms):
    """Whole-job DOF/s: all ranks' right-hand sides over the slowest rank's step time."""
    return world * N * nrhs / (ms * 1e-3)


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        load = [float(r[1]) for r in rows if float(r[3]) > 250.0] or sm
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows)}


def threaded_operator(A, threads):
    """The oracle's sparse matrix as a LinearOperator whose products run on
    `threads` host threads, one block of rows each (SciPy's sparse product
    releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    import scipy.sparse.linalg as spla

    A = A.tocsr()
    N = A.shape[0]
    bounds = np.linspace(0, N, threads + 1).astype(np.int64)
    parts = [A[bounds[i]:bounds[i + 1]] for i in range(threads)]
    pool = ThreadPoolExecutor(threads)

    def mv(x):
        x = np.ravel(x)
        out = np.empty(N)

        def one(i):
            out[bounds[i]:bounds[i + 1]] = parts[i] @ x

        list(pool.map(one, range(threads)))
        return out

    return spla.LinearOperator((N, N), matvec=mv, dtype=np.float64)


def cpu_converged(n, g, f, rtol, threads=None):
    """The oracle's FP64 CG on one right-hand side, run to convergence on the
    host cores; returns a dict with the measured time and iteration count."""
    from oracle import iterative, operator as op

    threads = threads or os.cpu_count() or 1
    A = threaded_operator(op.assemble(n, g), threads)
    t0 = time.perf_counter()
    u, it = iterative.cg(A, f, rtol=rtol, maxiter=50000)
    t = time.perf_counter() - t0
    relres = float(iterative.rel_residual(n, g, u, f)[0])
    return {"seconds": t, "iters": it, "rel_residual": relres, "threads": threads, "A": A,
            "converged": relres <= rtol * 1.01}


def cpu_chunk(A, f, iters):
    """Seconds for `iters` iterations of the oracle's CG (no early stop)."""
    from oracle import iterative

    t0 = time.perf_counter()
    iterative.cg(A, f, rtol=0.0, maxiter=iters)
    return time.perf_counter() - t0


def cpu_baseline_record(n, conv, rtol):
    N = n ** 3
    desc = ("oracle FP64 CG (not ACR), n=%d, one RHS (seed 100): %d iterations to rel. residual %.1e "
            "(measured %.2e, %s) in %.1f s; sparse products on %d host threads"
            % (n, conv["iters"], rtol, conv["rel_residual"], "converged" if conv["converged"] else "NOT converged",
               conv["seconds"], conv["threads"]))
    return {"value": N / conv["seconds"], "unit": "DOF/s", "cores": os.cpu_count(), "threads": conv["threads"],
            "kind": "oracle", "sample": desc}


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = WORKLOAD["n"]
    g = synthetic.gaussian_random_field(n, WORKLOAD["kappa_seed"])
    f = synthetic.uniform_rhs(n, 100)
    conv = cpu_converged(n, g, f, WORKLOAD["rtol"])
    # Each step: a bounded chunk of the same CG run (about ref_budget seconds),
    # scaled by the measured iteration count to 1e-10.
    per_it = conv["seconds"] / max(conv["iters"], 1)
    chunk = int(max(20, min(conv["iters"], args.ref_budget / per_it)))
    vals = []
    for s in range(args.warmup + args.steps):
        t = cpu_chunk(conv["A"], f, chunk)
        if s >= args.warmup:
            vals.append(WORKLOAD["N"] / (t * conv["iters"] / chunk))
    value = float(np.median(vals))
    cpu = cpu_baseline_record(n, conv, WORKLOAD["rtol"])
    cpu["value"] = value
    cpu["sample"] += ("; each timed step: %d iterations of the same CG, time scaled by %d/%d iterations"
                      % (chunk, conv["iters"], chunk))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": WORKLOAD["N"] * WORKLOAD["nrhs"] / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": WORKLOAD, "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# Kernel classes of the library's profile and the roof each is reported against.
TENSOR_CLASSES = ("gemm_tcgen05", "hodlr_expand")
ALU_CLASSES = ("gemm", "householder_qr", "pivoted_cholesky", "core_truncation", "rebuild_coef", "gauss_jordan")


def peaks_for(precision, peaks, source):
    """(tensor, alu, hbm) ceilings and their provenance."""
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    # FP32 products as three TF32 MMAs each: the tensor-pipe ceiling in FP32
    # flops is the TF32 dense rate / 3; TF32 = measured sustained BF16 x the
    # nominal TF32 : BF16 ratio (1.1 : 2.25 PFLOP/s dense).
    tensor = peaks["bf16_tflops_sustained"] * (1.1 / 2.25) / 3.0
    alu = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12 if precision == "f32" else 1.25
    return {
        "tensor": (tensor, "%s bf16_tflops_sustained x 1.1/2.25 (TF32) / 3 (3xTF32 passes)" % source),
        "alu": (alu, "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_mhz if precision == "f32"
                else "nominal FP64 rate of the recipe"),
        "hbm": (peaks["hbm_gbs"], "%s hbm_gbs" % source),
    }


def class_roof(name, kc, precision, peaks, source):
    """Roofline entry of one kernel class: achieved rate against its bound."""
    ms = kc["ms"]
    if ms <= 0:
        return None
    roofs = peaks_for(precision, peaks, source)
    gbs = kc["bytes"] / (ms * 1e-3) / 1e9
    tfs = kc["flops"] / (ms * 1e-3) / 1e12
    ai = kc["flops"] / kc["bytes"] if kc["bytes"] else 0.0
    ridge = roofs["alu"][0] * 1e12 / (roofs["hbm"][0] * 1e9)
    if name in TENSOR_CLASSES and precision == "f32":
        bound = "tensor"
    elif kc["flops"] > 0 and (name in ALU_CLASSES or ai >= ridge):
        bound = "alu"
    else:
        bound = "hbm"
    peak, src = roofs[bound]
    ach = gbs if bound == "hbm" else tfs
    return {"bound": bound, "achieved": ach, "peak": peak, "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
            "frac": ach / peak, "peak_source": src, "ms": ms, "launches": kc["launches"],
            "algorithmic_bytes_per_launch": kc["bytes"] / max(kc["launches"], 1),
            "algorithmic_flops_per_launch": kc["flops"] / max(kc["launches"], 1),
            "hbm_frac": gbs / roofs["hbm"][0], "arith_intensity": ai}


def roofline(kernels, precision, peaks, source):
    """Roofline of the dominant kernel class (largest device time)."""
    name, kc = max(kernels.items(), key=lambda kv: kv[1]["ms"])
    out = class_roof(name, kc, precision, peaks, source)
    if out is None:
        return None, name
    out.update({"kernel": name, "traffic": None, "share_of_device_time": None})
    return out, name


def class_table(kernels, precision, peaks, source):
    """Every kernel class with device time, its share and its roofline fraction."""
    tot = sum(v["ms"] for v in kernels.values()) or 1.0
    table = {}
    for name, kc in sorted(kernels.items(), key=lambda kv: -kv[1]["ms"]):
        e = class_roof(name, kc, precision, peaks, source)
        if e is None:
            continue
        table[name] = {"share": kc["ms"] / tot, "ms": round(kc["ms"], 3), "launches": kc["launches"],
                       "bound": e["bound"], "achieved": round(e["achieved"], 3), "unit": e["unit"],
                       "frac": round(e["frac"], 4), "hbm_frac": round(e["hbm_frac"], 4)}
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--tensor-cores", type=int, default=1, help="3xTF32 tensor-core GEMM tiles in the FP32 path")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="acr", choices=["acr", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--fp64-compare", type=int, default=1, help="also time one FP64 ACR step (the comparator)")
    ap.add_argument("--profile-steps", type=int, default=2, help="separate profiled steps for the class table")
    ap.add_argument("--ref-budget", type=float, default=4.0, help="seconds of CPU work per reference-arm step")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--e2e", type=int, default=1, help="also time the end-to-end host-buffer path")
    ap.add_argument("--profiler-range", type=int, default=0,
                    help="1: bracket the first timed step with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_main(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_1701_00182_gb300 as acr
    from paper_1701_00182_gb300 import build as b

    if rank == 0:
        b.build()
    if dist:
        dist.barrier()
    acr.load_library()

    n, nrhs = args.n, args.nrhs
    N = n ** 3
    wl = dict(WORKLOAD, n=n, N=N, nrhs=nrhs)
    if n != WORKLOAD["n"] or nrhs != WORKLOAD["nrhs"] or args.precision != "f32":
        # a reduced or variant run names its own sizes (the headline workload is n = 128, 64 RHS, FP32)
        wl["workload"] = ("ACR n=%d GRF kappa (ell=0.1, sigma=1, seed 1), leaf 64, tol 1e-6, %d uniform RHS, "
                          "%s factorisation + FP64 refinement to rel. residual 1e-10"
                          % (n, nrhs, args.precision.upper()))
    g_host = synthetic.gaussian_random_field(n, WORKLOAD["kappa_seed"])
    F_host = synthetic.multi_rhs(n, range(100, 100 + nrhs))
    g_dev = torch.from_numpy(g_host).cuda()
    B = torch.from_numpy(np.ascontiguousarray(F_host.T)).cuda()  # (nrhs, N): column-major N x nrhs
    X = torch.zeros_like(B)
    prec = acr.ACR_FP32 if args.precision == "f32" else acr.ACR_FP64

    def step(profile=0, kappa=g_dev, b=B, x=X, precision=prec, **kw):
        kw.setdefault("autotune", args.autotune)
        h = acr.acr_factor(n, kappa, WORKLOAD["tol"], WORKLOAD["leaf"], precision=precision, profile=profile,
                           nrhs_max=nrhs, graphs=1, tensor_cores=args.tensor_cores, **kw)
        it, rel, st = acr.acr_solve_ir(h, b.T, x.T, rtol=WORKLOAD["rtol"], maxit=60, check=False)
        s = acr.acr_get_stats(h)
        h.close()
        return it, rel, st, s

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    peaks, psrc = load_peaks()
    launches = 0
    iters = []
    worst = 0.0
    t_factor = 0.0
    last = None
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(args.steps):
            if args.profiler_range and i == 0:
                torch.cuda.profiler.start()
            it, rel, st, s = step()
            if args.profiler_range and i == 0:
                torch.cuda.synchronize()
                torch.cuda.profiler.stop()
            iters.append(it)
            worst = max(worst, float(np.max(rel)))
            launches += sum(v["launches"] for v in s["kernels"].values())
            t_factor += s["t_factor_ms"]
            last = s
        e1.record()
        torch.cuda.synchronize()
    clocks = clk.summary()
    ms = e0.elapsed_time(e1) / args.steps
    ms = reduce_step_time(ms, world, dist, "cuda")
    value = aggregate_value(world, N, nrhs, ms)

    # Per-kernel-class profile: the same step with CUDA events around every
    # launch (on the library's stream), kept out of the headline timing.
    kern = {}
    prof_ms = None
    if args.profile_steps > 0:
        torch.cuda.synchronize()
        p0 = time.perf_counter()
        for _ in range(args.profile_steps):
            _, _, _, s = step(profile=1)
            for k, v in s["kernels"].items():
                acc = kern.setdefault(k, {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
                for f in acc:
                    acc[f] += v[f] / args.profile_steps
        torch.cuda.synchronize()
        prof_ms = (time.perf_counter() - p0) / args.profile_steps * 1e3

    # end-to-end through the C ABI: host kappa and pinned host RHS, result read back every step
    e2e = None
    if args.e2e:
        B_pin = torch.from_numpy(np.ascontiguousarray(F_host.T)).pin_memory()
        X_pin = torch.empty_like(B_pin).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Bd = B_pin.cuda(non_blocking=True)
            Xd = torch.zeros_like(Bd)
            step(kappa=g_host, b=Bd, x=Xd)
            X_pin.copy_(Xd, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": world * N * nrhs / e2e_s, "unit": "DOF/s", "h2d_bytes_per_step": 8 * N * (nrhs + 1),
               "d2h_bytes_per_step": 8 * N * nrhs}

    rl, classes = None, None
    if kern:
        rl, dom = roofline(kern, args.precision, peaks, psrc)
        classes = class_table(kern, args.precision, peaks, psrc)
        if rl:
            rl["share_of_device_time"] = classes[dom]["share"]
    fp64 = None
    if args.fp64_compare and args.precision == "f32" and rank == 0:
        # plain FP64 ACR with its fastest correct settings: pivoted-QR core
        # truncation, heuristic GEMM tilings (FP64 autotuning costs minutes)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        it64, rel64, st64, s64 = step(precision=acr.ACR_FP64, core_svd=2, autotune=0)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - ta
        fp64 = {"s_per_step": t64, "value": N * nrhs / t64, "unit": "DOF/s", "t_factor_s": s64["t_factor_ms"] / 1e3,
                "t_solve_s": t64 - s64["t_factor_ms"] / 1e3, "ir_iters": it64,
                "max_rel_residual": float(np.max(rel64)), "status": st64, "core_truncation": "pivoted QR",
                "max_rank_by_cr_level": [max(r) for r in s64["max_rank_d"]],
                "mixed_speedup": value / world / (N * nrhs / t64)}
    cpu = None
    if args.cpu_baseline and rank == 0:
        conv = cpu_converged(n, g_host, F_host[:, 0].copy(), WORKLOAD["rtol"])
        cpu = cpu_baseline_record(n, conv, WORKLOAD["rtol"])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic", "config": wl,
            "t_factor_s": t_factor / args.steps / 1e3, "t_solve_s": ms / 1e3 - t_factor / args.steps / 1e3,
            "ir_iters": iters, "max_rel_residual": worst, "gpu_launches": launches, "clocks": clocks,
            "e2e": e2e, "roofline": rl, "cpu_baseline": cpu, "fp64_acr": fp64,
            "max_rank_by_cr_level": [max(r) for r in last["max_rank_d"]] if last else None,
            "max_rank_d": last["max_rank_d"] if last else None,
            "factor_bytes": last["factor_bytes"] if last else None,
            "profiled_ms_per_step": prof_ms, "classes": classes,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
