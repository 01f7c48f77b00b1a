"""Benchmark: ACR factor + solve of the n = 128 variable-coefficient workload on GB300.

Workload: -div(kappa grad u) = f, 7-point, Dirichlet, n = 128 (N = 2,097,152),
kappa = exp(g) with g a Gaussian random field (squared-exponential kernel,
length 0.1, sigma 1, seed 1); HODLR leaf 64, truncation tolerance 1e-6;
64 right-hand sides uniform on [-1, 1] (seeds 100..163) solved together.
One step = acr_factor in FP32 + FP64 iterative refinement (ACR as the
preconditioner) until every column has ||b - A x|| / ||b|| <= 1e-10.
Metric: DOF/s = N * nrhs / (factor + solve seconds) -- higher is better.

``--impl reference`` times the CPU FP64 oracle (conjugate gradients on the
same operator and RHS, host cores) on a bounded sample of the same workload.
Multi-GPU: replicas only (every rank solves its own copy; no collective on the
data path); the value is the sum over ranks.
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


def cg_sample(n, g, f, rtol, budget_s):
    """Oracle FP64 CG on one RHS with a wall-time budget; returns (DOF/s, description)."""
    from oracle import iterative, operator as op

    A = op.assemble(n, g)
    u = np.zeros_like(f)
    r = f.copy()
    p = r.copy()
    rr = r @ r
    f2 = f @ f
    t0 = time.perf_counter()
    it = 0
    while True:
        it += 1
        Ap = A @ p
        alpha = rr / (p @ Ap)
        u += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        if rr_new <= rtol * rtol * f2:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    relres = float(np.sqrt(rr_new / f2))
    if relres <= rtol:
        t_full, kind = t, "converged"
    else:
        t_full = t * np.log(rtol) / np.log(relres)
        kind = "extrapolated from rel. residual %.2e after %d iterations" % (relres, it)
    del iterative
    return n ** 3 / t_full, ("oracle FP64 CG (not ACR), n=%d, one RHS (seed 100) to %.0e: %d iterations in %.1f s, %s"
                            % (n, rtol, it, t, kind)), t_full


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = WORKLOAD["n"]
    g = synthetic.gaussian_random_field(n, WORKLOAD["kappa_seed"])
    f = synthetic.uniform_rhs(n, 100)
    vals = []
    desc = ""
    for s in range(args.warmup + args.steps):
        v, desc, _ = cg_sample(n, g, f, WORKLOAD["rtol"], args.ref_budget)
        if s >= args.warmup:
            vals.append(v)
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": WORKLOAD["N"] * WORKLOAD["nrhs"] / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": WORKLOAD,
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def roofline(kernels, precision, peaks, source):
    name, kc = max(kernels.items(), key=lambda kv: kv[1]["ms"])
    ms = kc["ms"]
    if ms <= 0:
        return None, name
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12 if precision == "f32" else 1.25  # TFLOP/s
    hbm = peaks["hbm_gbs"]
    gbs = kc["bytes"] / (ms * 1e-3) / 1e9
    tfs = kc["flops"] / (ms * 1e-3) / 1e12
    ai = kc["flops"] / kc["bytes"] if kc["bytes"] else 0.0
    ridge = alu_peak * 1e12 / (hbm * 1e9)
    per_launch = kc["bytes"] / max(kc["launches"], 1)
    if name == "gemm_tcgen05":
        # FP32 products as three TF32 MMAs each: the tensor-pipe ceiling in FP32
        # flops is the TF32 dense rate / 3; TF32 = measured sustained BF16 x the
        # nominal TF32 : BF16 ratio (1.1 : 2.25 PFLOP/s dense).
        tf32 = peaks["bf16_tflops_sustained"] * (1.1 / 2.25)
        peak = tf32 / 3.0
        out = {"bound": "tensor", "achieved": tfs, "peak": peak, "unit": "TFLOP/s", "frac": tfs / peak,
               "peak_source": "%s bf16_tflops_sustained x 1.1/2.25 (TF32) / 3 (3xTF32 passes)" % source}
    elif kc["flops"] > 0 and ai >= ridge:
        out = {"bound": "alu", "achieved": tfs, "peak": alu_peak, "unit": "TFLOP/s", "frac": tfs / alu_peak,
               "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_mhz
               if precision == "f32" else "nominal FP64 rate of the recipe"}
    else:
        out = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
               "peak_source": "%s hbm_gbs" % source}
    out.update({"kernel": name, "traffic": None, "algorithmic_bytes_per_launch": per_launch,
                "launches": kc["launches"], "share_of_device_time": None, "arith_intensity": ai})
    return out, name


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
    ap.add_argument("--fp64-compare", type=int, default=0, help="also time one FP64 ACR step (comparator)")
    ap.add_argument("--ref-budget", type=float, default=20.0, help="seconds of CPU work per oracle sample")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--e2e", type=int, default=1, help="also time the end-to-end host-buffer path")
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

    def step(profile=0, kappa=g_dev, b=B, x=X, precision=prec):
        h = acr.acr_factor(n, kappa, WORKLOAD["tol"], WORKLOAD["leaf"], precision=precision, profile=profile,
                           nrhs_max=nrhs, autotune=args.autotune, graphs=1,
                           tensor_cores=args.tensor_cores)
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
    kern = {}
    launches = 0
    iters = []
    worst = 0.0
    t_factor = 0.0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            it, rel, st, s = step(profile=1)
            iters.append(it)
            worst = max(worst, float(np.max(rel)))
            launches += sum(v["launches"] for v in s["kernels"].values())
            t_factor += s["t_factor_ms"]
            for k, v in s["kernels"].items():
                acc = kern.setdefault(k, {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
                for f in acc:
                    acc[f] += v[f]
        e1.record()
        torch.cuda.synchronize()
    clocks = clk.summary()
    ms = e0.elapsed_time(e1) / args.steps
    ms = reduce_step_time(ms, world, dist, "cuda")
    value = aggregate_value(world, N, nrhs, ms)

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

    rl, dom = roofline(kern, args.precision, peaks, psrc)
    tot_ms = sum(v["ms"] for v in kern.values())
    if rl:
        rl["share_of_device_time"] = kern[dom]["ms"] / tot_ms if tot_ms else None
    fp64 = None
    if args.fp64_compare and args.precision == "f32":
        torch.cuda.synchronize()
        ta = time.perf_counter()
        it64, rel64, st64, s64 = step(precision=acr.ACR_FP64)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - ta
        fp64 = {"s_per_step": t64, "value": N * nrhs / t64, "unit": "DOF/s", "t_factor_s": s64["t_factor_ms"] / 1e3,
                "ir_iters": it64, "max_rel_residual": float(np.max(rel64)), "status": st64,
                "max_rank_top": max(max(r) for r in s64["max_rank"])}
    cpu = None
    if args.cpu_baseline and rank == 0:
        v, desc, _ = cg_sample(n, g_host, F_host[:, 0].copy(), WORKLOAD["rtol"], args.ref_budget)
        cpu = {"value": v, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic", "config": wl,
            "t_factor_s": t_factor / args.steps / 1e3, "t_solve_s": ms / 1e3 - t_factor / args.steps / 1e3,
            "ir_iters": iters, "max_rel_residual": worst, "gpu_launches": launches, "clocks": clocks,
            "e2e": e2e, "roofline": rl, "cpu_baseline": cpu, "fp64_acr": fp64,
            "kernel_ms": {k: round(v["ms"], 3) for k, v in kern.items()},
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
