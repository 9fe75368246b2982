#!/usr/bin/env python
"""Benchmark: time-to-solution of (I - N) mu = -M gamma together with h at a
1e-10 relative residual, and Cauchy pair-evaluations per second, on the
unbounded domain exterior to 64 ellipses (centres U[-4,4]^2, semi-axes
U[0.1,0.4], min gap 0.05) with n = 1024 nodes per boundary (65,536 unknowns),
gamma = log|eta - alpha| with alpha the centre of the first ellipse.

One step = build the boundary handle from device-resident eta, eta', A (this
includes Eone = E q and the diagonals), run the fused FBIE computation (right-
hand side, GMRES to ||b - A mu|| <= 1e-10 ||b||, h and h_k), free the handle.
The headline form is FP32 pair sums inside GMRES with double-float (FP64-class,
on the FP32 pipe) refinement residuals; the plain FP64 GPU path, the FP32-inner
form with native FP64 residuals, and the adjoint equation are timed beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own seeded domain of the same shape
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-solution at 1e-10 rel. residual and matvec pair-evals/s vs plain FP64 GPU"
WORKLOAD = "64 ellipses, unbounded, n=1024 (65,536 unknowns): FBIE solve + h"
TOL = 1e-10
L2_FLUSH_BYTES = 256 << 20
SMS, SM_MAX_MHZ = 152, 2070.0
# Pipe peaks derived from unit counts and the maximum SM clock:
#   FP32: 128 lanes/SM; a pair costs 10 FP32-pipe instructions + 1 MUFU.
#   FP64: 2 DFMA lanes/SM (1.25 TFLOP/s nominal); a pair costs 13 FP64-pipe
#   instructions (10 arithmetic + 3 to refine the reciprocal seed).
#   double-float: ~97 FP32-pipe instructions per pair + 1 MUFU.
PEAK_PAIRS = {
    "pair32": SMS * SM_MAX_MHZ * 1e6 * 128 / 10,
    "pair64": SMS * SM_MAX_MHZ * 1e6 * 2 / 13,
    "pairdf": SMS * SM_MAX_MHZ * 1e6 * 128 / 97,
}
PEAK_BASIS = {
    "pair64": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2070 MHz / 13 FP64 instr per pair",
    "pair32": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz / 10 FP32 instr per pair",
    "pairdf": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz / 97 FP32 instr per double-float pair",
}
KERNEL_NAME = {"pair64": "pairsum64_kernel", "pair32": "pairsum32_kernel", "pairdf": "pairsumdf_kernel"}
MODES = {"mixed_df": 4, "mixed": 1, "fp64": 0, "df32": 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1024, help="nodes per boundary")
    ap.add_argument("--count", type=int, default=64, help="ellipses")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the comparison solves")
    ap.add_argument("--precision", choices=list(MODES), default="mixed_df")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed plumbing
def dist_init(want):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        else:
            backend = "gloo"
        dist.init_process_group(backend=backend)
        return dist, rank, ws, local
    return None, 0, 1, 0


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", idx, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        smax = max((num(r[1]) for r in rows if num(r[1]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        power = [num(r[2]) for r in rows if num(r[2]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(dom_full, count_sub=8):
    """Time the oracle (as it stands) on the sub-domain made of the first
    `count_sub` boundaries at the same n, and extrapolate to the full domain:
    assembly and products scale as N^2, the LU as N^3."""
    import numpy as np
    from oracle import gnk_dense as O
    from paper_1308_5351_gb300 import domains as Dm
    sub = Dm.build_domain(dom_full.curves[:count_sub], dom_full.n, bounded=dom_full.bounded)
    gam = Dm.gamma_log(sub, dom_full.holes[0])
    t0 = time.perf_counter()
    O.fbie(sub.et, sub.etp, sub.A, sub.n, gam)
    t_all = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    Mx = rng.normal(size=(sub.N, sub.N)) + 4 * sub.N ** 0.5 * np.eye(sub.N)
    bx = rng.normal(size=sub.N)
    t0 = time.perf_counter()
    np.linalg.solve(Mx, bx)
    t_lu = time.perf_counter() - t0
    t_asm = max(t_all - t_lu, 0.0)
    r = dom_full.N / sub.N
    est = t_asm * r ** 2 + t_lu * r ** 3
    sample = (f"oracle fbie (dense assembly + LU + h) on the first {count_sub} of "
              f"{dom_full.m1} boundaries (N={sub.N}): {t_all:.2f} s, of which LU {t_lu:.2f} s; "
              f"extrapolated to N={dom_full.N} as assembly*(N/Ns)^2 + LU*(N/Ns)^3")
    return est, t_all, sample


# ------------------------------------------------------------------ main
def main():
    args = parse()
    dist, rank, ws, local = dist_init(args.gpus)
    if args.impl == "reference":
        return run_reference(args, dist, rank, ws)

    import numpy as np
    import torch
    from paper_1308_5351_gb300 import build as B
    from paper_1308_5351_gb300 import domains as Dm
    from paper_1308_5351_gb300 import gnk as G

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        B.build()
    barrier(dist)
    G.load()

    dom = Dm.ellipses64(seed=2 + 1000 * rank, n=args.n, count=args.count)
    gam_np = Dm.gamma_log(dom, dom.holes[0])
    et, etp, A = (torch.as_tensor(a, device=dev) for a in (dom.et, dom.etp, dom.A))
    gam = torch.as_tensor(gam_np, device=dev)
    mu = torch.empty_like(gam)
    h = torch.empty_like(gam)
    hk = torch.empty(dom.m1, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    mode = MODES[args.precision]
    bprec = G.GNK_PREC_DF32 if args.precision in ("mixed_df", "df32") else G.GNK_PREC_FP64
    opts = G.options(tol=TOL, restart=20, maxit=50, precision=mode, inner_tol=1e-5)
    results = {}

    def step(o, build_prec):
        hnd = G.gnk_build_boundary_ex(dom.m1, dom.n, et, etp, A, None, None, dom.bounded,
                                      build_prec, stream)
        res = G.gnk_fbie(hnd, gam, mu, h, hk, o, stream)
        G.gnk_free_boundary(hnd)
        results["last"] = res
        return res

    for _ in range(args.warmup):
        flush.zero_()
        step(opts, bprec)
    torch.cuda.synchronize()

    kinds = (("pair64", G.PROF_PAIR64), ("pair32", G.PROF_PAIR32), ("pairdf", G.PROF_PAIRDF),
             ("reduce", G.PROF_REDUCE), ("circ", G.PROF_CIRC), ("krylov", G.PROF_KRYLOV))

    # ---- timed region
    launches0 = G.gnk_kernel_launches()
    G.gnk_profile_enable(True)
    clocks = ClockSampler()
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        res = step(opts, bprec)
        if res.status != 0 or res.relres > TOL:
            raise SystemExit(f"solve failed: {res.as_dict()}")
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    t_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    gpu_launches = G.gnk_kernel_launches() - launches0
    prof = {k: G.gnk_profile_query(i) for k, i in kinds}
    G.gnk_profile_enable(False)
    t_ms = max_over_ranks(dist, t_ms, dev)
    ms_per_step = t_ms / args.steps
    res = results["last"]
    mu_main = mu.clone()
    h_main = hk.clone()

    # ---- the same problem in the other forms (one timed run each, after one untimed)
    compare = {}
    kernel_rates = {}
    if not args.no_fp64:
        for name in ("fp64", "mixed", "mixed_df"):
            if name == args.precision:
                continue
            o = G.options(tol=TOL, restart=20, maxit=50, precision=MODES[name], inner_tol=1e-5)
            bp = G.GNK_PREC_DF32 if name in ("mixed_df", "df32") else G.GNK_PREC_FP64
            if name != "fp64":
                step(o, bp)
            flush.zero_()
            torch.cuda.synchronize()
            G.gnk_profile_enable(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step(o, bp)
            e1.record(stream)
            torch.cuda.synchronize()
            pk = {k: G.gnk_profile_query(i) for k, i in kinds}
            G.gnk_profile_enable(False)
            compare[name] = {
                "time_to_solution_s": e0.elapsed_time(e1) / 1e3, "iterations": r.iterations,
                "refinements": r.refinements, "relres": r.relres,
                "max_rel_diff_mu_vs_headline": float((mu - mu_main).abs().max() / mu_main.abs().max()),
                "max_abs_diff_hk_vs_headline": float((hk - h_main).abs().max()),
            }
            for k in ("pair64", "pair32", "pairdf"):
                if pk[k][1] > 0 and k not in kernel_rates:
                    kernel_rates[k] = pk[k][2] / (pk[k][1] / 1e3)
        # adjoint equation (I + N* + J) phi = gamma, headline precision
        etpp, Ap = (torch.as_tensor(a, device=dev) for a in (dom.etpp, dom.Ap))
        hnd = G.gnk_build_boundary_ex(dom.m1, dom.n, et, etp, A, etpp, Ap, dom.bounded, bprec, stream)
        phi = torch.empty_like(gam)
        G.gnk_solve_adjoint_ie(hnd, gam, phi, opts, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ra = G.gnk_solve_adjoint_ie(hnd, gam, phi, opts, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        G.gnk_free_boundary(hnd)
        compare["adjoint_" + args.precision] = {"time_to_solution_s": e0.elapsed_time(e1) / 1e3,
                                                "iterations": ra.iterations, "relres": ra.relres}
    for k in ("pair64", "pair32", "pairdf"):
        if prof[k][1] > 0:
            kernel_rates[k] = prof[k][2] / (prof[k][1] / 1e3)

    # ---- end to end through the C ABI with pinned host buffers
    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.complex128 if np.iscomplexobj(a) else torch.float64,
                        pin_memory=True)
        t.copy_(torch.as_tensor(a))
        return t.numpy()
    h_et, h_etp, h_A, h_gam = (pinned(a) for a in (dom.et, dom.etp, dom.A, gam_np))
    h_mu, h_h = pinned(np.zeros(dom.N)), pinned(np.zeros(dom.N))
    h_hk = pinned(np.zeros(dom.m1))

    def step_host():
        hnd = G.gnk_build_boundary_ex(dom.m1, dom.n, h_et, h_etp, h_A, None, None, dom.bounded,
                                      bprec, stream)
        r = G.gnk_fbie(hnd, h_gam, h_mu, h_h, h_hk, opts, stream)
        G.gnk_free_boundary(hnd)
        return r
    step_host()
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        step_host()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, (time.perf_counter() - t0) / args.steps, dev)
    h2d = 3 * 16 * dom.N + 8 * dom.N
    d2h = 8 * dom.N + 8 * dom.N + 8 * dom.m1

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (largest device time in the timed region)
    dom_kind = max(("pair64", "pair32", "pairdf"), key=lambda k: prof[k][1])
    n_l, ms_l, work = prof[dom_kind]
    achieved = work / (ms_l / 1e3) if ms_l > 0 else 0.0
    peak = PEAK_PAIRS[dom_kind]
    total_prof_ms = sum(v[1] for v in prof.values())
    pair_evals = sum(prof[k][2] for k in ("pair64", "pair32", "pairdf"))
    roofline = {
        "bound": "alu", "kernel": KERNEL_NAME[dom_kind],
        "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
        "frac": achieved / peak, "traffic": None,
        "launches": n_l, "avg_launch_ms": ms_l / max(n_l, 1),
        "share_of_instrumented_time": {k: v[1] / total_prof_ms for k, v in prof.items()},
        "peak_basis": PEAK_BASIS[dom_kind],
    }
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        est, t_sample, sample = oracle_sample(dom)
        cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
               "sample_seconds": t_sample}
    line = {
        "metric": METRIC, "value": ms_per_step / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed_df": "f32 + double-float f32 pairs, f64 vectors", "mixed": "f32 + f64",
                  "fp64": "f64", "df32": "double-float f32 pairs, f64 vectors"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": dom.N, "m1": dom.m1, "n": dom.n, "tol": TOL,
                   "restart": 20, "precision": args.precision,
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "pair_evals_per_s": pair_evals / (total_prof_ms / 1e3) if total_prof_ms else None,
        "pair_evals_per_s_by_kernel": {KERNEL_NAME[k]: v for k, v in kernel_rates.items()},
        "solve": {"precision": args.precision, "iterations": res.iterations,
                  "refinements": res.refinements, "matvecs_fp64_class": res.matvecs_fp64,
                  "matvecs_fp32": res.matvecs_fp32, "relres": res.relres},
        "compare": compare,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args, dist, rank, ws):
    """The oracle, as it stands, on the host cores: each step is the bounded
    sample of the same workload, extrapolated to the full domain."""
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    from paper_1308_5351_gb300 import domains as Dm
    dom = Dm.ellipses64(seed=2, n=args.n, count=args.count)
    for _ in range(args.warmup):
        oracle_sample(dom, count_sub=2)
    vals, sample = [], ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        est, _, sample = oracle_sample(dom, count_sub=4)
        vals.append(est)
    wall = time.perf_counter() - t0
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": args.n * args.count, "tol": "direct LU"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
