#!/usr/bin/env python
"""Benchmark: time-to-solution of (I - N) mu = -M gamma together with h at a
1e-10 relative residual, and Cauchy pair-evaluations per second, on the
unbounded domain exterior to 64 ellipses (centres U[-4,4]^2, semi-axes
U[0.1,0.4], min gap 0.05) with n = 1024 nodes per boundary (65,536 unknowns),
gamma = log|eta - alpha| with alpha the centre of the first ellipse.

One step = build the boundary handle from device-resident eta, eta', A (this
includes the quadtree, Eone = E q and the diagonals), run the fused FBIE
computation (right-hand side, GMRES to ||b - A mu|| <= 1e-10 ||b||, h and h_k),
free the handle.  The headline form evaluates every Cauchy sum by the fast
multipole method, as the paper does (order-32 expansions, FMM error ~1e-13 of
sum |w/d|; translations and near field in double-float on the FP32 pipe); the
final residual is re-checked with direct double-float sums.  The plain FP64
direct-sum GPU path, FP32 GMRES with FP64 / double-float / FMM refinement and
the adjoint equation are timed beside it.

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
def workload(count, n):
    """The workload name of the ellipse domains (64 ellipses, n = 1024 by default)."""
    return f"{count} ellipses, unbounded, n={n} ({count * n:,} unknowns): FBIE solve + h"
TOL = 1e-10
L2_FLUSH_BYTES = 256 << 20
SMS, SM_MAX_MHZ = 152, 2070.0
# Pipe peaks derived from unit counts and the maximum SM clock:
#   FP32: 128 lanes/SM; a pair costs 10 FP32-pipe instructions + 1 MUFU.
#   FP64: 2 DFMA lanes/SM (1.25 TFLOP/s nominal); a pair costs 13 FP64-pipe
#   instructions (10 arithmetic + 3 to refine the reciprocal seed).
#   double-float: ~97 FP32-pipe instructions per pair + 1 MUFU.
# The roofline compares the launches' algorithmic instructions on their limiting
# pipe (per pair: FP64 9 + 4R, FP32 6 + 4R, double-float 49 + 48R for R
# right-hand sides) with the pipe's peak instruction rate.
PEAK_INSTR = {
    "pair32": SMS * SM_MAX_MHZ * 1e6 * 128,
    "pair64": SMS * SM_MAX_MHZ * 1e6 * 2,
    "pairdf": SMS * SM_MAX_MHZ * 1e6 * 128,
    "fmm": SMS * SM_MAX_MHZ * 1e6 * 128,
    "fmm_near": SMS * SM_MAX_MHZ * 1e6 * 128,
    "fmm_l2p": SMS * SM_MAX_MHZ * 1e6 * 128,
    "fmm_up": SMS * SM_MAX_MHZ * 1e6 * 128,
    "fmm_l2l": SMS * SM_MAX_MHZ * 1e6 * 128,
}
PEAK_BASIS = {
    "pair64": "FP64 pipe: 152 SMs x 2 DFMA lanes x 2070 MHz; 9 + 4R FP64 instr per pair",
    "pair32": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz; 6 + 4R FP32 instr per pair (+1 MUFU)",
    "pairdf": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz; 49 + 48R FP32 instr per double-float pair",
    "fmm": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz; per M2L pair and lane 24 FP32 instr for each "
           "of the 32 double-float products of the real Pascal matrix + 98 for the two complex scalings",
    "fmm_up": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz; 742 FP32 instr per lane per binomial M2M "
              "transform, 36 x 47 per node for the powers and 48R per node and order in P2M",
    "fmm_l2l": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz; 840 FP32 instr per lane per Pascal-matrix L2L transform",
    "fmm_l2p": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz; 58R FP32 instr per node and order (Horner)",
    "fmm_near": "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz; 49 + 48R FP32 instr per double-float "
                "near-field pair",
}
KERNEL_NAME = {"pair64": "pairsum64_kernel", "pair32": "pairsum32x2_kernel", "pairdf": "pairsumdf2_kernel",
               "fmm": "fmm_m2l_kernel",
               "fmm_near": "fmm_near_bulk_kernel (near field streamed from the operator cache by bulk copies)",
               "fmm_l2p": "fmm_l2p_kernel", "fmm_up": "fmm_up_kernel (P2M and the M2M chain)",
               "fmm_l2l": "fmm_l2l_kernel"}
# DRAM bytes read + written per launch of the kernel at the headline size
# (64 ellipses, n = 1024; the R = 1 launches of the solve), from one ncu
# capture of the same command (ncu's default cache control: caches flushed
# before each captured launch), with the SHA-256 prefix of the kernel's source
# file at the time of the capture: a figure whose source has changed since is
# reported as null (stale).
TRAFFIC = {"fmm_near": (1.8917e8, "csrc/fmm.cu", "f9e02bb199254842"), "fmm": (1.07e6, "csrc/fmm.cu", "f9e02bb199254842"),
           "fmm_up": (3.465e7, "csrc/fmm.cu", "f9e02bb199254842"), "fmm_l2l": (0.89e6, "csrc/fmm.cu", "f9e02bb199254842"),
           "fmm_l2p": (5.28e6, "csrc/fmm.cu", "f9e02bb199254842")}
# kinds whose work is pair evaluations actually performed
PAIR_KINDS = ("pair64", "pair32", "pairdf", "fmm_near")
ROOF_KINDS = ("pair64", "pair32", "pairdf", "fmm", "fmm_near", "fmm_l2p", "fmm_up", "fmm_l2l")


def hbm_peak():
    """(GB/s, source) of the HBM roof: the measured copy bandwidth of this machine's
    GB300s when MEASURED_PEAKS.json is present, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "of fallback (6.8 TB/s, one earlier GB300 measurement)"


def source_sha(rel):
    import hashlib
    path = os.path.join(ROOT, "paper_1308_5351_gb300", rel)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_of(kind, args):
    """(bytes per launch or None, note) for the roofline's traffic field."""
    if kind not in TRAFFIC:
        return None, "no ncu capture of this kernel"
    if args.n != 1024 or args.count != 64:
        return None, "captured at the headline size only"
    val, rel, sha = TRAFFIC[kind]
    now = source_sha(rel)
    if sha is None or sha != now:
        return None, f"stale: {rel} changed since the ncu capture (now {now})"
    return val, f"ncu capture of {rel} at {sha}"
# instrumented kinds: pair sums (0, 1, 6) and the FMM kernels (7 to 11)
PROFILE_MASK = (1 << 0) | (1 << 1) | (1 << 6) | (1 << 7) | (1 << 8) | (1 << 9) | (1 << 10) | (1 << 11)
MODES = {"mixed_df": 4, "mixed": 1, "fp64": 0, "df32": 3, "fmm": 5, "mixed_fmm": 6}
FMM_MODES = ("fmm", "mixed_fmm")
DTYPES = {"mixed_df": "f32 + double-float f32 pairs, f64 vectors", "mixed": "f32 + f64",
          "fp64": "f64", "df32": "double-float f32 pairs, f64 vectors",
          "fmm": "f64-class: FMM with double-float f32 translations and near field, f64 vectors",
          "mixed_fmm": "f32 pairs + f64-class FMM"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--boundary-nodes", "--n", dest="n", type=int, default=1024,
                    help="nodes per boundary (use --boundary-nodes under torchrun)")
    ap.add_argument("--count", type=int, default=64, help="ellipses")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the comparison solves")
    ap.add_argument("--precision", choices=list(MODES), default="fmm")
    ap.add_argument("--workload", choices=["ellipses64", "close1024", "batched256", "stars20"],
                    default="ellipses64", help="ellipses64 is the headline; the others are extra lines")
    ap.add_argument("--domains", type=int, default=256, help="batched256: number of domains")
    ap.add_argument("--with-fp64", action="store_true",
                    help="close1024: also time the plain FP64 solve (minutes)")
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
            return
        # wait for the first sample, so that nvidia-smi's start-up (NVML
        # initialisation) is over before the timed region begins
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

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
ORACLE_SUB = 8          # boundaries of the oracle's timed sub-domain (N = 8 n)


def oracle_sample(dom_full, count_sub=ORACLE_SUB):
    """Time the oracle, as it stands, on the sub-domain made of the first
    `count_sub` boundaries at the same n: the dense assembly of its two
    matrices, the LU solve of its own system, and h; then extrapolate to the
    full domain (assembly and h scale as N^2, the LU as N^3).  Returns
    (extrapolated seconds, measured dict, sample description)."""
    import numpy as np
    from oracle import gnk_dense as O
    from paper_1308_5351_gb300 import domains as Dm
    sub = Dm.build_domain(dom_full.curves[:count_sub], dom_full.n, bounded=dom_full.bounded)
    gam = Dm.gamma_log(sub, dom_full.holes[0])
    t0 = time.perf_counter()
    K, M = O.matrices_K_M(sub.et, sub.etp, sub.A, sub.n)
    t1 = time.perf_counter()
    mu = np.linalg.solve(K, -(M @ gam))
    t2 = time.perf_counter()
    h = (M @ mu - K @ gam) / 2.0
    h.reshape(sub.m1, sub.n).mean(axis=1)
    t3 = time.perf_counter()
    t_asm, t_lu, t_h = t1 - t0, t2 - t1, t3 - t2
    r = dom_full.N / sub.N
    est = (t_asm + t_h) * r ** 2 + t_lu * r ** 3
    measured = {"N": sub.N, "boundaries": count_sub, "assembly_s": t_asm, "lu_solve_s": t_lu, "h_s": t_h,
                "total_s": t3 - t0}
    sample = (f"oracle (dense K and M assembly, LU solve of its own system, h) on the first {count_sub} of "
              f"{dom_full.m1} boundaries (N={sub.N}), measured {t3 - t0:.2f} s; full-size figure "
              f"extrapolated to N={dom_full.N} as (assembly + h)*(N/Ns)^2 + LU*(N/Ns)^3")
    return est, measured, sample


def oracle_pair_rate(dom):
    """One full direct FP64 Cauchy sum of the oracle's C routine (all host
    cores, OpenMP) on the whole domain: pair evaluations per second."""
    import numpy as np
    from oracle import cauchy_cpu as C
    w = np.random.default_rng(0).normal(size=dom.N) + 0j
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    C.cauchy_sum(dom.et, w, threads=threads)
    t = time.perf_counter() - t0
    rate = dom.N * (dom.N - 1) / t
    return rate, threads, (f"oracle C Cauchy sum (FP64, OpenMP, {threads} threads), one full product "
                           f"at N={dom.N}: {t:.2f} s")


def cpu_baseline_line(dom):
    """The cpu_baseline object: the oracle timed on the host cores."""
    est, measured, sample = oracle_sample(dom)
    rate, threads, pair_sample = oracle_pair_rate(dom)
    return {"value": est, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample,
            "value_is": "extrapolated to the full workload from the measured sample",
            "extrapolated_full_s": est, "measured": measured,
            "pair_evals_per_s": rate, "pair_sample": pair_sample}


def bench_config(args, N, m1, n, ws):
    """The config dict of both arms (the same workload)."""
    return {"workload": workload(m1, n), "N": N, "m1": m1, "n": n, "tol": TOL, "restart": 20,
            "precision": args.precision, "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


# ------------------------------------------------------------------ main
def main():
    args = parse()
    dist, rank, ws, local = dist_init(args.gpus)
    if args.impl == "reference":
        return run_reference(args, dist, rank, ws)
    if args.workload != "ellipses64":
        return run_extra(args, dist, rank, ws, local)

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
    if args.precision in FMM_MODES:
        bprec = G.GNK_PREC_FMM
    opts = G.options(tol=TOL, restart=20, maxit=50, precision=mode, inner_tol=1e-5)
    results = {}

    def step(o, build_prec):
        hnd = G.gnk_build_boundary_ex(dom.m1, dom.n, et, etp, A, None, None, dom.bounded,
                                      build_prec | G.GNK_BUILD_DEFER, stream)
        res = G.gnk_fbie(hnd, gam, mu, h, hk, o, stream)
        G.gnk_free_boundary(hnd)
        results["last"] = res
        return res

    kinds = (("pair64", G.PROF_PAIR64), ("pair32", G.PROF_PAIR32), ("pairdf", G.PROF_PAIRDF),
             ("fmm", G.PROF_FMM), ("fmm_near", G.PROF_FMMNEAR), ("fmm_l2p", G.PROF_FMML2P),
             ("fmm_up", G.PROF_FMMUP), ("fmm_l2l", G.PROF_FMML2L),
             ("reduce", G.PROF_REDUCE),
             ("circ", G.PROF_CIRC),
             ("krylov", G.PROF_KRYLOV))
    kind_id = dict(kinds)

    # warm-up; the last warm-up step records every kind, which gives the shares
    # of device time and picks the dominant kernel
    for w_ in range(args.warmup):
        flush.zero_()
        if w_ == args.warmup - 1:
            G.gnk_profile_enable(True)
        step(opts, bprec)
    torch.cuda.synchronize()
    prof_all = {k: G.gnk_profile_query_bytes(i) for k, i in kinds}
    G.gnk_profile_enable(False)
    dom_kind = max(ROOF_KINDS, key=lambda k: prof_all[k][1])

    # ---- timed region: event records only around the dominant kernel's
    # launches, so that the instrumentation hardly slows the step it measures
    launches0 = G.gnk_kernel_launches()
    G.gnk_profile_enable(True)
    G.gnk_profile_mask(1 << kind_id[dom_kind])
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
    prof = {k: G.gnk_profile_query_bytes(i) for k, i in kinds}
    G.gnk_profile_enable(False)
    t_ms = max_over_ranks(dist, t_ms, dev)
    ms_per_step = t_ms / args.steps
    res = results["last"]
    mu_main = mu.clone()
    h_main = hk.clone()
    # the final relative residual re-checked with direct double-float Cauchy sums
    hchk = G.gnk_build_boundary_ex(dom.m1, dom.n, et, etp, A, None, None, dom.bounded,
                                   G.GNK_PREC_DF32, stream)
    yv, kmu = torch.empty_like(gam), torch.empty_like(gam)
    G.gnk_apply_M(hchk, gam, yv, G.GNK_PREC_DF32, stream)
    G.gnk_apply_IminusN(hchk, mu, kmu, G.GNK_PREC_DF32, stream)
    G.gnk_free_boundary(hchk)
    relres_direct = float((kmu + yv).norm() / yv.norm())

    # ---- the same problem in the other forms (one timed run each, after one untimed)
    compare = {}
    kernel_rates = {}
    if not args.no_fp64:
        for name in ("fp64", "mixed", "mixed_df", "fmm", "mixed_fmm"):
            if name == args.precision:
                continue
            o = G.options(tol=TOL, restart=20, maxit=50, precision=MODES[name], inner_tol=1e-5)
            bp = G.GNK_PREC_DF32 if name in ("mixed_df", "df32") else G.GNK_PREC_FP64
            if name in FMM_MODES:
                bp = G.GNK_PREC_FMM
            if name != "fp64":
                step(o, bp)
            flush.zero_()
            torch.cuda.synchronize()
            G.gnk_profile_enable(True)
            G.gnk_profile_mask(PROFILE_MASK)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step(o, bp)
            e1.record(stream)
            torch.cuda.synchronize()
            pk = {k: G.gnk_profile_query_bytes(i) for k, i in kinds}
            G.gnk_profile_enable(False)
            compare[name] = {
                "time_to_solution_s": e0.elapsed_time(e1) / 1e3, "iterations": r.iterations,
                "refinements": r.refinements, "relres": r.relres,
                "max_rel_diff_mu_vs_headline": float((mu - mu_main).abs().max() / mu_main.abs().max()),
                "max_abs_diff_hk_vs_headline": float((hk - h_main).abs().max()),
            }
            for k in PAIR_KINDS:
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
    for k in PAIR_KINDS:
        src = prof if prof[k][1] > 0 else prof_all
        if src[k][1] > 0:
            kernel_rates[k] = src[k][2] / (src[k][1] / 1e3)

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
                                      bprec | G.GNK_BUILD_DEFER, stream)
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

    # ---- FMM products alone: (2I + diag(B1) - B) x by the FMM, back to back
    fmm_rate = None
    if args.precision in FMM_MODES:
        hnd = G.gnk_build_boundary_ex(dom.m1, dom.n, et, etp, A, None, None, dom.bounded, G.GNK_PREC_FMM,
                                      stream)
        xv, yv = torch.ones_like(gam), torch.empty_like(gam)
        for _ in range(3):
            G.gnk_apply_IminusN(hnd, xv, yv, G.GNK_PREC_FMM, stream)
        reps = 50
        G.gnk_profile_enable(True)
        G.gnk_profile_mask(1 << G.PROF_FMMNEAR)
        (_, t_f) = _timed(lambda: [G.gnk_apply_IminusN(hnd, xv, yv, G.GNK_PREC_FMM, stream)
                                   for _ in range(reps)], stream)
        nf = G.gnk_profile_query_ex(G.PROF_FMMNEAR)
        G.gnk_profile_enable(False)
        G.gnk_free_boundary(hnd)
        fmm_rate = {"products_per_s": reps / t_f, "ms_per_product": 1e3 * t_f / reps,
                    "near_pairs_per_product": nf[2] / max(nf[0], 1),
                    "near_pairs_per_s": nf[2] / t_f,
                    "what": "(2I + diag(B1) - B) x with E(q x) by the FMM, 50 products back to back "
                            "(one FMM product = one Cauchy sum over all N nodes)"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (largest device time in the last warm-up
    # step), from its launches in the timed region
    n_l, ms_l, work, instr, nbytes = prof[dom_kind]
    total_prof_ms = sum(v[1] for v in prof_all.values())
    if nbytes > 0:  # a memory-bound kernel (the near field from its operator cache)
        hbm, hbm_src = hbm_peak()
        achieved = nbytes / (ms_l / 1e3) / 1e9 if ms_l > 0 else 0.0
        bound = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                 "bytes_per_launch": nbytes / max(n_l, 1),
                 "peak_basis": f"HBM copy bandwidth, {hbm_src}; algorithmic bytes: the cached near-field "
                               "entries read (8 bytes per pair and part of z) + x in and z out per node"}
    else:
        achieved = instr / (ms_l / 1e3) if ms_l > 0 else 0.0
        peak = PEAK_INSTR[dom_kind]
        bound = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tinstr/s",
                 "frac": achieved / peak, "peak_basis": PEAK_BASIS[dom_kind] + " (derived from unit counts)"}
    roofline = {
        "kernel": KERNEL_NAME[dom_kind], **bound,
        "traffic": traffic_of(dom_kind, args)[0],
        "traffic_source": traffic_of(dom_kind, args)[1],
        "pair_evals_per_s": work / (ms_l / 1e3) if ms_l > 0 else 0.0,
        "launches": n_l, "avg_launch_ms": ms_l / max(n_l, 1),
        "share_of_instrumented_time": {k: v[1] / total_prof_ms for k, v in prof_all.items() if v[0] > 0},
        "instrumented": "timed region: the dominant kernel's launches; shares: every kind in the last "
                        "warm-up step",
    }
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_line(dom)
    line = {
        "metric": METRIC, "value": ms_per_step / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": bench_config(args, dom.N, dom.m1, dom.n, ws),
        "pair_evals_per_s": roofline["pair_evals_per_s"] if dom_kind in PAIR_KINDS else None,
        "pair_evals_per_s_note": "pairs actually evaluated by the dominant kernel per second of its live "
                                 "launch time (the FMM's far field is counted in products, not pairs)",
        "pair_evals_per_s_by_kernel": {KERNEL_NAME[k]: v for k, v in kernel_rates.items()},
        "fmm_product": fmm_rate,
        "solve": {"precision": args.precision, "iterations": res.iterations,
                  "refinements": res.refinements, "matvecs_fp64_class": res.matvecs_fp64,
                  "matvecs_fp32": res.matvecs_fp32, "relres": res.relres,
                  "relres_direct_df32": relres_direct},
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


# ------------------------------------------------------------------ extra workloads
def _timed(fn, stream):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def run_extra(args, dist, rank, ws, local):
    """Extra measurement lines (same JSON contract) for the other workloads:
    close1024  - 1024 close curves, n = 512 (524,288 unknowns), FBIE solve + h;
    batched256 - 256 domains, m+1 in 2..64, n in 128..1024, m+1 right-hand sides each;
    stars20    - gradient of h_1 - h_0 w.r.t. the Fourier coefficients of 16 star curves
                 (plus 4 graded polygons, n = 2048, N = 40,960) by one adjoint solve."""
    import numpy as np
    import torch
    from paper_1308_5351_gb300 import build as B
    from paper_1308_5351_gb300 import domains as Dm
    from paper_1308_5351_gb300 import gnk as G
    from oracle import gnk_dense as O
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        B.build()
    barrier(dist)
    G.load()
    stream = torch.cuda.current_stream(dev)
    line = {"metric": METRIC, "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    launches0 = G.gnk_kernel_launches()
    if args.workload == "close1024":
        dom = Dm.close_curves(seed=3 + 1000 * rank, n=512)
        gam_np = Dm.gamma_log(dom, dom.holes[0])
        et, etp, A = (torch.as_tensor(a, device=dev) for a in (dom.et, dom.etp, dom.A))
        gam = torch.as_tensor(gam_np, device=dev)
        mu, h = torch.empty_like(gam), torch.empty_like(gam)
        hk = torch.empty(dom.m1, dtype=torch.float64, device=dev)

        main = args.precision

        def step(prec):
            o = G.options(tol=TOL, restart=30, maxit=60, precision=MODES[prec], inner_tol=1e-5)
            bp = G.GNK_PREC_DF32 if prec in ("mixed_df", "df32") else G.GNK_PREC_FP64
            if prec in FMM_MODES:
                bp = G.GNK_PREC_FMM
            hnd = G.gnk_build_boundary_ex(dom.m1, dom.n, et, etp, A, None, None, False, bp, stream)
            r = G.gnk_fbie(hnd, gam, mu, h, hk, o, stream)
            G.gnk_free_boundary(hnd)
            return r
        for _ in range(args.warmup):
            step(main)
        times, res = [], None
        for _ in range(args.steps):
            res, t = _timed(lambda: step(main), stream)
            times.append(t)
        mu_np, h_np = mu.cpu().numpy(), h.cpu().numpy()
        # rows of the discrete equation (2I + diag(B1) - B) mu = -(D - diag(D1) + Lhat) gamma
        rows = np.random.default_rng(0).choice(dom.N, size=24, replace=False)
        lhs = O.rows_IminusN(dom.et, dom.etp, dom.A, dom.n, mu_np, rows)
        rhs = -O.rows_M(dom.et, dom.etp, dom.A, dom.n, gam_np, rows)
        compare = {}
        others = [p for p in ("mixed_df", "mixed_fmm") if p != main]
        if args.with_fp64:
            others.append("mixed")
        for other in others:
            _, t_o = _timed(lambda: step(other), stream)
            compare[other] = {"time_to_solution_s": t_o,
                              "max_rel_diff_mu_vs_headline": float(np.abs(mu.cpu().numpy() - mu_np).max()
                                                                   / np.abs(mu_np).max())}
        if args.with_fp64:
            _, t64 = _timed(lambda: step("fp64"), stream)
            compare["fp64"] = {"time_to_solution_s": t64,
                               "max_rel_diff_mu_vs_headline": float(np.abs(mu.cpu().numpy() - mu_np).max()
                                                                    / np.abs(mu_np).max())}
        # error against the dense oracle on the first 64 boundaries at n = 128
        sub = Dm.build_domain(dom.curves[:64], 128, bounded=False)
        gs = Dm.gamma_log(sub, dom.holes[0])
        sub_bp = G.GNK_PREC_FMM if main in FMM_MODES else G.GNK_PREC_DF32
        with G.Boundary.from_domain(sub, adjoint=False, device=dev, precision=sub_bp) as bs:
            ms, hs_, hks, rs = bs.fbie(torch.as_tensor(gs, device=dev), tol=TOL, precision=MODES[main],
                                       restart=30)
        mo, ho, hko = O.fbie(sub.et, sub.etp, sub.A, sub.n, gs)
        line.update({
            "value": statistics.median(times), "ms_per_step": 1e3 * statistics.median(times),
            "dtype": DTYPES[main],
            "config": {"workload": "1024 close curves (circles, ellipses, 32 graded squares; gaps to "
                                   "1e-3 r), unbounded, n=512 (524,288 unknowns): FBIE solve + h",
                       "N": dom.N, "tol": TOL, "restart": 30, "precision": main,
                       "l2": "working set larger than L2 (basis 130 MB)"},
            "solve": {"iterations": res.iterations, "refinements": res.refinements, "relres": res.relres},
            "sampled_row_residual_rel": float(np.abs(lhs - rhs).max() / np.abs(rhs).max()),
            "subset64_n128_vs_oracle": {"N": sub.N, "mu_rel_err": float(np.abs(ms.cpu().numpy() - mo).max()
                                                                        / np.abs(mo).max()),
                                        "h_err": float(np.abs(hs_.cpu().numpy() - ho).max()
                                                       / max(1.0, np.abs(ho).max()))},
            "compare": compare,
        })
    elif args.workload == "batched256":
        doms = Dm.batch_domains(seed=4 + 1000 * rank, count=args.domains)
        nrhs = [d.m1 for d in doms]
        gam_np = np.concatenate([Dm.gamma_log(d, d.holes[k]) for d in doms for k in range(d.m1)])
        bfmm = args.precision in FMM_MODES
        bprec = G.GNK_PREC_FMM if bfmm else G.GNK_PREC_MIXED_DF
        t0 = time.perf_counter()
        b = G.Batch(doms, nrhs, autotune=not bfmm, device=dev)
        t_build = time.perf_counter() - t0
        gam = torch.as_tensor(gam_np, device=dev)
        # the first FMM solve also builds each domain's tree and caches (kept with the batch)
        t_first = None
        for w_ in range(args.warmup):
            _, t_w = _timed(lambda: b.fbie(gam, tol=TOL, restart=20, inner_tol=1e-6, precision=bprec), stream)
            t_first = t_w if t_first is None else t_first
        times = []
        # per-kernel event records only for the persistent launches (the FMM path's
        # worker threads would serialise on the profiler's lock)
        G.gnk_profile_enable(not bfmm)
        for _ in range(args.steps):
            (mu, h, hk, res, rel), t = _timed(lambda: b.fbie(gam, tol=TOL, restart=20, inner_tol=1e-6,
                                                             precision=bprec), stream)
            times.append(t)
        prof = {k: G.gnk_profile_query(i) for k, i in (("pair32", G.PROF_PAIR32), ("pairdf", G.PROF_PAIRDF),
                                                        ("circ", G.PROF_CIRC))}
        G.gnk_profile_enable(False)
        # pair work of one batched product: sum_d nrhs_d N_d (N_d - 1); rate of a full product
        work = float(sum(r * d.N * (d.N - 1) for d, r in zip(doms, nrhs)))
        xs = torch.ones_like(gam)
        b.apply_IminusN(xs, G.GNK_PREC_FP32)
        _, t32 = _timed(lambda: b.apply_IminusN(xs, G.GNK_PREC_FP32), stream)
        _, tdf = _timed(lambda: b.apply_IminusN(xs, G.GNK_PREC_DF32), stream)
        # oracle check of the systems of the 4 smallest domains
        order = sorted(range(len(doms)), key=lambda i: doms[i].N)[:4]
        mu_np = mu.cpu().numpy()
        offs = np.cumsum([0] + [d.N * r for d, r in zip(doms, nrhs)])
        errs = []
        for i in order:
            d = doms[i]
            for k in range(nrhs[i]):
                a = offs[i] + k * d.N
                mo, _, _ = O.fbie(d.et, d.etp, d.A, d.n, gam_np[a:a + d.N])
                errs.append(float(np.abs(mu_np[a:a + d.N] - mo).max() / np.abs(mo).max()))
        tun = b.tuning()
        med = statistics.median(times)
        line.update({
            "value": med, "ms_per_step": 1e3 * med,
            "dtype": DTYPES["fmm"] if bfmm else "f32 + double-float f32 pairs, f64 vectors",
            "config": {"workload": "256 unbounded domains, m+1 ~ U{2..64}, n ~ U{128,256,512,1024}, "
                                   "m+1 right-hand sides log|eta - c_k| each: batched FBIE",
                       "systems": b.nsys, "vector_length": b.L, "nodes": int(sum(d.N for d in doms)),
                       "tol": TOL, "restart": 20, "precision": "fmm" if bfmm else "mixed_df",
                       "l2": "working set larger than L2"},
            "form": ("per-domain FMM handles (double-float direct sums below 4096 nodes) solved by 8 worker "
                     "threads on CUDA streams of their own" if bfmm else
                     "persistent FP32 / double-float launches over the whole batch, graph-captured cycles"),
            "first_solve_with_trees_s": t_first,
            "build_s": t_build, "tuning": tun,
            "solve": {"iterations": res.iterations, "refinements": res.refinements,
                      "max_relres": float(rel.max())},
            "pair_evals_per_batched_product": work,
            "kernel_time_s": {k: v[1] / 1e3 / args.steps for k, v in prof.items()},
            "full_product_s": {"fp32": t32, "df32": tdf},
            "pair_evals_per_s_full_product": {"fp32": work / t32, "df32": work / tdf},
            "oracle_check_smallest4_domains_max_rel_err_mu": max(errs),
        })
        b.close()
    else:  # stars20: gradient through the Fourier coefficients
        from paper_1308_5351_gb300 import autograd as AG
        rng = np.random.default_rng(5 + 1000 * rank)
        n, r0 = 2048, 0.3
        slots = [complex(x, y) for y in range(4) for x in range(5)]
        poly_slots = {3, 6, 13, 16}
        results = {}
        for kmax in (64, 128):
            k = np.arange(1, kmax + 1)
            params, centres, polys = [], [], []
            for sidx, c in enumerate(slots):
                if sidx in poly_slots:
                    polys.append(Dm.square(c, r0 * 0.8, ccw=False) if len(polys) % 2 == 0 else
                                 Dm.GradedPolygon([c + r0 * np.exp(-2j * np.pi * q / 3) for q in range(3)]))
                else:
                    centres.append(c)
                    params.append((torch.tensor(rng.normal(0, 0.05 / k), device=dev, requires_grad=True),
                                   torch.tensor(rng.normal(0, 0.05 / k), device=dev, requires_grad=True)))
            t_nodes = Dm.nodes(n)
            poly_et = [torch.as_tensor(pl.eval(t_nodes)[0], device=dev) for pl in polys]
            poly_etp = [torch.as_tensor(pl.eval(t_nodes)[1], device=dev) for pl in polys]
            m1 = len(centres) + len(polys)

            def J(ps):
                ets, etps = [], []
                for c, (ak, bk) in zip(centres, ps):
                    z, zp = AG.star_boundary(c, r0, ak, bk, n)
                    ets.append(z)
                    etps.append(zp)
                et = torch.cat(ets + poly_et)
                etp = torch.cat(etps + poly_etp)
                gam = torch.log(torch.abs(et - centres[0]))
                mu, h, hk = AG.fbie(et, etp, torch.ones_like(et), gam, m1, n, bounded=False,
                                    precision=MODES[args.precision], tol=1e-12, restart=30)
                return hk[1] - hk[0]
            for _ in range(args.warmup):  # untimed: first-call costs of the process and handles
                J(params).backward()
            for a_, b_ in params:
                a_.grad = None
                b_.grad = None
            val, t_fwd = _timed(lambda: J(params), stream)
            _, t_bwd = _timed(lambda: val.backward(), stream)
            grads = torch.cat([torch.cat([a.grad, b_.grad]) for a, b_ in params]).cpu().numpy()
            # central differences on three coefficients
            fd_err = 0.0
            for (si, which, kk) in ((0, 0, 0), (5, 1, 3), (11, 0, kmax - 1)):
                def shifted(delta):
                    ps = []
                    for t, (a, b_) in enumerate(params):
                        a2, b2 = a.detach().clone(), b_.detach().clone()
                        if t == si:
                            (a2 if which == 0 else b2)[kk] += delta
                        ps.append((a2, b2))
                    with torch.no_grad():
                        return float(J(ps))
                fd = (shifted(1e-6) - shifted(-1e-6)) / 2e-6
                an = float(params[si][which].grad[kk])
                fd_err = max(fd_err, abs(fd - an) / np.abs(grads).max())
            results[kmax] = {"parameters": int(grads.size), "forward_s": t_fwd, "backward_s": t_bwd,
                             "grad_norm": float(np.linalg.norm(grads)), "fd_max_err_3_coeffs_rel_to_max_grad": fd_err}
        tot = results[64]["forward_s"] + results[64]["backward_s"]
        line.update({
            "value": tot, "ms_per_step": 1e3 * tot, "dtype": DTYPES[args.precision],
            "config": {"workload": "16 star curves (a_k, b_k ~ N(0,(0.05/k)^2)) + 4 graded polygons, "
                                   "n=2048 (40,960 unknowns): d(h_1 - h_0)/d(a_k, b_k)",
                       "N": 20 * n, "tol": 1e-12, "precision": args.precision},
            "gradient": results,
        })
    line["gpu_launches"] = G.gnk_kernel_launches() - launches0
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args, dist, rank, ws):
    """The oracle, as it stands, on the host cores: each step is the bounded
    sample of the same workload (its first 8 boundaries), timed as measured and
    extrapolated to the full domain."""
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    from paper_1308_5351_gb300 import domains as Dm
    dom = Dm.ellipses64(seed=2, n=args.n, count=args.count)
    for _ in range(args.warmup):
        oracle_sample(dom)
    vals, meas, sample = [], [], ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        est, m, sample = oracle_sample(dom)
        vals.append(est)
        meas.append(m)
    wall = time.perf_counter() - t0
    v = statistics.median(vals)
    rate, threads, pair_sample = oracle_pair_rate(dom)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(args, dom.N, dom.m1, dom.n, ws),
        "cpu_baseline": {"value": v, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample,
                         "value_is": "median over the steps of the full-workload figure extrapolated from "
                                     "each step's measured sample",
                         "extrapolated_full_s": v,
                         "measured": {k: statistics.median(m[k] for m in meas) for k in meas[0]},
                         "pair_evals_per_s": rate, "pair_sample": pair_sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
