#!/usr/bin/env python
"""Benchmark of piCholesky k-fold cross-validation on GB300.

One step = the whole hot path on one batch of synthetic input: normal-equation
blocks, exact factors at the g sampled lambdas, the polynomial fit, and the
interpolated solves, refinement and hold-out scores at all q lambdas, ending
with the selected lambda.  The metric is fold x lambda hold-out evaluations per
second (k * q per step).

Own arm (default): the C ABI on cuda:LOCAL_RANK with X, Y resident in HBM.
Before the timed region the factorisation's launch shapes are autotuned
(results are bit-identical under every tuning), and eager calls are timed
against a CUDA-graph replay of one step; the faster launch mode is used.
Also reported: the same metric end to end from pinned host buffers (e2e),
exact-Cholesky cross-validation with the same kernels on the same GPU, the
error of the hold-out scores against the FP64 oracle on a sample, per-stage
device times, the roofline of the dominant kernel, SM clocks during the timed
region, the oracle timed on the host cores (cpu_baseline), and MChol
(Sec. 6.2) on the same data: alone at the paper's stopping width, and as the
range narrowing before piCholesky, each timed and compared with exact CV's
selected lambda; PINRMSE (the sampled hold-out errors interpolated
directly) likewise; and the warm start across folds (g' = 2 exact factors per
fold after the first).

Workloads: mixed_ecc (default: n = 32768, d = 2048, c = 10, k = 5, g = 6,
r = 3, q = 101, mixed precision, one refinement step against the interpolated
system), mixed_ecc_precond (the same with the exact-system refinement),
fp64_small (n = 2048, d = 256, FP64), batched_uneven (64 problems of uneven
size per CUDA-graph replay, streams and update strips autotuned).

--impl reference: the FP64 CPU oracle as it stands, one fold of the same
workload per step, on this machine's cores (rank 0 only).

Multi-GPU (torchrun): every rank runs its own replica of the problem (the
method's units are independent); the timed region is bracketed by barriers
and the maximum time over ranks is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fold×λ hold-out evals/sec vs exact-Cholesky CV on same GB300; err vs FP64"

WORKLOADS = {
    # n = 32768, d = 2048, c = 10 ECC targets of a 10-cluster mixture, k = 5, g = 6, r = 3, q = 101
    "mixed_ecc": dict(gen="mixed_ecc", cfg="MIXED_ECC", mode="mixed", basis="cheb_log", refine=1),
    # n = 2048, d = 256, c = 10, k = 5, g = 4, r = 2, q = 31, double precision
    "fp64_small": dict(gen="fp64_small", cfg="FP64_SMALL", mode="fp64", basis="mono", refine=0),
    # the mixed case with its refinement step taken against H_f + lambda I (the interpolated
    # factor as a preconditioner; moves the result toward exact CV; not the paper's method)
    "mixed_ecc_precond": dict(gen="mixed_ecc", cfg="MIXED_ECC", mode="mixed", basis="cheb_log", refine=1,
                              refine_target="exact"),
    # 64 problems, d ~ U[128, 1536], n = 8 d, c in {1, 10}, k = 5, g = 5, r = 3, q = 51, one CUDA graph
    "batched_uneven": dict(gen="batched_uneven", cfg=None, mode="mixed", basis="cheb_log", refine=1),
    # the mixed case's generator at d = 1024 (X 128 MB, coefficient planes 169 MB: both beyond the
    # L2 cache, a few GB on the device): the small case of the kernel profiles
    "mixed_ecc_d1024": dict(gen="mixed_ecc", cfg="MIXED_ECC", mode="mixed", basis="cheb_log", refine=1,
                            over=dict(d=1024)),
    # the large random-Fourier case as its own line (also a sub-line of the default run)
    "large_rff": dict(gen="large_rff", cfg="LARGE_RFF", mode="mixed", basis="cheb_log", refine=1),
}
BATCH = dict(count=64, k=5, g=5, r=3, q=51, lo=1e-3, hi=1e1, seed=3)

# GB300: 152 SMs x 128 FP32 lanes x 2 flops at the 2070 MHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="mixed_ecc")
    ap.add_argument("--refine", type=int, default=None, help="refinement steps (default: the workload's)")
    ap.add_argument("--solve-engine", type=int, choices=(0, 1, 2), default=None,
                    help="interpolated solves: 0 tensor cores, 1 CUDA cores, 2 automatic (the library's default)")
    ap.add_argument("--update-engine", type=int, choices=(0, 1), default=None,
                    help="trailing updates: 0 tensor cores, 1 CUDA cores (the library's default)")
    ap.add_argument("--no-exact", action="store_true", help="skip the exact-Cholesky comparison")
    ap.add_argument("--no-mchol", action="store_true", help="skip the MChol, PINRMSE and warm-start comparisons")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle sample (cpu_baseline, error)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large random-Fourier workload (n = 131072, d = 8192, c = 32) sub-line")
    ap.add_argument("--no-graph", action="store_true", help="time eager calls instead of one CUDA graph per step")
    ap.add_argument("--profile", action="store_true", help="warm-up + steps only, for ncu")
    ap.add_argument("--profile-grad", action="store_true",
                    help="as --profile, then two hold-out gradient calls at the grid's middle lambda")
    return ap.parse_args()


def max_over_ranks(ms, pg, device):
    """The slowest rank's duration (ms) of a timed region every rank ran;
    ``pg`` is torch.distributed with a process group, or None for one process."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, units_per_step, ms):
    """Units all ranks processed per second over the slowest rank's time (weak scaling:
    every rank runs the same work)."""
    return world * steps * units_per_step / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(name):
    from paper_1404_0466_gb300 import synth
    w = WORKLOADS[name]
    cfg = dict(getattr(synth, w["cfg"]), **w.get("over", {}))
    prob = getattr(synth, w["gen"])(**w.get("over", {}))
    return w, cfg, prob


def describe(name, w, cfg, refine):
    target = w.get("refine_target", "interpolated")
    return (f"{name}: n={cfg['n']} d={cfg['d']} c={cfg['c']} k={cfg['k']} g={cfg['g']} r={cfg['r']} "
            f"q={cfg['q']} basis={w['basis']} mode={w['mode']} refine={refine}"
            + (f" refine_target={target}" if refine and target != "interpolated" else ""))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        scratch = os.environ.get("BENCH_SCRATCH", os.path.join(ROOT, ".bench"))
        self.path = os.path.join(scratch, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            return summarise_clocks(fh)


def summarise_clocks(lines):
    """Median SM clock, the largest maximum clock and the throttle reasons that
    were active in any sample, from `nvidia-smi --query-gpu=<FIELDS>
    --format=csv,noheader` lines; lines that do not parse are skipped."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1].split()[0]))
            smax.append(float(parts[2].split()[0]))
        except (ValueError, IndexError):
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per stage (for the roofline of the dominant kernel)
# ---------------------------------------------------------------------------
def stage_work(cfg, mode, refine, target="interpolated", residual="tensor", update_engine=1):
    """Algorithmic work per step of each timed stage: (kind, amount, bound, executed).
    kind "flop": floating-point operations the method needs, counted once (an
    FMA counts 2), not the ones the kernel happens to execute; "byte": bytes
    that must cross HBM.  ``executed`` is the factor by which the kernel's own
    arithmetic exceeds that count (3 for the split-TF32 products, which run
    hi*hi + hi*lo + lo*hi; about 12 for double-float accumulation on the FP32
    pipes), reported beside the fraction and never folded into it.
    ``update_engine`` is the tuning's engine of the trailing updates (0 tensor
    cores, 1 CUDA cores, the library's default)."""
    n, d, c, k, g, r, q = (cfg[x] for x in ("n", "d", "c", "k", "g", "r", "q"))
    p = r + 1
    D = d * (d + 1) // 2
    nt = -(-d // 64)
    eb = 8 if mode == "fp64" else 4
    upd = sum((m * (m + 1) // 2) for m in range(nt)) * 2 * 64 ** 3 * k * g
    tensor = "tensor" if mode == "mixed" else "alu"
    split = 3 if mode == "mixed" else 1
    # per fold and lambda: the factor evaluated once (p multiply-adds per entry of the
    # lower triangle, 2 p D) and two triangular solves with c right-hand sides (2 d^2 c)
    eval_solve = k * q * (2 * d * d * c + 2 * p * D)
    work = {
        # SYRK of every fold block: n d (d + 1) flops
        "gram": ("flop", n * d * (d + 1), tensor, split),
        # X_j^T Y_j for every fold: 2 n d c flops
        "xty": ("flop", 2 * n * d * c, tensor, split),
        # trailing updates of k g blocked factorisations (lower tiles, 2 b^3 per tile update):
        # fp32 FMAs on the CUDA cores by default; with update_engine 0 (mixed mode) the bulk
        # of each step on the tensor cores in split TF32
        "chol_update": ("flop", upd, tensor, split) if (mode == "mixed" and update_engine == 0) else
                       ("flop", upd, "alu", 1),
        # the 64 x 64 diagonal tiles of k g factorisations, b^3 / 3 flops each, in FP64
        "chol_diag": ("flop", nt * k * g * 64 ** 3 // 3, "fp64", 1),
        # panel rows by substitution: b^3 flops per off-diagonal tile of the panel
        "chol_panel": ("flop", sum(range(nt)) * 64 ** 3 * k * g, "alu", 1),
        # per (fold, lambda, tile row): L~_ii from p planes (p b^2) and its inverse (b^3 / 3)
        "diag_inv": ("flop", k * q * nt * (64 ** 3 // 3 + p * 64 * 64), "alu", 1),
        # read g factors, write p coefficient sets, per fold (lower triangles); in mixed mode
        # the stage also splits the coefficients into the tensor-core operands (k_theta_split:
        # one read and four writes of the tile-major planes), counted as executed traffic
        "fit": ("byte", k * (g + p) * D * eb, "hbm",
                1 + (5 * p * (nt * (nt + 1) // 2) * 64 * 64 / ((g + p) * D) if mode == "mixed" else 0)),
        # the interpolated solves, once per refinement step more (the correction solve);
        # the kernel evaluates the factor in each of its two substitutions (4 p D)
        "solve": ("flop", eval_solve * (1 + refine), "alu",
                  (2 * d * d * c + 4 * p * D) / (2 * d * d * c + 2 * p * D)),
        # the residual B - L~ (L~^T W) per refinement step: the same two triangular
        # products and one evaluation of the factor per (fold, lambda); the kernel runs them
        # in double-float (error-free product + TwoSum: 11 and 13 flops per multiply-add)
        # and evaluates the factor in each of its two passes
        "resid": ("flop", eval_solve * refine, "alu",
                  (12 * d * d * c + 4 * p * D) / (2 * d * d * c + 2 * p * D)) if residual == "double_float" else
                 # on the tensor cores: one split-TF32 product per coefficient plane and pass
                 # (p (d^2 / 2) 2 c per lambda each, three products per split)
                 ("flop", eval_solve * refine, tensor, 3 * 2 * p * d * d * c / (2 * d * d * c + 2 * p * D)),
        # <W, G_f W> for every fold and lambda (the product G_f W, 2 d^2 c per system); in
        # mixed mode the kernel forms the hold-out residual Y_f - X_f W directly instead
        # (2 (n / k) d c per system, three products per split), in FP64 mode G_f W
        "score": ("flop", k * q * 2 * d * d * c, tensor, split * n / (k * d)) if mode == "mixed" else
                 ("flop", k * q * 2 * d * d * c, "alu", 1),
    }
    if target == "exact":
        # exact-system residual: G_f W and G_all W for every lambda, 2 d^2 c each
        work["resid"] = ("flop", k * q * refine * 2 * 2 * d * d * c, tensor, split)
    return work


def _peak(bound, mode, peaks):
    """Denominator of a stage's fraction: the measured HBM copy and bf16 figures
    (MEASURED_PEAKS.json), and this GPU's FP32 and FP64 FMA rates measured by
    pichol_probe_fma (all SMs of the device) when the bench has them."""
    pipes = peaks.get("pipes") or {}
    if bound == "hbm":
        return peaks.get("hbm_gbs"), "GB/s", "of measured (MEASURED_PEAKS.json hbm_gbs)"
    if bound == "tensor":
        # TF32 dense is half the bf16 rate on this part (nominal 1.1 vs 2.25 PFLOP/s)
        return peaks.get("bf16_tflops", 1919.0) * 0.5, "TFLOP/s", \
            "TF32 = 0.5 x measured bf16 burst (MEASURED_PEAKS.json), nominal ratio"
    if bound == "fp64" or mode == "fp64":
        if pipes.get("fp64_fma_tflops"):
            return pipes["fp64_fma_tflops"], "TFLOP/s", "of measured FP64 FMA rate (pichol_probe_fma, all SMs)"
        return 1.25, "TFLOP/s", "nominal GB300 FP64 (1.25 TFLOP/s); no measured figure"
    if pipes.get("fp32_fma_tflops"):
        return pipes["fp32_fma_tflops"], "TFLOP/s", "of measured FP32 FMA rate (pichol_probe_fma, all SMs)"
    return FP32_PEAK_TFLOPS, "TFLOP/s", "FP32 ALU: 152 SMs x 128 lanes x 2 flops x 2070 MHz (derived)"


def roofline_of(name, ms, launches, cfg, mode, refine, steps, peaks, work=None):
    """Roofline of one stage: achieved = algorithmic work per launch / average
    launch duration; frac = achieved / peak.  ``executed_per_algorithmic`` is
    how much arithmetic the kernel really runs per algorithmic flop, and
    ``issue_rate`` the executed rate (achieved x that factor)."""
    work = work if work is not None else stage_work(cfg, mode, refine)
    info = {"kernel_stage": name, "stage_ms_per_step": ms / steps, "launches_per_step": launches / steps}
    if name not in work or ms <= 0:
        info.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None})
        return info
    kind, amount, bound, executed = work[name]
    per_launch = amount / max(1, launches / steps)
    avg_s = ms / 1e3 / max(1, launches)
    peak, unit, note = _peak(bound, mode, peaks)
    achieved = per_launch / avg_s / (1e9 if kind == "byte" else 1e12)
    info.update({"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "peak_note": note,
                 "work": kind, "work_per_launch": per_launch,
                 "frac": (achieved / peak) if peak else None, "traffic": None,
                 "executed_per_algorithmic": executed, "issue_rate": achieved * executed})
    return info


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# stage's kernels from one ncu capture of the same code on the same workload,
# for kernels unchanged since that capture.
MEASURED_TRAFFIC = {
    # k_solve<float, 2, 10, 4> (packed FMAs), both launches of one step of the mixed case
    # (n = 32768, d = 2048): 1.03 GB read + 68.9 MB written, and 1.04 GB + 66.8 MB
    ("mixed_ecc", "solve"): 1.10e9,
}


def roofline(stage_ms, cfg, mode, refine, steps, peaks, work=None, workload=None):
    name, (ms, launches) = max(stage_ms.items(), key=lambda kv: kv[1][0])
    info = roofline_of(name, ms, launches, cfg, mode, refine, steps, peaks, work=work)
    info["traffic"] = MEASURED_TRAFFIC.get((workload, name))
    return info


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "note": "fallback"}


# ---------------------------------------------------------------------------
# oracle sample: error vs FP64 and cpu_baseline
# ---------------------------------------------------------------------------
def oracle_sample(prob, cfg, w, E_gpu, t_star):
    import numpy as np

    import oracle
    q = cfg["q"]
    idx = sorted(set([0, q // 4, q // 2, (3 * q) // 4, q - 1] + ([t_star] if t_star >= 0 else [])))
    tm = {}
    t0 = time.perf_counter()
    # the oracle follows the same refinement when it changes the result (exact-system target)
    pre = w["refine"] if w.get("refine_target") == "exact" else 0
    ref = oracle.cv(prob.X, prob.Y, k=cfg["k"], g=cfg["g"], r=cfg["r"], q=q, lo=cfg["lo"], hi=cfg["hi"],
                    basis=w["basis"], folds=[0], lam_idx=idx, timings=tm, precond_steps=pre)
    wall = time.perf_counter() - t0
    Eo = ref.E[0, idx]
    Eg = E_gpu[0, idx]
    err = float(np.max(np.abs(Eg - Eo) / np.abs(Eo)))
    # one fold of the method = fixed part (Hessian, factors, fit) + q evaluations
    per_eval = tm["eval"] / max(1, tm["n_eval"])
    fold_s = tm["setup"] + tm["fold"] + q * per_eval
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {
        "err_vs_fp64": {"max_rel_E": err, "sample": f"fold 0, grid indices {idx}"},
        "cpu_baseline": {"value": q / fold_s, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": (f"fold 0 of the workload: Hessian, {cfg['g']} factors and fit "
                                    f"({tm['setup'] + tm['fold']:.1f} s) and {len(idx)} of {q} lambdas "
                                    f"({per_eval:.2f} s each), extrapolated to the fold's {q} lambdas; "
                                    f"{wall:.1f} s of CPU work")},
    }


def oracle_exact_sample(prob, cfg, nlam=2):
    """The FP64 oracle's exact-Cholesky CV (the `Chol` comparator) on the host
    cores: fold 0 at nlam grid lambdas, extrapolated to the fold's q."""
    import oracle
    q = cfg["q"]
    idx = [q // 2 + i for i in range(nlam)]
    tm = {}
    t0 = time.perf_counter()
    oracle.cv(prob.X, prob.Y, k=cfg["k"], g=1, r=0, q=q, lo=cfg["lo"], hi=cfg["hi"], exact=True, folds=[0],
              lam_idx=idx, timings=tm)
    wall = time.perf_counter() - t0
    per_eval = tm["eval"] / max(1, tm["n_eval"])
    fold_s = tm["setup"] + tm["fold"] + q * per_eval
    return {"value": q / fold_s, "unit": "evals/s", "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "kind": "oracle exact CV",
            "sample": (f"fold 0: Hessian ({tm['setup'] + tm['fold']:.1f} s) and {len(idx)} of {q} lambdas "
                       f"({per_eval:.2f} s each: exact factor, solves, hold-out error), extrapolated; "
                       f"{wall:.1f} s of CPU work")}


def lapack_sample(prob, cfg):
    """Exact-Cholesky CV with NumPy's LAPACK and BLAS on the host cores (a
    competent CPU implementation, for context beside the plain oracle): fold
    0's Hessian by one GEMM, then Cholesky, two triangular solves and the
    hold-out error at a few grid lambdas, extrapolated to the fold's q."""
    import numpy as np
    import scipy.linalg as sla
    X = np.asarray(prob.X, dtype=np.float64)
    Y = np.asarray(prob.Y, dtype=np.float64)
    n, d = X.shape
    k, q = cfg["k"], cfg["q"]
    r0, r1 = 0, n // k
    t0 = time.perf_counter()
    Xt, Yt = X[r1:], Y[r1:]
    H = Xt.T @ Xt
    B = Xt.T @ Yt
    tau = float(np.einsum("ij,ij->", X, X)) / d
    t_fixed = time.perf_counter() - t0
    lam = tau * cfg["lo"] * (cfg["hi"] / cfg["lo"]) ** (np.arange(q) / max(1, q - 1))
    idx = [0, q // 2, q - 1]
    t1 = time.perf_counter()
    for t in idx:
        L = np.linalg.cholesky(H + lam[t] * np.eye(d))
        W = sla.solve_triangular(L.T, sla.solve_triangular(L, B, lower=True), lower=False)
        float(np.mean((Y[r0:r1] - X[r0:r1] @ W) ** 2))
    per = (time.perf_counter() - t1) / len(idx)
    fold_s = t_fixed + q * per
    return {"value": q / fold_s, "unit": "evals/s", "cores": os.cpu_count() or 1, "kind": "numpy LAPACK exact CV",
            "sample": (f"fold 0: Hessian by GEMM ({t_fixed:.2f} s), then {len(idx)} of {q} lambdas "
                       f"({per:.3f} s each: Cholesky, two triangular solves, hold-out error), extrapolated")}


# ---------------------------------------------------------------------------
# the reference arm: the oracle as it stands
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w, cfg, prob = workload(args.workload)
    k, q = cfg["k"], cfg["q"]
    refine = w["refine"] if args.refine is None else args.refine

    pre = refine if w.get("refine_target") == "exact" else 0

    def step(i):
        f = i % k
        oracle.cv(prob.X, prob.Y, k=k, g=cfg["g"], r=cfg["r"], q=q, lo=cfg["lo"], hi=cfg["hi"],
                  basis=w["basis"], folds=[f], precond_steps=pre)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    sec = time.perf_counter() - t0
    value = args.steps * q / sec
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": describe(args.workload, w, cfg, refine),
                   "reference_step": f"one fold (all {q} lambdas) of the FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"one fold per step, {q} lambdas each"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# own arm
# ---------------------------------------------------------------------------
def run_batched(args):
    """64 independent problems of uneven size per step, one CUDA graph replay."""
    import numpy as np
    import torch

    from paper_1404_0466_gb300 import binding, build, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    build.build()
    w = WORKLOADS["batched_uneven"]
    refine = w["refine"] if args.refine is None else args.refine
    B = BATCH
    probs = synth.batched_uneven(B["count"], seed=B["seed"], dtype=np.float32)
    specs = [dict(n=p.X.shape[0], d=p.X.shape[1], c=p.Y.shape[1], k=B["k"], g=B["g"], r=B["r"], q=B["q"],
                  lam_lo=B["lo"], lam_hi=B["hi"], basis=w["basis"], mode=w["mode"], refine_steps=refine)
             for p in probs]
    Xh = [torch.from_numpy(p.X).pin_memory() for p in probs]
    Yh = [torch.from_numpy(p.Y).pin_memory() for p in probs]
    Xs = [x.to(dev) for x in Xh]
    Ys = [y.to(dev) for y in Yh]
    batch = binding.Batch(specs, nstreams=8)
    stream = torch.cuda.current_stream()
    evals = sum(sp["k"] * sp["q"] for sp in specs)
    # the number of concurrent streams and the update strip chosen by the package's autotuner
    from paper_1404_0466_gb300 import autotune
    import torch.distributed as tdist
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tres = autotune.tune_batch(batch, Xs, Ys, reps=2, stream=stream, pg=tdist.group.WORLD if pg is not None else None)
    best, best_strip = tres.choice["streams"], tres.choice["update_strip"]
    tune = tres.timings
    batch.run(Xs, Ys)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run(Xs, Ys)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    n0 = batch.launch_count()
    sampler = ClockSampler()
    sampler.start()
    time.sleep(0.3)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    value = job_throughput(world, args.steps, evals, ms)
    # launches inside one graph replay = launches the captured run enqueued
    per_run = None
    n1 = batch.launch_count()
    batch.run(Xs, Ys)
    torch.cuda.synchronize()
    per_run = batch.launch_count() - n1
    # end to end: pinned host inputs copied in, scores copied out.  A second graph
    # of the same batch reads a second input buffer set; while one step's graph
    # runs, the next step's inputs are copied into the idle set on a second
    # stream (after the previous step, the last reader of that set, is done).
    Eh = [torch.empty(e.shape, dtype=torch.float64).pin_memory() for e in batch.E]
    XsB = [torch.empty_like(x) for x in Xs]
    YsB = [torch.empty_like(y) for y in Ys]
    graphB = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graphB):
        batch.run(XsB, YsB)
    sets = [(Xs, Ys, graph), (XsB, YsB, graphB)]
    cs = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    after = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(b):
        with torch.cuda.stream(cs):
            for x, xh in zip(sets[b][0], Xh):
                x.copy_(xh, non_blocking=True)
            for y, yh in zip(sets[b][1], Yh):
                y.copy_(yh, non_blocking=True)
            ready[b].record(cs)

    def e2e_steps(nsteps):
        cs.wait_stream(stream)
        copy_in(0)
        for i in range(nsteps):
            b = i % 2
            stream.wait_event(ready[b])
            if i + 1 < nsteps:
                if i >= 1:
                    cs.wait_event(after[1 - b])
                copy_in(1 - b)
            sets[b][2].replay()
            after[b].record(stream)
            for eh, e in zip(Eh, batch.E):
                eh.copy_(e, non_blocking=True)

    e2e_steps(2)                       # untimed: first use of the second buffer set and stream
    torch.cuda.synchronize()
    e0.record(stream)
    e2e_steps(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ems = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    del graphB, XsB, YsB
    if rank != 0:
        return 0
    h2d = sum(x.numel() * 4 for x in Xh) + sum(y.numel() * 4 for y in Yh)
    # per-kernel durations: one eager run on a single stream with stage timing, so the
    # kernels of different problems do not overlap; work summed over the problems
    batch.set_streams(1)
    batch.set_timing(1024)
    batch.run(Xs, Ys)
    torch.cuda.synchronize()
    stage_ms, work = {}, {}
    for i, sp in enumerate(specs):
        st, _ = batch.stage_times(i)
        for nm, (ms_, la) in st.items():
            if la:
                a, b = stage_ms.get(nm, (0.0, 0))
                stage_ms[nm] = (a + ms_, b + la)
        cfg_i = dict(sp, lo=B["lo"], hi=B["hi"])
        for nm, (kind, amount, bound, ex) in stage_work(cfg_i, w["mode"], refine).items():
            work[nm] = (kind, work.get(nm, (kind, 0, bound, ex))[1] + amount, bound, ex)
    batch.set_timing(0)
    peaks = load_peaks()
    pipes = {"fp32_fma_tflops": binding.probe_fma(False, 1 << 14), "fp64_fma_tflops": binding.probe_fma(True, 1 << 12),
             "method": "8 independent FMA chains per thread, 8 CTAs of 256 threads per SM (pichol_probe_fma)"}
    peaks["pipes"] = pipes
    top = max(stage_ms, key=lambda nm: stage_ms[nm][0])
    roof = roofline_of(top, *stage_ms[top], None, w["mode"], refine, 1, peaks, work=work)
    kern_roof = {nm: {kk: v for kk, v in roofline_of(nm, ms_, la, None, w["mode"], refine, 1, peaks, work=work).items()
                      if kk in ("achieved", "frac", "bound", "stage_ms_per_step", "launches_per_step", "issue_rate")}
                 for nm, (ms_, la) in stage_ms.items() if nm in work}
    # error against the FP64 oracle and the oracle's own speed, on four problems spread
    # over the batch's size range (fold 0, five lambdas each, extrapolated to the fold)
    import oracle
    by_size = sorted(range(len(probs)), key=lambda i: probs[i].X.shape[1])
    pick = [by_size[(2 * j + 1) * len(probs) // 8] for j in range(4)]
    errs = []
    fold_s = 0.0
    t0 = time.perf_counter()
    idx = [0, B["q"] // 4, B["q"] // 2, 3 * B["q"] // 4, B["q"] - 1]
    for i in pick:
        tm = {}
        ref = oracle.cv(probs[i].X, probs[i].Y, k=B["k"], g=B["g"], r=B["r"], q=B["q"], lo=B["lo"], hi=B["hi"],
                        basis=w["basis"], folds=[0], lam_idx=idx, timings=tm)
        fold_s += tm["setup"] + tm["fold"] + B["q"] * tm["eval"] / max(1, tm["n_eval"])
        got = batch.E[i].cpu().numpy()
        errs.append(float(np.max(np.abs(got[0, idx] - ref.E[0, idx]) / np.abs(ref.E[0, idx]))))
    wall = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    dims = [probs[i].X.shape[1] for i in pick]
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": (f"batched_uneven: {B['count']} problems, d ~ U[128,1536], n = 8 d, c in {{1,10}}, "
                                f"k={B['k']} g={B['g']} r={B['r']} q={B['q']} basis={w['basis']} mode=mixed "
                                f"refine={refine}; one CUDA graph per step, {best} streams, update strips of {best_strip} "
                                f"(autotune.tune_batch, ms: {json.dumps(tune)})"),
                   "l2": "inputs larger than L2 (%d MB of X)" % (h2d // 2 ** 20), "parallelism": f"replicas x{world}"},
        "e2e": {"value": job_throughput(world, args.steps, evals, ems), "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": sum(e.numel() * 8 for e in Eh), "ms_per_step": ems / args.steps,
                "pipelining": "next step's inputs copied on a second stream into a second buffer set"},
        "gpu_launches": per_run * args.steps,
        "clocks": clocks,
        "err_vs_fp64": {"max_rel_E": max(errs), "sample": f"problems {pick} (d = {dims}), fold 0, grid indices {idx}"},
        "cpu_baseline": {"value": len(pick) * B["q"] / fold_s, "unit": "evals/s", "cores": cores,
                         "kind": "oracle",
                         "sample": (f"fold 0 of problems {pick} (d = {dims}, spread over the batch's sizes): "
                                    f"Hessian, factors and fit, and {len(idx)} of {B['q']} lambdas, extrapolated "
                                    f"to the fold's {B['q']} lambdas; {wall:.1f} s of CPU work")},
        "roofline": dict(roof, traffic=None,
                         timing="per-launch durations from one eager run of the batch on one stream"),
        "kernels_roofline": kern_roof,
        "measured_pipes": pipes,
    }
    print(json.dumps(line), flush=True)
    batch.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


def mchol_compare(binding, params, cfg, X, Y, stream, exact, E, t_star):
    """MChol over the workload's range [lo, hi] tau (c = the range's centre in
    log10, s = its half-width), timed from the normal-equation blocks on:
      * alone at the paper's stopping width s0 = 0.0025 (Sec. 6.3), the
        selected lambda being the last level's winner;
      * narrowed to a half-width of at most 0.1 decade, then piCholesky over
        that range with the workload's g, r, q.
    Each selection is compared with exact CV's (and piCholesky's over the full
    range) as |log10(lambda / lambda_exact)|, the accuracy measure of the
    paper's accuracy-versus-time figure."""
    import math

    import numpy as np
    import torch
    c0 = 0.5 * (math.log10(cfg["lo"]) + math.log10(cfg["hi"]))
    s0 = 0.5 * (math.log10(cfg["hi"]) - math.log10(cfg["lo"]))
    ctx = binding.Context(**dict(params, exact_batch=max(3, cfg["g"])))
    out = ctx._outputs(False)
    lam_grid = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"c": c0, "s": s0}

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for name, s_min, with_pichol in (("alone", 0.0025, False), ("then_pichol", 0.1, True)):
        tr = None

        def run():
            nonlocal tr
            ctx.hessian(X, Y)
            tr = ctx.mchol(c0, s0, s_min)
            if with_pichol:
                ctx.factor_samples()
                ctx.fit()
                ctx.eval_holdout(out=out)

        ms = timed(run)
        # per-stage device time of one more run
        ctx.set_timing(4096)
        ctx.stage_times()
        run()
        mst, mcomplete = ctx.stage_times()
        ctx.set_timing(0)
        info = ctx.info()
        trh = tr.cpu().numpy()
        tau = float(trh[0, 1] / 10.0 ** c0)
        last = trh[-1]
        best = int(np.argmin(last[3:6]))
        entry = {"ms": ms, "levels": int(trh.shape[0]), "s_min": s_min,
                 "stages_ms": {nm: round(v[0], 3) for nm, v in mst.items() if v[1] > 0},
                 "stage_timing_complete": mcomplete,
                 "exact_factorisations": int(trh.shape[0]) * 3 * cfg["k"],
                 "lambda_rel": float(last[best] / tau), "Ebar": float(last[3 + best]),
                 "device_status": binding.STATUS.get(info.code)}
        if with_pichol:
            lam = ctx.lambdas().cpu().numpy()
            Ew = out[0].cpu().numpy()
            tw = int(out[1].cpu().item())
            entry.update({"window_rel": [float(lam[0] / tau), float(lam[-1] / tau)],
                          "t_star": tw, "lambda_rel": float(lam[tw] / tau) if tw >= 0 else None,
                          "Ebar": float(Ew.mean(axis=0)[tw]) if tw >= 0 else None,
                          "evals": cfg["k"] * cfg["q"] + int(trh.shape[0]) * 3 * cfg["k"]})
        res[name] = entry
    # the full-range grid, for the comparisons below
    ctx.hessian(X, Y)
    lam_grid = ctx.lambdas().cpu().numpy()
    tau = float(lam_grid[0] / cfg["lo"])
    torch.cuda.synchronize()
    ctx.close()
    ref = []
    if exact:
        ref.append(("exact", float(lam_grid[exact["t_star"]] / tau)))
    if t_star >= 0:
        ref.append(("pichol_full_range", float(lam_grid[t_star] / tau)))
    for name in ("alone", "then_pichol"):
        lr = res[name]["lambda_rel"]
        for rn, rl in ref:
            res[name][f"abs_log10_vs_{rn}"] = abs(math.log10(lr / rl)) if lr else None
    if exact:
        res["exact_ms"] = exact["ms_per_step"]
        res["exact_min_Ebar"] = exact["min_E_exact"]
    return res


def pinrmse_compare(binding, params, cfg, X, Y, stream, exact, t_star):
    """PINRMSE (the supplementary comparator) on the same data: the exact
    hold-out errors at the g sampled lambdas interpolated over the grid, timed
    from the normal-equation blocks on, with its selection's distance from
    exact CV's and piCholesky's in grid steps and decades."""
    import math

    import torch
    ctx = binding.Context(**dict(params, exact_batch=max(3, cfg["g"])))
    out = ctx._outputs(False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run():
        ctx.hessian(X, Y)
        ctx.factor_samples()
        ctx.eval_pinrmse(out=out)

    run()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    tp = int(out[1].cpu().item())
    step = (math.log10(cfg["hi"]) - math.log10(cfg["lo"])) / (cfg["q"] - 1)
    res = {"ms": ms, "t_star": tp, "device_status": binding.STATUS.get(ctx.info().code)}
    for name, ref in (("exact", exact["t_star"] if exact else None), ("pichol", t_star if t_star >= 0 else None)):
        if ref is not None and tp >= 0:
            res[f"grid_steps_from_{name}"] = tp - ref
            res[f"abs_log10_vs_{name}"] = abs(tp - ref) * step
    ctx.close()
    return res


def warm_compare(binding, params, cfg, X, Y, stream, exact, E, t_star, warm=2):
    """The warm start across folds (warm_samples = g'): one step of the same
    workload with fold 0 fitted from its g factors and every other fold from
    g' factors and fold 0's coefficients; timed, and its hold-out errors and
    selection compared with the plain piCholesky step's and exact CV's."""
    import math

    import numpy as np
    import torch
    ctx = binding.Context(**dict(params, warm_samples=warm, exact_batch=cfg["g"]))
    out = ctx._outputs(False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.run(X, Y, out=out)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        ctx.run(X, Y, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    Ew = out[0].cpu().numpy()
    tw = int(out[1].cpu().item())
    fin = np.isfinite(Ew) & np.isfinite(E)
    step = (math.log10(cfg["hi"]) - math.log10(cfg["lo"])) / (cfg["q"] - 1)
    res = {"warm_samples": warm, "ms": ms, "value": cfg["k"] * cfg["q"] / (ms / 1e3), "unit": "evals/s",
           "exact_factorisations": cfg["g"] + (cfg["k"] - 1) * warm,
           "max_rel_E_vs_plain": float(np.max(np.abs(Ew[fin] - E[fin]) / E[fin])) if fin.any() else None,
           "t_star": tw, "t_star_plain": t_star, "device_status": binding.STATUS.get(ctx.info().code)}
    if exact and tw >= 0:
        res["grid_steps_from_exact"] = tw - exact["t_star"]
        res["abs_log10_vs_exact"] = abs(tw - exact["t_star"]) * step
    ctx.close()
    return res


def _golden_large_rff():
    """Fold-0 hold-out errors of the large random-Fourier workload stored by
    tests/golden/make_large_rff_golden.py (which runs only the FP64 oracle)."""
    path = os.path.join(ROOT, "tests", "golden", "large_rff_fold0.txt")
    idx, E = [], []
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if parts and parts[0].isdigit() and len(parts) == 3:
                idx.append(int(parts[0]))
                E.append(float(parts[2]))
    return idx, E


def large_rff_compare(binding, steps=3, tuning=None):
    """The large single problem (n = 131072, d = 8192 random-Fourier features,
    c = 32, k = 5, g = 6, r = 3, q = 101, mixed, one refinement step): step
    time and evals/s from device-resident inputs, per-stage times, the
    interpolated solve's coefficient stream in GB/s, fold-0 errors against the
    stored FP64-oracle values, and exact-Cholesky CV on the same GPU.
    ``tuning``: engine choices passed to Context.set_tuning (the command line's
    --solve-engine / --update-engine), else the library's defaults."""
    import numpy as np
    import torch

    from paper_1404_0466_gb300 import synth
    cfg = dict(synth.LARGE_RFF)
    prob = synth.large_rff()
    k, q, g, r, d, c = (cfg[x] for x in ("k", "q", "g", "r", "d", "c"))
    X = torch.from_numpy(prob.X).cuda()
    Y = torch.from_numpy(prob.Y).cuda()
    del prob
    params = dict(n=cfg["n"], d=d, c=c, k=k, g=g, r=r, q=q, lam_lo=cfg["lo"], lam_hi=cfg["hi"], basis="cheb_log",
                  mode="mixed", refine_steps=1)
    ctx = binding.Context(exact_batch=g, **params)
    if tuning:
        ctx.set_tuning(**tuning)
    out = ctx._outputs(False)
    stream = torch.cuda.current_stream()
    ctx.run(X, Y, out=out)
    torch.cuda.synchronize()
    ctx.set_timing(4096)
    ctx.stage_times()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.run(X, Y, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st, complete = ctx.stage_times()
    ctx.set_timing(0)
    info = ctx.info()
    idx, Eg = _golden_large_rff()
    E = out[0].cpu().numpy()
    err = float(np.max(np.abs(E[0, idx] - np.array(Eg)) / np.array(Eg)))
    # Coefficient bytes one solve launch streams.  The library's automatic engine choice
    # takes the tensor cores when one fold's planes exceed 64 MiB: one launch per
    # substitution, each CTA (fold, 64 columns of the stacked lambdas) reading the
    # off-diagonal tiles' p planes once, as TF32 hi and lo.  Otherwise the CUDA-core
    # solve: one launch for both substitutions, each CTA (fold, lambda pair) reading the
    # fp32 planes once per substitution.
    nt = -(-d // 64)
    offdiag, p = nt * (nt + 1) // 2 - nt, r + 1
    se = (tuning or {}).get("solve_engine", 2)
    tensor_engine = se == 0 or (se == 2 and (nt * (nt + 1) // 2) * p * 64 * 64 * 4 > 64 * 1024 * 1024)
    if tensor_engine:
        ncb = -(-(q * c) // (64 if p <= 4 else 32))
        theta_bytes = k * ncb * offdiag * p * 2 * 64 * 64 * 4
        what = ("off-diagonal coefficient planes (TF32 hi and lo) read by one tensor-core substitution "
                "launch: each (fold, 64-column) CTA reads its fold's planes once")
    else:
        theta_bytes = k * ((q + 1) // 2) * 2 * offdiag * p * 64 * 64 * 4
        what = ("off-diagonal coefficient planes read by one CUDA-core solve launch: each (fold, lambda "
                "pair) CTA reads its fold's planes in both substitutions")
    sms, sla = st.get("solve", (0.0, 0))
    solve_ms = sms / steps / max(1, sla / steps)
    res = {"workload": (f"large_rff: n={cfg['n']} d={d} c={c} k={k} g={g} r={r} q={q} basis=cheb_log mode=mixed "
                        f"refine=1"),
           "value": k * q / (ms / 1e3), "unit": "evals/s", "ms_per_step": ms, "steps": steps,
           "stages_ms_per_step": {nm: round(v[0] / steps, 3) for nm, v in st.items() if v[1] > 0},
           "stage_timing_complete": complete,
           "solve_theta_stream": {"bytes_per_launch": theta_bytes, "ms_per_launch": solve_ms,
                                  "GBps": theta_bytes / (solve_ms / 1e3) / 1e9 if solve_ms > 0 else None,
                                  "engine": "tensor cores" if tensor_engine else "CUDA cores",
                                  "what": what + "; L2 holds none of a fold's planes at this size"},
           "err_vs_fp64": {"max_rel_E": err, "sample": f"fold 0, grid indices {idx}, stored oracle values"},
           "tuning": ctx.tuning(),
           "device_status": binding.STATUS.get(info.code)}
    ctx.close()
    del ctx, out
    torch.cuda.empty_cache()
    ctxe = binding.Context(**dict(params, refine_steps=0))
    oute = ctxe._outputs(False)
    ctxe.hessian(X, Y)
    e0.record(stream)
    ctxe.eval_holdout_exact(out=oute)
    e1.record(stream)
    torch.cuda.synchronize()
    gram = sum(res["stages_ms_per_step"].get(nm, 0.0) for nm in ("gram", "xty"))
    xms = e0.elapsed_time(e1) + gram
    res["exact_cv"] = {"ms_per_step": xms, "value": k * q / (xms / 1e3), "unit": "evals/s",
                       "note": "Gram stages taken from the piCholesky step (the same kernels)"}
    res["speedup_vs_exact"] = xms / ms
    ctxe.close()
    del ctxe, oute, X, Y
    torch.cuda.empty_cache()
    return res


def run_own(args):
    import numpy as np
    import torch

    from paper_1404_0466_gb300 import binding, build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    build.build()
    w, cfg, prob = workload(args.workload)
    refine = w["refine"] if args.refine is None else args.refine
    k, q = cfg["k"], cfg["q"]
    dt = torch.float64 if w["mode"] == "fp64" else torch.float32
    Xh = torch.from_numpy(prob.X).to(dt).pin_memory()
    Yh = torch.from_numpy(prob.Y).to(dt).pin_memory()
    X = Xh.to(dev)
    Y = Yh.to(dev)
    params = dict(n=cfg["n"], d=cfg["d"], c=cfg["c"], k=k, g=cfg["g"], r=cfg["r"], q=q, lam_lo=cfg["lo"],
                  lam_hi=cfg["hi"], basis=w["basis"], mode=w["mode"], refine_steps=refine,
                  refine_target=w.get("refine_target", "interpolated"))
    # the piCholesky context needs factor slots for the g samples only
    ctx = binding.Context(exact_batch=cfg["g"], **params)
    out = ctx._outputs(False)
    stream = torch.cuda.current_stream()

    def step():
        ctx.run(X, Y, out=out)

    def barrier():
        if pg is not None:
            pg.barrier()

    # the launch shapes chosen by the package's autotuner on this problem (every result is
    # bit-identical under each; --profile keeps the defaults so that profiled runs stay short);
    # under torchrun every rank applies rank 0's choice
    tune_res = None
    if not args.profile:
        from paper_1404_0466_gb300 import autotune
        import torch.distributed as tdist
        tune_res = autotune.tune_context(ctx, X, Y, reps=2, stream=stream,
                                         pg=tdist.group.WORLD if pg is not None else None)
    if args.solve_engine is not None:
        ctx.set_tuning(solve_engine=args.solve_engine)
    if args.update_engine is not None:
        ctx.set_tuning(update_engine=args.update_engine)
    tuning = dict(ctx.tuning(), autotuned_ms=(tune_res.timings if tune_res else {}), tuner="autotune.tune_context")
    ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = ctx.info()
    if info.code != 0:
        raise RuntimeError(f"device status after warm-up: {binding.STATUS.get(info.code)}")
    if args.profile:
        for _ in range(args.steps):
            step()
        if args.profile_grad:
            import math
            lg = math.log(float(ctx.lambdas()[q // 2].item()))
            for _ in range(2):
                ctx.holdout_grad(lg)
        torch.cuda.synchronize()
        return 0

    # ---- timed region: K steps, inputs resident in HBM -------------------
    # Launch mode: eager calls, or one step of the same public calls captured
    # into a CUDA graph and replayed (the library's calls are capturable; the
    # stage-timing events are then part of the graph and after the replays hold
    # the last step's launch durations).  Unless --no-graph forces eager calls,
    # both are timed on a few steps and the faster is used.
    mode_ms = {}
    if not args.no_graph:
        gtry = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gtry):
            step()
        for name, fn in (("eager", step), ("graph", gtry.replay)):
            fn()
            ta.record(stream)
            for _ in range(3):
                fn()
            tb.record(stream)
            torch.cuda.synchronize()
            mode_ms[name] = ta.elapsed_time(tb) / 3
        del gtry
        use_graph = mode_ms["graph"] < mode_ms["eager"]
        if pg is not None:
            flag = torch.tensor([1 if use_graph else 0], device=dev)
            pg.broadcast(flag, 0)
            use_graph = bool(flag.item())
        args.no_graph = not use_graph
    if args.no_graph:
        ctx.set_timing(args.steps * 400 + 64)
        ctx.stage_times()
        run, stage_steps = step, args.steps
        n0 = ctx.launch_count()
    else:
        ctx.set_timing(400)
        n_cap = ctx.launch_count()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        launches_per_step = ctx.launch_count() - n_cap
        graph.replay()
        torch.cuda.synchronize()
        run, stage_steps = graph.replay, 1
    sampler = ClockSampler()
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = (ctx.launch_count() - n0) if args.no_graph else launches_per_step * args.steps
    stages, complete = ctx.stage_times()
    # the graph's event-record nodes refer to the timing events: they are freed
    # (set_timing(0)) only after the graph is
    ms = max_over_ranks(ms, pg, dev)
    value = job_throughput(world, args.steps, k * q, ms)
    E = out[0].cpu().numpy()
    t_star = int(out[1].cpu().item())
    info = ctx.info()

    if not args.no_graph:
        del run, graph
        torch.cuda.synchronize()
    ctx.set_timing(0)

    # ---- end to end: pinned host in, scores and argmin out -----------------
    # The next step's X, Y are copied on a separate stream into the other half
    # of a double buffer (the normal-equation blocks are X and Y's only reader),
    # started after this step's fit so that they overlap the solves and
    # refinement rather than the factorisation; every copy is inside the timed
    # region.
    e2e = None
    if not args.no_e2e:
        Eh = torch.empty((k, q), dtype=torch.float64).pin_memory()
        th = torch.empty((1,), dtype=torch.int32).pin_memory()
        Xb, Yb = [X, torch.empty_like(X)], [Y, torch.empty_like(Y)]
        cs = torch.cuda.Stream(device=dev)
        ready = [torch.cuda.Event(), torch.cuda.Event()]    # inputs of buffer b copied
        formed = torch.cuda.Event()                           # this step's Hessian formed

        def e2e_steps(nsteps):
            cs.wait_stream(stream)
            with torch.cuda.stream(cs):
                Xb[0].copy_(Xh, non_blocking=True)
                Yb[0].copy_(Yh, non_blocking=True)
                ready[0].record(cs)
            for i in range(nsteps):
                b = i % 2
                stream.wait_event(ready[b])
                ctx.hessian(Xb[b], Yb[b])
                ctx.factor_samples()
                ctx.fit()
                if i + 1 < nsteps:
                    # the copy streams through L2: start it after the factorisation, whose
                    # working set it would evict, beside the ALU-bound evaluation
                    formed.record(stream)
                    cs.wait_event(formed)
                    with torch.cuda.stream(cs):
                        Xb[1 - b].copy_(Xh, non_blocking=True)
                        Yb[1 - b].copy_(Yh, non_blocking=True)
                        ready[1 - b].record(cs)
                ctx.eval_holdout(out=out)
                Eh.copy_(out[0], non_blocking=True)
                th.copy_(out[1], non_blocking=True)

        e2e_steps(2)                                          # untimed: first use of the buffers and stream
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        e2e_steps(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1), pg, dev)
        # the host link alone: one copy of X from the pinned buffer
        e0.record(stream)
        Xb[1].copy_(Xh, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        h2d_ms = e0.elapsed_time(e1)
        # one call end to end with nothing overlapped: copy X, Y in, run the path,
        # copy the scores out, wait (the latency a single caller sees)
        lat = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Xb[1].copy_(Xh, non_blocking=True)
            Yb[1].copy_(Yh, non_blocking=True)
            ctx.run(Xb[1], Yb[1], out=out)
            Eh.copy_(out[0], non_blocking=True)
            th.copy_(out[1], non_blocking=True)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": job_throughput(world, args.steps, k * q, ems), "unit": "evals/s",
               "h2d_bytes_per_step": Xh.numel() * Xh.element_size() + Yh.numel() * Yh.element_size(),
               "d2h_bytes_per_step": Eh.numel() * 8 + 4, "ms_per_step": ems / args.steps,
               "pipelining": "next step's inputs copied on a second stream during this step's evaluation",
               "h2d_GBps_alone": Xh.numel() * Xh.element_size() / (h2d_ms / 1e3) / 1e9,
               "call_latency_ms": min(lat),
               "call_latency_note": "one call, host clock, copies in, path, scores out, synchronised; "
                                    "no overlap (best of 3)"}
        del Xb, Yb

    # ---- the hold-out gradient in log(lambda) at one lambda -----------------
    grad = None
    if rank == 0:
        import math
        lg = math.log(float(ctx.lambdas()[q // 2].item()))
        ctx.holdout_grad(lg)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            ctx.holdout_grad(lg)
        e1.record(stream)
        torch.cuda.synchronize()
        grad = {"ms": e0.elapsed_time(e1) / 10, "folds": k, "log_lambda": lg,
                "what": "E_f and dE_f/dlog(lambda) of every fold at one lambda through the interpolated factor "
                        "(pichol_holdout_grad after the step's fit)"}
        # per-stage device time of one call (separate calls with stage timing on)
        ctx.set_timing(64)
        ctx.stage_times()
        ctx.holdout_grad(lg)
        gst, _ = ctx.stage_times()
        ctx.set_timing(0)
        grad["stages_ms"] = {nm: round(v[0], 4) for nm, v in gst.items() if v[1] > 0}

    # ---- exact-Cholesky CV with the same kernels ---------------------------
    exact = None
    if not args.no_exact and rank == 0:
        del ctx
        torch.cuda.empty_cache()
        ctxe = binding.Context(**dict(params, refine_steps=0, refine_target="interpolated"))
        oute = ctxe._outputs(False)
        ctxe.hessian(X, Y)
        ctxe.eval_holdout_exact(out=oute)
        torch.cuda.synchronize()
        reps = 2
        e0.record(stream)
        for _ in range(reps):
            ctxe.hessian(X, Y)
            ctxe.eval_holdout_exact(out=oute)
        e1.record(stream)
        torch.cuda.synchronize()
        xms = e0.elapsed_time(e1) / reps
        Ex = oute[0].cpu().numpy()
        tx = int(oute[1].cpu().item())
        gram_ms = sum(stages[st][0] for st in ("gram", "xty") if st in stages) / stage_steps
        exact = {"value": k * q / (xms / 1e3), "unit": "evals/s", "ms_per_step": xms,
                 "speedup_excluding_gram": (xms - gram_ms) / (ms / args.steps - gram_ms),
                 "t_star": tx, "t_star_pichol": t_star,
                 "min_E_exact": float(np.mean(Ex, axis=0)[tx]),
                 "min_E_pichol": float(np.mean(E, axis=0)[t_star]) if t_star >= 0 else None,
                 "selected_lambda_equal": tx == t_star}
        fin = np.isfinite(E)
        exact["max_rel_E_vs_exact"] = float(np.max(np.abs(E[fin] - Ex[fin]) / Ex[fin])) if fin.any() else None
        exact["rel_min_E_vs_exact"] = (abs(exact["min_E_pichol"] - exact["min_E_exact"]) / exact["min_E_exact"]
                                       if exact["min_E_pichol"] is not None else None)
        ctxe.close()

    # ---- MChol (Sec. 6.2), alone and as the range for piCholesky; PINRMSE --
    mchol = pinrmse = warm = None
    if not args.no_mchol and rank == 0:
        mchol = mchol_compare(binding, params, cfg, X, Y, stream, exact, E, t_star)
        pinrmse = pinrmse_compare(binding, params, cfg, X, Y, stream, exact, t_star)
        warm = warm_compare(binding, params, cfg, X, Y, stream, exact, E, t_star)

    large = None
    if rank == 0 and not args.no_large and args.workload == "mixed_ecc":
        del X, Y
        torch.cuda.empty_cache()
        try:
            eng = {nm: v for nm, v in (("solve_engine", args.solve_engine), ("update_engine", args.update_engine))
                   if v is not None}
            large = large_rff_compare(binding, tuning=eng)
        except Exception as exc:                      # context only: never costs the line
            large = {"unavailable": f"{type(exc).__name__}: {exc}"}

    if rank != 0:
        return 0
    sample = None if args.no_cpu else oracle_sample(prob, cfg, w, E, t_star)
    lapack = None if args.no_cpu else lapack_sample(prob, cfg)
    oracle_exact = None
    if not args.no_cpu:
        try:
            oracle_exact = oracle_exact_sample(prob, cfg)
        except Exception as exc:                      # context only: never costs the line
            oracle_exact = {"unavailable": f"{type(exc).__name__}: {exc}"}
    # the FP32 and FP64 pipes measured on this GPU: the denominators of the ALU-bound stages
    pipes = {"fp32_fma_tflops": binding.probe_fma(False, 1 << 14), "fp64_fma_tflops": binding.probe_fma(True, 1 << 12),
             "method": "8 independent FMA chains per thread, 8 CTAs of 256 threads per SM (pichol_probe_fma)",
             # context for the tcgen05 stages (their denominator stays the TF32 figure derived from
             # the measured bf16 GEMM): the tensor pipe's own rate on operands in shared memory
             "tf32_mma_tflops": {str(n): binding.probe_mma(n, 1 << 15) for n in (64, 128, 256)},
             "tf32_mma_method": "tcgen05.mma kind::tf32, M = 128, K = 8, one CTA per SM issuing back to back "
                                "(pichol_probe_mma)"}
    peaks = load_peaks()
    peaks["pipes"] = pipes
    stage_ms = {s: v for s, v in stages.items() if v[1] > 0}
    work = stage_work(cfg, w["mode"], refine, w.get("refine_target", "interpolated"),
                      update_engine=tuning.get("update_engine", 1))
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if w["mode"] == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": describe(args.workload, w, cfg, refine),
                   "l2": "inputs larger than L2 (X is %d MB)" % (Xh.numel() * Xh.element_size() // 2 ** 20),
                   "parallelism": f"replicas x{world}", "tuning": tuning},
        "e2e": e2e,
        "gpu_launches": launches,
        # (the stored DRAM traffic was measured with the library's default engines)
        "roofline": roofline(stage_ms, cfg, w["mode"], refine, stage_steps, peaks, work=work,
                             workload=args.workload if args.solve_engine is None and args.update_engine is None
                             else None),
        "kernels_roofline": {nm: {kk: v for kk, v in roofline_of(nm, ms_, la, cfg, w["mode"], refine, stage_steps,
                                                                peaks, work=work).items()
                                  if kk in ("bound", "achieved", "peak", "unit", "frac", "stage_ms_per_step", "issue_rate")}
                             for nm, (ms_, la) in stage_ms.items()
                             if nm in work},
        "stages_ms_per_step": {s: round(v[0] / stage_steps, 4) for s, v in stage_ms.items()},
        "launch_mode": ("eager calls" if args.no_graph else "one CUDA graph replay per step")
                       + (f" (tuned, ms per step: {', '.join(f'{k}: {v:.3f}' for k, v in mode_ms.items())})"
                          if mode_ms else ""),
        "stage_timing_complete": complete,
        "clocks": clocks,
        "exact_cv": exact,
        "speedup_vs_exact": (value / world / exact["value"]) if exact else None,
        "holdout_grad": grad,
        "mchol": mchol,
        "pinrmse": pinrmse,
        "warm_start": warm,
        "large_rff": large,
        "device_status": binding.STATUS.get(info.code), "unusable_pairs": info.unusable,
    }
    if sample:
        line["cpu_baseline"] = sample["cpu_baseline"]
        line["err_vs_fp64"] = sample["err_vs_fp64"]
    if lapack:
        line["cpu_lapack_exact"] = lapack
    if oracle_exact:
        line["cpu_oracle_exact"] = oracle_exact
    line["measured_pipes"] = pipes
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.profile_grad:
        args.profile = True
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_uneven":
        return run_batched(args)
    return run_own(args)


if __name__ == "__main__":
    sys.exit(main())
