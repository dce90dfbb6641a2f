"""PiTSBiCG throughput on GB300: PiT solves/s at rel err <= 1e-6 against the FP64 path.

Workload (default): 2D heat u_t = nu Lap u on the unit square, 128 x 128
interior points, nu = 1e-2, T = 1, N = 512 slices, fine = 50 RK4 steps per
slice in FP32, coarse = one implicit-Euler step, FP64 Krylov vectors and
scalars, float-float true residuals with iterative refinement (stopping at
1e-7 relative to ||G^-1 B|| so that the error against the FP64 path stays
below 1e-6); initial values = 8 seeded Gaussian bumps per member; a batch of
8 independent members per step (--batch).

One step = one PiTSBiCG solve (Algorithm 1 with refinement) of a batch of
independent initial values, through pit_bicgstab_solve on device-resident
inputs.  `value` = solves/s over all ranks (weak scaling: every rank solves
its own batch; no collective on the data path).  `e2e` = the same through the
host-pointer C-ABI call, with the H2D copy of y0 and the D2H copy of the
solution inside the timed region.  --workload advdiff | dense | serving
measure the other configurations.

--impl reference times the FP64 CPU oracle (test infrastructure, not the
product) on a bounded sample of the same workload.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import math
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
# directory for the clock samples taken during the timed region
CLOCKS_DIR = os.environ.get("PIT_BENCH_CLOCKS_DIR", ROOT)
sys.path.insert(0, ROOT)

from paper_2203_10148_gb300 import inputs  # noqa: E402
from paper_2203_10148_gb300.replicas import (dist_env, max_over_ranks, replica_seed,  # noqa: E402
                                             whole_job_rate)

GOLDEN_SOLVE = os.path.join(ROOT, "tests", "golden", "oracle_solve_heat2d_128_N512.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FINE_SRCS = [os.path.join(ROOT, "paper_2203_10148_gb300", "csrc", f)
             for f in ("heat2d.cu", "stencil_arith.cuh")]

FLOP_PER_POINT_STEP = 28       # RK4 Horner: 4 stages x (3 add + 2 FMA) = 4 x 7 flop
# pipe operations per point and fine step (FADD, FMUL, FFMA count one each):
# FP32 4 stages x 5; float-float 4 stages x 44 FP32 ops (four TwoSums of 6,
# 8 for the low parts, a 4-op product, a TwoSum of 6 and 2 to collect the low
# part) + a 3-op renormalisation per step; FP64 4 x 5 FP64 ops
OPS_PER_POINT_STEP = {"fine_fp32": 20, "fine_ff": 179, "fine_fp64": 20, "fine_split": 69}
# the method's own work per point and RK4 step (Horner form, 4 stages x
# (3 FADD + 2 FFMA)), whatever arithmetic carries it out: the roofline's frac
METHOD_OPS_PER_POINT_STEP = 20
# split RK4 (true residuals): 44 for the float-float first-order stage (the
# float-float stage above), 3 x 5 for the FP32 stages, 10 for the final sum
# periodic advection-diffusion: 4 stages x 14 (5 for the Laplacian, 2 x 3 for the
# upwind differences, 2 for the advection sum, 1 to combine)
ADV_OPS_PER_POINT_STEP = 56
# float-float advection-diffusion stage: 33 (Laplacian sum) + 16 (upwind
# differences) + 12 (three products with error terms) + 16 (their sum) + 15
# (u + cc L) = 92 FP32 operations, 4 stages; 90 when the coefficients are
# FP32 values (their low-part terms vanish), as in the synthetic workload
ADV_FF_OPS_PER_POINT_STEP = 360
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2          # 1.25 TFLOP/s nominal FP64 = 2 FMA/clk/SM at 2.07 GHz x 152 SMs
KERNEL_NAMES = {"fine_fp32": "k_heat2d_fine<float>", "fine_ff": "k_heat2d_fine<ff>",
                "fine_fp64": "k_heat2d_fine<double>", "fine_split": "k_heat2d_split"}
ADV_KERNEL_NAMES = {"fine_fp32": "k_advdiff_fine<float>", "fine_ff": "k_advdiff_fine<ff>",
                    "fine_fp64": "k_advdiff_fine<double>"}


def parse(argv=None):
    args = _parser().parse_args(argv)
    if args.batch is None:
        args.batch = 8 if args.workload == "heat2d" else 1
    if args.precision is None:
        args.precision = "fp64" if args.workload == "heat1d" else "mixed"
    if args.tol is None:
        args.tol = 1e-10 if args.workload == "heat1d" else 1e-7
    if args.tol_mode is None:
        args.tol_mode = "r0" if args.workload == "heat1d" else "rhs"
    args.N_given = args.N is not None
    if args.N is None:
        args.N = 512
    return args


def _parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=None,
                    help="independent members solved together per step (default: 8 for "
                         "heat2d, 1 for advdiff and dense)")
    ap.add_argument("--workload", default="heat2d",
                    choices=["heat2d", "heat1d", "dense", "advdiff", "serving"],
                    help="heat2d: 2D heat 128^2, N = 512 (the headline); dense: M = 1024, "
                         "N = 4096; advdiff: periodic 512^2, N = 256")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--N", type=int, default=None,
                    help="slices (default: 512 for heat2d, 256 for advdiff)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--inner-tol", type=float, default=1e-5)
    ap.add_argument("--requests", type=int, default=128,
                    help="serving: requests of the Poisson stream per step")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: arrivals per second")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent solves")
    ap.add_argument("--tol", type=float, default=None,
                    help="relative tolerance (default 1e-7 relative to ||G^-1 B||, error target "
                         "1e-6; heat1d: 1e-10 relative to ||R^0||)")
    ap.add_argument("--tol-mode", default=None, choices=["r0", "rhs"])
    ap.add_argument("--precision", default=None, choices=["mixed", "fp64"],
                    help="default: fp64 for heat1d (the plain method), mixed otherwise")
    ap.add_argument("--no-configs", action="store_true",
                    help="heat2d: skip the short lines of the other configurations")
    ap.add_argument("--residual", default="split", choices=["split", "ff", "fp64"],
                    help="arithmetic of the true residual's fine propagations (heat2d: split RK4 "
                         "where 8 nu dt/h^2 <= 1/8; other operators: split means float-float)")
    return ap


def workload(args, rank, step=0):
    if args.workload == "heat1d":
        seed = replica_seed(inputs.SEED_HEAT1D, rank, step)
        return inputs.heat1d(batch=args.batch, seed=seed)
    if args.workload == "dense":
        seed = replica_seed(inputs.SEED_DENSE, rank, step)
        return inputs.dense(batch=args.batch, seed=seed, tol=1e-6)
    if args.workload == "advdiff":
        seed = replica_seed(inputs.SEED_ADVDIFF2D, rank, step)
        return inputs.advdiff2d(batch=args.batch, seed=seed, tol=1e-6,
                                N=args.N if args.N_given else 256)
    seed = replica_seed(inputs.SEED_HEAT2D, rank, step)
    return inputs.heat2d(n=args.n, N=args.N, batch=args.batch, seed=seed, tol=1e-6)


# ---------------------------------------------------------------- helpers

def load_peaks():
    try:
        return json.load(open(PEAKS))
    except Exception:
        return None


def _fine_kernel_source(text, kernel="k_heat2d_fine"):
    """A 2D heat fine kernel's own code in heat2d.cu: its body (from its
    template line to the closing brace at column 0) and its launch code
    (k_heat2d_fine: from fine_smem to the split kernel's launch code;
    k_heat2d_split: from split_smem to make_args)."""
    if kernel == "k_heat2d_split":
        a = text.index("// ------------------------------------------- split RK4 (true residuals)")
        b = text.index("\n}\n", text.index("k_heat2d_split(Heat2dArgs a)", a)) + 3
        c = text.index("size_t split_smem(")
        d = text.index("Heat2dArgs make_args(")
        return text[a:b] + text[c:d]
    a = text.index("template <class V, int RX, int RY, bool CL>")
    b = text.index("\n}\n", a) + 3
    c = text.index("size_t fine_smem(")
    d = text.index("// Split RK4 (PIT_SPLIT): one CTA")
    return text[a:b] + text[c:d]


def src_hash(paths, kernel="k_heat2d_fine"):
    """Hash of the sources a committed ncu figure depends on: the whole of
    every file, except heat2d.cu, of which only the named kernel's code counts."""
    h = hashlib.sha256()
    for p in paths:
        text = open(p, "r").read()
        if os.path.basename(p) == "heat2d.cu":
            text = _fine_kernel_source(text, kernel)
        h.update(text.encode())
    return h.hexdigest()[:16]


def traffic_for(kernel, units):
    """DRAM bytes per launch of `units` point-slices, from a committed ncu
    capture (scaled by units), if the kernel sources are unchanged since."""
    try:
        t = json.load(open(TRAFFIC))
        e = t.get(kernel)
        base = "k_heat2d_split" if kernel == "k_heat2d_split" else "k_heat2d_fine"
        if e and e.get("source_sha") == src_hash(FINE_SRCS, base):
            return e["dram_bytes"] * units / e["units"]
    except Exception:
        pass
    return None


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, device_index=0):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9 or r[0] != str(device_index):
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle leg

def oracle_sample(w, slices):
    """Times the FP64 oracle's G^{-1}F on a bounded sample: the fine propagator
    on `slices` of the N slices (scaled to N) plus one full sequential sweep."""
    from oracle import OracleProblem
    o = OracleProblem.from_workload(w.member(0))
    X = np.tile(o.y0, (slices, 1))
    t0 = time.perf_counter()
    o.F(X)
    t_f = (time.perf_counter() - t0) * (w.N / slices)
    Q = np.zeros((w.N + 1, w.M))
    Q[0] = o.y0
    t0 = time.perf_counter()
    o.sweep_Ginv(Q)
    t_s = time.perf_counter() - t0
    return t_f, t_s


def _oracle_fine_seconds(args):
    """Seconds the FP64 oracle takes to propagate `slices` copies of y0 over
    one slice (run in a worker process of the all-cores timing)."""
    w, slices = args
    from oracle import OracleProblem
    o = OracleProblem.from_workload(w.member(0))
    X = np.tile(o.y0, (slices, 1))
    t0 = time.perf_counter()
    o.F(X)
    return time.perf_counter() - t0


_ORACLE_POOL = None


def oracle_pool():
    """One worker process per host core, started with spawn (safe after the
    GPU has been used), created once per run."""
    global _ORACLE_POOL
    if _ORACLE_POOL is None:
        import multiprocessing as mp
        try:
            ncores = len(os.sched_getaffinity(0))
        except AttributeError:
            ncores = os.cpu_count() or 1
        _ORACLE_POOL = (mp.get_context("spawn").Pool(ncores), ncores)
        import atexit
        atexit.register(_ORACLE_POOL[0].terminate)
    return _ORACLE_POOL


def oracle_sample_all_cores(w, per_core=2):
    """The fine propagator on per_core slices per host core, all cores at
    once (the paper's one-slice-per-CPU layout, Sec. 4): the slowest worker's
    time scaled to N slices; the coarse sweep stays sequential."""
    pool, ncores = oracle_pool()
    pool.map(_oracle_fine_seconds, [(w, 1)] * ncores)          # imports, first touch
    times = pool.map(_oracle_fine_seconds, [(w, per_core)] * ncores)
    return max(times) * (w.N / (per_core * ncores)), ncores


def oracle_matvecs():
    try:
        g = json.load(open(GOLDEN_SOLVE))
        return int(g["matvecs"]), g
    except Exception:
        return None, None


def cpu_baseline(w, slices=32, all_cores=True):
    mv, g = oracle_matvecs()
    t_f, t_s = oracle_sample(w, slices)
    t_mv = t_f + t_s
    out = {"unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": (f"FP64 numpy/scipy oracle, 1 thread: fine propagator on {slices} of "
                      f"{w.N} slices (x{w.N // slices}) + one full coarse sweep = "
                      f"{t_mv:.2f} s per G^-1F matvec; x {mv} matvecs of the oracle's own "
                      f"Algorithm 1 solve of this workload (tests/golden)"),
           "seconds_per_matvec": t_mv,
           "fine_slice_steps_per_s": w.N * w.fine[1] / t_f,
           # not a timed whole solve: the fine propagator is timed on `slices`
           # slices and scaled to N, and the matvec count is the oracle's own
           "extrapolated_from_slices": slices, "of_slices": w.N, "matvecs_assumed": mv}
    out["value"] = (1.0 / (t_mv * mv)) if mv else None
    if all_cores and mv:
        try:
            t_fp, ncores = oracle_sample_all_cores(w)
            t_mvp = t_fp + t_s
            out["all_cores"] = {
                "value": 1.0 / (t_mvp * mv), "unit": "solves/s", "cores": ncores,
                "seconds_per_matvec": t_mvp,
                "sample": (f"the same oracle in {ncores} spawned processes, 2 slices each at "
                           f"once (scaled to {w.N}), + the sequential coarse sweep")}
        except Exception as e:  # context only; never fail the line
            out["all_cores"] = {"value": None, "sample": f"failed: {e}"}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args, 0)
    vals, step_s = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(w, slices=8)
        if i >= args.warmup:
            step_s.append(time.perf_counter() - t0)
            vals.append(cb.get("all_cores", {}).get("value") or cb["value"])
    v = float(np.median(vals)) if vals and vals[0] else None
    # the reference arm is the oracle on all the host's cores (falling back to
    # one thread when the process pool is unavailable)
    ac = cb.get("all_cores", {})
    if ac.get("value"):
        cb = dict(cb, cores=ac["cores"], sample=ac["sample"] + "; one thread: " + cb["sample"],
                  seconds_per_matvec=ac["seconds_per_matvec"])
    cb["value"] = v
    line = {"impl": "reference", "metric": "PiT solves/s (rel err <= 1e-6 vs FP64 path)",
            "value": v, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup,
            # wall time of each timed step: the bounded oracle sample, not a
            # whole batch of solves (value extrapolates the sample to solves)
            "ms_per_step": 1e3 * float(np.mean(step_s)) if step_s else None,
            "oracle_ms_per_batch_estimated": (1e3 * w.batch / v) if v else None,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, w, 1),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_config(args, w, world):
    """The workload description both arms print (the reference arm names the
    same workload it samples)."""
    cfg = {"workload": w.name, "batch_per_gpu": w.batch, "grid": [w.nx, w.ny],
           "N": w.N, "fine": list(w.fine), "coarse": list(w.coarse),
           "precision": args.precision, "tol": args.tol, "tol_mode": args.tol_mode,
           "inner_tol": args.inner_tol,
           "true_residual": {"split": ("error-free splitting: 7 BF16 digit slices per operand, exact FP32 "
                                       "diagonal sums on the tensor cores" if w.kind == "dense" else
                                       "split RK4 (float-float first-order term, FP32 higher-order terms)")
                             if w.kind in ("dense", "heat2d") else "float-float",
                             "ff": "float-float", "fp64": "fp64"}[args.residual],
           "l2": "working set > L2 (9 Krylov vectors x %.0f MB)" % (w.batch * (w.N + 1) * w.M * 8 / 1e6),
           "parallelism": f"replicas x{world}"}
    if getattr(w, "coarse_inner", 0):
        cfg["coarse_chebyshev_steps"] = w.coarse_inner
    return cfg


# ----------------------------------------------------------------- roofline

SWEEP_KERNELS = {"heat1d": "k_heat1d_sweep_warp / k_heat1d_sweep (FP64), k_xform_tc + k_rec_* (mixed)",
                 "heat2d": "k_xform_tc x4 + k_rec_full (tcgen05 sine transforms, mixed)",
                 "advdiff2d": "k_advdiff_sweep (cooperative, Chebyshev steps, tagged halo exchange)",
                 "dense": "k_dense_sweep_tc (cooperative 8-CTA clusters, tcgen05) or k_dense_sweep"}


def sweep_cost(w, timing, total_ms, steps):
    """The coarse sweep, reported apart from the fine kernel's roofline as
    the latency-bound step it is: microseconds per sweep (one sweep covers
    the whole batch), sweeps per timed step and share of the timed steps."""
    cls = [k for k in ("sweep_mixed", "sweep_fp64") if timing.get(k, (0, 0.0))[0]]
    if not cls:
        return None
    calls = sum(timing[k][0] for k in cls)
    ms = sum(timing[k][1] for k in cls)
    return {"kernel": SWEEP_KERNELS.get(w.kind), "bound": "latency",
            "us_per_sweep": 1e3 * ms / calls, "sweeps_per_step": calls / max(steps, 1),
            "share": ms / total_ms}


def heat1d_uses_matrix(w):
    """The library's choice for the 1D heat FP64 fine batch: the propagator
    matrix where M^2 multiply-adds per slice undercut the m stepping
    instructions (PIT_HEAT1D_PHI=0 keeps the steps)."""
    if (os.environ.get("PIT_HEAT1D_PHI", "1").startswith("0") or w.M > 256
            or getattr(w, "precision", "fp64") != "fp64"):
        return False
    m = w.fine[1]
    E = 2 if w.M <= 64 else 4 if w.M <= 128 else 8
    return w.M * w.M < 0.5 * m * 32.0 * (5 * E + 8) and w.M * w.M * m <= 1e8


def roofline(w, timing, peaks, nsm, sub_timing=None):
    """Roofline of the dominant fine-propagator kernel class, from the
    per-class CUDA-event times recorded inside the timed solves; the FP32
    inner kernel's entry from `sub_timing` when the timed solves ran their
    iterations untimed (top-level timing)."""
    fine = {k: timing[k] for k in ("fine_fp32", "fine_ff", "fine_fp64", "fine_split")
            if timing.get(k, (0, 0.0))[0]}
    if not fine:
        return None
    dom = max(fine, key=lambda k: fine[k][1])
    calls, ms = timing[dom]
    avg_ms = ms / max(calls, 1)
    sm_max = (peaks or {}).get("sm_max_mhz", 2070.0)
    if w.kind == "dense":
        flop = 2.0 * w.batch * w.N * w.M * w.M                # one product Phi [x_0 .. x_N-1]
        if dom == "fine_fp32":
            bf16 = (peaks or {}).get("bf16_tflops", 1900.0)
            peak = 0.5 * bf16                                    # TF32 dense = BF16 / 2 (nominal)
            exe = 3.0 * flop                                     # three TF32 products (hi*hi, hi*lo, lo*hi)
            return {"bound": "tensor", "kernel": "k_dense_tf32x3 (tcgen05)", "achieved": exe / (avg_ms / 1e3) / 1e12,
                    "peak": peak, "unit": "TFLOP/s (TF32)", "frac": exe / (avg_ms / 1e3) / 1e12 / peak,
                    "traffic": None, "launch_ms": avg_ms, "launches": calls,
                    "algorithmic_tflops": flop / (avg_ms / 1e3) / 1e12,
                    "peak_source": "measured bf16 burst x 0.5 (nominal TF32/BF16 ratio), of measured"}
        tc = None
        t32 = (sub_timing or timing).get("fine_fp32", (0, 0.0))
        if t32[0]:
            # the inner solves' split-TF32 tcgen05 product (with its operand split)
            tms = t32[1] / t32[0]
            tpeak = 0.5 * (peaks or {}).get("bf16_tflops", 1900.0)
            tc = {"kernel": "k_gemm_tf32x3_p (tcgen05, persistent)", "launch_ms": tms,
                  "tflops_executed": 3.0 * flop / (tms / 1e3) / 1e12,
                  "frac_executed": 3.0 * flop / (tms / 1e3) / 1e12 / tpeak,
                  "peak": tpeak, "peak_source": "measured bf16 burst x 0.5 (nominal TF32/BF16 ratio)"}
        if dom == "fine_split":
            # product by error-free splitting: 7 BF16 digit slices per operand,
            # the 28 slice products of the diagonals s <= 8 on the tensor cores
            # (the launch time includes splitting the block vector)
            bf16 = (peaks or {}).get("bf16_tflops", 1900.0)
            exe = 28.0 * flop
            return {"bound": "tensor", "kernel": "k_gemm_oz (error-free splitting, tcgen05 BF16) + k_oz_split",
                    "tensor_product": tc,
                    "achieved": exe / (avg_ms / 1e3) / 1e12, "peak": bf16, "unit": "TFLOP/s (BF16 executed)",
                    "frac": exe / (avg_ms / 1e3) / 1e12 / bf16, "traffic": None,
                    "launch_ms": avg_ms, "launches": calls,
                    "algorithmic_tflops": flop / (avg_ms / 1e3) / 1e12,
                    "peak_source": "measured bf16 burst, of measured"}
        if dom == "fine_ff":
            # compensated float-float product: 12 FP32 lane-ops per multiply-add
            peak = FP32_LANES_PER_SM * nsm * sm_max * 1e6 / 1e12
            ops = 12.0 * flop / 2.0
            return {"bound": "alu", "kernel": "k_gemm_ff (float-float true residual)",
                    "tensor_product": tc,
                    "achieved": ops / (avg_ms / 1e3) / 1e12, "peak": peak,
                    "unit": "Tops/s (FP32 pipe lane-ops)",
                    "frac": ops / (avg_ms / 1e3) / 1e12 / peak, "traffic": None,
                    "launch_ms": avg_ms, "launches": calls,
                    "algorithmic_tflops": flop / (avg_ms / 1e3) / 1e12,
                    "peak_source": f"derived: 128 lanes/clk/SM x {nsm} SMs x {sm_max:.0f} MHz"}
        peak = FP64_LANES_PER_SM * 2 * nsm * sm_max * 1e6 / 1e12
        return {"bound": "alu", "kernel": "k_gemm_f64 (FP64 true residual)",
                "achieved": flop / (avg_ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s (FP64)",
                "frac": flop / (avg_ms / 1e3) / 1e12 / peak, "traffic": None, "launch_ms": avg_ms,
                "launches": calls, "peak_source": "derived: 4 FP64 flop/clk/SM x SMs x max SM clock"}
    point_steps = w.batch * w.N * w.fine[1] * w.M
    if w.kind == "heat1d":
        # one implicit-Euler step is a factored tridiagonal solve, two affine
        # scans of about 2 FMA per point each; at M = 63, N = 16 a launch is a
        # few microseconds of latency, far from any pipe's roofline
        flop = point_steps * 8.0
        peak = FP64_LANES_PER_SM * 2 * nsm * sm_max * 1e6 / 1e12
        ach = flop / (avg_ms / 1e3) / 1e12
        if dom == "fine_fp64" and heat1d_uses_matrix(w):
            # the m steps of a slice as one product with Phi = A^{-m} (M^2 FMA)
            mflop = 2.0 * w.batch * w.N * w.M * w.M
            mach = mflop / (avg_ms / 1e3) / 1e12
            return {"bound": "latency", "kernel": "k_heat1d_fine_phi (FP64 propagator matrix)",
                    "achieved": mach, "peak": peak, "unit": "TFLOP/s (FP64, 2 M^2 flop per slice)",
                    "frac": mach / peak, "traffic": None, "launch_ms": avg_ms, "launches": calls,
                    "equivalent_step_tflops": ach,
                    "note": "one CTA per slice, a row per thread: a few microseconds of launch and "
                            "load latency, far from the FP64 pipe's roofline",
                    "peak_source": "derived: 4 FP64 flop/clk/SM x SMs x max SM clock"}
        kname = "k_heat1d_fine_warp" if w.M <= 256 else "k_heat1d_fine"
        return {"bound": "latency", "kernel": "%s<%s>" % (kname, "double" if dom == "fine_fp64" else "float"),
                "achieved": ach, "peak": peak, "unit": "TFLOP/s (FP64, 8 flop per point-step)",
                "frac": ach / peak, "traffic": None, "launch_ms": avg_ms, "launches": calls,
                "note": ("one warp per slice, E points per lane: 5E + 8 FP64 warp instructions "
                         "per implicit-Euler step, issue-bound on one SM sub-partition's FP64 pipe")
                if w.M <= 256 else "latency-bound: one CTA per slice",
                "peak_source": "derived: 4 FP64 flop/clk/SM x SMs x max SM clock"}
    lanes = FP64_LANES_PER_SM if dom == "fine_fp64" else FP32_LANES_PER_SM
    peak = lanes * nsm * sm_max * 1e6 / 1e12
    if w.kind == "advdiff2d":
        method = ADV_OPS_PER_POINT_STEP
        executed = ADV_FF_OPS_PER_POINT_STEP if dom in ("fine_ff", "fine_split") else ADV_OPS_PER_POINT_STEP
    else:
        method = METHOD_OPS_PER_POINT_STEP
        executed = OPS_PER_POINT_STEP[dom]
    kdom = dom
    if w.kind == "heat2d" and dom == "fine_split":
        # the split residual needs z = 8 nu dt / h^2 <= 1/8; above it the
        # library runs the float-float kernel under the same timing class
        h = 1.0 / (w.nx + 1)
        z = 8.0 * w.nu * (w.T / w.N / w.fine[1]) / (h * h)
        if z > 0.125:
            kdom = "fine_ff"
            executed = OPS_PER_POINT_STEP["fine_ff"]
    secs = avg_ms / 1e3
    kname = KERNEL_NAMES[kdom] if w.kind == "heat2d" else ADV_KERNEL_NAMES.get(dom, ADV_KERNEL_NAMES["fine_ff"])
    units = w.batch * w.N * w.M                     # point-slices per launch
    tr = traffic_for(kname, units) if w.kind == "heat2d" else None
    # algorithmic bytes per point-slice: x_{n-1} read and the block-operator
    # row written once (x_n and x_{n-1} are the same array, read once over
    # the launch): FP64 in, FP64 out (residuals) or FP32 out (inner solves)
    alg_bytes = units * (8 + (4 if dom == "fine_fp32" else 8))
    roof = {"bound": "alu", "kernel": kname,
            "achieved": point_steps * method / secs / 1e12, "peak": peak,
            "unit": "Tops/s (%s pipe lane-ops of the method: %d per point-step)"
                    % ("FP64" if dom == "fine_fp64" else "FP32", method),
            "frac": point_steps * method / secs / 1e12 / peak,
            "frac_executed": point_steps * executed / secs / 1e12 / peak,
            "executed_ops_per_point_step": executed,
            "traffic": tr, "algorithmic_bytes": alg_bytes,
            "launch_ms": avg_ms, "launches": calls,
            "flop_rate_tflops": point_steps * FLOP_PER_POINT_STEP / secs / 1e12,
            "peak_source": f"derived: {lanes} lanes/clk/SM x {nsm} SMs x {sm_max:.0f} MHz (max SM clock)"}
    f32 = (sub_timing or timing)["fine_fp32"]
    if f32[0]:
        a32 = point_steps * method / (f32[1] / f32[0] / 1e3) / 1e12
        roof["fine_fp32"] = {"launch_ms": f32[1] / f32[0], "achieved": a32,
                             "frac": a32 / (FP32_LANES_PER_SM * nsm * sm_max * 1e6 / 1e12)}
    return roof


# ------------------------------------------------------------------ GPU leg

def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world,
                                device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_10148_gb300 import pit
    ctx = dict(torch=torch, pit=pit, rank=rank, world=world, local=local, dist=dist,
               dev=torch.device("cuda", local))
    line = measure_ours(args, ctx)
    if rank == 0 and world == 1 and args.workload == "heat2d" and not args.no_configs:
        line["configs"] = other_configs(args, ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


SUB_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "rel_err_max", "sweep",
            "rel_err_lambda_N", "iterations", "refinements", "matvecs", "status", "gpu_launches",
            "e2e", "fp64_path", "latency_s", "capacity_solves_per_s", "rel_err_max_sampled",
            "completed", "failed", "max_running", "fine_slice_steps_per_s", "invalid")


def _brief(line):
    """The parts of a workload's line that the headline line carries."""
    out = {k: line[k] for k in SUB_KEYS if k in line}
    out["workload"] = line["config"]["workload"]
    r = line.get("roofline") or {}
    out["roofline"] = {k: r.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit", "frac",
                                             "frac_executed", "launch_ms", "launches", "note")
                       if k in r}
    if "breakdown" in line:
        out["breakdown_share"] = {k: round(v["share"], 4) for k, v in line["breakdown"].items()
                                  if v["calls"]}
    if "serial_fine" in line:
        out["serial_fine"] = {k: v for k, v in line["serial_fine"].items() if k != "note"}
    return out


def other_configs(args, ctx):
    """Short lines of the other configurations after the headline's: the
    plain FP64 1D heat method (M = 63, N = 16), periodic advection-diffusion
    512^2 (N = 256), the dense-propagator mode (M = 1024, N = 4096) and
    serving (a Poisson stream at 200 requests/s), each with its own timed
    steps, accuracy against the FP64 path, end-to-end rate and roofline."""
    out = {}
    plans = [("heat1d_M63_N16_fp64", ["--workload", "heat1d", "--steps", "20", "--warmup", "3"]),
             ("advdiff2d_512x512_N256", ["--workload", "advdiff", "--steps", "3", "--warmup", "3"]),
             ("dense_M1024_N4096", ["--workload", "dense", "--steps", "3", "--warmup", "3"])]
    for name, argv in plans:
        sub = parse(argv + ["--residual", args.residual, "--no-cpu"] +
                    (["--no-e2e"] if args.no_e2e else []))
        t0 = time.perf_counter()
        try:
            out[name] = _brief(measure_ours(sub, ctx))
        except Exception as e:   # a failed sub-line must not lose the headline
            out[name] = {"failed": str(e)}
        out[name]["wall_s"] = time.perf_counter() - t0
    sub = parse(["--workload", "serving", "--steps", "2", "--warmup", "1", "--requests", "64",
                 "--no-cpu", "--residual", args.residual])
    t0 = time.perf_counter()
    try:
        out["serving_poisson_200rps"] = _brief(measure_serving(sub, ctx))
    except Exception as e:
        out["serving_poisson_200rps"] = {"failed": str(e)}
    out["serving_poisson_200rps"]["wall_s"] = time.perf_counter() - t0
    return out


def measure_ours(args, ctx):
    """One workload through pit_bicgstab_solve: the timed steps, accuracy,
    roofline, comparators and the end-to-end leg; returns rank 0's line."""
    torch, pit = ctx["torch"], ctx["pit"]
    rank, world, local, dist, dev = ctx["rank"], ctx["world"], ctx["local"], ctx["dist"], ctx["dev"]
    fp64 = args.precision == "fp64"
    stream = torch.cuda.Stream(device=dev)
    w = workload(args, rank)
    shape = (w.batch, w.N + 1, w.M)
    K, W = args.steps, args.warmup
    # distinct initial values per step, resident on the device
    y0s = [torch.from_numpy(workload(args, rank, step=s).y0.copy()).to(dev) for s in range(K + W)]
    prob = pit.Problem(w, args.precision)
    X = torch.zeros(shape, dtype=torch.float64, device=dev)
    if fp64:
        solve_kw = dict(tol=args.tol, tol_mode=args.tol_mode, max_iter=500)
    else:
        solve_kw = dict(tol=args.tol, tol_mode=args.tol_mode, max_iter=200, refine_max=8,
                        inner_tol=args.inner_tol, residual_precision=args.residual)

    def one(step):
        prob.set_y0(y0s[step])
        return prob.bicgstab_solve(X, stream=stream.cuda_stream, **solve_kw)[1]

    # timing on from the warm-up on (the graphs are captured in the timing
    # mode there); the clock sampler starts before the warm-up too, so its
    # start-up does not fall into the timed region.  The timed solves time
    # their top-level launches only (true residuals, sweeps outside the
    # iterations, each launch of the iterations as a whole: the iterations
    # run as the same loop graph as untimed); per-operator times come from a
    # few fully timed solves after the timed region
    tmode = 2
    prob.set_timing(tmode)
    clk = ClockSampler(os.path.join(CLOCKS_DIR,
                                    f"clocks_rank{rank}.csv"))
    with clk:
        with torch.cuda.stream(stream):
            for s in range(W):
                one(s)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        prob.set_timing(tmode)         # resets the per-class sums
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        infos = []
        launches0 = pit.kernel_launches()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for s in range(K):
                infos.append(one(W + s))
                ev[s + 1].record(stream)
        torch.cuda.synchronize()
    launches = pit.kernel_launches() - launches0
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(K)]
    total_ms = ev[0].elapsed_time(ev[K])
    timing = prob.timing()
    prob.set_timing(False)
    # per-class breakdown: with top-level timing, from a few fully timed
    # solves after the timed region (steps of the same y0 sequence)
    timing_full, full_ms, full_steps = timing, total_ms, K
    if tmode == 2:
        full_steps = min(K, 3)
        prob.set_timing(True)
        with torch.cuda.stream(stream):
            one(W)                       # captures the per-iteration graphs
        torch.cuda.synchronize()
        prob.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for s in range(full_steps):
                one(W + s)
            e1.record(stream)
        torch.cuda.synchronize()
        full_ms = e0.elapsed_time(e1)
        timing_full = prob.timing()
        prob.set_timing(False)
    total_ms = max_over_ranks([total_ms], dev)[0]
    solves = w.batch * K * world
    value = whole_job_rate(w.batch * K, world, total_ms / 1e3)
    slice_steps = sum(i["fine_slice_steps"] for inf in infos for i in inf) * world
    # accuracy of the last step against the FP64 serial fine trajectory (FP64 path)
    lam = torch.empty(shape, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t_ser = time.perf_counter()
    prob.serial_fine("fp64", out=lam)
    torch.cuda.synchronize()
    t_ser64 = time.perf_counter() - t_ser
    # the no-PiT comparator: the same trajectory stepped slice after slice
    # in FP32 (one launch per slice for the whole batch), and its accuracy
    lam32 = torch.empty(shape, dtype=torch.float64, device=dev)
    t_ser32 = e32 = None
    if not fp64:
        t_ser = time.perf_counter()
        prob.serial_fine("mixed", out=lam32)
        torch.cuda.synchronize()
        t_ser32 = time.perf_counter() - t_ser
        e32 = (((lam32 - lam).reshape(w.batch, -1).norm(dim=1)
                / lam.reshape(w.batch, -1).norm(dim=1)).max().item())
    # the no-PiT comparators that meet the 1e-6 bar: the serial trajectory in
    # float-float and in the split RK4 arithmetic (heat2d; float-float elsewhere)
    ser = {}
    for prec in ("ff", "split"):
        if fp64 or (prec == "split" and w.kind != "heat2d"):
            continue
        torch.cuda.synchronize()
        t_ser = time.perf_counter()
        prob.serial_fine(prec, out=lam32)
        torch.cuda.synchronize()
        ser[prec] = (time.perf_counter() - t_ser,
                     (((lam32 - lam).reshape(w.batch, -1).norm(dim=1)
                       / lam.reshape(w.batch, -1).norm(dim=1)).max().item()))
    del lam32
    d = (X - lam).reshape(w.batch, -1)
    rel = (d.norm(dim=1) / lam.reshape(w.batch, -1).norm(dim=1)).max().item()
    relN = ((X[:, -1] - lam[:, -1]).norm(dim=1) / lam[:, -1].norm(dim=1)).max().item()
    statuses = sorted({i["status_name"] for inf in infos for i in inf})

    line = None
    if rank == 0:
        peaks = load_peaks()
        clocks = clk.summary(local)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        # the FP64 path's fine kernel runs inside the iterations: its launches
        # are timed in the fully timed solves after the timed region
        roof = (roofline(w, timing_full, peaks, nsm) if fp64 else
                roofline(w, timing, peaks, nsm, sub_timing=timing_full))
        breakdown = {k: {"calls": c, "ms": m, "share": m / full_ms}
                     for k, (c, m) in timing_full.items() if k != "inner"}
        line = {"metric": "PiT solves/s (rel err <= 1e-6 vs FP64 path)", "value": value,
                "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if fp64 else "f32 fine / f64 krylov",
                "data": "synthetic",
                "config": bench_config(args, w, world),
                "fine_slice_steps_per_s": slice_steps / (total_ms / 1e3),
                "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                               "p99": float(np.percentile(step_ms, 99))},
                "rel_err_max": rel, "rel_err_lambda_N": relN, "status": statuses,
                "iterations": [i["iterations"] for inf in infos for i in inf],
                "refinements": [i["refinements"] for inf in infos for i in inf],
                "matvecs": [i["matvecs"] for inf in infos for i in inf],
                "gpu_launches": int(launches), "roofline": roof, "breakdown": breakdown,
                "sweep": sweep_cost(w, timing_full, full_ms, full_steps),
                "timing_note": ("timed region: CUDA events around the top-level launches (true "
                                "residuals, sweeps outside the iterations) and around each launch of "
                                "the BiCGStab iterations, which run as the uninstrumented loop graph; "
                                + ("roofline of the fine kernel (inside the iterations), "
                                   if fp64 else
                                   "roofline of the residual kernel from those events; ")
                                + "per-class breakdown, sweep cost and the FP32 inner kernel's entry from "
                                f"{full_steps} fully timed solves (per-operator CUDA events) after the "
                                "timed region"),
                "timed_region_classes": {k: {"calls": c, "ms": m} for k, (c, m) in timing.items() if c},
                "serial_fine": {"fp64_s_per_batch": t_ser64, "fp32_s_per_batch": t_ser32,
                                "fp32_rel_err": e32, "batch": w.batch,
                                **{f"{k}_s_per_batch": v[0] for k, v in ser.items()},
                                **{f"{k}_rel_err": v[1] for k, v in ser.items()},
                                # the fastest serial trajectory within 1e-6 of FP64 (FP64 itself
                                # included) against one PiT step of the same batch
                                "pit_speedup_vs_best_serial_within_1e6": (
                                    min([v[0] for v in ser.values() if v[1] <= 1e-6] + [t_ser64])
                                    / (total_ms / 1e3 / K)),
                                "note": "slice after slice on this GPU (no parallel in time), "
                                        "one launch per slice for the whole batch"},
                "clocks": clocks}
        if rel > 1e-6:
            line["invalid"] = f"rel err {rel:.3e} > 1e-6"

    # end-to-end through host buffers
    if not args.no_e2e:
        hx = torch.empty(shape, dtype=torch.float64).pin_memory()
        hy0 = [torch.from_numpy(workload(args, rank, step=s).y0.copy()).pin_memory()
               for s in range(K + W)]
        hx_np = hx.numpy()

        def one_host(step):
            prob.set_y0(hy0[step].numpy())
            return prob.bicgstab_solve(hx_np, **solve_kw)[1]

        for s in range(W):
            one_host(s)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for s in range(K):
            one_host(W + s)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks([e2e_s], dev)[0]
        if rank == 0:
            line["e2e"] = {"value": solves / e2e_s, "unit": "solves/s",
                           "h2d_bytes_per_step": w.batch * w.M * 8,
                           "d2h_bytes_per_step": w.batch * (w.N + 1) * w.M * 8}

    # the plain FP64 GPU path on the same workload, for comparison
    if rank == 0 and not args.no_fp64_path and not fp64:
        # same workload and batch, every step in FP64 on the device
        w1 = workload(args, 0)
        p64 = pit.Problem(w1, "fp64")
        X64 = torch.zeros((w1.batch, w1.N + 1, w1.M), dtype=torch.float64, device=dev)
        p64.bicgstab_solve(X64, tol=args.tol, tol_mode="rhs", max_iter=200)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, i64 = p64.bicgstab_solve(X64, tol=args.tol, tol_mode="rhs", max_iter=200)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        lam64 = torch.empty_like(X64[:1])
        p64.close()
        pm = pit.Problem(w1.member(0), "fp64")
        pm.serial_fine("fp64", out=lam64)
        pm.close()
        e64 = ((X64[:1] - lam64).norm() / lam64.norm()).item()
        line["fp64_path"] = {"value": w1.batch / t64, "unit": "solves/s", "batch": w1.batch,
                             "iterations": i64[0]["iterations"], "matvecs": i64[0]["matvecs"],
                             "rel_err_member0": e64}

    if rank == 0 and not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline(workload(args, 0))
        except Exception as e:  # the baseline is context; never fail the bench line
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1,
                                    "kind": "oracle", "sample": f"failed: {e}"}
    prob.close()
    return line


# -------------------------------------------------------------- serving leg

def serving_steps(args, rank, steps):
    """Requests of each step: consecutive pieces of one seeded Poisson stream
    (arrival times relative to the start of their step)."""
    out = []
    for st in range(steps):
        first = (rank * 100003 + st) * args.requests
        t, ws = 0.0, []
        for j in range(args.requests):
            gap, w = inputs.serving_request(first + j, rate=args.rate)
            t += gap
            w.arrival = t
            ws.append(w)
        out.append(ws)
    return out


def run_serving(args):
    """Open-loop serving: each step submits `--requests` requests of the Poisson
    stream at their arrival times to one server and waits for all results."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world,
                                device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_10148_gb300 import pit
    ctx = dict(torch=torch, pit=pit, rank=rank, world=world, local=local, dist=dist,
               dev=torch.device("cuda", local))
    line = measure_serving(args, ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def measure_serving(args, ctx):
    torch, pit = ctx["torch"], ctx["pit"]
    rank, world, local, dist = ctx["rank"], ctx["world"], ctx["local"], ctx["dist"]

    K, W = args.steps, args.warmup
    steps = serving_steps(args, rank, W + K + 1)
    opts = dict(tol=args.tol, tol_mode="rhs", max_iter=200, refine_max=8,
                inner_tol=args.inner_tol, residual_precision=args.residual)
    srv = pit.Server(hbm_budget_bytes=0, max_slots=args.slots)

    def one(ws, open_loop=True):
        t0 = time.perf_counter()
        tickets = []
        for w in ws:
            if open_loop:
                dt = w.arrival - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            tickets.append(srv.submit(w, **opts))
        return [srv.wait(t) for t in tickets]

    for s in range(W):
        one(steps[s])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    srv.stats(reset=True)
    launches0 = pit.kernel_launches()
    clk = ClockSampler(os.path.join(CLOCKS_DIR,
                                    f"clocks_rank{rank}.csv"))
    results = []
    with clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(K):
            results.append(one(steps[W + s]))
        torch.cuda.synchronize()
        total_s = time.perf_counter() - t0
    launches = pit.kernel_launches() - launches0
    st = srv.stats(reset=True)
    # capacity: one more step submitted at once (closed loop)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    burst = one(steps[W + K], open_loop=False)
    burst_s = time.perf_counter() - t1
    total_s, burst_s = max_over_ranks([total_s, burst_s], torch.device("cuda", local))
    nreq = args.requests * K
    ok = sum(1 for step in results for r in step if r[0] == pit.PIT_OK)
    value = ok * world / total_s
    slice_steps = sum(i["fine_slice_steps"] for step in results for r in step for i in r[2])
    # accuracy: the sampled requests with the least fine work, against the FP64 GPU path
    last = steps[W + K - 1]
    order = sorted(range(len(last)), key=lambda j: last[j].N * last[j].fine[1] * last[j].M)
    rel = 0.0
    for j in order[:4]:
        w = last[j]
        with pit.Problem(w, "fp64") as p:
            lam = p.serial_fine("fp64")
        X = results[-1][j][1]
        rel = max(rel, float(np.linalg.norm(X - lam) / np.linalg.norm(lam)))
    line = None
    if rank == 0:
        peaks = load_peaks()
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        sm_max = (peaks or {}).get("sm_max_mhz", 2070.0)
        peak = FP32_LANES_PER_SM * nsm * sm_max * 1e6 / 1e12
        pts = sum(i["fine_slice_steps"] * w.M for step_w, step in zip(steps[W:W + K], results)
                  for w, r in zip(step_w, step) for i in r[2])
        ach = pts * OPS_PER_POINT_STEP["fine_fp32"] / total_s / 1e12
        mix = [w for step in steps[W:W + K] for w in step]
        h2d = sum(w.y0.size * 8 for w in mix) / K
        d2h = sum(w.batch * (w.N + 1) * w.M * 8 for w in mix) / K
        line = {"metric": "PiT solves/s & p50/p99 latency, serving (rel err <= 1e-6 vs FP64 path)",
                "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": total_s * 1e3 / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 fine / f64 krylov", "data": "synthetic",
                "config": {"workload": f"serving_poisson_{args.rate:g}rps_{args.requests}req_per_step",
                           "mix": "50% heat1d M~U{63..4095} IE 100 steps/slice, 50% heat2d n~U{32..256} "
                                  "RK4 m=max(50, dT nu/(0.2 h^2)); N~U{16..1024}; nu log-uniform [1e-3, 1e-1]",
                           "slots": args.slots, "hbm_budget_bytes": st["hbm_budget"],
                           "tol": args.tol, "tol_mode": "rhs", "inner_tol": args.inner_tol,
                           "timer": "host wall clock around the open-loop stream, device synchronised",
                           "l2": "working set > L2 (concurrent requests' Krylov vectors)",
                           "parallelism": f"replicas x{world}"},
                "latency_s": {"p50": st["latency_p50"], "p99": st["latency_p99"],
                              "mean": st["latency_mean"], "queue_p50": st["queue_p50"],
                              "queue_p99": st["queue_p99"], "service_p50": st["service_p50"],
                              "service_p99": st["service_p99"]},
                "fine_slice_steps_per_s": slice_steps * world / total_s,
                "capacity_solves_per_s": args.requests * world / burst_s,
                "completed": st["completed"], "failed": st["failed"], "requests": nreq,
                "max_running": st["max_running"], "hbm_reserved_peak": st["hbm_reserved_peak"],
                "pool_peak_bytes": st["pool_peak"], "rel_err_max_sampled": rel,
                "gpu_launches": int(launches),
                "roofline": {"bound": "alu", "kernel": "whole serving run (all fine kernels)",
                             "achieved": ach, "peak": peak, "unit": "Tops/s (FP32 pipe lane-ops)",
                             "frac": ach / peak, "traffic": None,
                             "note": "fine slice-steps x points x 20 lane-ops (FP32 count) / wall time",
                             "peak_source": f"derived: 128 lanes/clk/SM x {nsm} SMs x {sm_max:.0f} MHz"},
                "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h),
                        "note": "the serving value is host to host: y0 in, X out per request"},
                "clocks": clk.summary(local)}
        if rel > 1e-6:
            line["invalid"] = f"rel err {rel:.3e} > 1e-6"
        if not args.no_cpu:
            try:
                line["cpu_baseline"] = serving_cpu_baseline(last, results[-1])
            except Exception as e:
                line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1,
                                        "kind": "oracle", "sample": f"failed: {e}"}
    srv.close()
    return line


def serving_cpu_baseline(ws, res, budget_s=20.0):
    """Oracle seconds per request, estimated on a bounded sample: for requests
    of the stream (in order, until about `budget_s` of CPU time), the oracle's
    G^{-1}F on up to 8 slices scaled to N plus one full sweep, times the number
    of matvecs the GPU solve of that request took."""
    tot, cnt, t_start = 0.0, 0, time.perf_counter()
    for w, r in zip(ws, res):
        if time.perf_counter() - t_start > budget_s and cnt >= 2:
            break
        if w.N * w.fine[1] * w.M > 4e8:
            continue
        t_f, t_s = oracle_sample(w, min(w.N, 8))
        tot += (t_f + t_s) * r[2][0]["matvecs"]
        cnt += 1
    return {"value": cnt / tot if tot else None, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 numpy/scipy oracle, 1 thread, {cnt} requests of the stream (fine "
                       f"work <= 4e8 point-steps per matvec): G^-1F on up to 8 slices scaled to N "
                       f"+ one full sweep, x the GPU solve's matvec count")}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
