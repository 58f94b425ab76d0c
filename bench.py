"""Benchmark: QTW-CG time to relative residual 1e-14 on the 128^3 7-point Poisson system.

Other configurations: --workload c1 c3 c4 c5 (2-D Poisson 64^2 latency case,
power-law graph Laplacian, 256-system batch vs one-by-one, differentiable
diffusion solve checked by TW finite differences), one JSON line each.

One step = one complete solve (initialisation + CG iterations until the FP64
relative residual drops below 1e-14) of the 3-D Poisson system (n = 2,097,152,
nnz = 14,581,760, b = 2U-1 seeded, x0 = 0) in quasi triple-word arithmetic,
through the C ABI (mwcg_solve).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mwcg|reference]

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload (a few CG iterations per step) and extrapolates to the
oracle's own iteration count for the full solve (tests/golden/fullsize_c2.json,
written from the oracle).  The solver has a single-GPU path; with N > 1
(torchrun) every rank solves its own replica and rank 0 reports the max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "QTW-CG time-to-1e-14 residual (3-D Poisson 128^3, 7-point)"
WORKLOAD = "c2"
GOLDEN = os.path.join(ROOT, "tests", "golden", "fullsize_c2.json")
# Nominal FP64 rate of the GB300 (context only): 2 FP64 operations per clock
# per SM (FMA counted as one operation, as the paper counts), 152 SMs, 2070 MHz.
FP64_OPS_PER_CLK_SM = 2
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_OPS = FP64_OPS_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6
# The paper's FP64 operation counts (FMA = 1) per stored entry and per row of
# the fused SpMV + p^T q kernel: FP64 x MW product + MW add per entry, minus the
# add saved on each row's first product, plus the dot leaf (MW product) and its
# accumulation.  Reported as `paper_ops_per_s`; part of this work runs on the
# integer pipe, so it is not a fraction of any one pipe.
SPMV_OPS = {  # arith: (per nnz, per row)
    "fp64": (1, 1 + 1),
    "dw": (6 + 11, 7 + 11 - 11),
    "qdw": (3 + 8, 4 + 8 - 8),
    "qtw": (12 + 21, 24 + 21 - 21),
}
SPMV_OPS["qdw_nn"] = SPMV_OPS["qdw"]
SPMV_OPS["qtw_nn"] = SPMV_OPS["qtw"]
# FP64 instructions the SpMV kernel executes per operation (thread level:
# DADD, DFMA, DMUL), from the device sequences: TwoSum errors (and the
# double-word TwoProd errors) come from the integer pipe, a power-of-two
# matrix entry scales the words exactly on the integer pipe, and the QTW SpMV
# adds the product's last word on the integer pipe and the DW SpMV the closing
# QuickTwoSum of its products.  Keys: FP64 x MW product
# with a general entry ("dx") and with a power-of-two entry ("dx2"), MW add,
# MW product.  These counts reproduce ncu's executed-instruction counters
# (profiles/k_spmv_*_c2.md).
SPMV_INSTR = {
    "qtw": {"dx": (1, 3, 2), "dx2": (0, 0, 0), "add": (6, 0, 0), "mul": (5, 6, 3)},
    "dw": {"dx": (0, 1, 1), "dx2": (0, 0, 0), "add": (6, 0, 0), "mul": (0, 2, 1)},   # QuickTwoSum on the integer pipe
    "qdw": {"dx": (0, 1, 1), "dx2": (0, 0, 0), "add": (3, 0, 0), "mul": (0, 2, 1)},
}
SPMV_INSTR["qtw_nn"] = SPMV_INSTR["qtw"]
SPMV_INSTR["qdw_nn"] = SPMV_INSTR["qdw"]
WORDS = {"fp64": 1, "dw": 2, "qdw": 2, "qtw": 3, "tw": 3, "qdw_nn": 2, "qtw_nn": 3, "qw": 4, "qqw": 4, "qqw_nn": 4,
         "qqf": 4, "qf": 4}
# FP32 pipe: 128 lanes per SM (FMA = 1 operation).
FP32_PEAK_OPS = 128 * SMS * SM_MAX_MHZ * 1e6
# FP32 operations of the QQF SpMV + p^T q kernel: per stored entry the FP64 x
# QQF product (the full QQF product with the split: 6 TwoProd x 2 + 8 TwoSum
# x 6 + 4 FMA + 8 adds = 72, plus the split's 2 exact subtractions) and the
# QQF add (6 TwoSum x 6 + 4 = 40), less the add saved on each row's first
# product; per row the dot leaf (product 72 + add 40).
QQF_SPMV_OPS = (72 + 2 + 40, 72 + 40 - 40)
# QF: every product and addition followed by VecSum4 (3 TwoSums, 18 operations).
FP32_SPMV_OPS = {"qqf": QQF_SPMV_OPS, "qf": (72 + 2 + 18 + 40 + 18, 72 + 18 + 40 + 18 - (40 + 18))}


def is_pow2(v):
    """The device's power-of-two test (mwi::is_pow2): zero fraction, normal exponent."""
    u = np.ascontiguousarray(v, dtype=np.float64).view(np.uint64)
    e = (u >> np.uint64(52)) & np.uint64(0x7FF)
    return ((u & np.uint64((1 << 52) - 1)) == 0) & (e >= 1) & (e <= 2046)


def spmv_fp64_instr(arith, A, V):
    """(DADD, DFMA, DMUL) thread-level FP64 instructions of one k_spmv launch
    (mode 1) with V lanes per row, or None when no model exists for `arith`.
    Every stored entry is one FP64 x MW product; a row of L > 0 entries adds
    L - 1 products (each lane sums its entries, the lane tree combines the
    lanes); each of the n rows gives a dot leaf, and the n leaves are summed by
    n - 1 additions (slot accumulation, block tree, grid tree).  FP64: a lane's
    first product is a DMUL, the rest are FMAs, the lane tree DADDs."""
    lens = np.diff(np.asarray(A.row_ptr, dtype=np.int64))
    n, nnz = int(A.n), int(A.nnz)
    if arith == "fp64":
        first = int(np.minimum(lens, V).sum())
        tree = int(np.maximum(np.minimum(lens, V) - 1, 0).sum())
        return (tree + max(n - 1, 0), nnz - first, first + n)
    m = SPMV_INSTR.get(arith)
    if m is None:
        return None
    p2 = int(is_pow2(A.val).sum())
    adds = (nnz - int((lens > 0).sum())) + max(n - 1, 0)
    tot = [0, 0, 0]
    for key, cnt in (("dx", nnz - p2), ("dx2", p2), ("add", adds), ("mul", n)):
        for j in range(3):
            tot[j] += m[key][j] * cnt
    return tuple(tot)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    return ws, rk


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank timing over all ranks (the job's time).  With N
    GPUs every rank solves its own replica of the workload (the headline
    system is one coupled solve, so there is no data-path collective); only
    this timing reduction crosses ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max([num(r[3]) for r in rows if num(r[3]) is not None], default=None)}


# The headers the CG kernels are built from: a committed ncu summary carries
# their digest, and its counters are used only while the digest still matches.
KERNEL_SOURCES = ("mw_int.cuh", "mw_device.cuh", "mw_float.cuh", "cg_kernels.cuh", "cg_float.cuh")


def _kernel_source_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2510_13536_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _profile_fields(arith):
    """The key/value lines of the committed ncu summary of k_spmv, or None when
    the summary is missing or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"k_spmv_{arith}_c2.md")
    try:
        kv = {}
        for line in open(path):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        return kv if kv.get("kernel_source_digest") == _kernel_source_digest() else None
    except OSError:
        return None


def _profiled_traffic(arith):
    """DRAM bytes per k_spmv launch from the committed ncu summary (or None)."""
    kv = _profile_fields(arith)
    try:
        return float(kv["dram_bytes_per_launch"]) if kv else None
    except (KeyError, ValueError):
        return None


def _profiled_fp64_pipe(arith):
    """Fraction of cycles the FP64 pipe was active in that capture (or None)."""
    kv = _profile_fields(arith)
    if not kv:
        return None
    for k, v in kv.items():
        if k.startswith("FP64 pipe active"):
            try:
                return float(v.split("%")[0].strip()) / 100.0
            except ValueError:
                return None
    return None


def _golden_plan():
    """Summation plan of the recorded full solve (the GB300 solver's plan)."""
    try:
        return tuple(json.load(open(GOLDEN))["plan"])
    except Exception:
        return (1, 256, 456)


def _golden_iters(arith):
    try:
        g = json.load(open(GOLDEN))
        return int(g[arith]["iters"]), "oracle full solve (tests/golden/fullsize_c2.json)"
    except Exception:
        return None, None


def oracle_sample(A, b, arith, iters_sample, total_iters, plan):
    """Time the CPU oracle (single thread) on `iters_sample` CG iterations of
    the workload and project a complete solve of `total_iters` iterations.
    Returns (projected seconds, seconds per iteration, init seconds, seconds
    actually spent, residual history of the timed run)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.cg(arith, A, b, tol=0.0, maxit=1, plan=plan)
    t_init1 = time.perf_counter() - t0                      # init + 1 iteration
    t0 = time.perf_counter()
    *_, hist = oracle.cg(arith, A, b, tol=0.0, maxit=1 + iters_sample, plan=plan, history=True)
    t_run = time.perf_counter() - t0                        # init + 1 + k iterations
    per_it = max(t_run - t_init1, 1e-9) / iters_sample
    init = max(t_init1 - per_it, 0.0)
    return init + per_it * total_iters, per_it, init, t_init1 + t_run, hist


CPU_SAMPLE_ITERS = 40       # oracle iterations timed for cpu_baseline (about 10 s of CPU work at c2)


def cpu_baseline(torch, mw, M, A, b_np, b_dev, arith, tol, gpu_iters, k=CPU_SAMPLE_ITERS):
    """The oracle (as it stands, one thread) timed on the first k CG iterations
    of the same solve, projected to the solve's iteration count; the GPU's
    first k + 1 residuals are checked bit for bit against the timed run's."""
    gi, src = _golden_iters(arith)
    tot = gi if gi is not None else gpu_iters
    src = src or "the GPU's iteration count (equal to the oracle's by the parity tests)"
    est, per_it, init, spent, hist = oracle_sample(A, b_np, arith, k, tot, M.plan)
    r = mw.solve(M, b_dev, arith, 0.0, 1 + k, history=True)
    same = bool(np.array_equal(r.history.cpu().numpy().view(np.uint64), np.asarray(hist).view(np.uint64)))
    return {"value": est, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"{k + 1} CG iterations + init of the full system timed (one thread, {spent:.1f} s), "
                      f"{per_it:.4f} s per iteration projected to {tot} iterations ({src}); the oracle is "
                      f"the test oracle built -O3 -ffp-contract=off, not tuned",
            "iterations_timed": k + 1, "projected": True, "seconds_timed": spent,
            "history_bits_match_gpu": same}


# FP64 instructions (DADD, DFMA, DMUL) per element of the vector kernels:
# k_update = x += alpha p and r += (-alpha) q (two muladds: MW product + MW
# add), the normalisation of r (QTW VecSum3: two TwoSums; QDW QuickTwoSum),
# the dot leaf r r and its accumulation; k_pupdate = p = r + beta p (one
# muladd).  The same sequences as the SpMV model's table (SPMV_INSTR), less
# one DMUL in QTW's leaf r r, whose two cross products a1 b2 and a2 b1 are the
# same product (computed once; ncu counts 8 DMUL per element).
VEC_INSTR = {
    "qtw": {"update": (35, 18, 8), "p_update": (11, 6, 3)},
    "dw": {"update": (18, 6, 3), "p_update": (6, 2, 1)},     # products' QuickTwoSum on the integer pipe
    "qdw": {"update": (9, 6, 3), "p_update": (3, 2, 1)},      # r's QuickTwoSum on the integer pipe
    "fp64": {"update": (1, 2, 1), "p_update": (0, 1, 0)},
}


def vector_rooflines(arith, n, kms, probe, elem):
    """FP64-pipe and HBM fractions of k_update and k_pupdate (as spmv_roofline)."""
    m = VEC_INSTR.get(arith)
    r_add, r_fma, r_mul = probe["dadd_ops_per_s"], probe["dfma_ops_per_s"], probe["dmul_ops_per_s"]
    hbm = _measured_hbm_gbs() * 1e9
    out = {}
    for name, ms, passes in (("update_dot", kms[1], 6), ("p_update", kms[2], 3)):
        t = ms * 1e-3
        d = {"kernel_ms": ms, "alg_bytes_per_launch": passes * elem * n,
             "hbm_frac_of_measured": passes * elem * n / t / hbm}
        if m is not None:
            a, f, mu = m["update" if name == "update_dot" else "p_update"]
            d["fp64_instr_per_launch"] = {"dadd": a * n, "dfma": f * n, "dmul": mu * n}
            d["fp64_pipe_frac"] = (a * n / r_add + f * n / r_fma + mu * n / r_mul) / t
        out[name] = d
    return out


def spmv_roofline(arith, A, plan, spmv_ms, probe, elem):
    """Roofline of the dominant kernel, k_spmv (SpMV + p^T q + alpha), from its
    mean duration over 30 launches (CUDA events on the launching stream).

    Two ceilings: HBM (algorithmic bytes / the measured copy bandwidth) and the
    pipe that executes the arithmetic.  For the FP64-word arithmetics that is
    the FP64 pipe, whose rate depends on the instruction: the executed
    DADD / DFMA / DMUL counts (spmv_fp64_instr) over the rates the probe
    measured in this run give the time the pipe needs; `frac` is that time over
    the kernel's duration, reported as DADD-equivalent instructions per second
    against the measured DADD rate.  For QQF it is the FP32 pipe (operations of
    the sequences over 128 lanes x SMs x clock).  `bound` is the larger of the
    two fractions' ceilings."""
    t = spmv_ms * 1e-3
    n, nnz = int(A.n), int(A.nnz)
    alg_bytes = 12 * nnz + 8 * (n + 1) + 2 * elem * n      # val + col, row_ptr (int64), p once, q written
    hbm = _measured_hbm_gbs() * 1e9
    hbm_frac = alg_bytes / t / hbm
    kv = _profile_fields(arith) or {}

    def pct(prefix):
        for k2, v in kv.items():
            if k2.startswith(prefix):
                try:
                    return float(v.split("%")[0].strip()) / 100.0
                except ValueError:
                    return None
        return None

    out = {"kernel": f"k_spmv<{arith.upper()}> (SpMV + p^T q + alpha)", "kernel_ms": spmv_ms,
           "alg_bytes_per_launch": alg_bytes, "hbm_gbs": alg_bytes / t / 1e9, "hbm_peak_gbs": hbm / 1e9,
           "hbm_frac_of_measured": hbm_frac, "traffic": _profiled_traffic(arith),
           "fp64_pipe_active_ncu": pct("FP64 pipe active"), "int_pipe_active_ncu": pct("ALU (integer) pipe")}
    if arith in SPMV_OPS:
        per_nnz, per_row = SPMV_OPS[arith]
        ops = per_nnz * nnz + per_row * n
        out["paper_ops_per_launch"] = ops
        out["paper_ops_per_s"] = ops / t
    if arith in FP32_SPMV_OPS:
        ops = FP32_SPMV_OPS[arith][0] * nnz + FP32_SPMV_OPS[arith][1] * n
        f32 = ops / t / FP32_PEAK_OPS
        out["fp32_ops_per_launch"] = ops
        out["fp32_frac_of_derived_peak"] = f32
        alu = {"achieved": ops / t / 1e12, "peak": FP32_PEAK_OPS / 1e12, "unit": "T FP32 op/s (FMA = 1)",
               "frac": f32, "peak_source": "128 FP32 lanes/clk/SM x 152 SMs x 2070 MHz (derived)"}
    else:
        instr = spmv_fp64_instr(arith, A, plan[0])
        if instr is None:
            out.update({"bound": "hbm", "achieved": alg_bytes / t / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                        "frac": hbm_frac, "fp64_model": None})
            return out
        dadd, dfma, dmul = instr
        r_add, r_fma, r_mul = probe["dadd_ops_per_s"], probe["dfma_ops_per_s"], probe["dmul_ops_per_s"]
        pipe_s = dadd / r_add + dfma / r_fma + dmul / r_mul
        out["fp64_instr_per_launch"] = {"dadd": dadd, "dfma": dfma, "dmul": dmul}
        out["fp64_pipe_s_per_launch"] = pipe_s
        out["fp64_frac_of_nominal"] = (dadd + dfma + dmul) / t / FP64_PEAK_OPS
        alu = {"achieved": pipe_s * r_add / t / 1e12, "peak": r_add / 1e12,
               "unit": "T FP64 instructions/s (DADD-equivalent: DFMA and DMUL weighted by the measured rates)",
               "frac": pipe_s / t,
               "peak_source": "DADD rate measured in this run (mwcg_probe_peak); nominal 2 op/clk/SM x 152 x "
                              "2070 MHz = 0.629 T"}
    if alu["frac"] >= hbm_frac:
        out.update({"bound": "alu", **alu})
    else:
        out.update({"bound": "hbm", "achieved": alg_bytes / t / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                    "frac": hbm_frac, "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
                    "alu_frac": alu["frac"]})
    return out


def _timed(torch, fn, reps=1):
    s = torch.cuda.current_stream()
    best = None
    out = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        out = fn()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return out, best


def run_c1(torch, mw, P, cpu):
    A, b, tol, maxit = P.workload("c1")
    M = mw.CSRMatrix.from_csr(A)
    db = torch.as_tensor(b, device="cuda")
    out = {"workload": "c1: " + P.WORKLOADS["c1"], "plan": list(M.plan)}
    for ar in ("dw", "fp64"):
        mw.solve(M, db, ar, tol, maxit)
        r, ms = _timed(torch, lambda: mw.solve(M, db, ar, tol, maxit), reps=5)
        err = float(np.max(np.abs(mw.collapse(r.x).cpu().numpy() - 1.0)))
        out[ar] = {"time_s": ms / 1e3, "iters": r.iters, "status": r.status, "relres": r.relres,
                   "iters_per_s": r.iters / (ms / 1e3), "us_per_iter": ms * 1e3 / max(r.iters, 1),
                   "max_forward_error": err}
        if cpu:
            import oracle
            t0 = time.perf_counter()
            _, it, _, _ = oracle.cg(ar, A, b, tol=tol, maxit=maxit, plan=M.plan)
            out[ar]["cpu_oracle_s"] = time.perf_counter() - t0
            out[ar]["cpu_oracle_iters"] = it
    return out


def run_c3(torch, mw, P, cpu):
    out = {"workload": "c3: " + P.WORKLOADS["c3"]}
    A, b, tol, maxit = P.workload("c3")
    M = mw.CSRMatrix.from_csr(A)
    db = torch.as_tensor(b, device="cuda")
    lens = np.diff(A.row_ptr)
    out.update({"n": A.n, "nnz": A.nnz, "mean_row": float(lens.mean()), "max_row": int(lens.max()),
                "plan": list(M.plan)})
    # Autotuner check: SpMV kernel time under every lane split V (same G).
    import ctypes
    from paper_2510_13536_gb300 import _capi
    auto = M.plan
    sweep = {}
    for ar in ("qtw", "dw", "fp64"):
        sweep[ar] = {}
        for V in (1, 2, 4, 8, 16, 32):
            M.plan = (V, auto[1], auto[2])
            x = torch.zeros((mw.words(ar), A.n), dtype=torch.float64, device="cuda")
            kms = (ctypes.c_double * 3)()
            _capi.check(_capi.load().mwcg_profile_kernels(
                M.handle, ctypes.c_void_p(db.data_ptr()), ctypes.c_void_p(x.data_ptr()), mw.arith_id(ar), 5,
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), kms))
            sweep[ar][V] = kms[0]
    M.plan = auto
    out["spmv_ms_by_V"] = sweep
    out["auto_V"] = auto[0]
    for ar in ("fp64", "dw", "qtw"):
        r, ms = _timed(torch, lambda: mw.solve(M, db, ar, tol, maxit))
        out[ar] = {"time_s": ms / 1e3, "iters": r.iters, "status": r.status, "relres": r.relres,
                   "ms_per_iter": ms / max(r.iters, 1)}
    At, bt, tol_t, maxit_t = P.workload("c3_twin")
    Mt = mw.CSRMatrix.from_csr(At)
    dbt = torch.as_tensor(bt, device="cuda")
    for ar in ("fp64", "dw", "qtw"):
        r, ms = _timed(torch, lambda: mw.solve(Mt, dbt, ar, tol_t, maxit_t))
        x = mw.collapse(r.x).cpu().numpy()
        xs = P.random_signs(At.n, P.SEED_BASE + 3 + 200)
        out[ar + "_twin"] = {"time_s": ms / 1e3, "iters": r.iters, "status": r.status, "relres": r.relres,
                             "forward_error": float(np.linalg.norm(x - xs) / np.sqrt(At.n))}
    return out


NORM_POLICIES = [(1, "r"), (0, ""), (2, "r"), (1, "r+x"), (1, "r+p"), (1, "r+q"), (1, "r+sum"),
                 (1, "r+x+p+q+sum"), (2, "r+x+p+q+sum"), (2, "r+p"), (4, "r+p"), (8, "r+p")]


def _forward_error(x, xs):
    """||x - x*||_2 / ||x*||_2 with x multi-word: the leading word's difference
    from x* = +-1 is exact (Sterbenz) wherever it matters, the lower words add."""
    e = x[0] - xs
    for k in range(1, x.shape[0]):
        e = e + x[k]
    return float(np.linalg.norm(e) / np.linalg.norm(xs))


def run_norm(torch, mw, P, cpu):
    """Normalisation frequency and placement of the quasi arithmetics (the open
    question of Sec. VI): iterations, time and forward error per policy, on
    exact-solution systems; DW and TW (normalised by every operation) alongside."""
    out = {"policies": "(every k iterations, places): r/x after their AXPYs, p after its update, "
                       "q = A p per row, sum = the SpMV running sum after every addition"}
    from paper_2510_13536_gb300 import _capi
    for name, (tq, tt, maxit) in (("norm_poisson", (1e-26, 1e-38, 6000)),
                                  ("norm_diffusion", (1e-26, 1e-38, 40000))):
        A, b, xs = P.exact_solution_system(name)
        M = mw.CSRMatrix.from_csr(A)
        db = torch.as_tensor(b, device="cuda")
        res = {"workload": P.NORM_SYSTEMS[name], "n": A.n, "nnz": A.nnz, "plan": list(M.plan), "runs": []}
        for ar, tol in (("qdw", tq), ("qtw", tt)):
            for every, places in NORM_POLICIES:
                mask = sum(_capi.NORM[k] for k in places.split("+") if k)
                M.normalization = (every, mask)
                mw.solve(M, db, ar, tol, 2)                      # graph build, module load
                r, ms = _timed(torch, lambda: mw.solve(M, db, ar, tol, maxit, history=True))
                h = r.history.cpu().numpy() if r.iters else np.array([np.nan])
                res["runs"].append({"arith": ar, "every": every, "places": places or "none", "tol": tol,
                                    "iters": r.iters, "status": r.status, "time_s": ms / 1e3,
                                    "ms_per_iter": ms / max(r.iters, 1), "min_relres": float(np.nanmin(h)),
                                    "forward_error": _forward_error(r.x.cpu().numpy(), xs)})
        M.normalization = (1, 1)
        for ar, tol in (("dw", tq), ("tw", tt)):
            mw.solve(M, db, ar, tol, 2)
            r, ms = _timed(torch, lambda: mw.solve(M, db, ar, tol, maxit, history=True))
            h = r.history.cpu().numpy() if r.iters else np.array([np.nan])
            res["runs"].append({"arith": ar, "every": "every op", "places": "all", "tol": tol,
                                "iters": r.iters, "status": r.status, "time_s": ms / 1e3,
                                "ms_per_iter": ms / max(r.iters, 1), "min_relres": float(np.nanmin(h)),
                                "forward_error": _forward_error(r.x.cpu().numpy(), xs)})
        out[name] = res
    return out


def run_pcg(torch, mw, P, cpu):
    """Jacobi-preconditioned CG against Algorithm 1 on three workloads: the
    3-D Poisson system (constant diagonal: the preconditioner only rescales),
    the variable-coefficient diffusion system and the power-law graph
    Laplacian (degrees 5..1000: the diagonal spans three orders of magnitude);
    FP64-word (FP64, DW, QTW) and FP32-word (QQF, QF) arithmetics."""
    out = {}
    for name in ("c2", "c5", "c3"):
        A, b, tol, maxit = P.workload(name)
        tol = 1e-14
        M = mw.CSRMatrix.from_csr(A)
        db = torch.as_tensor(b, device="cuda")
        res = {"workload": name + ": " + P.WORKLOADS[name], "tol": tol, "maxit": maxit, "plan": list(M.plan)}
        for ar in ("fp64", "dw", "qtw", "qqf", "qf"):
            for pc in ("none", "jacobi"):
                M.preconditioner = pc
                mw.solve(M, db, ar, tol, 2)                  # graph build, weights
                r, ms = _timed(torch, lambda: mw.solve(M, db, ar, tol, maxit))
                res[f"{ar}_{pc}"] = {"iters": r.iters, "status": r.status, "relres": r.relres, "time_s": ms / 1e3,
                                     "ms_per_iter": ms / max(r.iters, 1)}
            M.preconditioner = "none"
        out[name] = res
    return out


def run_words(torch, mw, P, cpu):
    """The precision ladder: every arithmetic on the exact-solution Poisson
    system (128^3, x* = +-1, b = A x* exact), each to a tolerance near its
    precision; iterations, time and the forward error measured in the words."""
    A, b, xs = P.exact_solution_system("norm_poisson")
    M = mw.CSRMatrix.from_csr(A)
    db = torch.as_tensor(b, device="cuda")
    out = {"workload": P.NORM_SYSTEMS["norm_poisson"], "plan": list(M.plan), "runs": []}
    for ar, tol in (("fp64", 1e-14), ("dw", 1e-26), ("qdw", 1e-26), ("tw", 1e-38), ("qtw", 1e-38),
                    ("qw", 1e-50), ("qqw", 1e-50)):
        mw.solve(M, db, ar, tol, 2)
        r, ms = _timed(torch, lambda: mw.solve(M, db, ar, tol, 20000))
        out["runs"].append({"arith": ar, "tol": tol, "iters": r.iters, "status": r.status, "relres": r.relres,
                            "time_s": ms / 1e3, "ms_per_iter": ms / max(r.iters, 1),
                            "forward_error": _forward_error(r.x.cpu().numpy(), xs)})
    return out


def run_qqf(torch, mw, P, cpu):
    """FP32-word arithmetic (QQF) against the FP64-word ones on the 128^3
    Poisson system to 1e-14 (time, iterations, per-kernel rooflines) and on
    its exact-solution twin to 1e-24 (forward error)."""
    import ctypes
    from paper_2510_13536_gb300 import _capi
    A, b, tol, maxit = P.workload("c2")
    M = mw.CSRMatrix.from_csr(A)
    db = torch.as_tensor(b, device="cuda")
    n, nnz = A.n, A.nnz
    out = {"workload": "c2: " + P.WORKLOADS["c2"], "runs": []}
    for ar in ("fp64", "dw", "qdw", "qtw", "qqf", "qf"):
        mw.solve(M, db, ar, tol, 2)
        r, ms = _timed(torch, lambda: mw.solve(M, db, ar, tol, maxit), reps=3)
        out["runs"].append({"arith": ar, "plan": list(M.plan), "iters": r.iters, "status": r.status,
                            "relres": r.relres, "time_s": ms / 1e3, "ms_per_iter": ms / max(r.iters, 1)})
    # Per-kernel durations (CUDA events around each launch) and their rooflines.
    s = torch.cuda.current_stream()
    hbm = _measured_hbm_gbs() * 1e9
    by = {"spmv_dot": 12 * nnz + 8 * (n + 1) + 2 * 16 * n,    # CSR + p gathered once + q written
          "update_dot": 6 * 16 * n,                         # x, r read and written; p, q read
          "p_update": 3 * 16 * n}                           # r read; p read and written
    for ar in ("qqf", "qf"):
        kms = (ctypes.c_double * 3)()
        xx = torch.zeros((2, n), dtype=torch.float64, device="cuda")
        _capi.check(_capi.load().mwcg_profile_kernels(M.handle, ctypes.c_void_p(db.data_ptr()),
                                                      ctypes.c_void_p(xx.data_ptr()), mw.arith_id(ar), 30,
                                                      ctypes.c_void_p(s.cuda_stream), kms))
        ops = FP32_SPMV_OPS[ar][0] * nnz + FP32_SPMV_OPS[ar][1] * n
        kern = {}
        for k, name in enumerate(("spmv_dot", "update_dot", "p_update")):
            t = kms[k] * 1e-3
            kern[name] = {"ms": kms[k], "alg_bytes": by[name], "hbm_gbs": by[name] / t / 1e9,
                          "hbm_frac_of_measured": by[name] / t / hbm}
        kern["spmv_dot"]["fp32_ops_full_products"] = ops
        kern["spmv_dot"]["fp32_frac_of_peak_full_products"] = ops / (kms[0] * 1e-3) / FP32_PEAK_OPS
        out[ar + "_kernels"] = kern
    # The ill-conditioned power-law graph Laplacian (n = 20000, kappa ~ 5e11):
    # QQF's ~96 bits run out on its cancelling rows, QF keeps QDW-class
    # convergence.
    Ap = P.power_law_laplacian(20000, seed=7, mean_deg=12, max_deg=300)
    bp = torch.as_tensor(P.rhs_uniform(Ap.n, 32), device="cuda")
    Mp = mw.CSRMatrix.from_csr(Ap)
    pl = []
    for ar in ("fp64", "qdw", "qqf", "qf"):
        mw.solve(Mp, bp, ar, 1e-14, 2)
        r, ms = _timed(torch, lambda: mw.solve(Mp, bp, ar, 1e-14, 40000))
        pl.append({"arith": ar, "iters": r.iters, "status": r.status, "relres": r.relres, "time_s": ms / 1e3})
    out["power_law_20000"] = {"workload": "power-law graph Laplacian n = 20000 (mean degree 12, max 300, "
                                          "lognormal weights, + 1e-8 I), b = 2U-1, tol 1e-14", "runs": pl}
    # Forward error on the exact-solution twin (x* = +-1, b = A x* exact).
    Ae, be, xs = P.exact_solution_system("norm_poisson")
    Me = mw.CSRMatrix.from_csr(Ae)
    dbe = torch.as_tensor(be, device="cuda")
    fe = []
    for ar, tl in (("dw", 1e-24), ("qdw", 1e-24), ("qqf", 1e-24), ("qf", 1e-24), ("fp64", 1e-14)):
        mw.solve(Me, dbe, ar, tl, 2)
        r, ms = _timed(torch, lambda: mw.solve(Me, dbe, ar, tl, 20000))
        x = r.x.double().cpu().numpy()
        fe.append({"arith": ar, "tol": tl, "iters": r.iters, "status": r.status, "time_s": ms / 1e3,
                   "forward_error": _forward_error(x, xs)})
    out["exact_solution_twin"] = {"workload": P.NORM_SYSTEMS["norm_poisson"], "runs": fe}
    if cpu:                               # the oracle on a bounded sample of the same QQF solve
        it_q = next(r["iters"] for r in out["runs"] if r["arith"] == "qqf")
        est, per_it, _init, spent, _h = oracle_sample(A, b, "qqf", 10, it_q, M.plan)
        out["cpu_baseline"] = {"value": est, "unit": "s", "cores": 1, "kind": "oracle", "projected": True,
                               "sample": f"11 QQF CG iterations + init of the full system timed (one thread, "
                                         f"{spent:.1f} s), {per_it:.3f} s per iteration projected to {it_q} "
                                         "iterations"}
    return out


def _measured_hbm_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def run_bicg(torch, mw, P, cpu):
    """BiCGStab on nonsymmetric upwind convection-diffusion systems (512^2,
    mesh Peclet 1 and 8), FP64 to QQW and the FP32-word QQF and QF, to 1e-14."""
    out = {}
    for beta in (1.0, 8.0):
        A = P.convection_diffusion_2d(512, beta)
        b = P.rhs_uniform(A.n, P.SEED_BASE + 8)
        M = mw.CSRMatrix.from_csr(A)
        db = torch.as_tensor(b, device="cuda")
        res = {"workload": f"2-D upwind convection-diffusion 512^2 (n = {A.n}), mesh Peclet {beta:g}, b = 2U-1, "
                           "tol 1e-14, maxit 20000", "plan": list(M.plan), "runs": []}
        for ar in ("fp64", "dw", "qdw", "qtw", "qqw", "qqf", "qf"):
            mw.solve_bicgstab(M, db, ar, 1e-14, 2)
            r, ms = _timed(torch, lambda: mw.solve_bicgstab(M, db, ar, 1e-14, 20000))
            res["runs"].append({"arith": ar, "iters": r.iters, "status": r.status, "relres": r.relres,
                                "time_s": ms / 1e3, "ms_per_iter": ms / max(r.iters, 1)})
        out[f"peclet_{beta:g}"] = res
    return out


def run_c4(torch, mw, P, cpu):
    specs = P.batch_specs(256, P.SEED_BASE + 4)
    systems = [P.build_batch_system(s) for s in specs]
    Ms = [mw.CSRMatrix.from_csr(A) for A, _ in systems]
    bs = [torch.as_tensor(b, device="cuda") for _, b in systems]
    ar = [s["arith"] for s in specs]
    tol, maxit = 1e-14, 20000
    nrows = sum(A.n for A, _ in systems)
    nnz = sum(A.nnz for A, _ in systems)
    # warm-up (graph instantiation of every handle, module load)
    mw.solve_batched(Ms[:4], bs[:4], ar[:4], tol, maxit)
    for M, b, a in zip(Ms, bs, ar):
        mw.solve(M, b, a, tol, 5)
    rb, ms_b = _timed(torch, lambda: mw.solve_batched(Ms, bs, ar, tol, maxit))
    rs, ms_s = _timed(torch, lambda: [mw.solve(M, b, a, tol, maxit) for M, b, a in zip(Ms, bs, ar)])
    dev = []
    for x1, x2 in zip(rb, rs):
        a = mw.collapse(x1.x)
        c = mw.collapse(x2.x)
        dev.append(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)))
    out = {"workload": "c4: 256 Laplacians, n U[1k,200k], 2-D/3-D, shift log-U[1e-6,1e-2], QDW/QTW, tol 1e-14",
           "systems": len(systems), "rows": nrows, "nnz": nnz, "cluster": mw.batched_cluster_size(),
           "batched": {"time_s": ms_b / 1e3, "solves_per_s": len(systems) / (ms_b / 1e3),
                       "converged": sum(r.status == 0 for r in rb), "iters_total": sum(r.iters for r in rb)},
           "sequential": {"time_s": ms_s / 1e3, "solves_per_s": len(systems) / (ms_s / 1e3),
                          "converged": sum(r.status == 0 for r in rs), "iters_total": sum(r.iters for r in rs)},
           "speedup": ms_s / ms_b, "max_rel_diff_batched_vs_sequential": max(dev)}
    return out


def run_c5(torch, mw, P, cpu, n_fd=32):
    A, b, tol, maxit = P.workload("c5")
    wv = P.c5_loss_weights(A.n)
    M = mw.CSRMatrix.from_csr(A)
    db = torch.as_tensor(b, device="cuda")
    dw = torch.as_tensor(wv, device="cuda")
    vals = torch.as_tensor(A.val, device="cuda").clone().requires_grad_(True)
    bb = db.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x = mw.solve_differentiable(M, vals, bb, "qtw", tol, maxit)
    L = torch.dot(dw, x)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    g_val = vals.grad.cpu().numpy()
    g_b = bb.grad.cpu().numpy()
    # Central differences in TW, symmetric pairs.
    rng = np.random.Generator(np.random.PCG64(P.SEED_BASE + 5 + 300))
    rp, cl = A.row_ptr, A.col
    errs = []
    Mfd = mw.CSRMatrix.from_csr(A)
    Mfd.plan = M.plan
    t0 = time.perf_counter()
    samples = []
    for _ in range(n_fd):
        i = int(rng.integers(A.n))
        k = int(rng.integers(rp[i], rp[i + 1]))
        j = int(cl[k])
        kt = [kk for kk in range(int(rp[j]), int(rp[j + 1])) if int(cl[kk]) == i][0]
        h = 1e-12 * abs(A.val[k])
        xs = []
        for sgn in (1, -1):
            v = A.val.copy()
            v[k] += sgn * h
            if kt != k:
                v[kt] += sgn * h
            Mfd.update_values(v)
            r = mw.solve(Mfd, db, "tw", 1e-28, 40000)
            xs.append(r.x.cpu().numpy())
        # L(+h) - L(-h) = sum_t w_t (x+_t - x-_t), differenced word by word (the
        # leading words agree to ~12 digits, so their difference is exact) and
        # summed with math.fsum: ~1e-16 relative accuracy on the difference.
        import math
        d = xs[0] - xs[1]
        dL = math.fsum((wv[None, :] * d).ravel().tolist())
        step = (A.val[k] + h) - A.val[k]                      # the step actually taken
        fd = dL / (2 * step)
        an = g_val[k] + (g_val[kt] if kt != k else 0.0)
        errs.append(abs(fd - an) / abs(an))
        samples.append({"i": i, "j": j, "fd": fd, "adjoint": an})
    t_fd = time.perf_counter() - t0
    out = {"workload": "c5: " + P.WORKLOADS["c5"], "n": A.n, "nnz": A.nnz, "arith": "qtw", "tol": tol,
           "forward_s": t_fwd, "backward_s": t_bwd, "backward_over_forward": t_bwd / t_fwd,
           "fd_entries": n_fd, "fd_max_rel_err": max(errs), "fd_median_rel_err": float(np.median(errs)),
           "fd_target": 1e-8, "fd_seconds": t_fd, "g_b_norm": float(np.linalg.norm(g_b)),
           "fd_samples": samples[:4]}
    return out


def qtw_over_dw_general(torch, mw, P):
    """QTW / DW time to 1e-14 on the c5 diffusion matrix, whose entries are
    not powers of two (the 128^3 Poisson entries are, and take an exact
    integer-pipe scaling path)."""
    A, b, _tol, maxit = P.workload("c5")
    M = mw.CSRMatrix.from_csr(A)
    db = torch.as_tensor(b, device="cuda")
    out = {"workload": "c5 matrix (" + P.WORKLOADS["c5"].split(",")[0] + "), b = c5's b, tol 1e-14",
           "pow2_entries_frac": float(is_pow2(A.val).mean())}
    for ar in ("dw", "qtw"):
        mw.solve(M, db, ar, 1e-14, 2)
        r, ms = _timed(torch, lambda: mw.solve(M, db, ar, 1e-14, maxit))
        out[ar] = {"time_s": ms / 1e3, "iters": r.iters, "status": r.status}
    out["ratio"] = out["qtw"]["time_s"] / out["dw"]["time_s"]
    return out


def run_workloads(args):
    """--workload c1|c3|c4|c5: the other configurations, one JSON line each."""
    import torch
    from paper_2510_13536_gb300 import build as _build
    _build.build()
    from paper_2510_13536_gb300 import problems as P
    from paper_2510_13536_gb300 import solver as mw
    for w in args.workload:
        t0 = time.perf_counter()
        if w == "c1":
            res = run_c1(torch, mw, P, not args.no_cpu)
        elif w == "c3":
            res = run_c3(torch, mw, P, not args.no_cpu)
        elif w == "c4":
            res = run_c4(torch, mw, P, not args.no_cpu)
        elif w == "c5":
            res = run_c5(torch, mw, P, not args.no_cpu, args.fd)
        elif w == "norm":
            res = run_norm(torch, mw, P, not args.no_cpu)
        elif w == "pcg":
            res = run_pcg(torch, mw, P, not args.no_cpu)
        elif w == "words":
            res = run_words(torch, mw, P, not args.no_cpu)
        elif w == "bicg":
            res = run_bicg(torch, mw, P, not args.no_cpu)
        elif w == "qqf":
            res = run_qqf(torch, mw, P, not args.no_cpu)
        else:
            raise SystemExit(f"unknown workload {w}")
        res["wall_s"] = time.perf_counter() - t0
        print(json.dumps({w: res}), flush=True)
    return 0


REF_SAMPLE_ITERS = 20      # oracle iterations per reference-arm step


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on one host core.  Each
    step times the initialisation and REF_SAMPLE_ITERS + 1 CG iterations of the
    headline solve; `value` projects the complete solve from the measured time
    per iteration and the oracle's own iteration count for it, while
    `ms_per_step` is the time the step actually took."""
    ws, rk = _dist()
    if rk != 0:
        return 0
    import oracle
    from paper_2510_13536_gb300 import problems as P
    A, b, tol, maxit = P.workload(WORKLOAD)
    iters, src = _golden_iters("qtw")
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration count for the full solve missing "
                                                               "(tests/golden/fullsize_c2.json)"}))
        return 0
    oracle.build()
    plan = _golden_plan()
    t0 = time.perf_counter()
    oracle.cg("qtw", A, b, tol=0.0, maxit=1, plan=plan)
    t_init1 = time.perf_counter() - t0                      # init + 1 iteration, once
    k = REF_SAMPLE_ITERS
    ests, step_s = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.cg("qtw", A, b, tol=0.0, maxit=1 + k, plan=plan)
        t_run = time.perf_counter() - t0
        per_it = max(t_run - t_init1, 1e-9) / k
        if s >= args.warmup:
            ests.append(max(t_init1 - per_it, 0.0) + per_it * iters)
            step_s.append(t_run)
    v = statistics.median(ests)
    cb = {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "projected": True, "iterations_timed": k + 1,
          "sample": f"{k + 1} QTW CG iterations + init of the full 128^3 system per step, one thread, "
                    f"{statistics.median(step_s):.2f} s per step; the solve's time projected to {iters} "
                    f"iterations ({src}); the test oracle built -O3 -ffp-contract=off, not tuned"}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": 0, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.mean(step_s) * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "value_is": "projected time-to-1e-14 of the complete solve (init + iterations x measured s/iteration); "
                       "ms_per_step is the bounded sample each step actually ran",
           "config": {"workload": WORKLOAD + ": " + P.WORKLOADS[WORKLOAD], "arith": "qtw", "tol": tol},
           "cpu_baseline": cb, "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_gpu(args):
    import torch
    import torch.distributed as dist

    ws, rk = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2510_13536_gb300 import build as _build
    _build.build()
    from paper_2510_13536_gb300 import problems as P
    from paper_2510_13536_gb300 import solver as mw

    A, b_np, tol, maxit = P.workload(WORKLOAD)
    if args.maxit is not None:
        maxit = args.maxit
    M = mw.CSRMatrix.from_csr(A)
    if args.plan:
        M.plan = tuple(int(v) for v in args.plan.split(","))
    if args.kernels_only:
        import ctypes
        from paper_2510_13536_gb300 import _capi
        dev0 = torch.device("cuda", torch.cuda.current_device())
        bb = torch.as_tensor(b_np, device=dev0)
        xx = torch.zeros((WORDS[args.arith], A.n), dtype=torch.float64, device=dev0)
        kms = (ctypes.c_double * 3)()
        _capi.check(_capi.load().mwcg_profile_kernels(
            M.handle, ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(xx.data_ptr()), mw.arith_id(args.arith),
            int(args.kernels_only), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), kms))
        per_nnz, per_row = SPMV_OPS.get(args.arith, (0, 0))
        ops = per_nnz * A.nnz + per_row * A.n
        print(json.dumps({"kernels_only": int(args.kernels_only), "arith": args.arith, "plan": list(M.plan),
                          "kernel_ms": {"spmv_dot": kms[0], "update_dot": kms[1], "p_update": kms[2]},
                          "spmv_fp64_ops_per_launch": ops,
                          "spmv_frac_of_fp64_peak": ops / (kms[0] * 1e-3) / FP64_PEAK_OPS if kms[0] else None}))
        return 0
    dev = torch.device("cuda", torch.cuda.current_device())
    b = torch.as_tensor(b_np, device=dev)
    arith = args.arith
    w = WORDS[arith]
    x = torch.zeros((w, A.n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def one_solve(ar=arith, xx=None):
        xx = x if xx is None else xx
        xx.zero_()
        return mw.solve(M, b, ar, tol, maxit, x0=xx)

    for _ in range(args.warmup):
        r = one_solve()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iters = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for s in range(args.steps):
            x.zero_()
            starts[s].record(stream)
            r = mw.solve(M, b, arith, tol, maxit, x0=x)
            ends[s].record(stream)
            iters.append(r.iters)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    step_ms = [starts[s].elapsed_time(ends[s]) for s in range(args.steps)]
    ms = statistics.mean(step_ms)
    ms = max_over_ranks(ms, dev)
    clocks = clk.summary()
    it = iters[-1]
    status, relres = r.status, r.relres
    if args.only_solve:
        if rk == 0:
            print(json.dumps({"metric": METRIC, "value": ms / 1e3, "unit": "s", "ms_per_step": ms, "iters": it,
                              "status": status, "relres": relres, "steps": args.steps, "warmup": args.warmup,
                              "maxit": maxit, "plan": list(M.plan), "clocks": clocks, "only_solve": True}))
        return 0

    # DW solve of the same system (QTW / DW time ratio).
    xdw = torch.zeros((2, A.n), dtype=torch.float64, device=dev)
    one_solve("dw", xdw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dw_ms = []
    dw_it = 0
    for _ in range(2):
        xdw.zero_()
        e0.record(stream)
        rd = mw.solve(M, b, "dw", tol, maxit, x0=xdw)
        e1.record(stream)
        torch.cuda.synchronize()
        dw_ms.append(e0.elapsed_time(e1))
        dw_it = rd.iters

    # Per-kernel durations (CUDA events around each launch, no graph).
    import ctypes
    from paper_2510_13536_gb300 import _capi
    kms = (ctypes.c_double * 3)()
    x.zero_()
    _capi.check(_capi.load().mwcg_profile_kernels(M.handle, ctypes.c_void_p(b.data_ptr()),
                                                  ctypes.c_void_p(x.data_ptr()), mw.arith_id(arith), 30,
                                                  ctypes.c_void_p(stream.cuda_stream), kms))
    spmv_ms = kms[0]
    fp32 = arith in FP32_SPMV_OPS         # FP32 words: the FP32 pipe, 16 bytes per element
    elem = 16 if fp32 else 8 * w

    # FP64 / integer pipe rates measured now on this GPU (the FP64 roofline's
    # denominators: the pipe's rate depends on the instruction).
    probe = {}
    scratch = torch.empty(torch.cuda.get_device_properties(dev).multi_processor_count * 8 * 256,
                          dtype=torch.float64, device=dev)
    for kind, name in ((0, "dfma_ops_per_s"), (1, "dadd_ops_per_s"), (2, "int32_ops_per_s"),
                       (3, "dadd_as_fma_ops_per_s"), (4, "dmul_ops_per_s")):
        v = ctypes.c_double(0.0)
        _capi.check(_capi.load().mwcg_probe_peak(kind, ctypes.c_void_p(scratch.data_ptr()), scratch.numel() * 8,
                                                 ctypes.c_void_p(stream.cuda_stream), ctypes.byref(v)))
        probe[name] = v.value
    roofline = spmv_roofline(arith, A, M.plan, spmv_ms, probe, elem)
    roofline["vector_kernels"] = vector_rooflines(arith, A.n, kms, probe, elem)

    # End to end through the C ABI with host buffers (pinned), copies included.
    bh = torch.empty(A.n, dtype=torch.float64, pin_memory=True)
    bh.copy_(torch.as_tensor(b_np))
    xh = torch.zeros((w, A.n), dtype=torch.float32 if fp32 else torch.float64, pin_memory=True)
    e2e_s = []
    for _ in range(2):
        xh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _xh, ith, rrh, sth = mw.solve_host(M, bh.numpy(), arith, tol, maxit, x0=xh.numpy())
        e2e_s.append(time.perf_counter() - t0)
    e2e = {"value": min(e2e_s), "unit": "s", "h2d_bytes_per_step": 8 * A.n + elem * A.n,
           "d2h_bytes_per_step": elem * A.n + 160}

    # CPU oracle on a bounded sample (rank 0, N = 1 only), and the two other
    # metrics of the workload family: batched vs one-by-one solves/s (c4) and
    # the gradient against TW finite differences (c5), outside the timed region.
    cpu = batched = grad = None
    if rk == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(torch, mw, M, A, b_np, b, arith, tol, it)
    if rk == 0 and ws == 1 and not args.no_extras:
        batched = run_c4(torch, mw, P, False)
        grad = run_c5(torch, mw, P, False, args.fd_bench)
        grad["qtw_over_dw"] = qtw_over_dw_general(torch, mw, P)

    # The automatic plan each arithmetic of this line ran with, and the SpMV
    # timings (ms per lane count V) the autotuner measured to choose it.
    autotune = {}
    for ar in dict.fromkeys((arith, "dw")):
        pl, tm = M.tuning(ar)
        autotune[ar] = {"plan": list(pl), "spmv_ms_by_V": {str(v): t for v, t in tm.items()}}

    alg_bytes_iter = 12 * A.nnz + 8 * (A.n + 1) + 11 * elem * A.n
    out = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + ": " + P.WORKLOADS[WORKLOAD], "arith": arith, "tol": tol,
                   "maxit": maxit, "plan": list(M.plan), "parallelism": "replicas only" if ws > 1 else "1 GPU",
                   "l2": "working set (CSR 192 MB + 4 vectors of 50 MB) larger than the 129 MB L2"},
        "iters": it, "status": status, "relres": relres, "iters_per_s": it / (ms / 1e3),
        "hbm_gbs_algorithmic": alg_bytes_iter * it / (ms / 1e3) / 1e9,
        "dw": {"time_s": min(dw_ms) / 1e3, "iters": dw_it},
        "qtw_over_dw_time": (ms / min(dw_ms)) if arith == "qtw" else None,
        "kernel_ms": {"spmv_dot": kms[0], "update_dot": kms[1], "p_update": kms[2]},
        "autotune": autotune,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": args.steps * (3 + 3 * it),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "batched": batched,
        "grad_fd": grad,
    }
    if rk == 0:
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mwcg", choices=["mwcg", "reference"])
    ap.add_argument("--arith", default="qtw", choices=["qtw", "dw", "qdw", "tw", "fp64", "qdw_nn", "qtw_nn", "qw", "qqw", "qf",
                                                       "qqw_nn", "qqf"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--only-solve", action="store_true",
                    help="time the solves only (no DW, profile, e2e or CPU legs); used for ncu captures")
    ap.add_argument("--maxit", type=int, default=None, help="override the iteration limit (ncu captures)")
    ap.add_argument("--kernels-only", type=int, default=0, metavar="N",
                    help="run N iterations with each kernel launched on its own (mwcg_profile_kernels) and print "
                         "their mean durations; used for ncu captures")
    ap.add_argument("--workload", nargs="+", default=None, choices=["c1", "c3", "c4", "c5", "norm", "pcg", "words", "bicg",
                                                                         "qqf"],
                    help="measure another configuration instead of the headline (one JSON line each)")
    ap.add_argument("--fd", type=int, default=32, help="finite-difference entries checked in --workload c5")
    ap.add_argument("--fd-bench", type=int, default=4,
                    help="finite-difference entries checked in the default line's grad_fd object")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (c4) and gradient (c5) objects of the default line")
    ap.add_argument("--plan", default=None, help="override the summation plan V,T,G (ncu / tuning runs)")
    args = ap.parse_args()
    if args.workload:
        return run_workloads(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
