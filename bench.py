#!/usr/bin/env python3
"""Benchmark of the sparse hot path on one node; prints ONE JSON line.

Step = one SpMV y = A x in every format (CSR, ELL, COO, hybrid) and value
type (FP64, FP32 values+vectors) on the three synthetic matrices of the SpMV
sweep: 3D 27-point stencil 128^3 (n = 2,097,152, nnz = 55,742,968), the
power-law matrix n = 10^6 (Zipf(2) row lengths clipped to [1, 10^4]) and the
banded matrix n = 10^6 (half-bandwidth 64, fill 0.3).  ELL on the power-law
matrix is rejected by the padding limit and is not part of the step.
SELL-P (slices of 64 rows) is timed the same way after the step and reported
under `extra_formats`, outside `value` (the sweep's formats are CSR, ELL, COO
and hybrid); on the power-law matrix it is rejected by the padding limit too.
CSR and COO plan parameters are chosen by the library's plan autotuner
(gko_matrix_tune, kernel kept) at setup, untimed; the plans are listed in
config.tuned_plans.
value = algorithmic bytes of all SpMVs / their summed device time (GB/s);
L2 is flushed (256 MB write) before every SpMV.  Matrices stay resident in
HBM; `e2e` repeats the step through the same C ABI calls with x copied in
from pinned host memory and y copied back inside the timed region.

--impl reference times the CPU oracle (plain C, FP64, OpenMP over rows) on
a bounded sample of the same workload on the host cores.
Multi-GPU (torchrun): every rank runs an independent replica (the SpMV
sweep has no exchange step); value is the sum over ranks of bytes divided by
the slowest rank's time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GB/s (% HBM peak) per format; solves/s + p99 latency at 1e-8 residual, mixed vs FP64"
WORKLOAD = ("SpMV format sweep: CSR/ELL/COO/hybrid x FP64/FP32 (int32 indices) on 27-pt stencil 128^3, "
            "power-law n=1e6 (Zipf s=2, clip [1,1e4], seed 0), banded n=1e6 (hb 64, fill 0.3, seed 0)")
FALLBACK_HBM_GBS = 6800.0
SWEEP_FORMATS = ("csr", "ell", "coo", "hybrid")
EXTRA_FORMATS = ("sellp",)  # timed the same way, reported beside the sweep, not part of `value`


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def workload_matrices(small=False):
    from paper_2006_14290_gb300 import inputs as I

    st = ("stencil27_96", I.stencil3d_27pt(96)) if small else ("stencil27_128", I.stencil3d_27pt(128))
    return [st, ("powerlaw_1m", I.powerlaw(1_000_000, seed=0)), ("banded_1m", I.banded(1_000_000, 64, 0.3, seed=0))]


def spmv_bytes(fmt, n_rows, n_cols, nnz, ell_nnz, tail_nnz, sv, sx, sy):
    """Algorithmic bytes of one y = A x (beta = 0): values + indices once,
    x once, y written once; padding, x re-reads and misses excluded."""
    if fmt == "csr":
        return nnz * (sv + 4) + 4 * (n_rows + 1) + sx * n_cols + sy * n_rows
    if fmt in ("ell", "sellp"):
        return nnz * (sv + 4) + sx * n_cols + sy * n_rows
    if fmt == "coo":
        return nnz * (sv + 8) + sx * n_cols + sy * n_rows
    return ell_nnz * (sv + 4) + tail_nnz * (sv + 8) + sx * n_cols + sy * n_rows


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if local_rank < len(ids) and ids[local_rank].strip().isdigit():
        return int(ids[local_rank])
    return local_rank


# Sources that define the SpMV kernels, their launch plans and the matrix
# layouts: the DRAM traffic recorded in profiles/traffic.json holds while
# these are unchanged (solver-only changes do not void it).
SPMV_SOURCES = ("common.cuh", "tma.cuh", "reduce.cuh", "spmv.cuh", "spmv_kernels.cuh", "spmv.cu",
                "spmv_f64.cu", "spmv_f32.cu", "spmv_bf16.cu", "matrix.cu")


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2006_14290_gb300", "csrc")
    for f in SPMV_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def traffic_record():
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != source_hash():
        return None
    return d


# ----------------------------------------------------------------- solvers --

def solver_suite(G, dev, stream):
    """Krylov solves to 1e-8 relative residual, FP64 vs mixed precision:
    CG on the 7-point Poisson problem 256^3 (b = A*1) and BiCGSTAB / GMRES(30)
    on 7-point upwind convection-diffusion 128^3 (cell Peclet 10, b = A*1);
    plus 1,000 CG iterations of fixed work (the paper's CG experiment)."""
    import torch
    from paper_2006_14290_gb300 import inputs as I

    out = {}

    def run(tag, solver, M, bd, n, nnz, prec, maxit=20000, tol=1e-8, restart=30, pc=0):
        fn = {"cg": G.gko_solve_cg, "bicgstab": G.gko_solve_bicgstab, "gmres": G.gko_solve_gmres}[solver]
        if solver == "bicgstab":
            maxit = 2000
        # the library's refinement defaults (GMRES: one restart cycle per step)
        opts = G.opts(precision=prec, restart=restart, preconditioner=pc)
        if tag == "bicgstab_convdiff128_mixed_f32":  # known not to converge: keep it short
            opts = G.opts(precision=prec, inner_maxit=500, max_outer=3)
        xd = torch.zeros(n, dtype=torch.float64, device=dev)
        fn(M, bd, xd, tol, maxit, opts, stream=stream)  # warm-up (also builds the low-precision copy)
        xd.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        res = fn(M, bd, xd, tol, maxit, opts, stream=stream)
        wall = time.perf_counter() - t0
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        sv = 8 if prec == G.PRECISION_F64 else (4 if prec == G.PRECISION_MIXED_F32 else 2)
        vb = 8 if prec == G.PRECISION_F64 else 4
        per_vec_passes = {"cg": 10, "bicgstab": 16, "gmres": 2 * 30 + 6}[solver] + (2 if pc else 0)
        spmvs = {"cg": 1, "bicgstab": 2, "gmres": 1}[solver]
        it_bytes = spmvs * (nnz * (sv + 4) + 4 * (n + 1) + 2 * vb * n) + per_vec_passes * vb * n
        out[tag] = {"status": int(res.status), "iterations": int(res.iterations),
                    "outer_iterations": int(res.outer_iterations), "rel_residual": float(res.rel_residual),
                    "time_ms": round(ms, 3), "wall_ms": round(wall * 1e3, 3), "solves_per_s": round(1e3 / ms, 3),
                    "GB_s_per_iteration": round(it_bytes * max(res.iterations, 1) / (ms * 1e-3) / 1e9, 1)}
        return ms

    def speedup(base, other):
        """Time ratio of two runs, only when both converged (a ratio against
        a breakdown or a stalled run says nothing)."""
        if out[base]["status"] != G.OK or out[other]["status"] != G.OK:
            return None
        return round(out[base]["time_ms"] / out[other]["time_ms"], 3)

    A = I.stencil3d_7pt(256)
    M = G.from_csr(A)
    n, nnz = A.n_rows, A.nnz
    del A
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    bd = torch.zeros_like(ones)
    G.gko_spmv(1.0, M, ones, 0.0, bd, stream=stream)
    run("cg_poisson256_f64", "cg", M, bd, n, nnz, G.PRECISION_F64)
    run("cg_poisson256_mixed_f32", "cg", M, bd, n, nnz, G.PRECISION_MIXED_F32)
    run("cg_poisson256_mixed_bf16", "cg", M, bd, n, nnz, G.PRECISION_MIXED_BF16)
    out["cg_poisson256_mixed_f32_speedup"] = speedup("cg_poisson256_f64", "cg_poisson256_mixed_f32")
    # fixed work: 1,000 iterations (tolerance 0 never stops early)
    xd = torch.zeros(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = G.gko_solve_cg(M, bd, xd, 0.0, 1000, G.opts(check_every=1000), stream=stream)
    dt = time.perf_counter() - t0
    out["cg_poisson256_1000_iterations"] = {"iterations": int(res.iterations), "time_ms": round(dt * 1e3, 3),
                                            "iterations_per_s": round(res.iterations / dt, 1)}
    del M, ones, bd, xd
    A = I.convdiff3d_7pt(128, 10.0)
    M = G.from_csr(A)
    n, nnz = A.n_rows, A.nnz
    del A
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    bd = torch.zeros_like(ones)
    G.gko_spmv(1.0, M, ones, 0.0, bd, stream=stream)
    for solver in ("bicgstab", "gmres"):
        tag = "bicgstab" if solver == "bicgstab" else "gmres30"
        run(f"{tag}_convdiff128_f64", solver, M, bd, n, nnz, G.PRECISION_F64)
        run(f"{tag}_convdiff128_mixed_f32", solver, M, bd, n, nnz, G.PRECISION_MIXED_F32)
        out[f"{tag}_convdiff128_mixed_f32_speedup"] = speedup(f"{tag}_convdiff128_f64", f"{tag}_convdiff128_mixed_f32")
    del M, ones, bd
    # unpreconditioned BiCGSTAB does not converge at cell Peclet 10 on 128^3
    # (the oracle diverges too); Peclet 1 is the converging companion case
    A = I.convdiff3d_7pt(128, 1.0)
    M = G.from_csr(A)
    del A
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    bd = torch.zeros_like(ones)
    G.gko_spmv(1.0, M, ones, 0.0, bd, stream=stream)
    run("bicgstab_convdiff128_P1_f64", "bicgstab", M, bd, n, nnz, G.PRECISION_F64)
    run("bicgstab_convdiff128_P1_mixed_f32", "bicgstab", M, bd, n, nnz, G.PRECISION_MIXED_F32)
    out["bicgstab_convdiff128_P1_mixed_f32_speedup"] = speedup("bicgstab_convdiff128_P1_f64",
                                                               "bicgstab_convdiff128_P1_mixed_f32")
    del M, ones, bd
    # Jacobi preconditioning on the variable-coefficient Poisson problem 128^3
    # (coefficients exp(N(0,1)) per cell, default_rng(0); b = A*1)
    A = I.varcoef3d_7pt(128, np.random.default_rng(0))
    M = G.from_csr(A)
    n, nnz = A.n_rows, A.nnz
    del A
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    bd = torch.zeros_like(ones)
    G.gko_spmv(1.0, M, ones, 0.0, bd, stream=stream)
    run("cg_varcoef128_f64", "cg", M, bd, n, nnz, G.PRECISION_F64)
    run("cg_varcoef128_jacobi_f64", "cg", M, bd, n, nnz, G.PRECISION_F64, pc=G.PRECOND_JACOBI)
    run("cg_varcoef128_jacobi_mixed_f32", "cg", M, bd, n, nnz, G.PRECISION_MIXED_F32, pc=G.PRECOND_JACOBI)
    out["cg_varcoef128_jacobi_speedup"] = speedup("cg_varcoef128_f64", "cg_varcoef128_jacobi_f64")
    out["cg_varcoef128_jacobi_mixed_f32_speedup"] = speedup("cg_varcoef128_f64", "cg_varcoef128_jacobi_mixed_f32")
    del M, ones, bd
    out["batched_cg"] = batched_suite(G, dev, stream)
    return out


def batched_suite(G, dev, stream):
    """4096 variable-coefficient 2D 5-point systems (sides log-uniform in
    [8, 64]) solved by batched CG to 1e-10 in one persistent graph-captured
    launch; FP64 and FP32 storage; warp/block threshold from the autotuner."""
    import torch
    from paper_2006_14290_gb300 import inputs as I

    sides = I.batch_sides(4096)
    systems, bs = [], []
    for i, sd in enumerate(sides):
        A, b = I.batch_system(i, int(sd))
        systems.append(A)
        bs.append(b)
    b = torch.from_numpy(np.concatenate(bs)).to(dev)
    res = {"systems": 4096, "rows": int(sum(S.n_rows for S in systems)), "nnz": int(sum(S.nnz for S in systems))}
    for storage, tag in ((G.F64, "f64"), (G.F32, "f32_storage")):
        B = G.Batch(systems, storage=storage)
        x0 = torch.zeros(B.total_rows, dtype=torch.float64, device=dev)
        chosen, tune_ms = B.tune(b, x0, 1e-10, 20000, stream=stream)
        x = torch.zeros_like(x0)
        B.cg(b, x, 1e-10, 20000, stream=stream)  # capture the graph
        times = []
        for _ in range(3):
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            code, it, rr, st = B.cg(b, x, 1e-10, 20000, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        res[tag] = {"status": int(code), "time_ms": round(ms, 3), "systems_per_s": round(4096 / (ms * 1e-3), 1),
                    "warp_rows_threshold": int(chosen), "tuned_ms": round(float(tune_ms), 3),
                    "iterations_total": int(it.sum()), "iterations_max": int(it.max()),
                    "max_rel_residual": float(rr.max())}
        del B
    return res


# ----------------------------------------------------------------- serving --

def serving_suite(G, windows=((2000.0, 0.25), (100.0, 1.0)), slots=8, budget_bytes=150 << 30):
    """Poisson arrivals of sparse solves against resident matrices.

    Pool: 8 variable-coefficient 7-point Poisson matrices (CG) and 8 upwind
    convection-diffusion matrices with cell Peclet ~ U[1, 20] (BiCGSTAB), cube
    sides rint(n^(1/3)) for n log-uniform in [1e3, 4e6], all from
    default_rng(0), uploaded before the window.  Requests: 70% CG / 30%
    BiCGSTAB on a uniformly chosen pool matrix, b = A*1, tolerance 1e-8
    (iteration caps CG 5000, BiCGSTAB 500; CG Jacobi-preconditioned, as the
    variable coefficients call for), admitted by a 150 GB budget over
    `slots` concurrent solves.  Each arrival window runs FP64 and mixed FP32.
    """
    import torch
    from paper_2006_14290_gb300 import inputs as I

    rng = np.random.default_rng(0)
    pool = []
    for kind in ("cg", "bicgstab"):
        for _ in range(8):
            n = float(np.exp(rng.uniform(np.log(1e3), np.log(4e6))))
            side = max(4, int(np.rint(n ** (1.0 / 3.0))))
            if kind == "cg":
                A = I.varcoef3d_7pt(side, rng)
            else:
                A = I.convdiff3d_7pt(side, float(rng.uniform(1.0, 20.0)))
            M = G.from_csr(A)
            ones = torch.ones(A.n_rows, dtype=torch.float64, device="cuda")
            bd = torch.zeros_like(ones)
            G.gko_spmv(1.0, M, ones, 0.0, bd)
            pool.append((kind, M, bd.cpu().numpy(), A.n_rows))
            del A
    out = {"pool_rows": [p[3] for p in pool], "slots": slots, "budget_GB": budget_bytes / 2**30}
    for rate, window in windows:
        arr = np.random.default_rng(1)
        times, picks = [], []
        t = 0.0
        while True:
            t += arr.exponential(1.0 / rate)
            if t > window:
                break
            times.append(t)
            k = 0 if arr.random() < 0.7 else 1
            picks.append(int(arr.integers(0, 8)) + 8 * k)
        for prec_name, prec in (("f64", G.PRECISION_F64), ("mixed_f32", G.PRECISION_MIXED_F32)):
            S = G.Server(slots=slots, budget_bytes=budget_bytes)
            ids = [S.add_matrix(p[1]) for p in pool]
            opts = G.opts(precision=prec, inner_maxit=1000)
            opts_cg = G.opts(precision=prec, inner_maxit=1000, preconditioner=G.PRECOND_JACOBI)
            t0 = time.perf_counter()
            rids = []
            for at, m in zip(times, picks):
                now = time.perf_counter() - t0
                if at > now:
                    time.sleep(at - now)
                kind = pool[m][0]
                rids.append(S.submit(ids[m], 0 if kind == "cg" else 1, pool[m][2], 1e-8,
                                     5000 if kind == "cg" else 500, opts_cg if kind == "cg" else opts))
            results = [S.result(r) for r in rids]
            wall = time.perf_counter() - t0
            st = S.stats()
            S.close()
            ok = sum(1 for r in results if r[0] == G.OK)
            cg_ok = sum(1 for r, m in zip(results, picks) if r[0] == G.OK and pool[m][0] == "cg")
            out[f"rate{int(rate)}_{prec_name}"] = {
                "requests": len(rids), "window_s": window, "converged": ok,
                "cg_converged": cg_ok, "cg_requests": sum(1 for m in picks if pool[m][0] == "cg"),
                "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                "solves_per_s": round(st["solves_per_s"], 2), "drain_s": round(wall, 3),
                "peak_concurrent": st["peak_active"]}
    return out


# ------------------------------------------------ subwarp microbenchmark --

def subwarp_microbench(G, dev, stream):
    """Section 3.3 method: time of 1000 subwarp reductions = t(2000 inner
    loops) - t(1000), median of 5, for the library primitive, CUDA
    cooperative groups and the full-warp shuffle, subwarp sizes 4..32, on
    4 blocks of 256 threads per SM; ratio S=4 / S=32 against log2(4)/log2(32)."""
    import torch

    props = torch.cuda.get_device_properties(dev)
    n = 256 * 4 * props.multi_processor_count
    out = {"threads": n, "theory_ratio_4_over_32": round(2 / 5, 3)}
    for dt in (torch.float32, torch.float64):
        data = torch.zeros(n, dtype=dt, device=dev)
        for impl, iname in ((0, "library"), (1, "cooperative_groups"), (2, "legacy_shfl")):
            per = {}
            for S in (4, 8, 16, 32):
                diffs = []
                for _ in range(5):
                    t = []
                    for loops in (1000, 2000):
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        G.gko_bench_subwarp_reduce(S, impl, data, loops, stream=stream)
                        b.record(stream)
                        torch.cuda.synchronize()
                        t.append(a.elapsed_time(b))
                    diffs.append(t[1] - t[0])
                per[S] = statistics.median(diffs) * 1e3  # us per 1000 reductions
            out[f"{'f32' if dt == torch.float32 else 'f64'}/{iname}"] = {
                "us_per_1000": {str(k): round(v, 2) for k, v in per.items()},
                "ratio_4_over_32": round(per[4] / per[32], 3) if per[32] > 0 else None}
    return out


# ------------------------------------------------------ cuSPARSE context --

def cusparse_context(mats, dev, stream, flush, steps, peak):
    """cuSPARSE CSR SpMV (torch.sparse CSR @ x, int32 indices) on the sweep
    matrices, timed like the sweep (L2 flushed, CUDA events): an outside
    reference point on the same GPU, not an oracle and not part of `value`."""
    import torch

    out = {}
    for name, A in mats:
        crow = torch.from_numpy(A.row_ptr.astype(np.int32)).to(dev)
        col = torch.from_numpy(A.col.astype(np.int32)).to(dev)
        for dt, tdt, sv in (("f64", torch.float64, 8), ("f32", torch.float32, 4)):
            try:
                val = torch.from_numpy(A.val).to(dev, tdt)
                M = torch.sparse_csr_tensor(crow, col, val, (A.n_rows, A.n_cols))
                x = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, A.n_cols)).to(dev, tdt)
                for _ in range(3):
                    y = M @ x
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps)]
                for k in range(steps):
                    flush.fill_(float(k))
                    ev[k][0].record(stream)
                    y = M @ x
                    ev[k][1].record(stream)
                torch.cuda.synchronize()
                ms = sum(a.elapsed_time(b) for a, b in ev) / steps
                nb = spmv_bytes("csr", A.n_rows, A.n_cols, A.nnz, 0, 0, sv, sv, sv)
                out[f"{name}/csr/{dt}"] = {"ms": round(ms, 4), "GB_s": round(nb / (ms * 1e-3) / 1e9, 1),
                                           "frac": round(nb / (ms * 1e-3) / 1e9 / peak, 4)}
                del M, val, x, y
            except (RuntimeError, TypeError) as e:
                out[f"{name}/csr/{dt}"] = {"unavailable": str(e).splitlines()[0][:160]}
        del crow, col
    return {"library": "cuSPARSE CSR SpMV through torch.sparse_csr_tensor @ x (torch " + torch.__version__ + ")",
            "cases": out}


# --------------------------------------------------------------- reference --

def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle as O

    O.lib()
    cores = O.set_threads(os.cpu_count() or 1)
    mats = workload_matrices()
    step_bytes = 0
    for name, A in mats:
        step_bytes += spmv_bytes("csr", A.n_rows, A.n_cols, A.nnz, 0, 0, 8, 8, 8)
    xs = {name: np.random.default_rng(0).uniform(-1, 1, A.n_cols) for name, A in mats}

    def one_step():
        for name, A in mats:
            O.spmv_csr(A, xs[name])

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    gbs = step_bytes * args.steps / dt / 1e9
    sample = (f"oracle FP64 CSR SpMV on the three sweep matrices per step ({args.steps} steps after "
              f"{args.warmup} warm-up), OpenMP over rows on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "host caches (CPU run)"},
            "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(mats, budget_s=12.0):
    """The oracle as it stands on the host cores, on a bounded sample."""
    import oracle as O

    O.lib()
    cores = O.set_threads(os.cpu_count() or 1)
    xs = {name: np.random.default_rng(0).uniform(-1, 1, A.n_cols) for name, A in mats}
    nbytes = 0
    reps = 0
    t0 = time.perf_counter()
    while reps < 20 and (time.perf_counter() - t0) < budget_s:
        for name, A in mats:
            O.spmv_csr(A, xs[name])
            nbytes += spmv_bytes("csr", A.n_rows, A.n_cols, A.nnz, 0, 0, 8, 8, 8)
        reps += 1
    dt = time.perf_counter() - t0
    return {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 CSR SpMV on the three sweep matrices, {reps} passes ({dt:.1f} s), OpenMP over rows"}


# ------------------------------------------------------------ multi-rank --

def ranks_max(values, device):
    """Element-wise maximum over all ranks (the slowest rank's times); the
    identity on one rank.  Works with NCCL (CUDA tensors) and gloo (CPU)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_gbs(world, bytes_per_rank, ms):
    """Whole-job throughput: every rank processes bytes_per_rank per step
    (replicas, weak scaling); time is the slowest rank's."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------- our path --

def build_cases(G, mats, dev, formats=("csr", "ell", "coo", "hybrid"), tune=True):
    """Every (matrix, format, value type) SpMV case of the sweep, resident on
    the device, with its algorithmic bytes and the number of kernel launches
    one gko_spmv call makes for it."""
    import torch

    convs = {"ell": lambda m: G.gko_matrix_convert_to_ell(m), "coo": G.gko_matrix_convert_to_coo,
             "hybrid": lambda m: G.gko_matrix_convert_to_hybrid(m), "sellp": lambda m: G.gko_matrix_convert_to_sellp(m)}
    cases, skipped = [], []
    for name, A in mats:
        M64 = G.from_csr(A)
        base = {"csr": M64} if "csr" in formats else {}
        for fmt in formats:
            if fmt == "csr":
                continue
            try:
                base[fmt] = convs[fmt](M64)
            except G.GkoError as e:
                if e.status != G.FORMAT_UNSUITABLE:
                    raise
                skipped.append(f"{name}/{fmt}: padding over the limit")
        x64 = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, A.n_cols)).to(dev)
        x32 = x64.float()
        for fmt, M in base.items():
            inf = M.info()
            for dt in ("f64", "f32"):
                H = M if dt == "f64" else G.gko_matrix_convert_values(M, G.F32)
                sv = 8 if dt == "f64" else 4
                ell_nnz = inf["nnz"] - inf["coo_nnz"] if fmt == "hybrid" else 0
                nb = spmv_bytes(fmt, A.n_rows, A.n_cols, A.nnz, ell_nnz, inf["coo_nnz"], sv, sv, sv)
                x = x64 if dt == "f64" else x32
                y = torch.zeros(A.n_rows, dtype=x.dtype, device=dev)
                plan = None
                if tune and fmt in ("csr", "coo"):  # setup step: the plan autotuner, untimed; the kernel
                    # itself stays the histogram rule's, so profiled runs launch the same kernels
                    k, S, R, cap, _ = H.tune(x, y, reps=2, keep_kernel=True)
                    plan = {"kernel": k, "subwarp": S, "rows_per_subwarp": R, "stage_cap": cap}
                coo_launches = 2 if inf["coo_nnz"] > 0 and fmt in ("coo", "hybrid") else 0
                hp = H.plan() if fmt in ("csr", "coo") else None
                csr_launches = 2 if hp and hp["kernel"] in (2, 3) else 1 + (2 if hp and hp["n_long_rows"] > 0 else 0)
                if fmt == "coo" and hp["kernel"] == 1:
                    coo_launches = 1  # row-block COO: one launch, no tile fix-up
                launches = {"csr": csr_launches, "ell": 1, "sellp": 1,
                            "coo": coo_launches if coo_launches else 1, "hybrid": 1 + coo_launches}[fmt]
                cases.append({"label": f"{name}/{fmt}/{dt}", "M": H, "x": x, "y": y, "bytes": nb, "plan": plan,
                              "launches": launches, "nnz": int(A.nnz), "xh": x.cpu().pin_memory(),
                              "yh": torch.empty(A.n_rows, dtype=x.dtype).pin_memory()})
        del A
    return cases, skipped


def profile_cases(args):
    """One SpMV per case (after one untimed pass), for ncu: prints the cases
    in launch order with their launch counts, algorithmic bytes and nnz."""
    import torch
    from paper_2006_14290_gb300 import gko as G

    G.load()
    dev = torch.device("cuda", 0)
    cases, _ = build_cases(G, workload_matrices(small=args.small), dev, formats=SWEEP_FORMATS + EXTRA_FORMATS)
    for c in cases:
        G.gko_spmv(1.0, c["M"], c["x"], 0.0, c["y"])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("profile_cases")
    for c in cases:
        G.gko_spmv(1.0, c["M"], c["x"], 0.0, c["y"])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    G.gko_device_status()
    print(json.dumps([[c["label"], c["launches"], int(c["bytes"]), c["nnz"]] for c in cases]))

def run_ours(args):
    import torch

    rank, world, local_rank = env_rank()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    from paper_2006_14290_gb300 import gko as G

    G.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    mats = workload_matrices()

    cases, skipped = build_cases(G, mats, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(events=None):
        for i, c in enumerate(cases):
            flush.fill_(float(i))
            if events is not None:
                events[i][0].record(stream)
            G.gko_spmv(1.0, c["M"], c["x"], 0.0, c["y"], stream=stream)
            if events is not None:
                events[i][1].record(stream)

    # end to end: every SpMV through the host-buffer C ABI call (x copied in
    # from pinned host memory, y copied back), cases rotating over eight
    # streams so copies overlap other cases' SpMVs (2 / 3 / 4 / 8 streams,
    # wall clock: 2.86 / 3.72 / 3.80 / 3.98 TB/s).  No L2 flush here: a case's matrix was
    # last touched 21 SpMVs (gigabytes) earlier and x arrives by copy anyway.
    E2E_STREAMS = 8
    e2e_streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(E2E_STREAMS - 1)]

    def e2e_step():
        for i, c in enumerate(cases):
            G.gko_spmv_host(1.0, c["M"], c["xh"], 0.0, c["yh"], c["x"], c["y"],
                            stream=e2e_streams[i % E2E_STREAMS])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    sampler = ClockSampler(gpu_index(local_rank))
    sampler.start()
    time.sleep(0.3)
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in cases]
          for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.nvtx.range_push("timed_steps")
    t_start.record(stream)
    for k in range(args.steps):
        step(ev[k])
    t_end.record(stream)
    barrier()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    per_case_ms = [sum(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps)) / args.steps
                   for i in range(len(cases))]
    kernel_ms = sum(per_case_ms)
    wall_ms = t_start.elapsed_time(t_end) / args.steps
    step_bytes = sum(c["bytes"] for c in cases)

    # end to end: host x in, host y out, through the same C ABI call
    for _ in range(max(args.warmup, 3)):
        e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in e2e_streams[1:]:
        st.wait_event(e0)
    for _ in range(args.steps):
        e2e_step()
    for st in e2e_streams[1:]:
        stream.wait_stream(st)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    kernel_ms, e2e_ms = ranks_max([kernel_ms, e2e_ms], dev)

    # formats beyond the sweep (SELL-P): same protocol, own timing loop
    extra, extra_skipped = build_cases(G, mats, dev, formats=EXTRA_FORMATS)
    for _ in range(max(args.warmup, 3)):
        for c in extra:
            G.gko_spmv(1.0, c["M"], c["x"], 0.0, c["y"], stream=stream)
    xev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in extra]
           for _ in range(args.steps)]
    for k in range(args.steps):
        for i, c in enumerate(extra):
            flush.fill_(float(i))
            xev[k][i][0].record(stream)
            G.gko_spmv(1.0, c["M"], c["x"], 0.0, c["y"], stream=stream)
            xev[k][i][1].record(stream)
    torch.cuda.synchronize()
    extra_ms = [sum(xev[k][i][0].elapsed_time(xev[k][i][1]) for k in range(args.steps)) / args.steps
                for i in range(len(extra))]

    peak, peak_kind = measured_peaks()
    dom = int(np.argmax(per_case_ms))
    dom_case = cases[dom]
    achieved = dom_case["bytes"] / (per_case_ms[dom] * 1e-3) / 1e9
    traffic = None
    tr = traffic_record()
    if tr and dom_case["label"] in tr.get("per_case_bytes", {}):
        traffic = tr["per_case_bytes"][dom_case["label"]]
    value = whole_job_gbs(world, step_bytes, kernel_ms)
    if rank == 0:
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(kernel_ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed before every SpMV (256 MB write, excluded from time)",
                       "matrices": {n: {"n": int(A.n_rows), "nnz": int(A.nnz)} for n, A in mats},
                       "skipped": skipped, "frac_of_peak_value": round(value / world / peak, 4),
                       "tuned_plans": {c["label"]: c["plan"] for c in cases if c["plan"]},
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": dom_case["label"], "achieved": round(achieved, 1),
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "algorithmic_bytes": int(dom_case["bytes"])},
            "per_case": {c["label"]: {"ms": round(per_case_ms[i], 4),
                                      "GB_s": round(c["bytes"] / (per_case_ms[i] * 1e-3) / 1e9, 1),
                                      "frac": round(c["bytes"] / (per_case_ms[i] * 1e-3) / 1e9 / peak, 4)}
                         for i, c in enumerate(cases)},
            "e2e": {"value": round(whole_job_gbs(world, step_bytes, e2e_ms), 2), "unit": "GB/s",
                    "h2d_bytes_per_step": int(sum(c["x"].numel() * c["x"].element_size() for c in cases)),
                    "d2h_bytes_per_step": int(sum(c["y"].numel() * c["y"].element_size() for c in cases))},
            "extra_formats": {c["label"]: {"ms": round(extra_ms[i], 4),
                                           "GB_s": round(c["bytes"] / (extra_ms[i] * 1e-3) / 1e9, 1),
                                           "frac": round(c["bytes"] / (extra_ms[i] * 1e-3) / 1e9 / peak, 4)}
                              for i, c in enumerate(extra)},
            "extra_skipped": extra_skipped,
            "wall_ms_per_step_incl_flush": round(wall_ms, 4),
            "clocks": clocks,
            "gpu_launches": int(sum(c["launches"] for c in cases) * args.steps),
        }
        if not args.no_context:
            result["cusparse_context"] = cusparse_context(mats, dev, stream, flush, min(args.steps, 10), peak)
            result["subwarp_reduce"] = subwarp_microbench(G, dev, stream)
        if not args.no_solvers:
            result["solvers"] = solver_suite(G, dev, stream)
        if not args.no_serving:
            result["serving"] = serving_suite(G)
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(mats)
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solvers", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-context", action="store_true", help="skip the cuSPARSE context leg")
    ap.add_argument("--profile-cases", action="store_true",
                    help="run each SpMV case once (for ncu) and print the case order")
    ap.add_argument("--small", action="store_true", help="with --profile-cases: 27-point stencil at 96^3")
    args = ap.parse_args()
    if args.profile_cases:
        profile_cases(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
