#!/usr/bin/env python
"""LMA fit+predict throughput on one GB300 (or N GPUs under torchrun).

One step = the whole hot path on one batch of synthetic input, through one
C-ABI call (lma_fit_predict, mixed form): SE-ARD covariances, the support-set
projection, residual windows, blanket-first factorisations and solves, local
summaries reduced into the global summary, the FP64 global step and the
local-route prediction of every test point.

Workload (default): C4, the largest configuration that fits one GPU —
N = 2,000,000 inputs in [0,1]^8, |S| = 2,048, 2,000 Morton-ordered blocks of
1,000, Markov order B = 1, 100,000 test points (the EMSLP scale of the
paper's Table 3, synthetic).  `--config C1..C5` selects another.

Metric: training points per second of fit+predict, next to
  * TFLOP/s of the algorithmic flop count and the roofline of the dominant
    kernel (timed in a separate pass, so that no profiler event sits in the
    headline's timed region);
  * e2e: the same call with pinned host buffers (copies inside);
  * the plain FP64 GPU form (per-window launches), timed on the first blocks
    and extrapolated linearly in the block count (the fit is a sum of
    independent per-block terms, Definition 2);
  * the errors of the mixed form against the FP64 oracle's stored values
    (tests/golden, written by tests/golden/make_golden.py from oracle/ only);
  * the gradient of the log-likelihood (lma_loglik_grad) on C5;
  * the FP64 CPU oracle timed on the host cores on the first blocks.
`--impl reference` times that oracle alone (the reference arm).
`--mode step` runs only the warm-up and the timed steps (for profilers).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LMA fit+predict train-points/s"
DTYPE = "mixed: f32 factorisations with 3xTF32 tensor-core products, f64 support-set and global steps"
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
GOLDEN = {("C2", 1): "c2_b1", ("C2", 2): "c2_b2", ("C3", 2): "c3", ("C4", 1): "c4", ("C5", 2): "c5"}
PARTITION = {"C1": "sorted by x1", "C2": "k-means order", "C3": "k-means clusters, uneven",
             "C4": "Morton order", "C5": "Morton order"}


# ----------------------------------------------------------------------------
# algorithmic counts (flop = 2 per multiply-add; triangles count half)
def window_sizes(bptr, B):
    """(n_m, b_m, |D^B_m|) of every window D_m u D^B_m."""
    M = len(bptr) - 1
    out = []
    for m in range(M):
        last = min(m + B, M - 1)
        out.append((int(bptr[last + 1] - bptr[m]), int(bptr[m + 1] - bptr[m]), int(bptr[last + 1] - bptr[m + 1])))
    return out


def fit_flops(p, B):
    """N s^2 (V) + sum_m [s n^2 (R) + n^3/3 (Cholesky) + n^2 (s+1) (solve) + b s^2 (summary)]
    + 2 s^3/3 (the Cholesky factorisations of Sigma_SS and I + A)."""
    s, N = p.s, p.N
    f = N * s * s + 2.0 * s ** 3 / 3.0
    for n, b, nb in window_sizes(p.block_ptr, B):
        f += s * n * n + n ** 3 / 3.0 + n * n * (s + 1) + b * s * s
    return f


def grad_flops(p, B):
    """Algorithmic flops of lma_loglik_grad beyond the fit it repeats: per
    window W (n = |W|, b = |D_m|, r = 2(s+1) + b right-hand sides) the
    right-hand sides L^-1 Vt_W Lc^-T s^2 n (triangular), the backward solve
    r n^2, the matrix G = 1/2 (Phi Phi^T - ...) r n^2 (lower half), G Vt_W
    2 n^2 s; over the N points Vt-bar = ... (s^2, triangular) and
    K_DS-bar = Vt-bar L_SS^-1 (s^2) and their contraction with dK/dtheta
    (2 N s (d + 2)); L_SS-bar and the Cholesky adjoint 4 s^3 (FP64)."""
    s, N, d = p.s, p.N, p.d
    f = 2.0 * N * s * s + 2.0 * N * s * (d + 2) + 4.0 * s ** 3
    for n, b, nb in window_sizes(p.block_ptr, B):
        r = 2 * (s + 1) + b
        f += s * s * n + r * n * n + r * n * n + 2.0 * n * n * s
    return f


def predict_flops(p, B):
    """2 U s^2 (test projection and variance term) + per (test block, window)
    pair: the right-hand sides 2 n s, their solve n^2, the h accumulation 2 kept s."""
    s = p.s
    ws = window_sizes(p.block_ptr, B)
    tp = p.test_block_ptr
    f = 2.0 * p.U * s * s
    for nb in range(p.M):
        nu = int(tp[nb + 1] - tp[nb])
        if nu == 0:
            continue
        for m in range(max(0, nb - B), nb + 1):
            n, b, nbl = ws[m]
            kept = n if m == nb else b
            f += nu * (2.0 * n * s + n * n + 2.0 * kept * s)
    return f


def kernel_work(p, B, fused=True):
    """Algorithmic flops per step of the main kernels.  fused: lma_fit_predict's
    mixed form, whose windows carry the test right-hand sides as extra rows
    solved by the fit's sweep (no separate prediction sweep)."""
    s, M = p.s, p.M
    ws = window_sizes(p.block_ptr, B)
    tp = p.test_block_ptr
    nu = [int(tp[m + 1] - tp[m]) for m in range(M)]
    trows = [sum(nu[n] for n in range(m, min(m + B, M - 1) + 1)) for m in range(M)] if fused else [0] * M
    wide = mid = tri = below = 0.0
    SP, HP = 256, 128  # the 256-wide update applies [0, kb), the 128-wide one [kb, kh), the 64-wide steps [kh, k0)
    for (n, b, nb), t in zip(ws, trows):
        rows = n + s + 1 + t
        for k0 in range(0, n, 64):
            w = min(64, n - k0)
            kb, kh = (k0 // SP) * SP, (k0 // HP) * HP
            below += 2.0 * max(0, rows - k0 - w) * w * (k0 - kh)
            tri += 2.0 * max(0, rows - k0 - w) * w * w / 2.0
            if k0 == kb and kb > 0:
                c = min(SP, n - kb)
                wide += 2.0 * ((rows - kb) * c - c * (c - 1) / 2.0) * kb
            if k0 == kh and kh > kb:
                c = min(HP, n - kh)
                mid += 2.0 * ((rows - kh) * c - c * (c - 1) / 2.0) * (kh - kb)
    # the residual kernel's own tiles: the blanket's [0, L)^2 part (L = n_B rounded
    # down to 128) is copied from the windows that compute it (k_copy_shared_tiles)
    resid = sum(s * (n * n - ((nb // 128) * 128) ** 2) for n, _, nb in ws)
    gram = sum(b * (s + 1) * (s + 1) for _, b, _ in ws)
    psweep = prhs = pacc = 0.0
    for nb_ in range(M):
        for m in range(max(0, nb_ - B), nb_ + 1) if nu[nb_] else ():
            n, b, nbl = ws[m]
            psweep += nu[nb_] * n * n
            prhs += 2.0 * nu[nb_] * n * s
            pacc += 2.0 * nu[nb_] * (b if m < nb_ else n) * s
    proj = (p.N + p.U) * s * s           # V = L^-1 K_SD: s^2 / 2 multiply-adds per point (triangular)
    var = p.U * s * s                    # L_C^-1 h of every test point (triangular)
    f64 = 2.0 * s ** 3 / 3.0             # Cholesky of Sigma_SS and of I + A, s^3 / 6 multiply-adds each
    # the panel steps' update (columns [kh, k0), at most 64) of the rows below
    # the diagonal block and the panel solves run in k_chol_panel_pt
    # (k_chol_step_tc updates and factorises the diagonal block itself)
    return {"k_chol_panel_pt": below + tri, "k_chol_wide": wide,
            "k_chol_mid": mid, "k_resid_bf6": resid,
            "k_gram_bf6": gram, "k_pred_rhs_bf6": prhs, "k_pred_accum_tc": pacc, "k_proj": proj,
            "k_proj_tc": proj, "k_var_gemm": var,
            "k_f64_chain": f64, **({} if fused else {"k_pred_sweep_tc": psweep})}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel from one ncu capture, {kernel: {"bytes": B, "files": the csrc files that
# define and launch it, "sources": their hash then, "note": where}}; reported
# only while those files still hash to the value the capture was taken at.
NCU_TRAFFIC: dict = {
    # profiles/k_chol_wide_traffic_c4_n50000.md: DRAM bytes of the seven super-panel launches of the
    # C4 recipe at N = 50,000 (50 windows), averaged per launch and scaled by the window count to C4
    # (the hash is of lma_tc.cuh after two unrelated kernels were deleted from it; the super-panel
    # kernel and its pipeline are the captured code)
    "k_chol_wide": {"bytes": 47.57e9, "case": ("C4", 1), "files": ["lma_tc.cuh"], "sources": "dd86857e5a16a326",
                    "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the 7 launches of one step at "
                            "N=50,000 (1.189 GB per launch on average, 1.34x the algorithmic bytes), x40 windows"},
}


def sources_hash(files=None) -> str:
    """sha256 prefix of the given csrc/ files (default: all sources and the header)."""
    import glob
    if files:
        paths = [os.path.join(ROOT, "paper_1411_4510_gb300", "csrc", f) for f in files]
    else:
        paths = sorted(glob.glob(os.path.join(ROOT, "paper_1411_4510_gb300", "csrc", "*.cu*"))
                       + glob.glob(os.path.join(ROOT, "include", "*.h")))
    h = hashlib.sha256()
    for f in paths:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TENSOR_KERNELS = {"k_chol_panel_pt", "k_chol_wide", "k_chol_mid", "k_pred_sweep_tc",
                  "k_pred_accum_tc", "k_bwd_sweep_tc", "k_grad_G_tc",
                  "k_grad_gv_tc", "k_grad_rhs_tc"}
BF16X6_KERNELS = {"k_proj_tc", "k_gram_bf6", "k_resid_bf6", "k_pred_rhs_bf6"}   # bfloat16 x 6 split products (the variance term shares the name k_var_gemm)
FP64_KERNELS = {"k_f64_chain"}
# launches of the FP64 factorisations (whichever form the tuner chose), reported as one entry
F64_CHAIN = ("k_f64_potrf", "k_f64_panel", "k_f64_solve2", "k_f64_coop", "k_f64_flow")


def merge_f64(prof):
    """{kernel: (ms, launches)} with the FP64 factorisation launches summed into k_f64_chain."""
    if not prof:
        return prof
    out = {k: v for k, v in prof.items() if k not in F64_CHAIN}
    parts = [v for k, v in prof.items() if k in F64_CHAIN]
    if parts:
        out["k_f64_chain"] = (sum(v[0] for v in parts), sum(v[1] for v in parts))
    return out
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rate of the part
FP64_PEAK = 1.25             # nominal FP64 TFLOP/s of the part (no measured figure)


def roofline_of(name, flops, tot_ms, n_l, peaks, sustained=True, bf16_var=True):
    """Achieved algorithmic rate of one kernel over its launches against its peak."""
    achieved = flops / (tot_ms / 1e3) / 1e12
    pk = peaks or {}
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    if name in BF16X6_KERNELS or (name == "k_var_gemm" and bf16_var):
        key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        src = "measured" if key in pk else "fallback"
        peak = pk.get(key, 1700.0 if sustained else 1900.0)
        r = {"bound": "tensor",
             "peak_note": f"BF16 dense, {src} {'sustained' if sustained else 'burst'} (MEASURED_PEAKS.json), of "
                          f"{src}; the bf16x6 split issues six BF16 MMAs per algorithmic product, so frac <= 1/6",
             "tensor_pipe_frac_issued": 6.0 * achieved / peak}
    elif name in TENSOR_KERNELS:
        key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        src = "measured" if key in pk else "fallback"
        bf16 = pk.get(key, 1700.0 if sustained else 1900.0)
        peak = bf16 * TF32_PER_BF16
        r = {"bound": "tensor",
             "peak_note": f"TF32 dense = {src} bf16 {'sustained' if sustained else 'burst'} "
                          f"({bf16:.1f} TFLOP/s, MEASURED_PEAKS.json) x 1.1/2.25 (nominal TF32/BF16 ratio), "
                          f"of {src}; 3xTF32 issues three TF32 MMAs per algorithmic product, so frac <= 1/3",
             "tensor_pipe_frac_issued": 3.0 * achieved / peak}
    elif name in FP64_KERNELS:
        peak = FP64_PEAK
        r = {"bound": "alu", "peak_note": "FP64: the part's nominal 1.25 TFLOP/s (derived; a microbenchmark "
             "on the box measured 1.6 FP64 FMA/clk/SM = 1.0 TFLOP/s at 2070 MHz)"}
    else:
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        r = {"bound": "alu", "peak_note": "FP32 SIMT: 152 SM x 128 lanes x 2 flop x sm_max_mhz (derived)"}
    r.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
              "kernel": name, "launches_timed": n_l, "avg_launch_ms": tot_ms / n_l})
    return r


# ----------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.idx = gpu_index
        self.first = 0

    def __enter__(self):
        # nvidia-smi's start-up (driver attach, NVML init) slows the GPU work
        # running beside it, so the timed region starts only after the first
        # sample has arrived; samples from before that are not summarised.
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={CLOCK_Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.time() + 20.0
            while not self.lines and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
            time.sleep(0.1)
        except Exception:
            self.proc = None
        self.first = len(self.lines)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.first:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ----------------------------------------------------------------------------
def sub_problem(p, k, B=None):
    """The first k blocks of problem p (their training and test points, the
    same support set and hyperparameters); B clipped to k - 1."""
    from workloads.synth import Problem
    k = min(int(k), p.M)
    nsub = int(p.block_ptr[k])
    usub = int(p.test_block_ptr[k])
    B = p.B if B is None else B
    return Problem(name=f"{p.name}[:{k}]", X=p.X[:nsub], y=p.y[:nsub], block_ptr=p.block_ptr[:k + 1].copy(),
                   S=p.S, XU=p.XU[:usub], yU=p.yU[:usub], test_block_ptr=p.test_block_ptr[:k + 1].copy(),
                   log_ell=p.log_ell, log_sigma_s=p.log_sigma_s, log_sigma_n=p.log_sigma_n, jitter=p.jitter,
                   mean=p.mean, B=min(B, k - 1))


def cpu_baseline(p, B, n_blocks):
    """FP64 oracle (as it stands) on the first n_blocks blocks of the workload:
    fit + local-route prediction of their test points, on the host cores."""
    from oracle import lma_oracle as O2
    sub = sub_problem(p, n_blocks, B)
    t0 = time.perf_counter()
    f = O2.fit(sub)
    O2.predict(f)
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v):
            cores = int(os.environ[v])
    return dict(value=sub.N / dt, unit="train-points/s", cores=cores, kind="oracle",
                sample=f"first {sub.M} of {p.M} blocks ({sub.N} training points, {sub.U} test points), "
                       f"same |S|={p.s}, B={sub.B}; fit+predict in {dt:.1f} s (one sample per step)"), dt


def workload_config(p, B, world=1, reduced=False):
    tag = p.name if not reduced else f"{p.name} (reduced)"
    c = {"workload": f"{tag}: N={p.N} d={p.d} |S|={p.s} M={p.M} blocks "
                     f"({PARTITION.get(p.name, '')}, sizes {int(p.block_sizes().min())}-{int(p.block_sizes().max())}) "
                     f"B={B} U={p.U} (RFF SE draw, synthetic)",
         "N": p.N, "d": p.d, "s": p.s, "M": p.M, "B": B, "U": p.U,
         "l2": "flushed between timed steps (256 MiB write outside the step events); inputs and "
               "intermediates are larger than L2"}
    if world > 1:
        c["workload"] = (f"{world} draws of {p.name} joined, one draw per rank (N={p.N} per draw, M={p.M}, |S|={p.s}, "
                         f"B={B}, U={p.U}); rank r owns draw r's blocks plus B-block halos; local summaries, one "
                         f"all-reduce of the (|S|+1)^2 FP64 summary Gram, global step on every rank")
        c["parallelism"] = f"block-sharded x{world}"
    return c


def golden(p, B):
    """The oracle's stored values for this workload, if its inputs' fingerprints match."""
    name = GOLDEN.get((p.name, B))
    path = os.path.join(ROOT, "tests", "golden", f"{name}.json") if name else None
    if not path or not os.path.exists(path):
        return None
    g = json.load(open(path))
    fp = g["fingerprints"]
    sha = lambda a: hashlib.sha256(a.tobytes()).hexdigest()[:32]  # noqa: E731
    ok = (fp["X_sha"] == sha(p.X) and fp["block_ptr_sha"] == sha(p.block_ptr.astype("int64"))
          and fp["test_block_ptr_sha"] == sha(p.test_block_ptr.astype("int64"))
          and abs(fp["y_fsum"] - math.fsum(p.y)) <= 1e-10 * max(1.0, abs(fp["y_fsum"])))
    return g if ok else None


def accuracy(g, mean, var, loglik, yU):
    """Errors of the mixed form's outputs against the oracle's stored values."""
    import numpy as np
    rows = np.asarray(g["sample_rows"], dtype=np.int64)
    mo, vo = np.asarray(g["mean"]), np.asarray(g["var"])
    m, v = np.asarray(mean)[rows], np.asarray(var)[rows]
    out = {"reference": "FP64 oracle (tests/golden, written from oracle/)",
           "sample": f"test blocks {g['sampled_blocks']} ({rows.size} points)",
           "mean_rel_err": float(np.linalg.norm(m - mo) / np.linalg.norm(mo)),
           "mean_max_abs_err": float(np.max(np.abs(m - mo))),
           "var_rel_err": float(np.linalg.norm(v - vo) / np.linalg.norm(vo)),
           "var_max_rel_err": float(np.max(np.abs(v - vo) / np.abs(vo))),
           "rmse_sample": float(np.sqrt(np.mean((m - yU[rows]) ** 2))), "rmse_sample_oracle": g["rmse_sample"]}
    if loglik is not None:
        out["loglik_rel_err"] = abs(loglik - g["fit"]["loglik"]) / abs(g["fit"]["loglik"])
    if "rmse_all" in g:
        out["rmse_all"] = float(np.sqrt(np.mean((np.asarray(mean) - yU) ** 2)))
        out["rmse_all_oracle"] = g["rmse_all"]
    return out


def run_reference(args, p):
    """Reference arm: the FP64 CPU oracle timed on the host cores, one bounded
    sample of the workload (its first --ref-blocks blocks) per step."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(p, args.B, args.ref_blocks)
    vals, last = [], None
    for _ in range(args.steps):
        cb, dt = cpu_baseline(p, args.B, args.ref_blocks)
        vals.append(dt)
        last = cb
    ms = 1e3 * statistics.mean(vals)
    nsub = int(p.block_ptr[min(args.ref_blocks, p.M)])
    value = nsub / (ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "train-points/s",
           "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(p, args.B, world),
           "cpu_baseline": dict(last, value=value),
           "e2e": {"value": value, "unit": "train-points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def build_problem(args, world, rank):
    """The configured workload (N = 1), or for N > 1 the joined draws this rank
    needs: its own draw and its neighbours' (halo blocks)."""
    from workloads import make_problem, make_replicated
    kw = {k: getattr(args, k) for k in ("N", "M", "s", "U") if getattr(args, k) is not None}
    if world == 1:
        return make_problem(args.config, B=args.B, **kw), 0
    lo, hi = max(0, rank - 1), min(world - 1, rank + 1)
    return make_replicated(args.config, hi - lo + 1, B=args.B, first_draw=lo, **kw), rank - lo


def grad_only(args, p, full, dev, L):
    """--mode grad: lma_loglik_grad on the configured workload (inputs resident),
    args.warmup untimed and args.steps timed calls (host clock: the call
    synchronises and returns host values), one JSON line."""
    import torch
    prec = L.FP64 if args.precision == "fp64" else L.MIXED
    d = {k: torch.as_tensor(full[k], device=dev) for k in ("X", "y", "S")}
    kw = {k: v for k, v in full.items() if k not in ("X", "y", "S")}
    for _ in range(args.warmup):
        L.lma_loglik_grad(d["X"], d["y"], S=d["S"], precision=prec, **kw)
    torch.cuda.synchronize()
    n0 = L.lma_kernel_launch_count()
    tms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        L.lma_loglik_grad(d["X"], d["y"], S=d["S"], precision=prec, **kw)
        tms.append(1e3 * (time.perf_counter() - t0))
    ms = statistics.mean(tms)
    gfl = fit_flops(p, args.B if args.B is not None else p.B) + grad_flops(p, args.B if args.B is not None else p.B)
    print(json.dumps({"metric": "lma_loglik_grad train-points/s", "value": p.N / (ms / 1e3), "unit": "train-points/s",
                      "ms_per_call": ms, "steps": args.steps, "warmup": args.warmup, "tflops": gfl / (ms / 1e3) / 1e12,
                      "gpu_launches": int(L.lma_kernel_launch_count() - n0),
                      "config": workload_config(p, args.B if args.B is not None else p.B, 1,
                                                any(getattr(args, k) is not None for k in ("N", "M", "s", "U")))}))


# ----------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lma", choices=["lma", "reference"])
    ap.add_argument("--config", default="C4", choices=["C1", "C2", "C3", "C4", "C5"])
    ap.add_argument("--B", type=int, default=None, help="Markov order (default: the configuration's)")
    ap.add_argument("--N", type=int, default=None, help="reduced case: training points (keeps the recipe)")
    ap.add_argument("--M", type=int, default=None, help="reduced case: blocks")
    ap.add_argument("--s", type=int, default=None, help="reduced case: support points")
    ap.add_argument("--U", type=int, default=None, help="reduced case: test points")
    ap.add_argument("--mode", default="full", choices=["full", "step", "grad"],
                    help="step: warm-up and timed steps only (for profilers); grad: lma_loglik_grad on the "
                         "configured workload, warm-up and timed calls only (1 GPU)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="form of the timed steps")
    ap.add_argument("--ref-blocks", type=int, default=2,
                    help="blocks of the oracle's sample (cpu_baseline and the reference arm)")
    ap.add_argument("--fp64-blocks", default="4,8", help="block counts of the FP64 form's timed subsets")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--dominant", default="auto")
    ap.add_argument("--trace", default=None,
                    help="write the per-launch trace (kernel, start ms, end ms; CUDA events around every launch, "
                         "all streams) of the untimed profiled step to this JSON file (rank 0)")
    args = ap.parse_args()
    if args.impl == "lma":
        args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from workloads.synth import _DEFAULTS
    if args.B is None:
        args.B = _DEFAULTS[args.config]["B"]
    reduced = any(getattr(args, k) is not None for k in ("N", "M", "s", "U"))

    if args.impl == "reference":
        if rank == 0:
            from workloads import make_problem
            kw = {k: getattr(args, k) for k in ("N", "M", "s", "U") if getattr(args, k) is not None}
            run_reference(args, make_problem(args.config, B=args.B, **kw))
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1411_4510_gb300 import build
    build.build()
    import paper_1411_4510_gb300 as L
    from paper_1411_4510_gb300 import api, shard

    p, my = build_problem(args, world, rank)
    dev = torch.device("cuda", local)
    full = L.problem_args(p, B=args.B)
    if args.mode == "grad":
        grad_only(args, p, full, dev, L)
        return
    if world == 1:
        sh, sub, u0, u1, tptr = None, full, 0, p.U, p.test_block_ptr
    else:
        # the joined draws [lo, hi] of build_problem: this rank owns draw `my`
        per = p.M // (p.meta.get("copies", 1))
        sh = shard.plan_range(p.block_ptr, args.B, my * per, (my + 1) * per, rank, world)
        sub = shard.sub_problem(full, sh)
        u0, u1, tptr = shard.test_rows(p.test_block_ptr, sh)
    prec = L.FP64 if args.precision == "fp64" else L.MIXED
    hostsrc = dict(X=sub["X"], y=sub["y"], S=sub["S"], XU=p.XU[u0:u1])
    dsrc = {k: torch.as_tensor(v, device=dev) for k, v in hostsrc.items()}
    kw = {k: v for k, v in sub.items() if k not in ("X", "y", "S")}
    n_total = p.N if world == 1 else p.N // p.meta.get("copies", 1) * world
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step(pr=prec, host=None, keep=False):
        src = dsrc if host is None else host
        if sh is None:  # fit and predict in one call: the global step overlaps the prediction
            return L.lma_fit_predict(src["X"], src["y"], S=src["S"], XU=src["XU"], test_block_ptr=tptr,
                                     precision=pr, keep_model=keep, **kw)
        m = api.lma_fit_local(src["X"], src["y"], S=src["S"], win_begin=0, own_begin=sh.own_begin,
                              own_end=sh.own_end, precision=pr, **kw)
        G, ld = api.lma_model_local_summary(m, device=dev)
        G, ld = shard.allreduce_sum(G, ld)
        api.lma_model_set_global(m, G, ld, n_total)
        mean, var = L.lma_predict(m, src["XU"], tptr)
        return (mean, var, m) if keep else (mean, var)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the form the fit really ran in: a mixed fit whose FP32 window lost
    # positive definiteness is redone in FP64 by the library
    model_prec = L.lma_model_precision(step(keep=True)[2])
    torch.cuda.synchronize()

    def timed(nsteps, pr=prec, host=None, profile=None, keep_trace=False):
        """Mean CUDA-event milliseconds of nsteps steps (L2 flushed before each,
        outside its events), launches of this library, optional profile."""
        evs = []
        n0 = L.lma_kernel_launch_count()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            L.profile_start(profile)
        for _ in range(nsteps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            step(pr, host)
            b.record(st)
            evs.append((a, b))
        torch.cuda.synchronize()
        trace = L.profile_trace() if (profile and keep_trace) else None
        prof = L.profile_stop() if profile else None
        if world > 1:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, L.lma_kernel_launch_count() - n0, prof, trace

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---- headline: no profiler events in the timed region ------------------
    with ClockSampler(local) as clk:
        ms, launches, _, _ = timed(args.steps)
    clocks = clk.summary()
    step_ms = max_over_ranks(statistics.mean(ms))
    fit_f, pred_f = fit_flops(p, args.B), predict_flops(p, args.B)
    if world > 1:  # whole job: one draw per rank
        fit_f, pred_f = fit_f / p.meta.get("copies", 1) * world, pred_f / p.meta.get("copies", 1) * world
    n_units = p.N if world == 1 else n_total
    value = n_units / (step_ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "train-points/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE if model_prec == L.MIXED else "f64", "data": "synthetic",
           "config": workload_config(p if world == 1 else p, args.B, world, reduced),
           "tflops": (fit_f + pred_f) / (step_ms / 1e3) / 1e12,
           "algorithmic_gflop_per_step": {"fit": fit_f / 1e9, "predict": pred_f / 1e9},
           "gpu_launches": int(launches), "clocks": clocks,
           "ms_per_step_all": [round(x, 3) for x in ms]}
    if args.mode == "step":
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- per-kernel profile of one untimed step; dominant kernel's own pass --
    work = kernel_work(p, args.B, fused=(world == 1 and prec == L.MIXED))
    if world > 1:
        work = {k: v / p.meta.get("copies", 1) for k, v in work.items()}
    _, _, prof_all, trace = timed(1, profile="k_", keep_trace=bool(args.trace))
    prof_all = merge_f64(prof_all)
    if args.trace and rank == 0:
        with open(args.trace, "w") as fh:
            json.dump([{"kernel": k, "start_ms": a, "end_ms": b} for k, a, b in trace], fh)
    dominant = args.dominant
    if dominant == "auto":
        known = {k: v for k, v in (prof_all or {}).items() if k in work}
        dominant = max(known, key=lambda k: known[k][0]) if known else None
    peaks = load_peaks()
    roof = None
    if dominant:
        nrs = min(args.steps, 3)
        _, _, prof, _ = timed(nrs, profile="k_f64_" if dominant == "k_f64_chain" else dominant)
        prof = merge_f64(prof)
        if prof and dominant in prof:
            tot_ms, n_l = prof[dominant]
            roof = roofline_of(dominant, work[dominant] * nrs, tot_ms, n_l, peaks)
            roof["work_per_step_gflop"] = work[dominant] / 1e9
            roof["timing"] = (f"CUDA events around each of its launches over {nrs} further steps (a separate pass; "
                              f"the headline steps carry no profiler events)")
            t = NCU_TRAFFIC.get(dominant)
            if t and t["sources"] == sources_hash(t.get("files")) and world == 1 and (p.name, args.B) == t.get("case"):
                roof["traffic"] = t["bytes"]
                roof["traffic_note"] = t["note"]
    out["roofline"] = roof
    out["autotune"] = [{"key": k, "choice": c, "candidates_ms": m} for _, k, c, m in L.lma_autotune_report()]
    out["roofline_by_kernel"] = {k: {kk: vv for kk, vv in roofline_of(k, work[k], v[0], v[1], peaks).items()
                                     if kk in ("bound", "achieved", "peak", "frac", "avg_launch_ms")}
                                 for k, v in (prof_all or {}).items() if k in work and v[0] > 0}
    out["kernel_ms_one_step"] = {k: round(v[0], 4) for k, v in
                                 sorted((prof_all or {}).items(), key=lambda kv: -kv[1][0])}

    # ---- end to end through the C ABI with pinned host buffers -------------
    host = {k: torch.as_tensor(v).pin_memory() for k, v in hostsrc.items()}
    ems, _, _, _ = timed(max(3, args.steps // 2), host=host)
    e2e_ms = max_over_ranks(statistics.mean(ems))
    nsub, Msub = len(hostsrc["y"]), len(kw["block_ptr"]) - 1
    h2d = 8 * (nsub * p.d + nsub + p.s * p.d + (u1 - u0) * p.d) + 8 * (Msub + 1) * 2
    out["e2e"] = {"value": n_units / (e2e_ms / 1e3), "unit": "train-points/s", "ms_per_step": e2e_ms,
                  "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16 * (u1 - u0)}

    if world == 1:
        # ---- accuracy against the oracle's stored values -------------------
        res = step(keep=True)
        mean, var, model = res
        ll = L.lma_model_loglik(model)
        del model
        torch.cuda.synchronize()
        mean, var = mean.cpu().numpy(), var.cpu().numpy()
        g = golden(p, args.B) if not reduced else None
        out["accuracy_vs_oracle"] = accuracy(g, mean, var, ll, p.yU) if g else None

        # ---- plain FP64 GPU form, timed on the first blocks ----------------
        if not args.no_fp64 and prec == L.MIXED:
            pts = []
            for k in [int(x) for x in args.fp64_blocks.split(",")]:
                q = sub_problem(p, k, args.B)
                qa = L.problem_args(q)
                qd = {kk: torch.as_tensor(getattr(q, kk), device=dev) for kk in ("X", "y", "S", "XU")}
                qkw = {kk: v for kk, v in qa.items() if kk not in ("X", "y", "S")}

                def qstep(pr):
                    return L.lma_fit_predict(qd["X"], qd["y"], S=qd["S"], XU=qd["XU"],
                                             test_block_ptr=q.test_block_ptr, precision=pr, **qkw)
                qstep(L.FP64)
                torch.cuda.synchronize()
                tms = []
                for _ in range(2):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    m64, _ = qstep(L.FP64)
                    b.record(st)
                    torch.cuda.synchronize()
                    tms.append(a.elapsed_time(b))
                mmx, _ = qstep(L.MIXED)
                m64, mmx = m64.cpu().numpy(), mmx.cpu().numpy()
                pts.append((q.M, statistics.mean(tms), float(np.linalg.norm(mmx - m64) / np.linalg.norm(m64))))
            (k1, t1, _), (k2, t2, e2) = pts[0], pts[-1]
            slope = (t2 - t1) / max(1, k2 - k1)
            t_full = t1 + (p.M - k1) * slope
            out["fp64_gpu_form"] = {
                "value": p.N / (t_full / 1e3), "ms_per_step": t_full, "extrapolated": True,
                "timed": {f"first {k} blocks": round(t, 2) for k, t, _ in pts},
                "how": f"lma_fit_predict in the FP64 form (one window per launch) on the first {k1} and {k2} blocks "
                       f"of the workload (same |S|, B), extrapolated linearly in the block count to {p.M}",
                "tflops": (fit_f + pred_f) / (t_full / 1e3) / 1e12,
                "mixed_speedup": t_full / step_ms,
                "mixed_mean_rel_err_vs_fp64": e2, "err_sample": f"first {k2} blocks' test points"}

        # ---- gradient of the log-likelihood (C5) ---------------------------
        if not args.no_grad and not reduced:
            from workloads import make_problem
            q = make_problem("C5")
            qa = L.problem_args(q)
            qd = {kk: torch.as_tensor(qa[kk], device=dev) for kk in ("X", "y", "S")}
            qkw = {kk: v for kk, v in qa.items() if kk not in ("X", "y", "S")}
            L.lma_loglik_grad(qd["X"], qd["y"], S=qd["S"], **qkw)
            tms = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                llg, gr = L.lma_loglik_grad(qd["X"], qd["y"], S=qd["S"], **qkw)
                tms.append(1e3 * (time.perf_counter() - t0))
            gms = statistics.mean(tms)
            L.profile_start("k_")
            L.lma_loglik_grad(qd["X"], qd["y"], S=qd["S"], **qkw)
            gprof = L.profile_stop()
            gfl = fit_flops(q, q.B) + grad_flops(q, q.B)
            leg = {"workload": workload_config(q, q.B)["workload"], "ms_per_call": gms,
                   "tflops": gfl / (gms / 1e3) / 1e12, "algorithmic_gflop": gfl / 1e9,
                   "flop_note": "fit (fit_flops) + adjoint (grad_flops); the adjoint's window products (right-hand "
                                "sides, backward sweep, G, G Vt) run on the tensor cores in 3xTF32, its N x s products "
                                "on the CUDA cores in FP32 and the s x s part in FP64",
                   "kernel_ms_one_call": {k: round(v[0], 3) for k, v in sorted(gprof.items(), key=lambda kv: -kv[1][0])},
                   "train_points_per_s": q.N / (gms / 1e3), "fit_gflop": fit_flops(q, q.B) / 1e9,
                   "timing": "host wall clock around lma_loglik_grad (it synchronises and returns host values)"}
            gg = golden(q, q.B)
            if gg:
                go = np.asarray(gg["grad"])
                leg["loglik_rel_err_vs_oracle"] = abs(llg - gg["loglik"]) / abs(gg["loglik"])
                leg["grad_rel_err_vs_oracle"] = float(np.linalg.norm(gr - go) / np.linalg.norm(go))
                leg["grad_max_rel_err_vs_oracle"] = float(np.max(np.abs(gr - go) / np.maximum(np.abs(go), 1e-300)))
            out["grad_leg"] = leg

        # ---- the oracle on the host cores -----------------------------------
        if not args.no_cpu and rank == 0:
            out["cpu_baseline"], _ = cpu_baseline(p, args.B, args.ref_blocks)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
