"""Benchmark: all-eigenvector solve of a seeded synthetic Schur pencil.

One step = one pevc_solve of the whole hot path (pre-processing, tips,
diagonal solves, updates, correction if any, post-processing) on an
n x n pencil that is already resident in HBM.  The default workload is the
n = 20000 pencil (2x2 blocks on ~50 % of the diagonal, N(0,1) off-diagonal
entries) with the split-BF16 path; ``--prec fp64`` measures the FP64 path.

Metric: effective GFLOP/s = F / time with F = sum over eigenvectors of 2 c^2
~ 2 n^3 / 3 (the FP64-equivalent work of the substitution); ms per solve and
eigenvectors/s are reported beside it.  Inputs (S, T: 2 x 3.2 GB at
n = 20000) are far larger than the 129 MB L2, so no flush is needed.

Under torchrun every rank solves its own pencil on its own GPU (the solve
does not shard: replicas, weak scaling); value = total work / max time.
``--impl reference`` times the FP64 CPU oracle (test infrastructure, the
reference arm of this benchmark) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "all-eigenvector solve time & GFLOP/s at n=20000, split-BF16 vs FP64 at resid<=100nu"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def flops_all(n: int) -> float:
    c = np.arange(1, n + 1, dtype=np.float64)
    return float((2.0 * c * c).sum())


# DRAM bytes per launch at n = 20000 (dram__bytes_read.sum + dram__bytes_write.sum)
# from the ncu captures summarised in profiles/ (k_diag_n4000.md,
# k_update_tc_bf16x5.md): small cases, scaled to the n = 20000 launches by
# the units one launch processes (the diagonal kernel's CTAs; the update's
# element updates); valid only for the kernel sources they were taken on
# (their hash): any later change to them reports null.
TRAFFIC = {
    "k_diag": {"bytes_per_launch": 1.2848e+07, "n": 20000, "prec": "bf16x5",
               "sources": ("diag.cu", "diag.cuh", "diag_tile.cuh", "common.cuh"),
               "sha256_16": "48a0fb1c5854b9b1"},
    "k_update_tc": {"bytes_per_launch": 9.570e8, "n": 20000, "prec": "bf16x5",
                    "sources": ("update_tc.cu", "tc.cuh", "common.cuh", "split.cuh"),
                    "sha256_16": "66320edc2040f95c"},
}


def diag_alg_flops(n: int, tb: int, M: int) -> float:
    """Algorithmic FP64 flops of the diagonal solves of one solve: per column
    and diagonal tile of order tb below it, the rank updates of the rows above
    every block column, 2 FMAs (4 flops) per (row, block column): 2 tb (tb - 1)
    flops; stage i solves the columns of the tiles right of tile i (n - (i+1) tb
    of them with uniform tiles).  The tips (each tile's own triangle, under
    0.5 %) are not counted."""
    return float(sum(max(n - (i + 1) * tb, 0) * 2.0 * tb * (tb - 1) for i in range(max(M - 1, 0))))


def rooflines(prof, ms, n, prec, tile, peaks, peak_src, nsm, tc_kernel=True):
    """Rooflines of the two large kernels from the per-launch CUDA-event
    profile of the timed steps: the update (tensor-bound; FP64 pipe on the FP64
    path) and the diagonal solves (bound by the FP64 FMA units: nsm SMs x 2
    lanes/clk x 2 flops at the maximum SM clock).  Returns (the kernel with
    the larger share of the step, the other)."""
    mean = lambda k: float(np.mean([p[k] for p in prof]))
    upd_ms, upd_n, upd_flops = mean("update_ms"), int(round(mean("update_launches"))), mean("update_tensor_flops")
    dg_ms, dg_n = mean("diag_ms"), int(round(mean("diag_launches")))
    if prec == "fp64":
        clk = float(peaks.get("sm_max_mhz") or 2070.0) * 1e6
        upd = {"bound": "alu", "unit": "TFLOP/s",
               "achieved": upd_flops / (upd_ms * 1e-3) / 1e12 if upd_ms else None,
               "peak": round(nsm * 2 * 2 * clk / 1e12, 4),
               "peak_source": f"FP64 pipe: {nsm} SMs x 2 lanes/clk x 2 flops x {clk / 1e6:.0f} MHz "
                              "(DMMA and DFMA share it on GB300)",
               "kernel": "k_update_f64" if dg_n else
                         "k_dag (FP64 updates and diagonal solves in one persistent launch)"}
    else:
        pk = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        upd = {"bound": "tensor", "unit": "TFLOP/s",
               "achieved": upd_flops / (upd_ms * 1e-3) / 1e12 if upd_ms else None,
               "peak": pk, "peak_source": f"{peak_src} bf16 sustained" +
                                          (" (E4M3 products counted at half weight, the nominal FP8:BF16 "
                                           "rate ratio of 2)" if prec == "fp8x4" else ""),
               "kernel": "k_update_tc" if tc_kernel else "k_update_split"}
    clock = float(peaks.get("sm_max_mhz") or 2070.0) * 1e6
    dg = {"bound": "alu", "unit": "TFLOP/s",
          "achieved": diag_alg_flops(n, tile, dg_n) / (dg_ms * 1e-3) / 1e12 if dg_ms else None,
          "peak": round(nsm * 2 * 2 * clock / 1e12, 4),
          "peak_source": f"FP64 FMA units: {nsm} SMs x 2 lanes/clk x 2 flops x {clock / 1e6:.0f} MHz",
          "kernel": "k_diag"}
    for r, t, c in ((upd, upd_ms, upd_n), (dg, dg_ms, dg_n)):
        if r["achieved"]:
            r["achieved"] = round(r["achieved"], 2)
            r["frac"] = round(r["achieved"] / r["peak"], 4)
        r["traffic"] = measured_traffic(r["kernel"], n, prec)
        r["launches_per_step"] = c
        r["avg_launch_ms"] = round(t / max(c, 1), 4)
        r["share_of_step"] = round(t / ms, 3) if ms else None
    return (dg, upd) if dg_ms >= upd_ms else (upd, dg)


def measured_traffic(kernel: str, n: int = 20000, prec: str = "bf16x5"):
    import hashlib
    rec = TRAFFIC.get(kernel)
    if not rec or rec["n"] != n or rec["prec"] != prec:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_2003_04776_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes_per_launch"] if h.hexdigest()[:16] == rec["sha256_16"] else None


def column_kinds_all(block):
    """Kind (0 real, 1 Re and 2 Im of a pair) of every output column of an
    all-eigenvector solve; column c belongs to diagonal position c."""
    block = np.asarray(block)
    kinds = np.zeros(block.size, dtype=np.int64)
    kinds[block == 1] = 1
    kinds[block == 2] = 2
    return kinds


def gpu_residuals(St, Tt, V, kinds, lam_re, lam_im, block_cols: int = 1024, row_block: int = 0):
    """Relative residual ||beta S v - alpha T v||_inf / ((|beta| ||S||_inf +
    |alpha| ||T||_inf) ||v||_inf) of every eigenvector of an all-eigenvector
    solve, with (alpha, beta) = (lam, 1) from the generator's eigenvalues (a
    pair's first row carries +Im); a pair's two columns get its complex
    vector's value.  S V and T V are FP64 GEMMs on the GPU (cuBLAS through
    torch), restricted by the upper quasi-triangular structure: the columns
    [c0, c1) of V are zero below row c1, so only S[:c1+1, :c1+1] meets them.
    St, Tt, V hold the column-major arrays (row c of the tensor = column c).
    With row_block > 0 every block of row_block rows is normalised by its own
    norms instead, (|beta| ||S[K, :]||_inf + |alpha| ||T[K, :]||_inf) ||v||_inf,
    and the largest block value is returned: huge entries elsewhere in S or T
    then cannot hide an error in the rows they do not touch.
    Returns a numpy array with one value per column."""
    import torch
    n = V.shape[0]
    dev = V.device
    rS = St.abs().sum(dim=0)                          # row sums of |S|
    rT = Tt.abs().sum(dim=0)
    if row_block > 0:
        nb = (n + row_block - 1) // row_block
        pad = nb * row_block - n
        blk_max = lambda r: torch.cat([r, r.new_zeros(pad)]).view(nb, row_block).max(dim=1).values
        nS = blk_max(rS).repeat_interleave(row_block)[:n]   # per row: its block's norm
        nT = blk_max(rT).repeat_interleave(row_block)[:n]
    else:
        nS, nT = rS.max(), rT.max()
    kinds_t = torch.as_tensor(np.asarray(kinds), device=dev)
    pos = np.arange(n) - (np.asarray(kinds) == 2)
    a_t = torch.as_tensor(np.asarray(lam_re)[pos], dtype=torch.float64, device=dev)
    b_t = torch.as_tensor(np.abs(np.asarray(lam_im)[pos]), dtype=torch.float64, device=dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    c0 = 0
    while c0 < n:
        c1 = min(n, c0 + block_cols)
        if kinds[c1 - 1] == 1:
            c1 += 1                                   # keep a pair whole
        r1 = min(n, c1 + 1)
        X = V[c0:c1, :r1]
        WS = X @ St[:r1, :r1]                         # WS[c, r] = (S V)[r, c]
        WT = X @ Tt[:r1, :r1]
        k = kinds_t[c0:c1]
        a, b = a_t[c0:c1, None], b_t[c0:c1, None]
        nxt = lambda A: torch.cat([A[1:], torch.zeros_like(A[:1])])
        prv = lambda A: torch.cat([torch.zeros_like(A[:1]), A[:-1]])
        pair = (k == 1)[:, None]
        # real columns: beta S x - a T x; a pair's first column (x, y):
        # re = S x - a T x + b T y, im = S y - a T y - b T x
        re = WS - a * WT + torch.where(pair, b * nxt(WT), torch.zeros_like(WT))
        im = torch.where(pair, nxt(WS) - a * nxt(WT) - b * WT, torch.zeros_like(WT))
        rabs = torch.sqrt(re * re + im * im)
        y = torch.where(pair, nxt(X), torch.zeros_like(X))
        zmax = torch.sqrt(X * X + y * y).max(dim=1).values
        alpha = torch.sqrt(a[:, 0] ** 2 + torch.where(k == 0, torch.zeros_like(b[:, 0]), b[:, 0]) ** 2)
        if row_block > 0:
            den = (nS[None, :r1] + alpha[:, None] * nT[None, :r1]) * zmax[:, None]
            val = torch.where(rabs > 0, rabs / den, torch.zeros_like(rabs)).max(dim=1).values
        else:
            val = rabs.max(dim=1).values / ((nS + alpha * nT) * zmax)
        # a pair's second column takes the value of its first
        val = torch.where(k == 2, prv(val), val)
        out[c0:c1] = val
        c0 = c1
    return out.cpu().numpy()


def normalised_error(Vref, Vgot, kinds):
    """Largest componentwise difference of the GPU's columns from the
    oracle's, both normalised at the oracle's entry of largest modulus (pairs
    as complex vectors); Vref, Vgot: n x m numpy arrays of the same columns."""
    worst = 0.0
    q = 0
    m = Vref.shape[1]
    while q < m:
        if kinds[q] == 1:
            zr, zg, step = Vref[:, q] + 1j * Vref[:, q + 1], Vgot[:, q] + 1j * Vgot[:, q + 1], 2
        else:
            zr, zg, step = Vref[:, q].astype(complex), Vgot[:, q].astype(complex), 1
        i = int(np.argmax(np.abs(zr)))
        d = zg[i]
        e = np.inf if (d == 0 or not np.isfinite(d)) else float(np.abs(zg / d - zr / zr[i]).max())
        worst = max(worst, e)
        q += step
    return worst


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "200"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 6:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[2 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def cpu_oracle_sample(pencil, budget_s: float, threads: int, top: int = 0):
    """Time the oracle, OpenMP-parallel over eigenvectors on `threads` host
    threads, on a stratified sample of the pencil's eigenvectors (spread evenly
    over the diagonal, so large and small ones alike) sized for about
    `budget_s` seconds; extrapolate to all of them with the sum-of-c^2 work
    weights.  With `top` > 0 the eigenvectors of the first `top` diagonal
    positions (cheap: their work grows with c^2) are computed afterwards,
    untimed, for the accuracy check.  Returns (GFLOP/s, info, (select, V) of
    the timed sample, (select, V) of the top positions or None)."""
    import oracle
    n = pencil.n
    starts = np.flatnonzero(pencil.block != 2)
    per_thread = 0.5e9                      # rough single-thread oracle rate, for sizing only
    avg_work = 2.0 * n * n / 3.0
    k = int(budget_s * threads * per_thread / max(avg_work, 1.0))
    k = max(min(len(starts), 4 * threads), min(len(starts), k))
    picks = np.unique(np.linspace(0, len(starts) - 1, num=k).astype(int))
    sel = np.zeros(n, dtype=np.int32)
    work = 0.0
    for idx in picks:
        c = int(starts[idx])
        sel[c] = 1
        sz = 2 if pencil.block[c] == 1 else 1
        work += sum(2.0 * (cc + 1) ** 2 for cc in range(c, c + sz))
    t0 = time.perf_counter()
    st, V, sc, m = oracle.evc(pencil.S, pencil.T, select=sel, nthreads=threads)
    spent = time.perf_counter() - t0
    rate = work / spent / 1e9
    top_part = None
    if top > 0:
        tsel = np.zeros(n, dtype=np.int32)
        tsel[:min(top, n)] = 1
        if pencil.block[min(top, n) - 1] == 1:
            tsel[min(top, n)] = 1               # keep the last pair whole
        _, Vt, _, _ = oracle.evc(pencil.S, pencil.T, select=tsel, nthreads=threads)
        top_part = (tsel, Vt)
    info = {"columns": int(len(picks)), "seconds": round(spent, 2), "work_flops": work}
    return rate, info, (sel, V), top_part


def selected_columns(block, sel):
    """Output columns (of an all-eigenvector solve) of the selected
    eigenvectors, and their kinds: a pair's two columns follow its first row."""
    cols, kinds = [], []
    for c in np.flatnonzero(sel):
        if block[c] == 2:
            continue
        if block[c] == 1:
            cols += [c, c + 1]
            kinds += [1, 2]
        else:
            cols.append(c)
            kinds.append(0)
    return np.asarray(cols, dtype=np.int64), np.asarray(kinds, dtype=np.int64)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a bounded sample of the workload.
    A step is one timed sample (stratified eigenvectors of the benchmark's
    pencil, OpenMP over eigenvectors on every host core); value is the
    sample's rate extrapolated to the whole solve by the sum-of-c^2 work
    weights, ms_per_step the sample's own wall time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import pencilgen
    n = args.n
    p = pencilgen.config_pencil(3, n=n) if n == 20000 else pencilgen.make_pencil(n, pencilgen.config_seed(3))
    budget = max(4.0, 90.0 / max(args.steps + args.warmup, 1))
    threads = os.cpu_count() or 1
    rates, secs = [], []
    for s in range(args.warmup + args.steps):
        r, info, _, _ = cpu_oracle_sample(p, budget, threads)
        if s >= args.warmup:
            rates.append(r)
            secs.append(info["seconds"])
    val = float(np.median(rates))
    F = flops_all(n)
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * float(np.mean(secs)), 1),
            "ms_per_full_solve_extrapolated": round(F / (val * 1e9) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"schur-pencil n={n}, all eigenvectors", "n": n, "prec": "oracle-fp64"},
            "cpu_baseline": {"value": round(val, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": f"{info['columns']} eigenvectors per step (stratified over the diagonal), "
                                       f"{info['seconds']} s on {threads} threads, extrapolated by sum c^2"},
            "e2e": {"value": round(val, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pevc", choices=["pevc", "reference"])
    ap.add_argument("--prec", default="bf16x5", choices=["bf16x3", "bf16x5", "fp8x4", "fp64"])
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    # skip the FP64 and BF16x3 comparison arms (timed after the headline)
    ap.add_argument("--no-arms", action="store_true")
    # "real" is the headline workload; "cplx" times the complex-pencil solve
    # (FP64) on its own, as a separate line
    ap.add_argument("--workload", default="real", choices=["real", "cplx", "batched", "backtransform"])
    return ap.parse_args(argv)


def flops_cplx(n: int) -> float:
    """Real flops of all eigenvectors of a complex triangular pencil: per
    column c and row pair (i, l) above it, the complex products S_il x_l and
    T_il x_l (16 real flops), over c^2 / 2 pairs: sum 8 c^2, about 8 n^3 / 3."""
    return 8.0 * (n - 1) * n * (2 * n - 1) / 6.0


def run_complex(args):
    """The complex-pencil solve (pevc_solve_cplx, FP64) on one seeded pencil
    resident in HBM, timed with CUDA events like the headline workload."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import pencilgen
    import paper_2003_04776_gb300 as pevc
    n = args.n
    p = pencilgen.make_complex_pencil(n, pencilgen.config_seed(3))
    St = pevc.to_device_colmajor_c(p.S)
    Tt = pevc.to_device_colmajor_c(p.T)
    V = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    scale = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    plan = pevc.Plan(n, prec="fp64", stream=stream)

    def step():
        st, m = pevc.pevc_solve_cplx(plan.h, St.data_ptr(), n, Tt.data_ptr(), n, n, 0, V.data_ptr(), n,
                                     scale.data_ptr())
        if st:
            raise pevc.PevcError(st, "pevc_solve_cplx")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    plan.close()
    F = flops_cplx(n)
    tflops = F / (ms * 1e-3) / 1e12
    peak = 152 * 2 * 2 * 2070e6 / 1e12
    line = {"metric": "complex all-eigenvector solve throughput", "value": round(F / (ms * 1e-3) / 1e9, 2),
            "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"complex-schur-pencil n={n}, all eigenvectors", "n": n, "prec": "fp64",
                       "tile": 64},
            "roofline": {"bound": "alu", "achieved": round(tflops, 4), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tflops / peak, 4), "traffic": None,
                         "peak_source": "FP64 FMA units: 152 SMs x 2 lanes/clk x 2 flops x 2070 MHz",
                         "kernel": "whole solve (k_cx_update dominant)"},
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


class Batch:
    """The batched workload resident on the device: every pencil's S, T and
    output V in one buffer each (column-major n x n blocks, back to back), so
    that the host copies of the end-to-end step are one transfer per
    operand."""

    def __init__(self, pencils, pevc):
        import torch
        self.pencils = pencils
        self.n = [p.n for p in pencils]
        self.off = np.concatenate([[0], np.cumsum([n * n for n in self.n])]).astype(np.int64)
        total = int(self.off[-1])
        host_S = np.empty(total)
        host_T = np.empty(total)
        for b, p in enumerate(pencils):
            host_S[self.off[b]:self.off[b + 1]] = p.S.ravel(order="F")
            host_T[self.off[b]:self.off[b + 1]] = p.T.ravel(order="F")
        self.hS = torch.from_numpy(host_S).pin_memory()
        self.hT = torch.from_numpy(host_T).pin_memory()
        self.S = self.hS.to("cuda")
        self.T = self.hT.to("cuda")
        self.V = torch.empty(total, dtype=torch.float64, device="cuda")
        self.scale = torch.empty(int(sum(self.n)), dtype=torch.int32, device="cuda")
        self.soff = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        ptr = lambda t, o, es: t.data_ptr() + int(o) * es
        self.S_p = [ptr(self.S, o, 8) for o in self.off[:-1]]
        self.T_p = [ptr(self.T, o, 8) for o in self.off[:-1]]
        self.V_p = [ptr(self.V, o, 8) for o in self.off[:-1]]
        self.sc_p = [ptr(self.scale, o, 4) for o in self.soff[:-1]]
        self.ld = [max(n, 1) for n in self.n]
        self.pevc = pevc

    def view(self, t, b):
        """Pencil b's block of t as a tensor whose row c is column c."""
        n = self.n[b]
        return t[self.off[b]:self.off[b + 1]].view(n, n)

    def solve(self, plan):
        st, m_out, stat = self.pevc.pevc_solve_batched(plan.h, len(self.n), self.S_p, self.ld, self.T_p, self.ld,
                                                       self.n, None, self.V_p, self.ld, self.sc_p)
        if st:
            raise self.pevc.PevcError(st, "pevc_solve_batched")
        bad = [b for b, x in enumerate(stat) if x]
        if bad:
            raise self.pevc.PevcError(stat[bad[0]], f"pevc_solve_batched pencil {bad[0]}")
        return m_out


def batch_accuracy(batch):
    """Per pencil: the largest residual / (n u) over its columns (global
    norms, and per 64-row block with the block's own norms) and whether V is
    finite."""
    import torch
    res, res_rb, finite = [], [], []
    for b, p in enumerate(batch.pencils):
        St, Tt, V = batch.view(batch.S, b), batch.view(batch.T, b), batch.view(batch.V, b)
        kinds = column_kinds_all(p.block)
        finite.append(bool(torch.isfinite(V).all().item()))
        u = p.n * 2.0 ** -53
        res.append(float(gpu_residuals(St, Tt, V, kinds, p.lam_re, p.lam_im).max() / u))
        res_rb.append(float(gpu_residuals(St, Tt, V, kinds, p.lam_re, p.lam_im, row_block=64).max() / u))
    return np.asarray(res), np.asarray(res_rb), np.asarray(finite)


def run_batched(args):
    """The batched workload: 1024 pencils with n log-uniform in [32, 2048],
    odd indices stress pencils, all eigenvectors, in one pevc_solve_batched
    call per step on inputs resident in HBM.  Metric: pencils per second."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import pencilgen
    import paper_2003_04776_gb300 as pevc
    orders = pencilgen.batch_orders()
    pencils = [pencilgen.batch_pencil(b, int(n)) for b, n in enumerate(orders)]
    batch = Batch(pencils, pevc)
    stream = torch.cuda.current_stream()
    plan = pevc.Plan(int(orders.max()), prec=args.prec, tile=args.tile, batch_max=len(pencils), stream=stream)
    for _ in range(args.warmup):
        batch.solve(plan)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            batch.solve(plan)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    count = len(pencils)
    F = float(sum(flops_all(int(n)) for n in orders))
    line = {"metric": "batched all-eigenvector solves, 1024 pencils, n log-uniform [32, 2048], half stress",
            "value": round(count / (ms * 1e-3), 2), "unit": "pencils/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16-split+f64" if args.prec != "fp64" else "f64",
            "data": "synthetic",
            "config": {"workload": "batched schur pencils: 1024, n = round(exp(U[ln 32, ln 2048])), odd = stress",
                       "prec": args.prec, "tile": plan.info[0], "pencils": count,
                       "l2": "inputs %.1f GB >> 129 MB L2, no flush" % (2 * 8 * batch.off[-1] / 1e9)},
            "effective_gflops": round(F / (ms * 1e-3) / 1e9, 2), "clocks": clk.summary()}
    # end to end: the pencils from pinned host memory and V back, every step
    e_times = []
    hV = torch.empty(int(batch.off[-1]), dtype=torch.float64).pin_memory()
    for q in range(max(2, min(args.steps, 4))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.S.copy_(batch.hS, non_blocking=True)
        batch.T.copy_(batch.hT, non_blocking=True)
        batch.solve(plan)
        hV.copy_(batch.V, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if q:
            e_times.append(e0.elapsed_time(e1))
    ems = float(np.median(e_times))
    line["e2e"] = {"value": round(count / (ems * 1e-3), 2), "unit": "pencils/s", "ms_per_step": round(ems, 3),
                   "h2d_bytes_per_step": int(2 * 8 * batch.off[-1]), "d2h_bytes_per_step": int(8 * batch.off[-1])}
    plan.close()
    res, res_rb, finite = batch_accuracy(batch)
    line["accuracy"] = {"max_resid_over_nu": float(res.max()), "max_rowblock_resid_over_nu": float(res_rb.max()),
                        "resid_over_nu_percentiles_50_90_99": [float(np.percentile(res, q)) for q in (50, 90, 99)],
                        "pencils_nonfinite": int((~finite).sum()),
                        "checker": "every column of every pencil, FP64 GEMMs on the GPU (cuBLAS via torch)"}
    if not args.no_cpu_baseline:
        import oracle
        threads = os.cpu_count() or 1
        picks = list(range(0, count, 32))           # every 32nd pencil: plain ones (even indices)
        t0 = time.perf_counter()
        outs = [oracle.evc(pencils[b].S, pencils[b].T, nthreads=threads) for b in picks]
        spent = time.perf_counter() - t0
        Fs = float(sum(flops_all(int(orders[b])) for b in picks))
        rate = Fs / spent                            # flop/s of the oracle on the sample
        line["cpu_baseline"] = {"value": round(count / (F / rate), 4), "unit": "pencils/s", "cores": threads,
                                "kind": "oracle",
                                "sample": f"{len(picks)} pencils (every 32nd), {spent:.1f} s on {threads} threads, "
                                          "extrapolated to the batch by sum 2n^3/3"}
        errs = []
        for b, (st, Vo, sco, m) in zip(picks, outs):
            Vg = batch.view(batch.V, b).cpu().numpy().T
            errs.append(normalised_error(Vo, Vg, column_kinds_all(pencils[b].block)))
        line["accuracy"]["max_err_vs_oracle"] = float(max(errs))
        line["accuracy"]["err_pencils"] = f"{len(picks)} plain pencils (every 32nd)"
    print(json.dumps(line))
    return 0


def run_backtransform(args):
    """Back-transformation X = Z V of all eigenvectors of the n x n benchmark
    pencil (V from an FP64-accurate split solve, resident in HBM; Z dense,
    N(0, 1/n) entries -- the GEMM's speed does not depend on Z being
    orthogonal): the library's split GEMM against cuBLAS's FP64 GEMM, each
    timed with CUDA events (normalisation included)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import pencilgen
    import paper_2003_04776_gb300 as pevc
    n = args.n
    p = pencilgen.config_pencil(3, n=n)
    stream = torch.cuda.current_stream()
    St, Tt = pevc.to_device_colmajor(p.S), pevc.to_device_colmajor(p.T)
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    sc = torch.empty(n, dtype=torch.int32, device="cuda")
    plan = pevc.Plan(n, prec="bf16x5", stream=stream)
    st, m = plan.solve_colmajor(St, Tt, n, V, sc)
    assert st == 0 and m == n
    del St, Tt
    g = torch.Generator(device="cuda").manual_seed(pencilgen.config_seed(3) + 77)
    Z = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g) / n ** 0.5
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    res = {}
    for name, fl, steps in (("split", 0, max(1, args.steps)), ("cublas", pevc.BT_CUBLAS, 1)):
        call = lambda: pevc.pevc_backtransform(plan.h, Z.data_ptr(), n, n, V.data_ptr(), n, n, None, X.data_ptr(),
                                               n, fl)
        assert call() == 0                     # first use: workspace or handle
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record(stream)
            for _ in range(steps):
                assert call() == 0
            e1.record(stream)
            torch.cuda.synchronize()
        res[name] = (e0.elapsed_time(e1) / steps, clk.summary(), steps)
        if name == "split":
            Xs = X.clone()
    # the two results against each other (normalised eigenvectors)
    diff = float((Xs - X).abs().max().item())
    plan.close()
    F = 2.0 * n * n * n                       # nominal GEMM flops (the split GEMM skips V's zero chunks)
    ms, clk, steps = res["split"]
    peaks, src = load_peaks()
    slice_flops = 21 * sum(2.0 * n * min(n, ((c + 2 + 255) // 256) * 256) for c in range(n))
    line = {"metric": "back-transformation X = Z V of all eigenvectors, n=%d" % n,
            "value": round(F / (ms * 1e-3) / 1e9, 2), "unit": "GFLOP/s (2 n^3 nominal)", "n_gpus": 1,
            "steps": steps, "warmup": 1, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split(6)+f64", "data": "synthetic",
            "config": {"workload": f"X = Z V, V: the eigenvectors of the n={n} benchmark pencil, Z dense", "n": n},
            "roofline": {"bound": "tensor", "unit": "TFLOP/s",
                         "achieved": round(slice_flops / (ms * 1e-3) / 1e12, 2),
                         "peak": peaks.get("bf16_tflops_sustained"), "peak_source": f"{src} bf16 sustained",
                         "frac": round(slice_flops / (ms * 1e-3) / 1e12 / peaks.get("bf16_tflops_sustained", 1.0), 4),
                         "kernel": "k_bt_gemm (mma.sync BF16, 21 slice products per chunk; slicing included)"},
            "cublas_fp64": {"ms_per_step": round(res["cublas"][0], 3),
                            "value": round(F / (res["cublas"][0] * 1e-3) / 1e9, 2)},
            "speedup_over_cublas_fp64": round(res["cublas"][0] / ms, 2),
            "max_abs_diff_vs_cublas_normalised": diff, "clocks": clk}
    print(json.dumps(line))
    return 0


def accuracy_of(St, Tt, V, pencil):
    """Accuracy of an all-eigenvector solve, outside any timed region: the
    residual of every column (GPU FP64 GEMMs) and the count of non-finite
    entries of V."""
    import torch
    kinds = column_kinds_all(pencil.block)
    nonfinite = int((~torch.isfinite(V)).sum().item())
    res = gpu_residuals(St, Tt, V, kinds, pencil.lam_re, pencil.lam_im)
    return {"max_resid_over_nu": float(res.max() / (pencil.n * 2.0 ** -53)), "resid_columns": int(res.size),
            "nonfinite": nonfinite,
            "checker": "relative residual of every column, FP64 GEMMs on the GPU (cuBLAS via torch)"}


def timed_solves(pevc, St, Tt, n, prec, tile, stream, warmup, steps, V, scale, dist=None, clock_index=None):
    """warmup untimed solves, then `steps` solves bracketed by CUDA events on
    the solve's stream (barrier + synchronize on both sides under torchrun).
    Returns (ms per solve, per-step kernel profiles, plan info, clocks)."""
    import torch
    plan = pevc.Plan(n, prec=prec, tile=tile, stream=stream)
    plan.profile(True)

    def step():
        st, m = plan.solve_colmajor(St, Tt, n, V, scale)
        if st:
            raise pevc.PevcError(st, "pevc_solve")

    try:
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        prof = []
        clk = ClockSampler(clock_index if clock_index is not None else 0)
        with clk:
            ev0.record(stream)
            for _ in range(steps):
                step()
                prof.append(plan.kernel_profile())
            ev1.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = ev0.elapsed_time(ev1) / steps
        info = plan.info
        sweeps_run = plan.stats[7] if prec != "fp64" else 0.0   # correction sweeps of the last solve
    finally:
        plan.close()
    return ms, prof, info, clk.summary(), sweeps_run


def main():
    args = parse_args()

    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "cplx":
        return run_complex(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "backtransform":
        return run_backtransform(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import pencilgen
    import paper_2003_04776_gb300 as pevc

    n = args.n
    seed_pencil = pencilgen.config_pencil(3, index=rank, n=n)
    stream = torch.cuda.current_stream()
    St = pevc.to_device_colmajor(seed_pencil.S)
    Tt = pevc.to_device_colmajor(seed_pencil.T)
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    scale = torch.empty(n, dtype=torch.int32, device="cuda")

    ms, prof, info, clocks, _ = timed_solves(pevc, St, Tt, n, args.prec, args.tile, stream, args.warmup,
                                             args.steps, V, scale, dist, local)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    F = flops_all(n)
    value = F * world / (ms * 1e-3) / 1e9
    launches = int(np.mean([p["launches"] for p in prof]))

    # rooflines of the dominant kernel and the other large one (CUDA events
    # around each launch, on the solve's stream)
    peaks, peak_src = load_peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    tc = info[0] == 128 and not os.environ.get("PEVC_UPDATE_KERNEL", "").startswith("m")
    roof, roof_other = rooflines(prof, ms, n, args.prec, info[0], peaks, peak_src, nsm, tc)

    line = {"metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16-split+f64" if args.prec != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": f"schur-pencil n={n}, all eigenvectors, 2x2 blocks ~50%",
                       "n": n, "prec": args.prec, "tile": info[0], "slices": info[6],
                       "correction_sweeps": info[7], "parallelism": f"replicas{world}",
                       "l2": "inputs 2 x %.1f GB >> 129 MB L2, no flush" % (n * n * 8 / 1e9)},
            "eigvec_per_s": round(n * world / (ms * 1e-3), 1),
            "gpu_launches": launches, "roofline": roof, "roofline_other": roof_other, "clocks": clocks}

    if not args.no_e2e:
        # end to end through the public API for host data (pevc_solve_host):
        # S, T in pinned host memory (row-major storage of the transposes is
        # the column-major storage the library reads), the library copies
        # them in by column blocks behind the solve and the result back
        Sh = torch.from_numpy(np.ascontiguousarray(seed_pencil.S.T)).pin_memory()
        Th = torch.from_numpy(np.ascontiguousarray(seed_pencil.T.T)).pin_memory()
        Vh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        sch = torch.empty(n, dtype=torch.int32).pin_memory()
        steps_e2e = max(1, min(args.steps, 5))
        plan = pevc.Plan(n, prec=args.prec, tile=args.tile, stream=stream)

        def e2e_step():
            st, m = plan.solve_host(Sh, Th, Vh, sch)
            if st:
                raise pevc.PevcError(st, "pevc_solve_host")

        e2e_step()   # untimed: first use of the pinned buffers
        torch.cuda.synchronize()
        times = []
        for _ in range(steps_e2e):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        h2d, d2h = plan.host_bytes
        plan.close()
        ems = float(np.median(times))   # host copies vary from step to step
        line["e2e"] = {"value": round(F * world / (ems * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
                       "ms_per_step": round(ems, 3), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "api": "pevc_solve_host"}
        del Sh, Th, Vh, sch

    extra = rank == 0 and world == 1 and not args.no_arms
    if rank == 0:
        line["accuracy"] = accuracy_of(St, Tt, V, seed_pencil)

    # the comparison the target turns on: the plain FP64-DMMA path, and the
    # 3-slice BF16 and 4-slice FP8 split paths with their correction sweeps,
    # timed the same way
    if extra:
        for prec, key, steps in (("fp64", "fp64_path", 2), ("bf16x3", "bf16x3_path", 3), ("fp8x4", "fp8x4_path", 3)):
            if prec == args.prec:
                continue
            Va = torch.empty((n, n), dtype=torch.float64, device="cuda")
            ms_a, prof_a, info_a, clk_a, sw_a = timed_solves(pevc, St, Tt, n, prec, 0, stream, 1, steps, Va, scale)
            r_main, r_other = rooflines(prof_a, ms_a, n, prec, info_a[0], peaks, peak_src, nsm, info_a[0] == 128)
            upd = r_main if r_main["kernel"].startswith(("k_update", "k_dag")) else r_other
            line[key] = {"ms_per_step": round(ms_a, 3), "value": round(F / (ms_a * 1e-3) / 1e9, 2),
                         "unit": "GFLOP/s", "eigvec_per_s": round(n / (ms_a * 1e-3), 1), "steps": steps,
                         "warmup": 1, "tile": info_a[0], "slices": info_a[6], "correction_sweeps": int(sw_a),
                         "correction_sweeps_max": info_a[7],
                         "roofline_update": upd, "roofline_diag": r_other if upd is r_main else r_main,
                         "clocks": clk_a, "accuracy": accuracy_of(St, Tt, Va, seed_pencil)}
            del Va
        if "fp64_path" in line:
            line["split_speedup_over_fp64"] = round(line["fp64_path"]["ms_per_step"] / ms, 2)

    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r, inf, (sel, Vo), top = cpu_oracle_sample(seed_pencil, 20.0, threads, top=1024)
        line["cpu_baseline"] = {"value": round(r, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                                "sample": f"{inf['columns']} eigenvectors of the same pencil (stratified over the "
                                          f"diagonal), {inf['seconds']} s on {threads} threads (OpenMP over "
                                          "eigenvectors), extrapolated to all n by sum c^2"}
        # the GPU's columns against the oracle's: the timed sample and every
        # eigenvector of the first 1024 diagonal positions
        errs = []
        for s_, Vo_ in ((sel, Vo), top):
            cols, kinds = selected_columns(seed_pencil.block, s_)
            Vg = V[torch.as_tensor(cols, device="cuda")].cpu().numpy().T
            errs.append(normalised_error(Vo_, Vg, kinds))
        line["accuracy"]["max_err_vs_oracle"] = float(max(errs))
        line["accuracy"]["err_columns"] = (f"{inf['columns']} stratified eigenvectors and every eigenvector of the "
                                           "first 1024 diagonal positions, normalised at the oracle's largest entry")
        r1, inf1, _, _ = cpu_oracle_sample(seed_pencil, 6.0, 1)
        line["cpu_baseline_1core"] = {"value": round(r1, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                                      "sample": f"{inf1['columns']} eigenvectors (stratified), {inf1['seconds']} s "
                                                "on one thread (the xTGEVC analogue), extrapolated by sum c^2"}
    if rank == 0:
        kp = prof[-1]
        print("breakdown (last step): " + ", ".join(
            f"{k}={kp[k]:.2f}" if isinstance(kp[k], float) else f"{k}={kp[k]}" for k in sorted(kp)),
            file=sys.stderr)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
