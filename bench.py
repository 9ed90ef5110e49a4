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


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged
# over the launches of one n = 20000 solve) from the ncu captures summarised in
# profiles/k_update_tc_bf16x5.md and profiles/k_diag_n8000.md, valid only for
# the kernel sources they were taken on (their hash); any later change to them
# reports null.
TRAFFIC = {
    "k_diag": {"bytes_per_launch": 1.1207e7, "n": 20000, "prec": "bf16x5",
               "sources": ("diag.cu", "diag.cuh", "common.cuh"),
               "sha256_16": "c873c533c59ed5e8"},
    "k_update_tc": {"bytes_per_launch": 1.2159e9, "n": 20000, "prec": "bf16x5",
                    "sources": ("update_tc.cu", "tc.cuh", "common.cuh", "split.cuh"),
                    "sha256_16": "5acffce1442da583"},
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
        upd = {"bound": "alu", "unit": "TFLOP/s",
               "achieved": upd_flops / (upd_ms * 1e-3) / 1e12 if upd_ms else None,
               "peak": 1.02, "peak_source": "own DFMA/DMMA probe (FP64 tensor and ALU rates are equal on GB300)",
               "kernel": "k_update_f64"}
    else:
        pk = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        upd = {"bound": "tensor", "unit": "TFLOP/s",
               "achieved": upd_flops / (upd_ms * 1e-3) / 1e12 if upd_ms else None,
               "peak": pk, "peak_source": f"{peak_src} bf16 sustained",
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


def cpu_oracle_sample(pencil, budget_s: float, threads: int):
    """Time the oracle, OpenMP-parallel over eigenvectors on `threads` host
    threads, on a stratified sample of the pencil's eigenvectors (spread evenly
    over the diagonal, so large and small ones alike) sized for about
    `budget_s` seconds; extrapolate to all of them with the sum-of-c^2 work
    weights.  Returns (GFLOP/s, info)."""
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
    return rate, {"columns": int(len(picks)), "seconds": round(spent, 2), "work_flops": work}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import pencilgen
    n = args.n
    p = pencilgen.config_pencil(3, n=n) if n == 20000 else pencilgen.make_pencil(n, pencilgen.config_seed(3))
    budget = max(2.0, 60.0 / max(args.steps + args.warmup, 1))
    threads = os.cpu_count() or 1
    rates = []
    for s in range(args.warmup + args.steps):
        r, info = cpu_oracle_sample(p, budget, threads)
        if s >= args.warmup:
            rates.append(r)
    val = float(np.median(rates))
    F = flops_all(n)
    ms = F / (val * 1e9) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
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
    # "real" is the headline workload; "cplx" times the complex-pencil solve
    # (FP64) on its own, as a separate line
    ap.add_argument("--workload", default="real", choices=["real", "cplx"])
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


def main():
    args = parse_args()

    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "cplx":
        return run_complex(args)

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
    plan = pevc.Plan(n, prec=args.prec, tile=args.tile, stream=stream)
    plan.profile(True)

    def step():
        st, m = plan.solve_colmajor(St, Tt, n, V, scale)
        if st:
            raise pevc.PevcError(st, "pevc_solve")
        return m

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    prof = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            prof.append(plan.kernel_profile())
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    F = flops_all(n)
    value = F * world / (ms * 1e-3) / 1e9
    info = plan.info
    launches = int(np.mean([p["launches"] for p in prof]))

    # rooflines of the dominant kernel and the other large one (CUDA events
    # around each launch, on the solve's stream)
    peaks, peak_src = load_peaks()
    tc = info[0] == 128 and not os.environ.get("PEVC_UPDATE_KERNEL", "").startswith("m")
    roof, roof_other = rooflines(prof, ms, n, args.prec, info[0], peaks, peak_src,
                                 torch.cuda.get_device_properties(0).multi_processor_count, tc)

    line = {"metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16-split+f64" if args.prec != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": f"schur-pencil n={n}, all eigenvectors, 2x2 blocks ~50%",
                       "n": n, "prec": args.prec, "tile": info[0], "slices": info[6],
                       "correction_sweeps": info[7], "parallelism": f"replicas{world}",
                       "l2": "inputs 2 x %.1f GB >> 129 MB L2, no flush" % (n * n * 8 / 1e9)},
            "eigvec_per_s": round(n * world / (ms * 1e-3), 1),
            "gpu_launches": launches, "roofline": roof, "roofline_other": roof_other, "clocks": clk.summary()}

    if not args.no_e2e:
        # end to end through the public API: host S, T in pinned memory, result back to host
        Sh = torch.from_numpy(np.ascontiguousarray(seed_pencil.S.T)).pin_memory()
        Th = torch.from_numpy(np.ascontiguousarray(seed_pencil.T.T)).pin_memory()
        Vh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        sch = torch.empty(n, dtype=torch.int32).pin_memory()
        steps_e2e = max(1, min(args.steps, 5))

        def e2e_step():
            St.copy_(Sh, non_blocking=True)
            Tt.copy_(Th, non_blocking=True)
            step()
            Vh.copy_(V, non_blocking=True)
            sch.copy_(scale, non_blocking=True)

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
        ems = float(np.median(times))   # host copies vary from step to step
        line["e2e"] = {"value": round(F * world / (ems * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
                       "ms_per_step": round(ems, 3),
                       "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": n * n * 8 + n * 4}

    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r, inf = cpu_oracle_sample(seed_pencil, 20.0, threads)
        line["cpu_baseline"] = {"value": round(r, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                                "sample": f"{inf['columns']} eigenvectors of the same pencil (stratified over the "
                                          f"diagonal), {inf['seconds']} s on {threads} threads (OpenMP over "
                                          "eigenvectors), extrapolated to all n by sum c^2"}
    plan.close()
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
