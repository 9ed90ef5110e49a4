"""Host-side logic of bench.py (no GPU): the roofline of the dominant kernel,
the diagonal solves' algorithmic flops, the traffic records' source hashes (a
record reports only for the kernel sources it was measured on), and the
reference arm's JSON line and oracle sampling."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _prof(diag_ms, upd_ms):
    return [{"update_ms": upd_ms, "update_launches": 156, "update_tensor_flops": 7.9995e13,
             "diag_ms": diag_ms, "diag_launches": 157}]


def test_diag_flops_close_to_n2_tb():
    f = bench.diag_alg_flops(20000, 128, 157)
    assert abs(f / (20000.0 ** 2 * 128) - 1.0) < 0.02


def test_dominant_kernel_first():
    peaks = {"bf16_tflops_sustained": 1730.2, "sm_max_mhz": 2070.0}
    roof, other = bench.rooflines(_prof(110.0, 80.7), 205.8, 20000, "bf16x5", 128, peaks, "measured", 152)
    assert roof["kernel"] == "k_diag" and roof["bound"] == "alu"
    assert other["kernel"] == "k_update_tc" and other["bound"] == "tensor"
    assert abs(roof["peak"] - 152 * 4 * 2.07e9 / 1e12) < 1e-3
    assert 0.3 < roof["frac"] < 0.45
    assert abs(other["achieved"] - 7.9995e13 / 80.7e-3 / 1e12) < 0.1
    roof2, other2 = bench.rooflines(_prof(60.0, 80.7), 170.0, 20000, "bf16x5", 128, peaks, "measured", 152)
    assert roof2["kernel"] == "k_update_tc" and other2["kernel"] == "k_diag"
    for r in (roof, other):
        assert set(("bound", "achieved", "peak", "unit", "frac", "traffic")) <= set(r)


def test_traffic_records_apply_only_to_their_workload():
    # a record reports for its own workload (and only while the kernel sources
    # hash to the measured version; otherwise null)
    for k in ("k_update_tc", "k_diag"):
        v = bench.measured_traffic(k)
        assert v is None or v == bench.TRAFFIC[k]["bytes_per_launch"]
        assert bench.measured_traffic(k, n=4000) is None
        assert bench.measured_traffic(k, prec="fp64") is None
    assert bench.measured_traffic("k_post") is None


def _ref_args(n=256, steps=2, warmup=1):
    import argparse
    return argparse.Namespace(n=n, steps=steps, warmup=warmup, gpus=1)


def test_reference_line_keeps_the_contract(monkeypatch, capsys):
    import json
    monkeypatch.delenv("RANK", raising=False)
    calls = []

    def fake_sample(pencil, budget, threads):
        calls.append((pencil.n, budget, threads))
        return 12.5, {"columns": 3, "seconds": 0.1, "work_flops": 1e9}, None, None

    monkeypatch.setattr(bench, "cpu_oracle_sample", fake_sample)
    assert bench.run_reference(_ref_args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert len(calls) == 3 and all(c[0] == 256 for c in calls)          # warm-up + timed steps
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 12.5 and line["unit"] == "GFLOP/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["ms_per_step"] == 100.0                                  # the sample's own time per step
    assert abs(line["ms_per_full_solve_extrapolated"] - bench.flops_all(256) / 12.5e9 * 1e3) < 0.1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == 12.5 and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == 12.5 and e2e["unit"] == "GFLOP/s"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("schur-pencil n=256")


def test_reference_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda *a: (_ for _ in ()).throw(AssertionError("ran")))
    assert bench.run_reference(_ref_args()) == 0
    assert capsys.readouterr().out == ""


def test_cpu_oracle_sample_times_a_stratified_subset():
    import pencilgen
    p = pencilgen.make_pencil(200, 31)
    rate, info, (sel, V), top = bench.cpu_oracle_sample(p, 0.05, 2, top=17)
    assert rate > 0 and 1 <= info["columns"] <= 200
    cols, kinds = bench.selected_columns(p.block, sel)
    assert V.shape == (200, cols.size) and top[1].shape[1] == bench.selected_columns(p.block, top[0])[0].size
    assert top[0][:17].all() and not top[0][18:].any()
    # the work is the sum of 2 (c+1)^2 over the sampled columns (both columns of a pair)
    assert 0 < info["work_flops"] <= bench.flops_all(200) * 1.01


def test_clock_summary_parses_nvidia_smi_lines():
    cs = bench.ClockSampler()
    assert cs.summary()["reasons"] == ["unsampled"]
    for sm, act in ((1965, "Not Active"), (1980, "Active"), (1995, "Not Active"), ("[N/A]", "Not Active")):
        line = f"{sm}, 2070, Not Active, Not Active, Not Active, {act}"
        cs.samples.append([p.strip() for p in line.split(",")])
    s = cs.summary()
    assert s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]          # "Not Active" is not a reason
    cs.samples.append(["2070", "2070", "Active", "Not Active", "Active", "Not Active"])
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_parse_args_defaults_and_complex_workload():
    a = bench.parse_args([])
    assert (a.gpus, a.steps, a.warmup, a.impl, a.prec, a.n, a.workload) == (1, 5, 3, "pevc", "bf16x5", 20000, "real")
    b = bench.parse_args(["--workload", "cplx", "--n", "4000", "--steps", "2"])
    assert b.workload == "cplx" and b.n == 4000 and b.steps == 2
    # 8 n^3 / 3 to leading order; exact for the sum over columns of 8 c^2
    assert bench.flops_cplx(3) == 8.0 * (0 + 1 + 4)
    assert abs(bench.flops_cplx(20000) / (8 * 20000 ** 3 / 3) - 1) < 1e-4


def test_gpu_residual_checker_matches_the_oracle_residuals():
    """The benchmark's all-column residual (written for the GPU, run here on
    torch's CPU tensors) against oracle/check.py's, on the oracle's own
    eigenvectors of a plain and a stress pencil; a planted error in one
    column is seen by both."""
    import torch
    import oracle
    import pencilgen
    from oracle import check
    for n, stress in ((150, False), (130, True)):
        p = pencilgen.make_pencil(n, 4401 + n, stress=stress)
        st, V, sc, m = oracle.evc(p.S, p.T)
        assert st == 0 and m == n
        _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
        kinds, pos = check.column_kinds(blk)
        ref = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta)
        to_t = lambda A: torch.from_numpy(np.ascontiguousarray(np.asarray(A).T))
        got = bench.gpu_residuals(to_t(p.S), to_t(p.T), to_t(V), bench.column_kinds_all(p.block),
                                  p.lam_re, p.lam_im, block_cols=37)
        assert np.array_equal(bench.column_kinds_all(p.block), kinds)
        # the generator's eigenvalue differs from the rounded block's by O(u)
        assert np.all(np.abs(got - ref) <= 4 * n * check.U + 1e-3 * ref), (got - ref).max()
        V2 = V.copy()
        c = n // 2
        V2[c // 2, c] += 1e-6 * np.abs(V2[:, c]).max()
        bad = bench.gpu_residuals(to_t(p.S), to_t(p.T), to_t(V2), kinds, p.lam_re, p.lam_im, block_cols=64)
        assert bad[c] > 1e3 * n * check.U and np.delete(bad, [c - 1, c, c + 1]).max() <= 100 * n * check.U


def test_normalised_error_is_scale_free_and_sees_a_changed_entry():
    import pencilgen
    import oracle
    p = pencilgen.make_pencil(60, 4501)
    st, V, sc, m = oracle.evc(p.S, p.T)
    kinds = bench.column_kinds_all(p.block)
    W = V * -3.5                                   # a real multiple of every column
    assert bench.normalised_error(V, W, kinds) <= 1e-15
    q = int(np.flatnonzero(kinds == 1)[0])
    Z = (V[:, q] + 1j * V[:, q + 1]) * (0.3 - 2j)  # a complex multiple of one pair
    W[:, q], W[:, q + 1] = Z.real, Z.imag
    assert bench.normalised_error(V, W, kinds) <= 1e-14
    W[0, 5] += 1e-7
    assert bench.normalised_error(V, W, kinds) >= 1e-8


def test_row_block_residual_sees_an_error_that_huge_tiles_hide():
    """On a stress pencil (a 1e100 tile swamps ||S||_inf) an error planted in
    rows whose block holds no huge entry is invisible to the global residual
    and plain in the row-block one; the oracle's own vectors pass both."""
    import torch
    import oracle
    import pencilgen
    n = 192
    p = pencilgen.make_pencil(n, 4601, stress=True)
    S = p.S.copy()
    S[0:64, 128:192] *= 1e100                   # rows 0..63 hold the only huge tile
    st, V, sc, m = oracle.evc(S, p.T)
    assert st == 0
    kinds = bench.column_kinds_all(p.block)
    to_t = lambda A: torch.from_numpy(np.ascontiguousarray(np.asarray(A).T))
    good = bench.gpu_residuals(to_t(S), to_t(p.T), to_t(V), kinds, p.lam_re, p.lam_im, row_block=64)
    assert good.max() <= 100 * n * 2.0 ** -53
    c = 120 if kinds[120] != 2 else 121
    V2 = V.copy()
    V2[c - 40, c] += 1e-6 * np.abs(V2[:, c]).max()  # row 80: block 1, no huge entry
    glob = bench.gpu_residuals(to_t(S), to_t(p.T), to_t(V2), kinds, p.lam_re, p.lam_im)
    rb = bench.gpu_residuals(to_t(S), to_t(p.T), to_t(V2), kinds, p.lam_re, p.lam_im, row_block=64)
    assert glob[c] <= 100 * n * 2.0 ** -53 < 1e3 * n * 2.0 ** -53 < rb[c]
