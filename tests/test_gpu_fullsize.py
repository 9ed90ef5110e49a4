"""Parity at the full sizes of the benchmark workloads.

n = 20000, split BF16x5, in the configuration the benchmark times (default
tile, all eigenvectors), and n = 10000 overflow stress on the FP64 path.  The
GPU solves every eigenvector; then
  * the residual of every one of the n columns is held to 100 n u (FP64 GEMMs
    on the GPU through torch/cuBLAS as the checker, bench.gpu_residuals);
  * every eigenvector of the first TOP diagonal positions (where the
    normalised vectors carry their smallest entries and the split path its
    largest errors) and an evenly spaced sample of the rest are computed one
    by one by the oracle and compared componentwise after normalisation at
    the oracle's largest entry;
  * on the stress pencil, whose 1e100 tiles swamp ||S||_inf, the residual is
    also taken per block of 64 rows, normalised by that block's own norms, so
    an error in rows that meet no huge entry cannot hide behind them.
"""
import os
import sys

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

pytestmark = pytest.mark.gpu

TOP = 2000
SPREAD = 48


def _solve_all(pevc, p, prec):
    import torch
    n = p.n
    St = pevc.to_device_colmajor(p.S)
    Tt = pevc.to_device_colmajor(p.T)
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    scale = torch.empty(n, dtype=torch.int32, device="cuda")
    plan = pevc.Plan(n, prec=prec)
    try:
        st, m = plan.solve_colmajor(St, Tt, n, V, scale)
    finally:
        plan.close()
    torch.cuda.synchronize()
    assert st == 0 and m == n
    assert int((~torch.isfinite(V)).sum().item()) == 0, "Inf/NaN in V"
    return St, Tt, V, scale


def _oracle_sample(p):
    sel = np.zeros(p.n, dtype=np.int32)
    sel[:TOP] = 1
    for k in range(SPREAD):
        sel[int(round(TOP + k * (p.n - 1 - TOP) / (SPREAD - 1)))] = 1
    for c in np.flatnonzero(sel):              # select a pair by its first row
        if p.block[c] == 2:
            sel[c] = 0
            sel[c - 1] = 1
    return sel


def _compare_with_oracle(p, V, scale, sel):
    import torch
    ost, Vo, sco, mo = oracle.evc(p.S, p.T, select=sel, nthreads=os.cpu_count() or 1)
    assert ost == 0
    cols, kinds = bench.selected_columns(p.block, sel)
    assert mo == cols.size
    Vg = V[torch.as_tensor(cols, device="cuda")].cpu().numpy().T
    err, errs = check.compare_normalised(Vo, Vg, kinds)
    sc = scale[torch.as_tensor(cols, device="cuda")].cpu().numpy()
    return err, errs, np.abs(sc.astype(np.int64) - sco.astype(np.int64)).max()


def _checker_agrees(p, V, res, sel):
    """The GPU residual checker against the oracle's residual helper on the
    spread-out sampled columns."""
    import torch
    spread = sel.copy()
    spread[:TOP] = 0
    cols, _ = bench.selected_columns(p.block, spread)
    Vs = V[torch.as_tensor(cols, device="cuda")].cpu().numpy().T
    _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk, spread)
    ref = check.residuals(p.S, p.T, Vs, kinds, pos, a, b, beta)
    assert np.all(np.abs(res[cols] - ref) <= 1e-3 * ref + 4 * p.n * check.U), np.abs(res[cols] - ref).max()


def test_fullsize_split_bf16x5_n20000(pevc_lib):
    p = pencilgen.config_pencil(3)
    assert p.n == 20000
    St, Tt, V, scale = _solve_all(pevc_lib, p, "bf16x5")
    kinds_all = bench.column_kinds_all(p.block)
    res = bench.gpu_residuals(St, Tt, V, kinds_all, p.lam_re, p.lam_im)
    r = res.max() / (p.n * check.U)
    sel = _oracle_sample(p)
    err, errs, dsc = _compare_with_oracle(p, V, scale, sel)
    _checker_agrees(p, V, res, sel)
    print(f"n=20000 bf16x5: every column: max residual / (n u) {r:.3e}; oracle on {len(errs)} eigenvectors "
          f"(first {TOP} positions and {SPREAD} spread): max err {err:.3e}, median {np.median(errs):.3e}, "
          f"scale exponents within {dsc}")
    assert r <= 100.0
    assert err <= 1e-8
    assert dsc <= 1


def test_fullsize_stress_fp64_n10000(pevc_lib):
    p = pencilgen.config_pencil(2)
    assert p.n == 10000
    St, Tt, V, scale = _solve_all(pevc_lib, p, "fp64")
    kinds_all = bench.column_kinds_all(p.block)
    res = bench.gpu_residuals(St, Tt, V, kinds_all, p.lam_re, p.lam_im)
    res_rb = bench.gpu_residuals(St, Tt, V, kinds_all, p.lam_re, p.lam_im, row_block=64)
    assert int(scale.max().item()) > 1023             # growth beyond the FP64 range is represented
    sel = _oracle_sample(p)
    err, errs, dsc = _compare_with_oracle(p, V, scale, sel)
    _checker_agrees(p, V, res, sel)
    r, rb = res.max() / (p.n * check.U), res_rb.max() / (p.n * check.U)
    print(f"n=10000 stress fp64: every column: max residual / (n u) {r:.3e}, per 64-row block {rb:.3e}; "
          f"oracle on {len(errs)} eigenvectors: max err {err:.3e}, median {np.median(errs):.3e}, "
          f"scale exponents within {dsc}")
    assert r <= 100.0
    assert rb <= 100.0
    assert err <= 1e-6
    assert dsc <= 1
