"""Parity of the split-precision GPU paths with the FP64 oracle.

bf16x5: one pass, five BF16 slices per operand (15 slice products per update).
bf16x3: three slices (6 products) plus the residual correction sweep (the
residual with 5-slice products, the correction pass with 3).
fp8x4: four FP8 E4M3 slices of 4-bit digits (10 products) plus the same
sweep (the residual in BF16x5, the correction pass on E4M3 slices).
Bar: residual <= 100 n u and no Inf/NaN; componentwise error against the
oracle within the tolerance below (and printed).
"""
import os
import sys

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-8     # componentwise; the binding bar of the split paths is the residual (<= 100 n u)


def _run(pevc, S, T, prec, tile=0, select=None, correction=True, normalise=True):
    plan = pevc.Plan(S.shape[0], prec=prec, tile=tile, correction=correction, normalise=normalise)
    try:
        V, sc, st = plan.solve(S, T, select=select, check=False)
        stats = plan.stats
    finally:
        plan.close()
    return V, sc, st, stats


def _rowblock_res(p, V):
    """Largest residual per block of 64 rows, each normalised by its own
    rows' norms (all eigenvectors; see bench.gpu_residuals): 1e100 tiles
    elsewhere in S cannot hide an error from it."""
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    to_t = lambda A: torch.from_numpy(np.ascontiguousarray(np.asarray(A).T))
    r = bench.gpu_residuals(to_t(p.S), to_t(p.T), to_t(V), bench.column_kinds_all(p.block), p.lam_re, p.lam_im,
                            row_block=64)
    return r.max() / (p.n * check.U)


def _errors(p, V, select=None):
    ost, Vo, sco, m = oracle.evc(p.S, p.T, select=select, nthreads=os.cpu_count() or 1)
    assert ost == 0
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk, select)
    err, errs = check.compare_normalised(Vo, V, kinds)
    res = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta)
    return err, res.max() / (p.n * check.U)


@pytest.mark.parametrize("prec", ["bf16x5", "bf16x3", "fp8x4"])
@pytest.mark.parametrize("n,tile", [(1, 32), (5, 32), (64, 32), (100, 32), (257, 32), (300, 64), (500, 96),
                                    (513, 128)])
def test_split_matches_oracle(pevc_lib, prec, n, tile):
    p = pencilgen.make_pencil(n, 2000 + n + tile)
    V, sc, st, stats = _run(pevc_lib, p.S, p.T, prec, tile=tile)
    assert st == 0
    assert np.isfinite(V).all()
    err, res = _errors(p, V)
    print(f"{prec} n={n} tile={tile}: err {err:.3e} resid/(nu) {res:.3e} sweeps {stats[7]:.0f}")
    lo, hi = {"bf16x5": (0, 0), "bf16x3": (1, 1), "fp8x4": (1, 6)}[prec]   # correction sweeps run
    assert lo <= stats[7] <= hi
    assert res <= 100.0
    assert err <= TOL_SPLIT


@pytest.mark.parametrize("prec,tile", [("bf16x3", 64), ("fp8x4", 64), ("fp8x4", 128)])
def test_split_uncorrected_is_low_precision(pevc_lib, prec, tile):
    """Without the correction sweep the 3-slice BF16 pass carries ~2^-22
    errors and the 4-slice E4M3 pass ~2^-15; the sweep brings them to FP64
    level (this is what the sweep is for)."""
    p = pencilgen.make_pencil(400, 4001)
    V0, _, st0, _ = _run(pevc_lib, p.S, p.T, prec, tile=tile, correction=False)
    V1, _, st1, _ = _run(pevc_lib, p.S, p.T, prec, tile=tile, correction=True)
    assert st0 == st1 == 0
    e0, r0 = _errors(p, V0)
    e1, r1 = _errors(p, V1)
    print(f"{prec} tile {tile}: uncorrected err {e0:.3e} resid/(nu) {r0:.3e}; "
          f"corrected err {e1:.3e} resid/(nu) {r1:.3e}")
    assert np.isfinite(V0).all()
    assert e0 < (1e-2 if prec == "fp8x4" else 1e-3)
    assert r1 <= 100.0 and e1 <= TOL_SPLIT
    assert e1 < e0


@pytest.mark.parametrize("prec", ["bf16x5", "bf16x3", "fp8x4"])
def test_split_config0(pevc_lib, prec):
    p = pencilgen.config_pencil(0)
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, prec)
    assert st == 0
    err, res = _errors(p, V)
    print(f"config0 {prec}: err {err:.3e} resid/(nu) {res:.3e}")
    assert res <= 100.0 and err <= TOL_SPLIT


@pytest.mark.parametrize("prec", ["bf16x5", "bf16x3", "fp8x4"])
def test_split_selection(pevc_lib, prec):
    p = pencilgen.make_pencil(350, 4002)
    sel = np.zeros(p.n, dtype=np.int32)
    sel[::5] = 1
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, prec, tile=64, select=sel)
    assert st == 0
    err, res = _errors(p, V, select=sel)
    assert res <= 100.0 and err <= TOL_SPLIT


@pytest.mark.parametrize("prec", ["bf16x5", "bf16x3", "fp8x4"])
def test_split_stress_finite(pevc_lib, prec):
    p = pencilgen.make_pencil(700, pencilgen.config_seed(2), stress=True)
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, prec, tile=64)
    assert st == 0
    assert np.isfinite(V).all()
    assert sc.max() > 1023
    err, res = _errors(p, V)
    rb = _rowblock_res(p, V)
    print(f"stress {prec}: err {err:.3e} resid/(nu) {res:.3e} per 64-row block {rb:.3e}")
    assert res <= 100.0 and rb <= 100.0
    assert err <= 1e-6


@pytest.mark.parametrize("prec", ["bf16x5", "bf16x3", "fp8x4"])
def test_split_config1_full(pevc_lib, prec):
    p = pencilgen.config_pencil(1)
    V, sc, st, stats = _run(pevc_lib, p.S, p.T, prec)
    assert st == 0
    err, res = _errors(p, V)
    print(f"config1 {prec}: err {err:.3e} resid/(nu) {res:.3e} device ms {stats[0]:.1f}")
    assert res <= 100.0 and err <= TOL_SPLIT


@pytest.mark.parametrize("kernel", ["tc", "mma"])
@pytest.mark.parametrize("prec", ["bf16x5", "bf16x3", "fp8x4"])
@pytest.mark.parametrize("n,stress", [(700, False), (700, True), (1030, False)])
def test_split_update_kernels_tile128(pevc_lib, monkeypatch, kernel, prec, n, stress):
    """Tiles of order 128 run the update on the tcgen05 tensor cores (TMA-fed,
    tensor-memory accumulators) or, selected by PEVC_UPDATE_KERNEL=mma, on the
    mma.sync path; both must meet the same bar (ragged last tiles included)."""
    monkeypatch.setenv("PEVC_UPDATE_KERNEL", kernel)
    p = pencilgen.make_pencil(n, 5000 + n + int(stress), stress=stress)
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, prec, tile=128)
    assert st == 0
    assert np.isfinite(V).all()
    err, res = _errors(p, V)
    rb = _rowblock_res(p, V)
    print(f"{kernel} {prec} n={n} stress={stress}: err {err:.3e} resid/(nu) {res:.3e} per 64-row block {rb:.3e}")
    assert res <= 100.0 and rb <= 100.0
    assert err <= (1e-6 if stress else TOL_SPLIT)


@pytest.mark.parametrize("prec,correction", [("bf16x5", True), ("bf16x3", False), ("fp8x4", False),
                                             ("fp8x4", True)])
def test_split_tc_and_mma_updates_agree(pevc_lib, monkeypatch, prec, correction):
    """The tcgen05 update and the mma.sync one compute the same exact level
    sums (integer-valued products, FP32 accumulation that must not round:
    below 2^24 for BF16 slices, below 2^16 for E4M3 ones), so a solve through
    either agrees to FP64 rounding, also uncorrected, where an inexact
    accumulation would show at the 2^-15 level of the slices themselves.  The
    two differ only in the column maxima they record (the tcgen05 epilogue
    keeps an upper bound within 2^-20), which can move a power-of-two scale."""
    p = pencilgen.make_pencil(1030, 6100)
    out = {}
    for kernel in ("tc", "mma"):
        monkeypatch.setenv("PEVC_UPDATE_KERNEL", kernel)
        V, sc, st, _ = _run(pevc_lib, p.S, p.T, prec, tile=128, correction=correction)
        assert st == 0 and np.isfinite(V).all()
        out[kernel] = V
    kinds, _ = check.column_kinds(p.block)
    diff, _ = check.compare_normalised(out["mma"], out["tc"], kinds)
    same = np.array_equal(out["tc"], out["mma"])
    print(f"{prec} correction={correction}: tc vs mma {diff:.3e} (bitwise {same})")
    assert diff <= 1e-13
