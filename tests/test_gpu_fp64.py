"""Parity of the FP64 GPU path (libpevc through its C ABI) with the FP64 oracle.

Bar (normalised vectors, largest-modulus entry 1): componentwise within 1e-10
of the oracle, no Inf/NaN, residual <= 100 n u; stress pencils: finite and
residual <= 100 n u with the error against the oracle stated.
"""
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _run(pevc, S, T, prec="fp64", tile=0, select=None, normalise=True, correction=True):
    plan = pevc.Plan(S.shape[0], prec=prec, tile=tile, normalise=normalise, correction=correction)
    try:
        V, sc, st = plan.solve(S, T, select=select, check=False)
        stats = plan.stats
    finally:
        plan.close()
    return V, sc, st, stats


def _compare(p_S, p_T, block, V, sc, select=None, tol=TOL):
    ost, Vo, sco, m = oracle.evc(p_S, p_T, select=select, nthreads=os.cpu_count() or 1)
    assert ost == 0
    assert V.shape == Vo.shape
    kinds, pos = check.column_kinds(block, select)
    err, errs = check.compare_normalised(Vo, V, kinds)
    assert np.isfinite(V).all()
    assert err <= tol, f"max componentwise error vs oracle {err:.3e}"
    assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)
    return err


@pytest.mark.parametrize("n,tile", [(1, 32), (2, 32), (3, 32), (7, 32), (33, 32), (64, 32),
                                    (100, 32), (100, 64), (257, 32), (257, 64), (300, 128), (513, 96)])
def test_fp64_matches_oracle_small(pevc_lib, n, tile):
    p = pencilgen.make_pencil(n, 1000 + n + tile)
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, tile=tile)
    assert st == 0
    _compare(p.S, p.T, p.block, V, sc)


def test_fp64_config0(pevc_lib):
    """n = 256, all eigenvectors, autotuned tile."""
    p = pencilgen.config_pencil(0)
    V, sc, st, _ = _run(pevc_lib, p.S, p.T)
    assert st == 0
    err = _compare(p.S, p.T, p.block, V, sc)
    stt, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    res = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta)
    assert res.max() <= 100 * p.n * check.U
    print(f"config0 fp64: max err {err:.3e}, max resid/(n u) {res.max() / (p.n * check.U):.3e}")


def test_fp64_exact_golden(pevc_lib):
    import glob
    import importlib.util
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    for path in sorted(glob.glob(os.path.join(here, "golden", "exact_*.txt"))):
        S, T, block, Vx = mg.load(path)
        V, sc, st, _ = _run(pevc_lib, S, T, tile=32)
        assert st == 0
        kinds, _ = check.column_kinds(block)
        Vr = np.zeros_like(V)
        for c, k in enumerate(kinds):
            if k == 0:
                Vr[:, c] = Vx[:, c].real
            elif k == 1:
                Vr[:, c] = Vx[:, c].real
                Vr[:, c + 1] = Vx[:, c].imag
        err, _ = check.compare_normalised(Vr, V, kinds)
        assert err <= 1e-12, (path, err)


def test_fp64_selection(pevc_lib):
    p = pencilgen.make_pencil(300, 77)
    sel = np.zeros(p.n, dtype=np.int32)
    sel[::7] = 1
    sel[np.flatnonzero(p.block == 2)[::3]] = 1
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, tile=64, select=sel)
    assert st == 0
    _compare(p.S, p.T, p.block, V, sc, select=sel)


def test_fp64_unnormalised_representation(pevc_lib):
    p = pencilgen.make_pencil(200, 78)
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, tile=32, normalise=False)
    assert st == 0
    ost, Vo, sco, m = oracle.evc(p.S, p.T, normalise=False)
    kinds, _ = check.column_kinds(p.block)
    # 2^sc * V must represent the same vector as 2^sco * Vo
    for c in range(p.n):
        d = int(sc[c]) - int(sco[c])
        a = np.ldexp(V[:, c], d)
        assert np.allclose(a, Vo[:, c], rtol=0, atol=1e-10 * np.abs(Vo[:, c]).max())
    # consolidated to the exponent of the largest stored part: that part lies in
    # [1, 2), so a complex entry's modulus lies in [1, 2*sqrt(2))
    vecs, cols = check.as_complex(V, kinds)
    for z, c in zip(vecs, cols):
        mx = max(np.abs(z.real).max(), np.abs(z.imag).max())
        assert 1.0 <= mx < 2.0


def test_fp64_deterministic(pevc_lib):
    p = pencilgen.make_pencil(400, 79)
    V1, s1, st1, _ = _run(pevc_lib, p.S, p.T, tile=64)
    V2, s2, st2, _ = _run(pevc_lib, p.S, p.T, tile=64)
    assert st1 == st2 == 0
    assert np.array_equal(V1, V2) and np.array_equal(s1, s2)


def test_fp64_status_codes(pevc_lib):
    p = pencilgen.make_pencil(64, 80)
    i = int(np.flatnonzero(p.block == 1)[0])
    S = p.S.copy(order="F")
    S[i, i + 1] = abs(S[i, i + 1])
    S[i + 1, i] = abs(S[i + 1, i])      # real eigenvalues in a 2x2 block
    _, _, st, _ = _run(pevc_lib, S, p.T, tile=32)
    assert st == pevc_lib.ERR_NOT_SCHUR
    T = p.T.copy(order="F")
    T[i, i + 1] = 0.25                  # T_jj not diagonal
    _, _, st, _ = _run(pevc_lib, p.S, T, tile=32)
    assert st == pevc_lib.ERR_NOT_SCHUR
    S = p.S.copy(order="F")
    S[3, 40] = np.inf
    _, _, st, _ = _run(pevc_lib, S, p.T, tile=32)
    assert st == pevc_lib.ERR_NONFINITE
    S = p.S.copy(order="F")
    T = p.T.copy(order="F")
    j = int(np.flatnonzero(p.block == 0)[0])
    S[j, j] = 0.0
    T[j, j] = 0.0
    _, _, st, _ = _run(pevc_lib, S, T, tile=32)
    assert st == pevc_lib.ERR_INDEFINITE
    # the same entry unselected is no error
    sel = np.ones(p.n, dtype=np.int32)
    sel[j] = 0
    _, _, st, _ = _run(pevc_lib, S, T, tile=32, select=sel)
    assert st == 0


def test_fp64_invalid_arguments(pevc_lib):
    import torch
    plan = pevc_lib.Plan(16, tile=32)
    buf = torch.zeros(16 * 16, dtype=torch.float64, device="cuda")
    sc = torch.zeros(16, dtype=torch.int32, device="cuda")
    st, m = pevc_lib.pevc_solve(plan.h, buf.data_ptr(), 16, buf.data_ptr(), 16, 17, 0,
                                buf.data_ptr(), 16, sc.data_ptr())
    assert st == -6                     # n > n_max
    st, m = pevc_lib.pevc_solve(plan.h, buf.data_ptr(), 8, buf.data_ptr(), 16, 16, 0,
                                buf.data_ptr(), 16, sc.data_ptr())
    assert st == -3                     # lds < n
    st, m = pevc_lib.pevc_solve(plan.h, 0, 16, buf.data_ptr(), 16, 16, 0,
                                buf.data_ptr(), 16, sc.data_ptr())
    assert st == -2
    st, m = pevc_lib.pevc_solve(plan.h, buf.data_ptr(), 16, buf.data_ptr(), 16, 0, 0,
                                buf.data_ptr(), 16, sc.data_ptr())
    assert st == 0 and m == 0           # n = 0 is an empty problem
    plan.close()
    st, h = pevc_lib.pevc_plan(10, 1, 9, 0, 0, 0)
    assert st == -4
    st, h = pevc_lib.pevc_plan(10, 1, 0, 48, 0, 0)
    assert st == -5


def test_fp64_stress_finite_small(pevc_lib):
    """Overflow stress (T's diagonal 2^-40, clustered eigenvalues, 1e100 tiles)."""
    p = pencilgen.make_pencil(700, pencilgen.config_seed(2), stress=True)
    V, sc, st, _ = _run(pevc_lib, p.S, p.T, tile=64)
    assert st == 0
    assert np.isfinite(V).all()
    assert sc.max() > 1023
    stt, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    res = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta)
    assert res.max() <= 100 * p.n * check.U
    # per block of 64 rows, normalised by the block's own norms (the 1e100
    # tiles elsewhere cannot hide an error there)
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    to_t = lambda A: torch.from_numpy(np.ascontiguousarray(np.asarray(A).T))
    rb = bench.gpu_residuals(to_t(p.S), to_t(p.T), to_t(V), bench.column_kinds_all(p.block), p.lam_re, p.lam_im,
                             row_block=64).max()
    assert rb <= 100 * p.n * check.U
    ost, Vo, sco, m = oracle.evc(p.S, p.T, nthreads=os.cpu_count() or 1)
    err, errs = check.compare_normalised(Vo, V, kinds)
    print(f"stress n=700: max err vs oracle {err:.3e}, median {np.median(errs):.3e}, "
          f"per-block residual {rb / (p.n * check.U):.3e} n u")
    assert err <= 1e-6


def test_fp64_config1_full(pevc_lib):
    """n = 4000, all eigenvectors, autotuned tile, full oracle comparison."""
    p = pencilgen.config_pencil(1)
    V, sc, st, stats = _run(pevc_lib, p.S, p.T)
    assert st == 0
    err = _compare(p.S, p.T, p.block, V, sc)
    print(f"config1 fp64: max err {err:.3e}; device ms {stats[0]:.1f}")
