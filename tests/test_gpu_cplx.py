"""GPU parity of the complex-pencil path through the C ABI: pevc_solve_cplx,
pevc_solve_cplx_left and pevc_backtransform_cplx against the complex oracle
(eigenvectors of complex triangular pencils, the extension to complex data
that Section 7 names).

Bar: componentwise within 1e-10 of the oracle after normalisation at the
oracle's entry of largest modulus, residual <= 100 n u, scale exponents
within 1 of the oracle's, zeros below the tip, no Inf/NaN.
"""
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _check(p, V, sc, select=None):
    assert np.isfinite(V).all()
    st, Vo, sco, m = oracle.evc_cplx(p.S, p.T, select=select, nthreads=os.cpu_count() or 1)
    assert st == 0 and V.shape == Vo.shape
    err, _ = check.compare_normalised_cplx(Vo, V)
    idx = np.arange(p.n) if select is None else np.flatnonzero(select)
    res = check.cplx_residuals(p.S, p.T, V, np.diag(p.S)[idx], np.diag(p.T)[idx]).max() / (p.n * check.U)
    for q, c in enumerate(idx):
        assert np.all(V[c + 1:, q] == 0)
    print(f"cplx n={p.n}: err {err:.3e} resid/(nu) {res:.3e}")
    assert err <= TOL
    assert res <= 100.0
    assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)


@pytest.mark.parametrize("n", [1, 2, 5, 63, 64, 65, 129, 300, 701])
def test_cplx_matches_oracle(pevc_lib, n):
    p = pencilgen.make_complex_pencil(n, 7100 + n)
    plan = pevc_lib.Plan(n, prec="fp64")
    try:
        V, sc, st = plan.solve_cplx(p.S, p.T)
    finally:
        plan.close()
    assert st == 0
    _check(p, V, sc)


def test_cplx_stress_and_selection(pevc_lib):
    n = 700
    p = pencilgen.make_complex_pencil(n, 7200, stress=True)
    rng = np.random.default_rng(7201)
    sel = (rng.random(n) < 0.3).astype(np.int32)
    plan = pevc_lib.Plan(n, prec="bf16x5")          # the complex path is FP64 whatever the plan's precision
    try:
        V, sc, st = plan.solve_cplx(p.S, p.T)
        assert st == 0
        _check(p, V, sc)
        assert sc.max() > 1023
        Vs, scs, st = plan.solve_cplx(p.S, p.T, select=sel)
        assert st == 0
        _check(p, Vs, scs, select=sel)
        idx = np.flatnonzero(sel)
        assert np.array_equal(Vs, V[:, idx]) and np.array_equal(scs, sc[idx])
    finally:
        plan.close()


def test_cplx_exact_fixtures(pevc_lib):
    import importlib.util
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    plan = pevc_lib.Plan(16, prec="fp64")
    try:
        for name in ("cexact_n5_s7", "cexact_n8_s13", "cexact_n6_s29_inf"):
            S, T, Vx = mg.load_cplx(os.path.join(here, "golden", name + ".txt"))
            V, sc, st = plan.solve_cplx(S, T)
            assert st == 0
            err, _ = check.compare_normalised_cplx(Vx, V)
            assert err <= 1e-13, name
    finally:
        plan.close()


def test_cplx_unnormalised_plan(pevc_lib):
    n = 200
    p = pencilgen.make_complex_pencil(n, 7300)
    plan = pevc_lib.Plan(n, prec="fp64", normalise=False)
    try:
        W, e, st = plan.solve_cplx(p.S, p.T)
    finally:
        plan.close()
    assert st == 0
    st, Vo, sco, m = oracle.evc_cplx(p.S, p.T)
    err, _ = check.compare_normalised_cplx(Vo, W)
    assert err <= TOL
    # 2^e W has the oracle's growth: its largest modulus is 2^scale within a factor 2
    for q in range(n):
        big = np.abs(W[:, q]).max()
        assert abs(e[q] + np.frexp(big)[1] - 1 - sco[q]) <= 1


def test_cplx_status_codes_and_arguments(pevc_lib):
    import torch
    n = 40
    p = pencilgen.make_complex_pencil(n, 7400)
    plan = pevc_lib.Plan(n, prec="fp64")
    try:
        S = p.S.copy(order="F")
        S[3, 20] = np.nan
        assert plan.solve_cplx(S, p.T, check=False)[2] == pevc_lib.ERR_NONFINITE
        S = p.S.copy(order="F")
        T = p.T.copy(order="F")
        S[7, 7] = 0
        T[7, 7] = 0
        assert plan.solve_cplx(S, T, check=False)[2] == pevc_lib.ERR_INDEFINITE
        sel = np.ones(n, dtype=np.int32)
        sel[7] = 0
        V, sc, st = plan.solve_cplx(S, T, select=sel)
        assert st == 0 and V.shape[1] == n - 1 and np.isfinite(V).all()
        buf = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
        scb = torch.zeros(n, dtype=torch.int32, device="cuda")
        b, s = buf.data_ptr(), scb.data_ptr()
        f = pevc_lib.pevc_solve_cplx
        assert f(plan.h, b, n - 1, b, n, n, 0, b, n, s)[0] == -3
        assert f(plan.h, b, n, b, n, n + 1, 0, b, n + 1, s)[0] == -6
        assert f(plan.h, b, n, b, n, n, 0, b, n - 1, s)[0] == -9
        assert f(plan.h, b + 8, n, b, n, n, 0, b, n, s)[0] == -2
        assert f(plan.h, b, n, b, n, 0, 0, b, n, s) == (0, 0)
    finally:
        plan.close()


@pytest.mark.parametrize("n", [1, 5, 64, 65, 300])
def test_cplx_left_matches_oracle(pevc_lib, n):
    from oracle.left import evc_left_cplx
    p = pencilgen.make_complex_pencil(n, 7500 + n)
    plan = pevc_lib.Plan(n, prec="fp64")
    try:
        U, sc, st = plan.solve_cplx_left(p.S, p.T)
        V, _, st2 = plan.solve_cplx(p.S, p.T)        # the plan stays usable for right solves
    finally:
        plan.close()
    assert st == 0 and st2 == 0
    assert np.isfinite(U).all()
    ost, Uo, sco, m = evc_left_cplx(p.S, p.T, nthreads=os.cpu_count() or 1)
    assert ost == 0 and U.shape == Uo.shape
    err, _ = check.compare_normalised_cplx(Uo, U)
    res = check.cplx_left_residuals(p.S, p.T, U, np.diag(p.S), np.diag(p.T)).max() / (n * check.U)
    for c in range(n):
        assert np.all(U[:c, c] == 0)
    print(f"cplx left n={n}: err {err:.3e} resid/(nu) {res:.3e}")
    assert err <= TOL and res <= 100.0
    assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)


def test_cplx_left_selection_and_stress(pevc_lib):
    from oracle.left import evc_left_cplx
    n = 400
    p = pencilgen.make_complex_pencil(n, 7600, stress=True)
    sel = (np.arange(n) % 5 == 3).astype(np.int32)
    plan = pevc_lib.Plan(n, prec="fp64")
    try:
        U, sc, st = plan.solve_cplx_left(p.S, p.T, select=sel)
    finally:
        plan.close()
    assert st == 0 and np.isfinite(U).all()
    ost, Uo, sco, m = evc_left_cplx(p.S, p.T, select=sel, nthreads=os.cpu_count() or 1)
    assert U.shape == Uo.shape
    err, _ = check.compare_normalised_cplx(Uo, U)
    idx = np.flatnonzero(sel)
    res = check.cplx_left_residuals(p.S, p.T, U, np.diag(p.S)[idx], np.diag(p.T)[idx]).max() / (n * check.U)
    assert err <= TOL and res <= 100.0


def test_cplx_backtransform_matches_oracle(pevc_lib):
    from oracle.backtransform import backtransform_cplx, random_unitary
    n = 300
    p = pencilgen.make_complex_pencil(n, 7800)
    Q, Z = random_unitary(n, 7801), random_unitary(n, 7802)
    A, B = Q @ p.S @ Z.conj().T, Q @ p.T @ Z.conj().T
    plan = pevc_lib.Plan(n, prec="fp64")
    try:
        V, sc, st = plan.solve_cplx(p.S, p.T)
        X, st2 = plan.backtransform_cplx(Z, V)
        Xr, st3 = plan.backtransform_cplx(Z, V, normalise=False)
    finally:
        plan.close()
    assert st == 0 and st2 == 0 and st3 == 0
    st, Vo, sco, m = oracle.evc_cplx(p.S, p.T, nthreads=os.cpu_count() or 1)
    Xo = backtransform_cplx(Z, Vo)
    err, _ = check.compare_normalised_cplx(Xo, X)
    res = check.cplx_residuals(A, B, X, np.diag(p.S), np.diag(p.T)).max() / (n * check.U)
    assert err <= TOL and res <= 100.0
    ref = Z @ V
    assert np.abs(Xr - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_cplx_stress_every_tile_and_repeated_eigenvalue(pevc_lib):
    """Every off-diagonal tile scaled by 1e100 over several tiles (segments of
    different exponents meet in every update), and an exactly repeated
    eigenvalue (a zero pivot raised to smin): scale exponents within 1 of the
    oracle's."""
    p = pencilgen.make_complex_pencil(300, 7900, stress=True, big_frac=1.0)
    ep = pencilgen.exact_complex_pencil(10, 652)
    S2, T2 = ep.as_complex()
    S2[6, 6], T2[6, 6] = S2[1, 1], T2[1, 1]
    plan = pevc_lib.Plan(300, prec="fp64")
    try:
        V, sc, st = plan.solve_cplx(p.S, p.T)
        V2, sc2, st2 = plan.solve_cplx(S2, T2)
    finally:
        plan.close()
    assert st == 0 and st2 == 0
    _check(p, V, sc)
    assert np.isfinite(V2).all() and 40 <= sc2[6] <= 70
    ost, Vo2, sco2, m2 = oracle.evc_cplx(S2, T2)
    assert np.all(np.abs(sc2.astype(np.int64) - sco2.astype(np.int64)) <= 1)
