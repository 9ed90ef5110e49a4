"""pevc_solve_left through the C ABI against the oracle: left eigenvectors
u^H (beta S - alpha T) = 0.

Bar: componentwise within 1e-10 (FP64) or 1e-8 (split BF16x5) of the oracle
after normalisation, left residual <= 100 n u, no Inf/NaN, zeros above the
eigenvector's block.
"""
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check
from oracle.left import evc_left

pytestmark = pytest.mark.gpu


def _compare(p, U, select, tol):
    assert np.isfinite(U).all()
    ost, Uo, sco, m = evc_left(p.S, p.T, select=select, nthreads=os.cpu_count() or 1)
    assert ost == 0 and U.shape == Uo.shape
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk, select)
    err, _ = check.compare_normalised(Uo, U, kinds)
    res = check.left_residuals(p.S, p.T, U, kinds, pos, a, b, beta).max() / (p.n * check.U)
    for c, k in enumerate(kinds):
        if k != 2:
            assert np.all(U[:pos[c], c] == 0)
    print(f"left n={p.n}: err {err:.3e} resid/(nu) {res:.3e}")
    assert err <= tol
    assert res <= 100.0
    return sco


@pytest.mark.parametrize("prec,n,tile,tol", [("fp64", 1, 32, 1e-10), ("fp64", 5, 32, 1e-10),
                                             ("fp64", 300, 32, 1e-10), ("fp64", 257, 64, 1e-10),
                                             ("bf16x5", 700, 128, 1e-8), ("fp8x4", 500, 96, 1e-8)])
def test_left_matches_oracle(pevc_lib, prec, n, tile, tol):
    p = pencilgen.make_pencil(n, 6100 + n)
    plan = pevc_lib.Plan(n, prec=prec, tile=tile)
    try:
        U, sc, st = plan.solve_left(p.S, p.T)
    finally:
        plan.close()
    assert st == 0
    sco = _compare(p, U, None, tol)
    if prec == "fp64":
        assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)


def test_left_selection_and_stress(pevc_lib):
    n = 240
    rng = np.random.default_rng(6201)
    sel = (rng.random(n) < 0.35).astype(np.int32)
    p = pencilgen.make_pencil(n, 6200)
    plan = pevc_lib.Plan(n, prec="fp64", tile=32)
    try:
        U, sc, st = plan.solve_left(p.S, p.T, select=sel)
        assert st == 0
        _compare(p, U, sel, 1e-10)
        q = pencilgen.make_pencil(n, 6202, stress=True)
        U2, sc2, st2 = plan.solve_left(q.S, q.T)
        assert st2 == 0
        assert np.isfinite(U2).all()
        st, blk, a, b, beta, _ = oracle.eigpairs(q.S, q.T)
        kinds, pos = check.column_kinds(blk)
        res = check.left_residuals(q.S, q.T, U2, kinds, pos, a, b, beta).max() / (n * check.U)
        print(f"left stress n={n}: resid/(nu) {res:.3e}")
        assert res <= 100.0
    finally:
        plan.close()


def test_left_then_right_on_one_plan(pevc_lib):
    """A left solve leaves the plan usable for right solves (and the other way)."""
    n = 200
    p = pencilgen.make_pencil(n, 6300)
    plan = pevc_lib.Plan(n, prec="fp64", tile=32)
    try:
        V1, _, st1 = plan.solve(p.S, p.T)
        U, _, st2 = plan.solve_left(p.S, p.T)
        V2, _, st3 = plan.solve(p.S, p.T)
    finally:
        plan.close()
    assert st1 == st2 == st3 == 0
    assert np.array_equal(V1, V2)


def test_left_argument_errors(pevc_lib):
    import torch
    n = 32
    plan = pevc_lib.Plan(n, prec="fp64", tile=32)
    try:
        buf = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        sc = torch.zeros(n, dtype=torch.int32, device="cuda")
        b, s = buf.data_ptr(), sc.data_ptr()
        f = pevc_lib.pevc_solve_left
        assert f(None, b, n, b, n, n, 0, b, n, s)[0] == -1
        assert f(plan.h, b, n - 1, b, n, n, 0, b, n, s)[0] == -3
        assert f(plan.h, b, n, b, n, n + 1, 0, b, n + 1, s)[0] == -6
        assert f(plan.h, b, n, b, n, n, 0, b, n - 1, s)[0] == -9
        assert f(plan.h, b, n, b, n, 0, 0, b, n, s) == (0, 0)
    finally:
        plan.close()
