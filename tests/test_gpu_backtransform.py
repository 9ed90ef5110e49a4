"""pevc_backtransform through the C ABI: X = Z V, the eigenvectors of the
original pencil (A, B) = (Q S Z^T, Q T Z^T), against the oracle.

Bar: componentwise within 1e-10 of the oracle after normalisation at the
oracle's largest entry, residual of (A, B) <= 100 n u, no Inf/NaN.
"""
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check
from oracle.backtransform import backtransform, random_orthogonal

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _split_bound(Z, V, K=256, bits=46):
    """Entrywise bound of |X - Z V| for the library's split GEMM: every entry
    of Z (row r) and V (column c) is cut to 48 bits relative to a power of two
    at most twice the largest |entry| of its row (column) in its chunk of K,
    so a chunk's term errs by at most 2^-47 (max_chunk |Z_r.| sum |V_.c| +
    max_chunk |V_.c| sum |Z_r.|); 2^-46 leaves a factor 2, and the FP64
    sums of the chunks add a few units of rounding of |Z| |V|."""
    B = np.zeros((Z.shape[0], V.shape[1]))
    for k0 in range(0, Z.shape[0], K):
        Zc, Vc = np.abs(Z[:, k0:k0 + K]), np.abs(V[k0:k0 + K, :])
        B += Zc.max(axis=1, keepdims=True) * Vc.sum(axis=0, keepdims=True)
        B += Zc.sum(axis=1, keepdims=True) * Vc.max(axis=0, keepdims=True)
    return 2.0 ** -bits * B + 1e-14 * (np.abs(Z) @ np.abs(V))


def _case(n, seed, stress=False, select=None):
    p = pencilgen.make_pencil(n, seed, stress=stress)
    Q = random_orthogonal(n, seed + 11)
    Z = random_orthogonal(n, seed + 12)
    ost, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    assert ost == 0
    kinds, pos = check.column_kinds(blk, select)
    return p, Z, Q @ p.S @ Z.T, Q @ p.T @ Z.T, kinds, pos, (a, b, beta)


def _check(p, Z, A, B, kinds, pos, ev, X, select=None):
    assert np.isfinite(X).all()
    ost, Vo, sco, m = oracle.evc(p.S, p.T, select=select, nthreads=os.cpu_count() or 1)
    assert ost == 0
    Xo = backtransform(Z, Vo, kinds)
    err, _ = check.compare_normalised(Xo, X, kinds)
    res = check.residuals(A, B, X, kinds, pos, *ev).max() / (p.n * check.U)
    print(f"n={p.n}: err {err:.3e} resid/(nu) {res:.3e}")
    assert err <= TOL
    assert res <= 100.0


@pytest.mark.parametrize("prec,n,tile", [("fp64", 300, 32), ("fp64", 257, 64), ("bf16x5", 700, 128)])
def test_backtransform_matches_oracle(pevc_lib, prec, n, tile):
    p, Z, A, B, kinds, pos, ev = _case(n, 4200 + n)
    plan = pevc_lib.Plan(n, prec=prec, tile=tile)
    try:
        V, sc, st = plan.solve(p.S, p.T)
        X, st = plan.backtransform(Z, V)              # kinds of the last solve
        Xk, st2 = plan.backtransform(Z, V, kinds=list(kinds))
    finally:
        plan.close()
    assert st == 0 and st2 == 0
    assert np.array_equal(X, Xk)
    _check(p, Z, A, B, kinds, pos, ev, X)


def test_backtransform_selection_and_unnormalised(pevc_lib):
    n = 240
    rng = np.random.default_rng(4301)
    sel = (rng.random(n) < 0.3).astype(np.int32)
    p, Z, A, B, kinds, pos, ev = _case(n, 4300, select=sel)
    plan = pevc_lib.Plan(n, prec="fp64", tile=32)
    try:
        V, sc, st = plan.solve(p.S, p.T, select=sel)
        assert V.shape[1] == len(kinds)
        X, st = plan.backtransform(Z, V)
        Xr, st2 = plan.backtransform(Z, V, normalise=False)
    finally:
        plan.close()
    assert st == 0 and st2 == 0
    _check(p, Z, A, B, kinds, pos, ev, X, select=sel)
    ref = Z @ V
    assert np.all(np.abs(Xr - ref) <= _split_bound(Z, V))


def test_backtransform_stress_pencil_finite(pevc_lib):
    n = 200
    p, Z, A, B, kinds, pos, ev = _case(n, 4400, stress=True)
    plan = pevc_lib.Plan(n, prec="fp64", tile=32)
    try:
        V, sc, st = plan.solve(p.S, p.T)
        X, st = plan.backtransform(Z, V)
    finally:
        plan.close()
    assert st == 0
    assert np.isfinite(X).all()
    res = check.residuals(A, B, X, kinds, pos, *ev).max() / (n * check.U)
    print(f"stress n={n}: resid/(nu) {res:.3e}")
    assert res <= 100.0


def test_backtransform_emulated_gemm(pevc_lib):
    n = 400
    p, Z, A, B, kinds, pos, ev = _case(n, 4500)
    plan = pevc_lib.Plan(n, prec="fp64", tile=64)
    try:
        V, sc, st = plan.solve(p.S, p.T)
        X, st = plan.backtransform(Z, V, emulated=True, check=False)
    finally:
        plan.close()
    if st == pevc_lib.ERR_UNSUPPORTED:
        pytest.skip("fixed-point FP64 emulation not available in this cuBLAS")
    assert st == 0
    _check(p, Z, A, B, kinds, pos, ev, X)


def test_backtransform_argument_errors(pevc_lib):
    import torch
    n = 64
    p = pencilgen.make_pencil(n, 4600)
    plan = pevc_lib.Plan(n, prec="fp64", tile=32)
    try:
        V, sc, st = plan.solve(p.S, p.T)
        m = V.shape[1]
        buf = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        ptr = buf.data_ptr()
        bt = pevc_lib.pevc_backtransform
        assert bt(None, ptr, n, n, ptr, n, m, None, ptr, n) == -1
        assert bt(plan.h, ptr, n - 1, n, ptr, n, m, None, ptr, n) == -3
        assert bt(plan.h, ptr, n, n + 1, ptr, n + 1, m, None, ptr, n + 1) == -4
        assert bt(plan.h, ptr, n, n, ptr, n, n + 1, None, ptr, n) == -7
        assert bt(plan.h, ptr, n, n, ptr, n, m - 1, None, ptr, n) == -8     # not the last solve's count
        assert bt(plan.h, ptr, n, n, ptr, n, 2, [1, 0], ptr, n) == -8       # a pair without its second column
        assert bt(plan.h, ptr, n, n, ptr, n, m, None, ptr, n, 128) == -11
        assert bt(plan.h, ptr, n, n, ptr, n, 0, None, ptr, n) == 0
    finally:
        plan.close()


def test_backtransform_split_gemm_many_chunks_against_cublas_and_oracle(pevc_lib):
    """n = 1500 (six chunks of 256 along the inner dimension, the last one
    ragged; a selection so that V has columns of every height): the split
    GEMM within its entrywise bound of Z V, within 1e-10 of the oracle after
    normalisation, and faster than cuBLAS's FP64 GEMM on the same call."""
    import time
    import torch
    n = 1500
    sel = (np.arange(n) % 3 != 1).astype(np.int32)
    p, Z, A, B, kinds, pos, ev = _case(n, 4700, select=sel)
    plan = pevc_lib.Plan(n, prec="fp64")
    try:
        V, sc, st = plan.solve(p.S, p.T, select=sel)
        assert st == 0
        X, st = plan.backtransform(Z, V)
        Xr, st2 = plan.backtransform(Z, V, normalise=False)
        Xc, st3 = plan.backtransform(Z, V, normalise=False, cublas=True)
        assert st == 0 and st2 == 0 and st3 == 0
        # timing of the GEMMs alone, device-resident operands
        Zt, Vt = pevc_lib.to_device_colmajor(Z), pevc_lib.to_device_colmajor(V)
        m = V.shape[1]
        Xt = torch.empty((m, n), dtype=torch.float64, device="cuda")
        ms = {}
        for name, fl in (("split", pevc_lib.NO_NORMALISE), ("cublas", pevc_lib.NO_NORMALISE | pevc_lib.BT_CUBLAS)):
            args = (plan.h, Zt.data_ptr(), n, n, Vt.data_ptr(), n, m, [int(k) for k in kinds], Xt.data_ptr(), n, fl)
            assert pevc_lib.pevc_backtransform(*args) == 0
            t0 = time.perf_counter()
            for _ in range(3):
                assert pevc_lib.pevc_backtransform(*args) == 0
            ms[name] = (time.perf_counter() - t0) / 3 * 1e3
    finally:
        plan.close()
    ref = Z @ V
    assert np.all(np.abs(Xr - ref) <= _split_bound(Z, V))
    assert np.max(np.abs(Xc - ref)) <= 1e-12 * np.max(np.abs(ref))
    _check(p, Z, A, B, kinds, pos, ev, X, select=sel)
    print(f"back-transform n={n}, m={V.shape[1]}: split {ms['split']:.2f} ms, cuBLAS FP64 {ms['cublas']:.2f} ms")
    assert ms["split"] < ms["cublas"]
