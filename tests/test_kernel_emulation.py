"""The library's CUDA C++ kernels, run on a CPU model of the CUDA thread model
(tests/emu/), against the oracle.

The emulation compiles the kernel sources and the host driver as host C++
(one host thread per CUDA thread, barriers for __syncthreads, per-warp
exchange slots for shuffles and votes) and calls the library's own C entry
points with host arrays.  It checks the kernels' logic -- index maps, warp
exchanges, scale bookkeeping, the stage walk -- between GPU runs, and covers
code that has not yet run on a GPU.  It is not a parity claim: the GPU tests
are.  The FP64 real path, the split-precision path with its mma.sync update,
the complex path, the back-transform normalisation and the bounded-wait
self-test are covered; the tcgen05 / TMA update is not.
Sizes are small, since every warp exchange is a host barrier.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check
from oracle.backtransform import backtransform, backtransform_cplx
from oracle.left import evc_left_cplx

HERE = os.path.dirname(os.path.abspath(__file__))


def _emu_build():
    import importlib.util
    spec = importlib.util.spec_from_file_location("pevc_emu_build", os.path.join(HERE, "emu", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


vp, ci = ctypes.c_void_p, ctypes.c_int


@pytest.fixture(scope="module")
def emu():
    L = ctypes.CDLL(_emu_build().build())
    L.pevc_plan.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, ctypes.c_uint, vp]
    for f in ("pevc_solve", "pevc_solve_cplx", "pevc_solve_cplx_left"):
        getattr(L, f).argtypes = [vp, vp, ci, vp, ci, ci, vp, vp, ci, vp, ctypes.POINTER(ci)]
    L.pevc_destroy.argtypes = [vp]
    L.emu_bt_normalise.argtypes = [vp, ci, ci, ci, vp]
    L.emu_bt_normalise_c.argtypes = [vp, ci, ci, ci]
    return L


def _call(L, fn, S, T, dtype, tile=32, sel=None, flags=0):
    n = S.shape[0]
    h = vp()
    assert L.pevc_plan(ctypes.byref(h), n, 1, 0, tile, flags, None) == 0
    S = np.asfortranarray(S, dtype=dtype)
    T = np.asfortranarray(T, dtype=dtype)
    V = np.zeros((n, n), dtype=dtype, order="F")
    sc = np.zeros(n, dtype=np.int32)
    m = ci(0)
    s = None if sel is None else np.ascontiguousarray(sel, dtype=np.int32)
    st = getattr(L, fn)(h, S.ctypes.data, n, T.ctypes.data, n, n, None if s is None else s.ctypes.data,
                        V.ctypes.data, n, sc.ctypes.data, ctypes.byref(m))
    L.pevc_destroy(h)
    return st, V[:, :m.value].copy(), sc[:m.value].copy()


def test_emulated_fp64_real_solve_matches_oracle(emu):
    # two tiles of 32 (a ragged last one), real and complex-pair columns, and a selection
    p = pencilgen.make_pencil(45, 9100)
    sel = (np.arange(45) % 3 == 0).astype(np.int32)
    for s in (None, sel):
        st, V, sc = _call(emu, "pevc_solve", p.S, p.T, np.float64, tile=32, sel=s)
        assert st == 0
        ost, Vo, sco, m = oracle.evc(p.S, p.T, select=s)
        _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
        kinds, pos = check.column_kinds(blk, s)
        err, _ = check.compare_normalised(Vo, V, kinds)
        res = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta).max() / (45 * check.U)
        assert V.shape == Vo.shape and err <= 1e-12 and res <= 100.0
        assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)


@pytest.mark.parametrize("n,tile,stress,every", [(70, 32, False, 1), (90, 64, True, 1), (140, 128, False, 3)])
def test_emulated_stage_walk_matches_scheduler_bitwise(emu, n, tile, stress, every):
    """The stage walk (one launch per stage kind, host-ordered) against the
    device-side scheduler (one persistent launch, tasks taken by ticket and
    ordered by ready counters): the updates land in every tile in the same
    order and the kernels' arithmetic is shared, so the same bits, over real
    and complex-pair columns, 1x1 and 2x2 blocks, ragged tiles, stress
    scaling and a selection that leaves partial chunks."""
    p = pencilgen.make_pencil(n, 9700 + n, stress=stress)
    sel = None if every == 1 else (np.arange(n) % every != 1).astype(np.int32)
    st1, V1, sc1 = _call(emu, "pevc_solve", p.S, p.T, np.float64, tile=tile, sel=sel, flags=8)    # PEVC_STAGE_WALK
    st2, V2, sc2 = _call(emu, "pevc_solve", p.S, p.T, np.float64, tile=tile, sel=sel, flags=32)   # PEVC_DEVICE_WALK
    assert st1 == 0 and st2 == 0
    assert np.array_equal(V1, V2) and np.array_equal(sc1, sc2)
    ost, Vo, sco, m = oracle.evc(p.S, p.T, select=sel)
    kinds, _ = check.column_kinds(p.block, sel)
    assert check.compare_normalised(Vo, V1, kinds)[0] <= (1e-6 if stress else 1e-12)


@pytest.mark.parametrize("prec,n,tile,every", [(0, 70, 32, 1), (0, 90, 32, 3), (3, 45, 0, 1)])
def test_emulated_host_solve_matches_device_solve_bitwise(emu, prec, n, tile, every):
    """pevc_solve_host (S and T streamed in by column blocks from the right,
    upper tiles only; each block's pre-pass, slices and tips on its arrival)
    against pevc_solve on the same pencil: the same bits (FP64, and split
    BF16x5 with its mma.sync update), the lower triangles of the host arrays
    filled with garbage the method must not read, a selection, and the bytes
    copied each way."""
    emu.pevc_solve_host.argtypes = [vp, vp, ci, vp, ci, ci, vp, vp, ci, vp, ctypes.POINTER(ci)]
    emu.pevc_last_host_bytes.argtypes = [vp, vp]
    p = pencilgen.make_pencil(n, 9800 + n)
    sel = None if every == 1 else (np.arange(n) % every != 1).astype(np.int32)
    h = vp()
    assert emu.pevc_plan(ctypes.byref(h), n, 1, prec, tile, 0, None) == 0
    S, T = np.asfortranarray(p.S), np.asfortranarray(p.T)
    V1, V2 = np.zeros((n, n), order="F"), np.full((n, n), np.nan, order="F")   # every entry must be written
    sc1, sc2 = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
    m1, m2 = ci(0), ci(0)
    s = None if sel is None else sel.ctypes.data
    st1 = emu.pevc_solve(h, S.ctypes.data, n, T.ctypes.data, n, n, s, V1.ctypes.data, n, sc1.ctypes.data,
                         ctypes.byref(m1))
    # below the subdiagonal: entries the method never reads
    Sg, Tg = S.copy(order="F"), T.copy(order="F")
    low = np.tril(np.ones((n, n), dtype=bool), -2)
    Sg[low] = 7.0e300
    Tg[low] = -3.0e300
    st2 = emu.pevc_solve_host(h, Sg.ctypes.data, n, Tg.ctypes.data, n, n, s, V2.ctypes.data, n, sc2.ctypes.data,
                              ctypes.byref(m2))
    nb = (ctypes.c_longlong * 2)()
    assert emu.pevc_last_host_bytes(h, nb) == 0
    emu.pevc_destroy(h)
    assert st1 == 0 and st2 == 0 and m1.value == m2.value
    m = m1.value
    assert np.array_equal(V1[:, :m], V2[:, :m]) and np.array_equal(sc1[:m], sc2[:m])
    # upper tiles only: between the upper triangle and the whole matrix, both S and T
    assert n * (n + 1) * 8 <= nb[0] <= 2 * n * n * 8
    # V: the rows above each column tile's end (the zeros below are written on the host)
    assert m * 8 <= nb[1] - m * 4 <= m * n * 8


def test_emulated_complex_solve_matches_oracle(emu):
    # two tiles of 64 (the second ragged), then a stress pencil in one tile
    for n, seed, stress in ((65, 9200, False), (40, 9201, True)):
        p = pencilgen.make_complex_pencil(n, seed, stress=stress)
        st, V, sc = _call(emu, "pevc_solve_cplx", p.S, p.T, np.complex128)
        assert st == 0 and np.isfinite(V).all()
        ost, Vo, sco, m = oracle.evc_cplx(p.S, p.T)
        err, _ = check.compare_normalised_cplx(Vo, V)
        res = check.cplx_residuals(p.S, p.T, V, np.diag(p.S), np.diag(p.T)).max() / (n * check.U)
        assert err <= 1e-12 and res <= 100.0
        assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)


def test_emulated_complex_left_solve_matches_oracle(emu):
    n = 70
    p = pencilgen.make_complex_pencil(n, 9300)
    sel = (np.arange(n) % 4 != 1).astype(np.int32)
    st, U, sc = _call(emu, "pevc_solve_cplx_left", p.S, p.T, np.complex128, sel=sel)
    assert st == 0
    ost, Uo, sco, m = evc_left_cplx(p.S, p.T, select=sel)
    assert U.shape == Uo.shape
    err, _ = check.compare_normalised_cplx(Uo, U)
    idx = np.flatnonzero(sel)
    res = check.cplx_left_residuals(p.S, p.T, U, np.diag(p.S)[idx], np.diag(p.T)[idx]).max() / (n * check.U)
    assert err <= 1e-12 and res <= 100.0
    assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)


def test_emulated_complex_stress_over_several_tiles(emu):
    """Two tiles with the off-diagonal tile scaled by 1e100 and T's diagonal
    by 2^-40: the updates consolidate segments of different exponents, guard
    the right update and protect the left one, and the post-pass brings every
    column to one power of two -- all visible in the scale exponents."""
    p = pencilgen.make_complex_pencil(100, 9900, stress=True, big_frac=1.0)
    st, V, sc = _call(emu, "pevc_solve_cplx", p.S, p.T, np.complex128)
    assert st == 0 and np.isfinite(V).all()
    ost, Vo, sco, m = oracle.evc_cplx(p.S, p.T)
    assert sco.max() > 1023
    err, _ = check.compare_normalised_cplx(Vo, V)
    res = check.cplx_residuals(p.S, p.T, V, np.diag(p.S), np.diag(p.T)).max() / (100 * check.U)
    assert err <= 1e-12 and res <= 100.0
    assert np.all(np.abs(sc.astype(np.int64) - sco.astype(np.int64)) <= 1)


def test_emulated_complex_repeated_eigenvalue(emu):
    """An exactly repeated eigenvalue: the zero pivot is raised to smin, so the
    vector is finite and grows by about 1/u, as in the oracle."""
    ep = pencilgen.exact_complex_pencil(10, 652)
    S, T = ep.as_complex()
    S[6, 6], T[6, 6] = S[1, 1], T[1, 1]
    st, V, sc = _call(emu, "pevc_solve_cplx", S, T, np.complex128)
    assert st == 0 and np.isfinite(V).all()
    ost, Vo, sco, m = oracle.evc_cplx(S, T)
    assert 40 <= sc[6] <= 70 and abs(int(sc[6]) - int(sco[6])) <= 1
    assert check.cplx_residuals(S, T, V, np.diag(S), np.diag(T)).max() <= 100 * 10 * check.U


@pytest.mark.parametrize("big", [1.0, 1e200, 2.0 ** 1020])
def test_emulated_backtransform_normalisation(emu, big):
    """The entry of largest modulus becomes exactly 1, also for columns whose
    squared modulus would overflow (unnormalised inputs reach 2^1022)."""
    rng = np.random.default_rng(9400)
    n, m = 300, 4
    X = np.asfortranarray(rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) * big
    X[:, 2] = 0.0                                          # an all-zero column stays zero
    Y = X.copy(order="F")
    emu.emu_bt_normalise_c(Y.ctypes.data, n, n, m)
    assert np.abs(Y - backtransform_cplx(np.eye(n), X)).max() <= 1e-15
    R = np.asfortranarray(np.stack([X[:, 0].real, X[:, 0].imag, X[:, 1].real, X[:, 2].real], axis=1))
    kinds = [1, 2, 0, 0]
    k = np.asarray(kinds, dtype=np.int8)
    Rr = R.copy(order="F")
    emu.emu_bt_normalise(Rr.ctypes.data, n, n, m, k.ctypes.data)
    assert np.abs(Rr - backtransform(np.eye(n), R, kinds)).max() <= 1e-15


def test_emulated_watchdog_selftest(emu):
    """The bounded-wait self-test on the modelled mbarrier: the wait completes
    when the arrival happens and gives up with ERR_TIMEOUT when it is withheld;
    a solve on the same plan afterwards is unaffected."""
    emu.pevc_watchdog_selftest.argtypes = [vp, ci, ctypes.c_longlong]
    h = vp()
    assert emu.pevc_plan(ctypes.byref(h), 40, 1, 0, 32, 0, None) == 0
    try:
        assert emu.pevc_watchdog_selftest(h, 0, 2_000_000) == 0
        assert emu.pevc_watchdog_selftest(h, 1, 2_000_000) == 4          # PEVC_ERR_TIMEOUT
        assert emu.pevc_watchdog_selftest(h, 2, 10) == -2
        assert emu.pevc_watchdog_selftest(h, 1, 0) == -3
    finally:
        emu.pevc_destroy(h)
    p = pencilgen.make_pencil(24, 9500)
    st, V, sc = _call(emu, "pevc_solve", p.S, p.T, np.float64)
    assert st == 0 and np.isfinite(V).all()


def _check_real(p, V, sc, sel=None):
    ost, Vo, sco, m = oracle.evc(p.S, p.T, select=sel)
    _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk, sel)
    err, _ = check.compare_normalised(Vo, V, kinds)
    res = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta).max() / (p.n * check.U)
    assert V.shape == Vo.shape and err <= 1e-12 and res <= 100.0


def test_emulated_real_left_static_and_batched_entry_points(emu):
    """The host logic of three more entry points, on the emulated kernels:
    left eigenvectors (flips and output permutation), the no-allocation solve
    (its one file-scope workspace), and the batched solve (child workspaces,
    per-pencil statuses, one pencil with an error among good ones)."""
    from oracle.left import evc_left
    p = pencilgen.make_pencil(40, 9600)
    # left eigenvectors
    emu.pevc_solve_left.argtypes = [vp, vp, ci, vp, ci, ci, vp, vp, ci, vp, ctypes.POINTER(ci)]
    st, U, sc = _call(emu, "pevc_solve_left", p.S, p.T, np.float64)
    assert st == 0
    ost, Uo, sco, m = evc_left(p.S, p.T)
    _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    err, _ = check.compare_normalised(Uo, U, kinds)
    assert U.shape == Uo.shape and err <= 1e-12
    assert check.left_residuals(p.S, p.T, U, kinds, pos, a, b, beta).max() <= 100 * 40 * check.U
    # the no-allocation solve
    emu.pevc_solve_static.argtypes = [vp, ci, vp, ci, ci, vp, vp, ci, vp, ctypes.POINTER(ci), ctypes.c_uint, vp]
    S, T = np.asfortranarray(p.S), np.asfortranarray(p.T)
    V = np.zeros((40, 40), order="F")
    scs = np.zeros(40, dtype=np.int32)
    m = ci(0)
    emu.emu_alloc_count.restype = ctypes.c_longlong
    allocs = emu.emu_alloc_count()
    # n = 0 is the set-up call (it only looks up the static workspace)
    assert emu.pevc_solve_static(None, 1, None, 1, 0, None, None, 1, None, ctypes.byref(m), 0, None) == 0
    assert emu.pevc_solve_static(S.ctypes.data, 40, T.ctypes.data, 40, 40, None, V.ctypes.data, 40,
                                 scs.ctypes.data, ctypes.byref(m), 0, None) == 0
    assert emu.emu_alloc_count() == allocs            # no cudaMalloc / cudaMallocHost on this path
    _check_real(p, V[:, :m.value], scs[:m.value])
    assert emu.emu_alloc_count() == allocs
    # the batched solve: three pencils of different orders, the middle one not in Schur form
    pens = [pencilgen.make_pencil(n, 9610 + n) for n in (20, 33, 47)]
    Sb = [np.asfortranarray(q.S) for q in pens]
    Tb = [np.asfortranarray(q.T) for q in pens]
    # two adjacent 1x1 blocks become the 2x2 block S = [[0, 1], [1, 0]], T = I: real eigenvalues +-1
    c = next(int(r) for r in range(32) if pens[1].block[r] == 0 and pens[1].block[r + 1] == 0)
    Sb[1][c:c + 2, c:c + 2] = [[0.0, 1.0], [1.0, 0.0]]
    Tb[1][c:c + 2, c:c + 2] = np.eye(2)
    Vb = [np.zeros((q.n, q.n), order="F") for q in pens]
    scb = [np.zeros(q.n, dtype=np.int32) for q in pens]
    P, I = vp * 3, ci * 3
    emu.pevc_solve_batched.argtypes = [vp, ci, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    h = vp()
    assert emu.pevc_plan(ctypes.byref(h), 47, 3, 0, 32, 0, None) == 0
    mo, so = I(), I()
    st = emu.pevc_solve_batched(h, 3, P(*[x.ctypes.data for x in Sb]), I(20, 33, 47),
                                P(*[x.ctypes.data for x in Tb]), I(20, 33, 47), I(20, 33, 47), None,
                                P(*[x.ctypes.data for x in Vb]), I(20, 33, 47), P(*[x.ctypes.data for x in scb]),
                                mo, so)
    emu.pevc_destroy(h)
    assert st == 0
    assert so[0] == 0 and so[2] == 0 and so[1] == 1          # PEVC_ERR_NOT_SCHUR for the middle pencil only
    for q, Vq, sq, mq in ((pens[0], Vb[0], scb[0], mo[0]), (pens[2], Vb[2], scb[2], mo[2])):
        _check_real(q, Vq[:, :mq], sq[:mq])


# PEVC_SPLIT_BF16X5; PEVC_SPLIT_BF16X3 and PEVC_SPLIT_FP8X4 (+ correction);
# PEVC_SPLIT_FP8X4 with PEVC_NO_CORRECTION (about 15 bits)
@pytest.mark.parametrize("prec,n,flags,tol", [(3, 45, 0, 1e-8), (1, 36, 0, 1e-8), (2, 40, 0, 1e-8), (2, 40, 2, 1e-5)])
def test_emulated_split_solve_matches_oracle(emu, prec, n, flags, tol):
    """The split-precision path with its mma.sync update (BF16 or E4M3 slices,
    FP32 level accumulators, FP64 recombination), the slicing kernels it
    shares with the tcgen05 update, and the correction sweep of BF16x3 and
    FP8x4 (residual in BF16x5)."""
    p = pencilgen.make_pencil(n, 9800 + n)
    h = vp()
    assert emu.pevc_plan(ctypes.byref(h), n, 1, prec, 32, flags, None) == 0
    S, T = np.asfortranarray(p.S), np.asfortranarray(p.T)
    V = np.zeros((n, n), order="F")
    sc = np.zeros(n, dtype=np.int32)
    m = ci(0)
    st = emu.pevc_solve(h, S.ctypes.data, n, T.ctypes.data, n, n, None, V.ctypes.data, n, sc.ctypes.data,
                        ctypes.byref(m))
    emu.pevc_destroy(h)
    assert st == 0 and np.isfinite(V).all()
    ost, Vo, sco, mo = oracle.evc(p.S, p.T)
    _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    err, _ = check.compare_normalised(Vo, V[:, :m.value], kinds)
    res = check.residuals(p.S, p.T, V[:, :m.value], kinds, pos, a, b, beta).max() / (n * check.U)
    print(f"emulated split prec {prec} flags {flags}: err {err:.3e} resid/(nu) {res:.3e}")
    assert err <= tol and (res <= 100.0 or flags)


def test_epilogue_and_protection_helpers(emu):
    """The scalar helpers the tcgen05 epilogue and the protection are built
    from (common.cuh), compiled as host code, against exact rational
    arithmetic: the int64 -> binary64 assembly rounds to nearest, ties to even,
    the power-of-two scalings are exact, and the exponent bounds bound."""
    from fractions import Fraction
    cd, cll = ctypes.c_double, ctypes.c_longlong
    f = emu
    f.emu_i64_scaled_fast.argtypes = [cll, ci, ctypes.POINTER(ci)]
    f.emu_i64_scaled_fast.restype = cd
    f.emu_i64_scaled.argtypes = [cll, ci]
    f.emu_i64_scaled.restype = cd
    f.emu_pow2_scale_fast.argtypes = [cd, ci, ctypes.POINTER(ci)]
    f.emu_pow2_scale_fast.restype = cd
    f.emu_pow2_scale.argtypes = [cd, ci]
    f.emu_pow2_scale.restype = cd
    f.emu_exp_ub.argtypes = [cd]
    for name in ("emu_protect_update", "emu_protect_update_ub"):
        getattr(f, name).argtypes = [cd, cd, cd]
    f.emu_protect_division.argtypes = [cd, ci, cd]
    f.emu_max_nonneg.argtypes = [cd, cd]
    f.emu_max_nonneg.restype = cd
    rng = np.random.default_rng(9950)
    OMEGA = Fraction(2) ** 1022
    slow = ci(0)
    ties = [(2 ** 53 + 1) << s for s in (1, 3, 9)] + [(2 ** 53 + 3) << 1, -((2 ** 54 + 2) << 2) - 4]
    ts = [int(x) for x in (rng.integers(-2 ** 62, 2 ** 62, 3000) >> rng.integers(0, 62, 3000))] + ties + [0, 1, -1]
    for t in ts:
        for e in (int(rng.integers(-1140, 1040)), int(rng.integers(-60, 60))):
            exact = Fraction(t) * Fraction(2) ** e
            r = f.emu_i64_scaled_fast(t, e, ctypes.byref(slow))
            big = exact != 0 and (abs(exact) < Fraction(2) ** -1022 or abs(exact) >= Fraction(2) ** 1024)
            if slow.value == 0:
                assert r == float(exact), (t, e)        # correctly rounded, ties to even
            else:
                assert big or abs(exact) < Fraction(2) ** -1021
            if Fraction(2) ** -1022 <= abs(exact) < Fraction(2) ** 1023:
                assert f.emu_i64_scaled(t, e) == float(exact)
    ys = np.concatenate([_ldexp_samples(rng, 2000), [0.0, -0.0, 5e-324, -2.2250738585072014e-308]])
    for y in ys.tolist():
        sh = int(rng.integers(-1100, 1100))
        r = f.emu_pow2_scale_fast(y, sh, ctypes.byref(slow))
        if slow.value == 0:
            assert r == math_ldexp(y, sh)
        assert f.emu_pow2_scale(y, sh) == math_ldexp(y, sh)
        if y != 0 and np.isfinite(y):
            eu = f.emu_exp_ub(y)
            assert abs(y) < 2.0 ** eu if eu < 1024 else True
            if abs(y) >= 2.2250738585072014e-308:
                assert eu == np.frexp(abs(y))[1]
    for _ in range(3000):
        y, t, x = (abs(float(v)) for v in _ldexp_samples(rng, 3))
        for fn in ("emu_protect_update", "emu_protect_update_ub"):
            k = getattr(f, fn)(y, t, x)
            assert k >= 0 and Fraction(y) + Fraction(t) * Fraction(x) <= OMEGA * Fraction(2) ** k
        b, tt, sh = min(abs(y), 2.0 ** 1000), max(t, 2.0 ** -1000), int(rng.integers(0, 6))
        kd = f.emu_protect_division(b, sh, tt)
        assert kd >= 0 and Fraction(b) * Fraction(2) ** sh <= Fraction(tt) * OMEGA * Fraction(2) ** kd
        assert f.emu_max_nonneg(y, t) == max(y, t)


def _ldexp_samples(rng, count):
    """Signed magnitudes spread over the whole binary64 range, subnormals included."""
    v = np.ldexp(rng.uniform(0.5, 1.0, count), rng.integers(-1074, 1024, count))
    v = np.where(np.isfinite(v), v, 1.0)
    return v * rng.choice([-1.0, 1.0], count)


def math_ldexp(x, e):
    import math
    try:
        return math.ldexp(x, e)
    except OverflowError:
        return math.copysign(float("inf"), x)


def test_epilogue_flush_helpers(emu):
    """The correction sweeps' product helpers (update_tc.cu): a scaled product
    t 2^e in the normal range is the correctly rounded value, as on the fast
    path; one whose magnitude is below 2^-1022 becomes a zero of its sign
    without the exact path; overflow still asks for the exact path."""
    from fractions import Fraction
    cd, cll = ctypes.c_double, ctypes.c_longlong
    emu.emu_i64_scaled_ftz.argtypes = [cll, ci, ctypes.POINTER(ci)]
    emu.emu_i64_scaled_ftz.restype = cd
    emu.emu_pow2_scale_ftz.argtypes = [cd, ci, ctypes.POINTER(ci)]
    emu.emu_pow2_scale_ftz.restype = cd
    rng = np.random.default_rng(9960)
    slow = ci(0)
    tiny, huge = Fraction(2) ** -1022, Fraction(2) ** 1024
    ts = [int(x) for x in (rng.integers(-2 ** 62, 2 ** 62, 2000) >> rng.integers(0, 62, 2000))] + [0, 1, -1, 2 ** 53 + 1]
    seen = {"normal": 0, "flushed": 0, "overflow": 0}
    for t in ts:
        for e in (int(rng.integers(-1140, 1040)), int(rng.integers(-1100, -1000)), int(rng.integers(-60, 60))):
            exact = Fraction(t) * Fraction(2) ** e
            r = emu.emu_i64_scaled_ftz(t, e, ctypes.byref(slow))
            if t != 0 and abs(exact) < tiny:
                assert r == 0.0 and math.copysign(1.0, r) == math.copysign(1.0, t) and slow.value == 0, (t, e)
                seen["flushed"] += 1
            elif abs(exact) >= huge:
                assert slow.value == 1, (t, e)
                seen["overflow"] += 1
            elif slow.value == 0:
                assert r == float(exact), (t, e)         # correctly rounded, as the fast path
                seen["normal"] += 1
            else:
                assert abs(exact) >= Fraction(2) ** 1023   # rounds up into overflow
            if t != 0:
                y = float(t)
                ey = Fraction(y) * Fraction(2) ** e
                ry = emu.emu_pow2_scale_ftz(y, e, ctypes.byref(slow))
                if abs(ey) < tiny:
                    assert ry == 0.0 and math.copysign(1.0, ry) == math.copysign(1.0, y) and slow.value == 0
                elif abs(ey) >= huge:
                    assert slow.value == 1
                else:
                    assert ry == float(ey) and slow.value == 0
    assert min(seen.values()) > 20, seen


def test_emulated_split_backtransform_gemm(emu):
    """The split back-transformation GEMM (slices of Z per row and of V per
    column, per chunk of 256, BF16 mma.sync, exact level sums, FP64 chunk
    sums) on the emulation: two chunks, the second ragged, columns of every
    height; X within the entrywise bound the slicing implies."""
    import sys
    sys.path.insert(0, HERE)
    from test_gpu_backtransform import _split_bound
    from oracle.backtransform import random_orthogonal
    n, m = 270, 40
    p = pencilgen.make_pencil(n, 4950)
    st, V, sc, mm = oracle.evc(p.S, p.T)
    V = np.asfortranarray(V[:, ::7][:, :m])          # columns of heights spread over both chunks
    m = V.shape[1]
    Z = np.asfortranarray(random_orthogonal(n, 4951))
    X = np.zeros((n, m), order="F")
    emu.pevc_backtransform.argtypes = [vp, vp, ci, ci, vp, ci, ci, vp, vp, ci, ctypes.c_uint]
    h = vp()
    assert emu.pevc_plan(ctypes.byref(h), n, 1, 0, 32, 0, None) == 0
    kinds = (ci * m)(*[0] * m)
    rc = emu.pevc_backtransform(h, Z.ctypes.data, n, n, V.ctypes.data, n, m, kinds, X.ctypes.data, n, 1)
    emu.pevc_destroy(h)
    assert rc == 0
    assert np.all(np.abs(X - Z @ V) <= _split_bound(Z, V))
