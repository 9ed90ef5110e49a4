"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

* exact kernels of beta*S - alpha*T over the Gaussian rationals (brute force,
  stored fixtures and fresh tiny pencils);
* the eigenvalues the generator placed (independent of the oracle's formula);
* the properties of ProtectDivision / ProtectUpdate (paper, Section 4),
  checked in exact rational arithmetic;
* special cases that reduce to library routines (T = I, scipy's QZ-based
  generalized eigensolver) and to unit vectors (diagonal pencils);
* the residual bar, conjugate-pair structure and zeros below the tip
  (Section 2, Lemma);
* robustness: on stress pencils the non-robust substitution overflows while
  the oracle stays finite and records growth beyond the binary64 range.
"""
import glob
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check, exact

HERE = os.path.dirname(os.path.abspath(__file__))
OMEGA = Fraction(2) ** 1022


def _real_columns(Vc, kinds):
    n = Vc.shape[0]
    Vr = np.zeros((n, len(kinds)))
    for c, k in enumerate(kinds):
        if k == 0:
            Vr[:, c] = Vc[:, c].real
        elif k == 1:
            Vr[:, c] = Vc[:, c].real
            Vr[:, c + 1] = Vc[:, c].imag
    return Vr


# ---------------------------------------------------------------- exact pins

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(HERE, "golden", "exact_*.txt"))))
def test_oracle_matches_golden_exact(path):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    S, T, block, Vx = mg.load(path)
    st, V, sc, m = oracle.evc(S, T)
    assert st == 0 and m == S.shape[0]
    kinds, pos = check.column_kinds(block)
    err, _ = check.compare_normalised(_real_columns(Vx, kinds), V, kinds)
    assert err <= 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_oracle_matches_fresh_exact(n):
    worst = 0.0
    for seed in range(12):
        ep = pencilgen.exact_pencil(n, 100 + seed)
        S, T = ep.as_float()
        Vx, dims = exact.exact_eigenvectors(ep)
        assert all(d == 1 for d in dims)
        st, V, sc, m = oracle.evc(S, T)
        assert st == 0
        kinds, _ = check.column_kinds(ep.block)
        err, _ = check.compare_normalised(_real_columns(Vx, kinds), V, kinds)
        worst = max(worst, err)
    assert worst <= 1e-13


def test_oracle_first_max_normalisation_exact():
    """The oracle puts exactly 1 at its largest-modulus entry and 0 below the tip."""
    p = pencilgen.config_pencil(0, n=64)
    st, V, sc, m = oracle.evc(p.S, p.T)
    kinds, pos = check.column_kinds(p.block)
    vecs, cols = check.as_complex(V, kinds)
    for z, c in zip(vecs, cols):
        mags = np.abs(z)
        i = int(np.argmax(mags))
        assert z[i] == 1.0
        tip_last = pos[c] + (1 if kinds[c] == 1 else 0)
        assert np.all(z[tip_last + 1:] == 0)


# ------------------------------------------------------------ eigenvalues

def test_eigpairs_match_generated_eigenvalues():
    for seed, stress in ((1, False), (2, True)):
        p = pencilgen.make_pencil(300, seed, stress=stress)
        st, blk, a, b, beta, sigma = oracle.eigpairs(p.S, p.T)
        assert st == 0
        assert np.array_equal(blk, p.block)
        lam = (a + 1j * b) / beta
        first = np.flatnonzero(p.block != 2)
        ref = p.lam_re[first] + 1j * p.lam_im[first]
        assert np.all(np.abs(lam[first] - ref) <= 1e-12 * (1 + np.abs(ref)))
        assert np.all(b[p.block == 1] > 0)
        assert np.all(beta >= 0)


def test_eigpairs_status_codes():
    p = pencilgen.config_pencil(0, n=16)
    i = int(np.flatnonzero(p.block == 1)[0])
    S = p.S.copy(order="F")
    S[i + 1, i] = -S[i + 1, i] * 0 + 1e-30 * np.sign(S[i, i + 1] or 1)  # 2x2 block with real eigenvalues
    S[i, i + 1] = abs(S[i, i + 1])
    S[i + 1, i] = abs(S[i + 1, i])
    st, *_ = oracle.eigpairs(S, p.T)
    assert st == oracle.ERR_NOT_SCHUR
    T = p.T.copy(order="F")
    T[i, i + 1] = 0.5                                            # T_jj not diagonal
    st, *_ = oracle.eigpairs(p.S, T)
    assert st == oracle.ERR_NOT_SCHUR
    S = p.S.copy(order="F")
    S[0, 5] = np.nan
    st, *_ = oracle.eigpairs(S, p.T)
    assert st == oracle.ERR_NONFINITE
    S = p.S.copy(order="F")
    T = p.T.copy(order="F")
    j = int(np.flatnonzero(p.block == 0)[0])
    S[j, j] = 0.0
    T[j, j] = 0.0
    st, V, sc, m = oracle.evc(S, T)
    assert st == oracle.ERR_INDEFINITE


# ------------------------------------------------ ProtectUpdate / Division

def _random_magnitudes(rng, count):
    e = rng.integers(-1074, 1024, size=count)
    m = rng.uniform(0.5, 1.0, size=count)
    vals = np.ldexp(m, e)
    vals = np.where(np.isfinite(vals), vals, np.finfo(float).max)
    return vals


def test_protect_update_properties():
    rng = np.random.default_rng(7)
    ys = _random_magnitudes(rng, 4000)
    ts = _random_magnitudes(rng, 4000)
    xs = _random_magnitudes(rng, 4000)
    edge = [0.0, 5e-324, 2.2250738585072014e-308, 1.0, 2.0 ** 1022, np.finfo(float).max]
    cases = list(zip(ys, ts, xs))
    for y in edge:
        for t in edge:
            for x in edge:
                cases.append((y, t, x))
    for y, t, x in cases:
        k = oracle.protect_upd(y, t, x)
        assert k >= 0
        val = Fraction(y) + Fraction(t) * Fraction(x)
        assert val <= OMEGA * Fraction(2) ** k           # xi (y + t x) <= Omega, xi = 2^-k
        if k > 0:                                        # at most 3 bits beyond the minimum
            assert val > OMEGA * Fraction(2) ** (k - 4)


def test_protect_division_properties():
    rng = np.random.default_rng(8)
    bs = _random_magnitudes(rng, 4000)
    ts = _random_magnitudes(rng, 4000)
    edge = [5e-324, 2.2250738585072014e-308, 1e-200, 1.0, 2.0 ** 1022]
    cases = list(zip(bs, ts)) + [(b, t) for b in edge + [0.0] for t in edge]
    for b, t in cases:
        if b > 2.0 ** 1022:
            continue                                     # precondition |b| <= Omega
        k = oracle.protect_div(b, t)
        assert k >= 0
        assert Fraction(b) <= Fraction(t) * OMEGA * Fraction(2) ** k
        if k > 0:
            assert Fraction(b) > Fraction(t) * OMEGA * Fraction(2) ** (k - 3)


def test_protect_properties_million_samples():
    """The same two properties on 10^6 draws each across the whole binary64
    range (subnormals included), checked in floating point after the exact
    power-of-two scaling: one rounding in the check, hence the 4u slack."""
    rng = np.random.default_rng(10)
    N = 1_000_000
    y, t, x = (_random_magnitudes(rng, N) for _ in range(3))
    zero = rng.random((3, N)) < 0.02                  # some exact zeros
    y[zero[0]] = 0.0
    t[zero[1]] = 0.0
    x[zero[2]] = 0.0
    L = oracle.lib()
    ku = np.fromiter((L.orc_protect_upd(a, b, c) for a, b, c in zip(y.tolist(), t.tolist(), x.tolist())),
                     dtype=np.int64, count=N)
    assert ku.min() >= 0
    # 2^-k (y + t x) <= Omega, with t x formed after scaling t (no overflow)
    lhs = np.ldexp(y, -ku) + np.ldexp(t, -ku) * x
    assert np.all(lhs <= 2.0 ** 1022 * (1 + 4 * 2.0 ** -53))
    # not over-scaled: with k > 0, 2^-(k-4) (y + t x) > Omega
    pos = ku > 0
    with np.errstate(over="ignore"):                  # an overflowing product is above Omega all the same
        big = np.maximum(np.ldexp(y[pos], 4 - ku[pos]), np.ldexp(t[pos], 4 - ku[pos]) * x[pos])
        assert np.all(2 * big > 2.0 ** 1022)
    b = np.minimum(_random_magnitudes(rng, N), 2.0 ** 1022)   # precondition |b| <= Omega
    b[rng.random(N) < 0.02] = 0.0
    d = _random_magnitudes(rng, N)
    kd = np.fromiter((L.orc_protect_div(p_, q_) for p_, q_ in zip(b.tolist(), d.tolist())), dtype=np.int64, count=N)
    assert kd.min() >= 0
    # 2^-k b <= t Omega, compared as 2^-k b / 2^1022 <= t (both sides exact or one rounding)
    assert np.all(np.ldexp(b, -kd - 1022) <= d * (1 + 4 * 2.0 ** -53))
    pos = kd > 0
    assert np.all(np.ldexp(b[pos], 3 - kd[pos] - 1022) > d[pos] * (1 - 4 * 2.0 ** -53))


def test_complex_division_accuracy_and_range():
    rng = np.random.default_rng(9)
    for _ in range(3000):
        a = complex(*np.ldexp(rng.uniform(-1, 1, 2), rng.integers(-250, 250, 2)))
        b = complex(*np.ldexp(rng.uniform(-1, 1, 2), rng.integers(-250, 250, 2)))
        if b == 0:
            continue
        q = oracle.cdiv(a, b)
        # exact quotient in rationals
        ar, ai, br, bi = map(Fraction, (a.real, a.imag, b.real, b.imag))
        d = br * br + bi * bi
        qr = (ar * br + ai * bi) / d
        qi = (ai * br - ar * bi) / d
        mod = math.sqrt(float(qr * qr + qi * qi)) if (qr or qi) else 0.0
        if mod == 0 or not math.isfinite(mod) or mod < 1e-290:
            continue
        err = math.hypot(q.real - float(qr), q.imag - float(qi))
        assert err <= 8 * 2.0 ** -53 * mod
    # extreme operands where the textbook formula overflows or underflows
    q = oracle.cdiv(complex(1e300, 1e300), complex(1e300, 1e-300))
    assert abs(q - complex(1, 1)) < 1e-15
    q = oracle.cdiv(complex(1e-300, 1e-300), complex(1e-300, 2e-300))
    assert abs(q - complex(0.6, -0.2)) < 1e-15


# -------------------------------------------- special cases and invariants

def test_identity_T_reduces_to_standard_eigenproblem():
    import scipy.linalg as sl
    p = pencilgen.config_pencil(0, n=120)
    T = np.asfortranarray(np.eye(p.n))
    S = p.S.copy(order="F")
    # with T = I the diagonal blocks of S carry the eigenvalues directly
    for i in range(p.n):
        if p.block[i] == 0:
            S[i, i] = p.lam_re[i]
        elif p.block[i] == 1:
            mu, nu = p.lam_re[i], p.lam_im[i]
            S[i:i + 2, i:i + 2] = [[mu, nu], [-nu, mu]]
    st, V, sc, m = oracle.evc(S, T)
    assert st == 0
    w, VR = sl.eig(S)
    st, blk, a, b, beta, _ = oracle.eigpairs(S, T)
    kinds, pos = check.column_kinds(blk)
    vecs, cols = check.as_complex(V, kinds)
    worst = 0.0
    for z, c in zip(vecs, cols):
        lam = (a[pos[c]] + 1j * b[pos[c]]) / beta[pos[c]]
        j = int(np.argmin(np.abs(w - lam)))
        zr = VR[:, j]
        i = int(np.argmax(np.abs(z)))
        worst = max(worst, np.abs(zr / zr[i] - z).max())
    assert worst < 1e-8


def test_scipy_generalized_cross_check():
    import scipy.linalg as sl
    p = pencilgen.make_pencil(250, 31)
    st, V, sc, m = oracle.evc(p.S, p.T)
    w, VR = sl.eig(p.S, p.T)
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    vecs, cols = check.as_complex(V, kinds)
    worst = 0.0
    for z, c in zip(vecs, cols):
        lam = (a[pos[c]] + 1j * b[pos[c]]) / beta[pos[c]]
        j = int(np.argmin(np.abs(w - lam)))
        zr = VR[:, j]
        i = int(np.argmax(np.abs(z)))
        worst = max(worst, np.abs(zr / zr[i] - z).max())
    assert worst < 1e-8


def test_diagonal_pencil_gives_unit_vectors():
    n = 9
    S = np.asfortranarray(np.diag(np.arange(1.0, n + 1)))
    T = np.asfortranarray(np.eye(n))
    st, V, sc, m = oracle.evc(S, T)
    assert st == 0
    assert np.array_equal(V, np.eye(n))
    assert np.all(sc == 0)


def test_residual_and_pair_structure():
    for n, seed in ((256, pencilgen.config_seed(0)), (500, 12)):
        p = pencilgen.make_pencil(n, seed)
        st, V, sc, m = oracle.evc(p.S, p.T, nthreads=4)
        assert st == 0 and np.isfinite(V).all()
        st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
        kinds, pos = check.column_kinds(blk)
        res = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta)
        assert res.max() <= 100 * n * check.U
        # the conjugate vector solves the conjugate problem, and [x y] has rank 2
        for c in np.flatnonzero(kinds == 1)[:20]:
            z = V[:, c] - 1j * V[:, c + 1]
            al = complex(a[pos[c]], -b[pos[c]])
            r = beta[pos[c]] * (p.S @ z) - al * (p.T @ z)
            assert np.abs(r).max() <= 100 * n * check.U * (np.abs(p.S).sum(1).max() + abs(al) * np.abs(p.T).sum(1).max())
            sv = np.linalg.svd(V[:, c:c + 2], compute_uv=False)
            assert sv[1] > 1e-8 * sv[0]


def test_selection_matches_full_and_closes_pairs():
    p = pencilgen.config_pencil(0, n=100)
    st, Vfull, scfull, m = oracle.evc(p.S, p.T)
    sel = np.zeros(p.n, dtype=np.int32)
    pairs = np.flatnonzero(p.block == 1)
    ones = np.flatnonzero(p.block == 0)
    sel[ones[::3]] = 1
    sel[pairs[::2] + 1] = 1                       # second row only: the pair is selected
    st, Vs, scs, ms = oracle.evc(p.S, p.T, select=sel)
    assert st == 0
    kinds, pos = check.column_kinds(p.block, sel)
    assert ms == len(kinds)
    expect = []
    for c in range(p.n):
        if p.block[c] == 0 and sel[c]:
            expect.append(c)
        elif p.block[c] == 1 and (sel[c] or sel[c + 1]):
            expect += [c, c + 1]
    assert np.array_equal(Vs, Vfull[:, expect])
    assert np.array_equal(scs, scfull[expect])


def test_unnormalised_output_represents_same_vectors():
    p = pencilgen.config_pencil(0, n=80)
    st, V, sc, m = oracle.evc(p.S, p.T)
    st, W, e, m = oracle.evc(p.S, p.T, normalise=False)
    kinds, _ = check.column_kinds(p.block)
    err, _ = check.compare_normalised(V, W, kinds)
    assert err < 1e-15
    # scale of the normalised output is the growth exponent of the largest entry
    for c, k in enumerate(kinds):
        if k == 0:
            assert sc[c] == e[c] + math.frexp(np.abs(W[:, c]).max())[1] - 1


# --------------------------------------------------------------- stress

def test_stress_plain_overflows_robust_finite():
    p = pencilgen.make_pencil(600, pencilgen.config_seed(2), stress=True)
    st, V, sc, m = oracle.evc(p.S, p.T, nthreads=4)
    assert st == 0
    assert np.isfinite(V).all()
    assert sc.max() > 1023                      # growth beyond the binary64 range is represented
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    res = check.residuals(p.S, p.T, V, kinds, pos, a, b, beta)
    assert res.max() <= 100 * p.n * check.U
    stp, Vp, scp, mp = oracle.evc(p.S, p.T, plain=True, normalise=False)
    assert not np.isfinite(Vp).all()


def test_infinite_eigenvalue_vector():
    ep = pencilgen.exact_pencil(7, 44, two_by_two=False)
    r = 3
    ep.T[r][r] = Fraction(0)
    ep.S[r][r] = Fraction(5, 4)
    S, T = ep.as_float()
    Vx, dims = exact.exact_eigenvectors(ep)
    assert all(d == 1 for d in dims)
    st, V, sc, m = oracle.evc(S, T)
    assert st == 0
    kinds, _ = check.column_kinds(ep.block)
    err, _ = check.compare_normalised(_real_columns(Vx, kinds), V, kinds)
    assert err < 1e-13
    # the vector of the infinite eigenvalue lies in the kernel of T
    assert np.abs(T @ V[:, r]).max() < 1e-14


# ---------------------------------------------------------------------------
# Back-transformation (Section 1): x = Z v is an eigenvector of (A, B) =
# (Q S Z^T, Q T Z^T).  The pins use the residual of the original pencil, which
# does not go through oracle.backtransform.
# ---------------------------------------------------------------------------

def _original_pencil(p, seed):
    from oracle.backtransform import random_orthogonal
    Q = random_orthogonal(p.n, seed)
    Z = random_orthogonal(p.n, seed + 1)
    return Q, Z, Q @ p.S @ Z.T, Q @ p.T @ Z.T


def test_backtransform_gives_eigenvectors_of_original_pencil():
    from oracle.backtransform import backtransform
    p = pencilgen.config_pencil(0, n=60)
    st, Vo, sc, m = oracle.evc(p.S, p.T)
    assert st == 0
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    Q, Z, A, B = _original_pencil(p, 777)
    X = backtransform(Z, Vo, kinds)
    res = check.residuals(A, B, X, kinds, pos, a, b, beta)
    assert res.max() <= 100 * p.n * check.U, res.max() / (p.n * check.U)
    # normalisation: the entry of largest modulus of every eigenvector is exactly 1
    for c, k in enumerate(kinds):
        if k == 0:
            assert np.max(np.abs(X[:, c])) == 1.0
        elif k == 1:
            z = X[:, c] + 1j * X[:, c + 1]
            i = int(np.argmax(np.abs(z)))
            assert z[i] == 1.0


def test_backtransform_planted_transpose_fails_the_residual():
    from oracle.backtransform import backtransform
    p = pencilgen.config_pencil(0, n=60)
    st, Vo, sc, m = oracle.evc(p.S, p.T)
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    Q, Z, A, B = _original_pencil(p, 779)
    X = backtransform(Z.T, Vo, kinds)            # the mistake: Z^T instead of Z
    res = check.residuals(A, B, X, kinds, pos, a, b, beta)
    assert res.max() > 1e-6


def test_backtransform_with_identity_returns_the_vectors():
    from oracle.backtransform import backtransform
    p = pencilgen.config_pencil(0, n=50)
    st, Vo, sc, m = oracle.evc(p.S, p.T)
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, _ = check.column_kinds(blk)
    X = backtransform(np.eye(p.n), Vo, kinds)
    assert np.array_equal(X, Vo)


# ---------------------------------------------------------------------------
# Left eigenvectors: u^H (beta S - alpha T) = 0.  Pinned by the left residual
# (from the definition), exact Gaussian-rational null vectors of
# (beta S - alpha T)^H, the support below the block, and a planted mistake.
# ---------------------------------------------------------------------------

def test_left_oracle_residual_and_support():
    from oracle.left import evc_left
    for n, stress in ((80, False), (60, True)):
        p = pencilgen.make_pencil(n, 880 + n, stress=stress)
        st, U, sc, m = evc_left(p.S, p.T)
        assert st == 0 and m == n
        st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
        kinds, pos = check.column_kinds(blk)
        res = check.left_residuals(p.S, p.T, U, kinds, pos, a, b, beta)
        assert np.isfinite(U).all()
        assert res.max() <= 100 * n * check.U, res.max() / (n * check.U)
        for c, k in enumerate(kinds):
            if k != 2:
                assert np.all(U[:pos[c], c] == 0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_left_oracle_matches_fresh_exact(n):
    from oracle.left import evc_left
    worst = 0.0
    for seed in range(8):
        ep = pencilgen.exact_pencil(n, 300 + seed)
        S, T = ep.as_float()
        Ux, dims = exact.exact_left_eigenvectors(ep)
        assert all(d == 1 for d in dims)
        st, U, sc, m = evc_left(S, T)
        assert st == 0
        kinds, _ = check.column_kinds(ep.block)
        err, _ = check.compare_normalised(_real_columns(Ux, kinds), U, kinds)
        worst = max(worst, err)
    assert worst <= 1e-13


def test_left_oracle_planted_conjugation_fails_the_residual():
    from oracle.left import evc_left
    p = pencilgen.make_pencil(70, 891)
    st, U, sc, m = evc_left(p.S, p.T)
    st, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    kinds, pos = check.column_kinds(blk)
    assert (kinds == 1).any()
    Ubad = U.copy()
    Ubad[:, kinds == 2] *= -1.0          # the mistake: the imaginary part not negated
    res = check.left_residuals(p.S, p.T, Ubad, kinds, pos, a, b, beta)
    assert res[kinds == 1].max() > 1e-6


# ---------------------------------------------------------------------------
# Invariances of the eigenvector problem (pins from the mathematics, which a
# misplaced index, a transposed operand or a mishandled scale would break).
# ---------------------------------------------------------------------------

def test_power_of_two_scaling_of_the_pencil_leaves_the_vectors():
    """(2^a S, 2^b T) has the eigenvalues 2^(a-b) lambda and the same eigenvectors."""
    p = pencilgen.make_pencil(150, 640)
    st, V, sc, m = oracle.evc(p.S, p.T)
    kinds, _ = check.column_kinds(p.block)
    for a, b in ((7, 0), (0, -5), (300, 300), (-200, 100)):
        st2, V2, sc2, m2 = oracle.evc(np.ldexp(p.S, a), np.ldexp(p.T, b))
        assert st2 == 0
        err, _ = check.compare_normalised(V, V2, kinds)
        assert err <= 1e-13, (a, b, err)


def test_diagonal_similarity_maps_the_vectors():
    """(D S D^-1, D T D^-1) with D diagonal has the eigenvectors D v (row i
    scaled by d_i).  A misplaced row index in the update (an off-by-one row,
    say) breaks this; a transposed read, which lands on the zero lower
    triangle, keeps it and is caught by the residual pins instead."""
    p = pencilgen.make_pencil(120, 641)
    rng = np.random.default_rng(642)
    d = np.ldexp(1.0, rng.integers(-6, 7, p.n))        # powers of two: D S D^-1 is exact
    S2 = np.asfortranarray(p.S * d[:, None] / d[None, :])
    T2 = np.asfortranarray(p.T * d[:, None] / d[None, :])
    st, V, sc, m = oracle.evc(p.S, p.T)
    st2, V2, sc2, m2 = oracle.evc(S2, T2)
    assert st == st2 == 0
    kinds, _ = check.column_kinds(p.block)
    err, _ = check.compare_normalised(V2, d[:, None] * V, kinds)
    assert err <= 1e-12


def test_cplx_scalar_multiple_and_conjugation():
    """(c S, c T) for a complex c has the same eigenvectors (beta' S' - alpha' T'
    = c^2 (beta S - alpha T)); (conj S, conj T) has the conjugate ones."""
    p = pencilgen.make_complex_pencil(130, 643)
    st, V, sc, m = oracle.evc_cplx(p.S, p.T)
    c = complex(0.6, -0.8) * 3.0
    st2, V2, _, _ = oracle.evc_cplx(c * p.S, c * p.T)
    st3, V3, _, _ = oracle.evc_cplx(np.conj(p.S), np.conj(p.T))
    assert st == st2 == st3 == 0
    assert check.compare_normalised_cplx(V, V2)[0] <= 1e-12
    assert check.compare_normalised_cplx(np.conj(V), V3)[0] <= 1e-15


def test_cplx_diagonal_similarity_maps_the_vectors():
    p = pencilgen.make_complex_pencil(100, 644)
    rng = np.random.default_rng(645)
    d = np.ldexp(1.0, rng.integers(-6, 7, p.n)) * np.exp(1j * rng.uniform(0, 2 * np.pi, p.n))
    S2 = np.asfortranarray(p.S * d[:, None] / d[None, :])
    T2 = np.asfortranarray(p.T * d[:, None] / d[None, :])
    st, V, sc, m = oracle.evc_cplx(p.S, p.T)
    st2, V2, sc2, m2 = oracle.evc_cplx(S2, T2)
    assert st == st2 == 0
    assert check.compare_normalised_cplx(V2, d[:, None] * V)[0] <= 1e-12


def test_repeated_eigenvalue_needs_the_perturbed_pivot():
    """An eigenvalue repeated exactly makes a pivot of the substitution exactly
    zero; the pivot raised to smin keeps every vector finite and within the
    residual bar (the vector of a pencil perturbed by about u)."""
    ep = pencilgen.exact_pencil(12, 650, two_by_two=False)
    S, T = ep.as_float()
    S[7, 7], T[7, 7] = S[2, 2], T[2, 2]                   # (alpha_7, beta_7) = (alpha_2, beta_2): pivot exactly 0
    st, V, sc, m = oracle.evc(S, T)
    assert st == 0 and np.isfinite(V).all()
    st, blk, a, b, beta, _ = oracle.eigpairs(S, T)
    kinds, pos = check.column_kinds(blk)
    assert check.residuals(S, T, V, kinds, pos, a, b, beta).max() <= 100 * 12 * check.U
    # reading 9: the zero pivot is raised to smin = u (|beta||S_22| + |alpha||T_22|), so the vector grows
    # by about 1/u = 2^53 (a floor of 2^-1022 alone would make it grow by about 2^1022)
    assert 40 <= sc[7] <= 70, sc[7]


def test_huge_entries_need_the_prescaling():
    """Entries near 2^1010: beta S - alpha T would overflow without the
    power-of-two pre-scaling of (alpha, beta); the vectors are those of the
    unscaled pencil."""
    p = pencilgen.make_pencil(90, 651)
    st, V, sc, m = oracle.evc(p.S, p.T)
    st2, V2, sc2, m2 = oracle.evc(np.ldexp(p.S, 1010), np.ldexp(p.T, 1010))
    assert st2 == 0 and np.isfinite(V2).all()
    kinds, _ = check.column_kinds(p.block)
    assert check.compare_normalised(V, V2, kinds)[0] <= 1e-13


def _growth_pencil():
    """n = 3, T = I: x_1 = -S_12 / (lambda_1 - lambda_2) reaches Omega
    (2^600 / 2^-450), and the update of row 0 multiplies it by S_01 = 2^600, the
    largest entry of column 1 above the diagonal, in the row just above it."""
    l2 = 2.0 ** -400
    l1 = l2 * (1.0 + 2.0 ** -50)                          # lambda_1 - lambda_2 = 2^-450, exact
    S = np.array([[0.5, 2.0 ** 600, 0.0], [0.0, l1, 2.0 ** 600], [0.0, 0.0, l2]], order="F")
    return S, np.asfortranarray(np.eye(3))


def test_column_bound_covers_the_row_above_the_diagonal():
    S, T = _growth_pencil()
    st, V, sc, m = oracle.evc(S, T)
    assert st == 0 and np.isfinite(V).all()
    assert sc[2] > 1023                                   # the growth is represented, not overflowed
    st, blk, a, b, beta, _ = oracle.eigpairs(S, T)
    kinds, pos = check.column_kinds(blk)
    assert check.residuals(S, T, V, kinds, pos, a, b, beta).max() <= 100 * 3 * check.U


def test_conditioning_bound_holds_for_an_independent_fp64_method():
    """The conditioning-relative bar of the batched workload's parity test
    (per eigenvector: max(1e-10, 16 * sensitivity to a 2^-52 row-normwise
    perturbation)) admits LAPACK's own eigenvectors (dggev, through scipy),
    a backward-stable FP64 method independent of the oracle, on batched
    pencils whose vectors are among the worse conditioned; and a planted
    error of 1e-8 in one entry is outside it."""
    import scipy.linalg as sl
    orders = pencilgen.batch_orders()
    for b in (478, 1006, 388):
        p = pencilgen.batch_pencil(b, int(orders[b]))
        st, Vo, sco, m = oracle.evc(p.S, p.T, nthreads=os.cpu_count() or 1)
        assert st == 0
        kinds, pos = check.column_kinds(p.block)
        sens = check.perturbation_sensitivity(p.S, p.T, Vo, kinds,
                                              lambda S, T: oracle.evc(S, T, nthreads=os.cpu_count() or 1), 7700 + b)
        bound = np.maximum(1e-10, 16.0 * sens)
        w, VR = sl.eig(p.S, p.T)
        ref, cols = check.as_complex(Vo, kinds)
        lam = p.lam_re + 1j * p.lam_im
        for q, (z, c) in enumerate(zip(ref, cols)):
            x = VR[:, int(np.argmin(np.abs(w - lam[pos[c]])))]
            i = int(np.argmax(np.abs(z)))
            assert np.abs(x / x[i] - z / z[i]).max() <= bound[q], (b, c)
        assert sens.max() < 1e-8
        V2 = Vo.copy()
        V2[0, -1] += 1e-8 * np.abs(V2[:, -1]).max()
        assert check.compare_normalised(Vo, V2, kinds)[1][-1] > bound[-1]
