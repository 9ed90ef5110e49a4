"""Pins of the complex-pencil oracle (the extension to complex data types that
the paper names in Section 7) against facts fixed outside the oracle:

* exact kernels of beta*S - alpha*T over the Gaussian rationals (stored
  fixtures and fresh tiny pencils, including an infinite eigenvalue);
* a real triangular pencil passed as complex reduces to the real oracle's
  1x1-block path, and T = I or a diagonal pencil reduce to library routines
  and unit vectors;
* scipy's QZ-based generalized eigensolver on generated complex pencils;
* the residual bar, zeros below the tip, selection and unnormalised output;
* robustness: on stress pencils the non-robust substitution overflows while
  the oracle stays finite and records growth beyond the binary64 range;
* planted mistakes (a conjugated vector, a transposed operand) fail the
  residual check, so it can catch them.
"""
import glob
import importlib.util
import math
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check, exact

HERE = os.path.dirname(os.path.abspath(__file__))
BAR = 100 * check.U


def _golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def _diag(S, T):
    return np.diag(S).copy(), np.diag(T).copy()


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(HERE, "golden", "cexact_*.txt"))))
def test_cplx_oracle_matches_golden_exact(path):
    S, T, Vx = _golden().load_cplx(path)
    st, V, sc, m = oracle.evc_cplx(S, T)
    assert st == 0 and m == S.shape[0]
    err, _ = check.compare_normalised_cplx(Vx, V)
    assert err <= 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_cplx_oracle_matches_fresh_exact(n):
    worst = 0.0
    for seed in range(10):
        ep = pencilgen.exact_complex_pencil(n, 300 + seed, infinite=(seed % 3 == 2))
        S, T = ep.as_complex()
        Vx, dims = exact.exact_complex_eigenvectors(ep)
        assert all(d == 1 for d in dims)
        st, V, sc, m = oracle.evc_cplx(S, T)
        assert st == 0
        err, _ = check.compare_normalised_cplx(Vx, V)
        worst = max(worst, err)
        # first-maximum normalisation: the exact vector's entry of largest
        # modulus is exactly 1 in the oracle's output too (when it is unique)
        for c in range(n):
            a = np.abs(Vx[:, c])
            if np.sum(a == a.max()) == 1:
                assert V[int(np.argmax(a)), c] == 1.0
    assert worst <= 1e-13


def test_cplx_infinite_eigenvalue_lies_in_kernel_of_T():
    ep = pencilgen.exact_complex_pencil(7, 77, infinite=True)
    S, T = ep.as_complex()
    st, V, sc, m = oracle.evc_cplx(S, T)
    assert st == 0
    assert np.abs(T @ V[:, -1]).max() < 1e-14
    assert V[-1, -1] != 0


def test_real_pencil_as_complex_matches_real_oracle():
    ep = pencilgen.exact_pencil(60, 8, two_by_two=False)
    S, T = ep.as_float()
    st, Vr, scr, m = oracle.evc(S, T)
    assert st == 0
    st, Vc, scc, mc = oracle.evc_cplx(S.astype(complex), T.astype(complex))
    assert st == 0 and mc == m
    assert np.all(Vc.imag == 0)
    assert np.abs(Vc.real - Vr).max() <= 1e-13
    assert np.all(np.abs(scc.astype(np.int64) - scr.astype(np.int64)) <= 1)


def test_cplx_identity_T_reduces_to_standard_eigenproblem():
    import scipy.linalg as sl
    p = pencilgen.make_complex_pencil(150, 61)
    S = p.S.copy(order="F")
    S[np.arange(p.n), np.arange(p.n)] = p.lam
    T = np.asfortranarray(np.eye(p.n, dtype=complex))
    st, V, sc, m = oracle.evc_cplx(S, T)
    assert st == 0
    w, VR = sl.eig(S)
    worst = 0.0
    for c in range(p.n):
        j = int(np.argmin(np.abs(w - p.lam[c])))
        z = V[:, c]
        i = int(np.argmax(np.abs(z)))
        worst = max(worst, np.abs(VR[:, j] / VR[i, j] - z).max())
    assert worst < 1e-8


def test_cplx_scipy_generalized_cross_check():
    import scipy.linalg as sl
    p = pencilgen.make_complex_pencil(200, 62)
    st, V, sc, m = oracle.evc_cplx(p.S, p.T, nthreads=4)
    assert st == 0
    w, VR = sl.eig(p.S, p.T)
    worst = 0.0
    for c in range(p.n):
        j = int(np.argmin(np.abs(w - p.lam[c])))
        assert abs(w[j] - p.lam[c]) < 1e-8 * max(1.0, abs(p.lam[c]))
        z = V[:, c]
        i = int(np.argmax(np.abs(z)))
        worst = max(worst, np.abs(VR[:, j] / VR[i, j] - z).max())
    assert worst < 1e-8


def test_cplx_diagonal_pencil_gives_unit_vectors():
    n = 7
    d = np.arange(1, n + 1) * (1 + 1j)
    S = np.asfortranarray(np.diag(d))
    T = np.asfortranarray(np.diag(np.full(n, 2.0 - 1j)))
    st, V, sc, m = oracle.evc_cplx(S, T)
    assert st == 0
    assert np.array_equal(V, np.eye(n, dtype=complex))
    assert np.all(sc == 0)


def test_cplx_eigpairs_are_the_scaled_diagonal():
    p = pencilgen.make_complex_pencil(64, 63)
    st, alpha, beta, sigma = oracle.eigpairs_cplx(p.S, p.T)
    assert st == 0 and np.all(sigma == 0)
    assert np.array_equal(alpha, np.diag(p.S)) and np.array_equal(beta, np.diag(p.T))
    big = p.S * 2.0 ** 900
    st, alpha, beta, sigma = oracle.eigpairs_cplx(big, p.T)
    assert st == 0 and sigma.min() > 0
    for c in range(p.n):
        assert alpha[c] == big[c, c] * 2.0 ** -int(sigma[c])
        assert beta[c] == p.T[c, c] * 2.0 ** -int(sigma[c])
        # max(|beta|, |alpha|) * max entry <= 2^1000 with |.| = |re| + |im|
        mag = lambda z: abs(z.real) + abs(z.imag)   # noqa: E731
        mx = max(np.max(np.abs(big.real) + np.abs(big.imag)), 1.0)
        assert max(mag(alpha[c]), mag(beta[c])) * mx <= 2.0 ** 1000


def test_cplx_residual_and_support():
    for n, seed in ((256, 64), (500, 65)):
        p = pencilgen.make_complex_pencil(n, seed)
        st, V, sc, m = oracle.evc_cplx(p.S, p.T, nthreads=4)
        assert st == 0 and np.isfinite(V).all()
        a, b = _diag(p.S, p.T)
        res = check.cplx_residuals(p.S, p.T, V, a, b)
        assert res.max() <= BAR * n
        for c in range(n):
            assert np.all(V[c + 1:, c] == 0) and V[c, c] != 0


def test_cplx_selection_matches_full():
    p = pencilgen.make_complex_pencil(90, 66)
    st, Vf, scf, m = oracle.evc_cplx(p.S, p.T)
    sel = (np.arange(p.n) % 3 == 1).astype(np.int32)
    st, Vs, scs, ms = oracle.evc_cplx(p.S, p.T, select=sel)
    assert st == 0 and ms == int(sel.sum())
    idx = np.flatnonzero(sel)
    assert np.array_equal(Vs, Vf[:, idx]) and np.array_equal(scs, scf[idx])
    st, V0, sc0, m0 = oracle.evc_cplx(p.S, p.T, select=np.zeros(p.n, dtype=np.int32))
    assert st == 0 and m0 == 0


def test_cplx_unnormalised_output_represents_same_vectors():
    p = pencilgen.make_complex_pencil(80, 67)
    st, V, sc, m = oracle.evc_cplx(p.S, p.T)
    st, W, e, m = oracle.evc_cplx(p.S, p.T, normalise=False)
    err, _ = check.compare_normalised_cplx(V, W)
    assert err < 1e-15
    for c in range(p.n):
        assert sc[c] == e[c] + math.frexp(np.abs(W[:, c]).max())[1] - 1


def test_cplx_stress_plain_overflows_robust_finite():
    p = pencilgen.make_complex_pencil(600, 68, stress=True)
    st, V, sc, m = oracle.evc_cplx(p.S, p.T, nthreads=4)
    assert st == 0
    assert np.isfinite(V).all()
    assert sc.max() > 1023
    a, b = _diag(p.S, p.T)
    res = check.cplx_residuals(p.S, p.T, V, a, b)
    assert res.max() <= BAR * p.n
    stp, Vp, scp, mp = oracle.evc_cplx(p.S, p.T, plain=True, normalise=False)
    assert not np.isfinite(Vp).all()


def test_cplx_planted_mistakes_fail_the_residual():
    p = pencilgen.make_complex_pencil(120, 69)
    st, V, sc, m = oracle.evc_cplx(p.S, p.T)
    a, b = _diag(p.S, p.T)
    assert check.cplx_residuals(p.S, p.T, V, a, b).max() <= BAR * p.n
    # conjugated vectors (a sign error in the imaginary parts)
    assert check.cplx_residuals(p.S, p.T, np.conj(V), a, b)[10:].min() > 1e-6
    # the vectors of the transposed pencil
    St, Tt = np.asfortranarray(p.S.T[::-1, ::-1]), np.asfortranarray(p.T.T[::-1, ::-1])
    st, Vt, _, _ = oracle.evc_cplx(St, Tt)
    assert check.cplx_residuals(p.S, p.T, Vt[::-1, ::-1], a, b)[10:].min() > 1e-6


def test_cplx_status_codes():
    p = pencilgen.make_complex_pencil(20, 70)
    S = p.S.copy(order="F")
    S[3, 9] = np.nan
    assert oracle.evc_cplx(S, p.T)[0] == oracle.ERR_NONFINITE
    S = p.S.copy(order="F")
    S[9, 3] = np.nan                   # below the diagonal: never read
    assert oracle.evc_cplx(S, p.T)[0] == 0
    S = p.S.copy(order="F")
    T = p.T.copy(order="F")
    S[5, 5] = 0
    T[5, 5] = 0
    assert oracle.evc_cplx(S, T)[0] == oracle.ERR_INDEFINITE
    sel = np.ones(20, dtype=np.int32)
    sel[5] = 0                          # the singular entry not selected
    st, V, sc, m = oracle.evc_cplx(S, T, select=sel)
    assert st == 0 and m == 19
    assert oracle.evc_cplx(np.zeros((0, 0), complex), np.zeros((0, 0), complex))[0] == 0


# ---------------------------------------------------------------------------
# Left eigenvectors of complex pencils: pinned by the left residual from the
# definition (no flip), exact null vectors of (beta S - alpha T)^H over the
# Gaussian rationals, the support above the tip, and a planted conjugation.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_cplx_left_oracle_matches_fresh_exact(n):
    from oracle.left import evc_left_cplx
    worst = 0.0
    for seed in range(8):
        ep = pencilgen.exact_complex_pencil(n, 500 + seed, infinite=(seed % 4 == 3))
        S, T = ep.as_complex()
        Ux, dims = exact.exact_complex_left_eigenvectors(ep)
        assert all(d == 1 for d in dims)
        st, U, sc, m = evc_left_cplx(S, T)
        assert st == 0 and m == n
        err, _ = check.compare_normalised_cplx(Ux, U)
        worst = max(worst, err)
    assert worst <= 1e-13


def test_cplx_left_oracle_residual_support_selection():
    from oracle.left import evc_left_cplx
    for n, stress in ((150, False), (300, True)):
        p = pencilgen.make_complex_pencil(n, 510 + n, stress=stress)
        st, U, sc, m = evc_left_cplx(p.S, p.T, nthreads=4)
        assert st == 0 and m == n and np.isfinite(U).all()
        a, b = _diag(p.S, p.T)
        res = check.cplx_left_residuals(p.S, p.T, U, a, b)
        assert res.max() <= BAR * n
        for c in range(n):
            assert np.all(U[:c, c] == 0)
            # the tip itself survives normalisation unless the growth exceeds the binary64 range
            assert U[c, c] != 0 or (stress and sc[c] > 1074)
    sel = (np.arange(n) % 4 == 2).astype(np.int32)
    st, Us, scs, ms = evc_left_cplx(p.S, p.T, select=sel, nthreads=4)
    idx = np.flatnonzero(sel)
    assert st == 0 and ms == idx.size
    assert np.array_equal(Us, U[:, idx]) and np.array_equal(scs, sc[idx])


def test_cplx_left_planted_conjugation_fails_the_residual():
    from oracle.left import evc_left_cplx
    p = pencilgen.make_complex_pencil(90, 520)
    st, U, sc, m = evc_left_cplx(p.S, p.T)
    a, b = _diag(p.S, p.T)
    assert check.cplx_left_residuals(p.S, p.T, U, a, b).max() <= BAR * p.n
    # the mistake: the flipped pencil transposed without conjugation
    Sp = np.asfortranarray(p.S.T[::-1, ::-1])
    Tp = np.asfortranarray(p.T.T[::-1, ::-1])
    st, Vp, _, _ = oracle.evc_cplx(Sp, Tp)
    Ubad = Vp[::-1, ::-1]
    assert check.cplx_left_residuals(p.S, p.T, Ubad, a, b)[:-10].min() > 1e-6


# ---------------------------------------------------------------------------
# Back-transformation of complex eigenvectors: x = Z v is an eigenvector of
# (A, B) = (Q S Z^H, Q T Z^H).  Pinned by the residual of the original pencil,
# which does not go through oracle.backtransform.
# ---------------------------------------------------------------------------

def test_cplx_backtransform_gives_eigenvectors_of_original_pencil():
    from oracle.backtransform import backtransform_cplx, random_unitary
    n = 160
    p = pencilgen.make_complex_pencil(n, 530)
    Q, Z = random_unitary(n, 531), random_unitary(n, 532)
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() < 1e-13
    A, B = Q @ p.S @ Z.conj().T, Q @ p.T @ Z.conj().T
    st, V, sc, m = oracle.evc_cplx(p.S, p.T)
    X = backtransform_cplx(Z, V)
    a, b = _diag(p.S, p.T)
    assert check.cplx_residuals(A, B, X, a, b).max() <= BAR * n
    for c in range(n):
        i = int(np.argmax(np.abs(X[:, c])))
        assert X[i, c] == 1.0
    # the planted mistake: conj(Z) instead of Z (a conjugation dropped or doubled)
    Xbad = backtransform_cplx(Z.conj(), V)
    assert check.cplx_residuals(A, B, Xbad, a, b)[5:].min() > 1e-6
    # Z = I returns the vectors themselves
    assert np.abs(backtransform_cplx(np.eye(n), V) - V).max() == 0.0


def test_cplx_repeated_eigenvalue_needs_the_perturbed_pivot():
    ep = pencilgen.exact_complex_pencil(10, 652)
    S, T = ep.as_complex()
    S[6, 6], T[6, 6] = S[1, 1], T[1, 1]                   # the same (alpha, beta): a pivot exactly 0
    st, V, sc, m = oracle.evc_cplx(S, T)
    assert st == 0 and np.isfinite(V).all()
    a, b = np.diag(S), np.diag(T)
    assert check.cplx_residuals(S, T, V, a, b).max() <= BAR * 10
    assert 40 <= sc[6] <= 70, sc[6]                        # growth about 1/u from smin (reading 9)


def test_cplx_huge_entries_need_the_prescaling():
    p = pencilgen.make_complex_pencil(80, 653)
    st, V, sc, m = oracle.evc_cplx(p.S, p.T)
    st2, V2, sc2, m2 = oracle.evc_cplx(p.S * 2.0 ** 1010, p.T * 2.0 ** 1010)
    assert st2 == 0 and np.isfinite(V2).all()
    assert check.compare_normalised_cplx(V, V2)[0] <= 1e-13


def test_cplx_column_bound_covers_the_row_above_the_diagonal():
    """The complex twin of the real growth pencil (the row just above the
    diagonal holds the column's largest entry)."""
    l2 = 2.0 ** -400 * (1 + 1j)
    l1 = l2 * (1.0 + 2.0 ** -50)
    S = np.array([[0.5, 2.0 ** 600 * 1j, 0.0], [0.0, l1, 2.0 ** 600], [0.0, 0.0, l2]], dtype=complex, order="F")
    T = np.asfortranarray(np.eye(3, dtype=complex))
    st, V, sc, m = oracle.evc_cplx(S, T)
    assert st == 0 and np.isfinite(V).all()
    assert sc[2] > 1023
    assert check.cplx_residuals(S, T, V, np.diag(S), np.diag(T)).max() <= BAR * 3
