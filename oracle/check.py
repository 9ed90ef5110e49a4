"""Residual and comparison helpers -- TEST INFRASTRUCTURE.

The relative residual of an eigenvector v of (S, T) for (alpha, beta) is
    ||beta S v - alpha T v||_inf / ((|beta| ||S||_inf + |alpha| ||T||_inf) ||v||_inf)
(matrix infinity norms are maximum row sums, vector norms maximum moduli);
Table 1 of the paper reports all vectors below 2u with this kind of measure.
The acceptance bar used here is 100 n u, u = 2^-53.
"""
from __future__ import annotations

import numpy as np

U = 2.0 ** -53


def column_kinds(blk, select=None):
    """Kind and diagonal position of each output column.

    Returns (kinds, pos): kinds[c] = 0 real, 1 first (real part) and 2 second
    (imaginary part) column of a complex pair; pos[c] = diagonal row of the
    block's first row.
    """
    blk = np.asarray(blk)
    n = blk.size
    kinds, pos = [], []
    c = 0
    while c < n:
        sz = 2 if blk[c] == 1 else 1
        sel = select is None or bool(select[c]) or (sz == 2 and bool(select[c + 1]))
        if sel:
            if sz == 1:
                kinds.append(0)
                pos.append(c)
            else:
                kinds += [1, 2]
                pos += [c, c]
        c += sz
    return np.asarray(kinds, dtype=np.int64), np.asarray(pos, dtype=np.int64)


def as_complex(V, kinds):
    """One complex vector per eigenvector (pairs combined), with its column."""
    out, cols = [], []
    for c, k in enumerate(kinds):
        if k == 0:
            out.append(V[:, c].astype(complex))
            cols.append(c)
        elif k == 1:
            out.append(V[:, c] + 1j * V[:, c + 1])
            cols.append(c)
    return out, cols


def residuals(S, T, V, kinds, pos, a, b, beta):
    """Relative residual of every eigenvector (one value per output column).

    S V and T V are formed with two real matrix products (library calls);
    a pair's complex vector z = x + i y gives S z = S x + i S y."""
    S = np.asarray(S)
    T = np.asarray(T)
    V = np.asarray(V)
    kinds = np.asarray(kinds)
    pos = np.asarray(pos)
    nS = np.abs(S).sum(axis=1).max()
    nT = np.abs(T).sum(axis=1).max()
    SV = S @ V
    TV = T @ V
    res = np.zeros(len(kinds))
    for c, k in enumerate(kinds):
        if k == 2:
            continue
        p = pos[c]
        al = complex(a[p], b[p])
        bt = beta[p]
        if k == 0:
            z, sz, tz = V[:, c].astype(complex), SV[:, c].astype(complex), TV[:, c].astype(complex)
        else:
            z = V[:, c] + 1j * V[:, c + 1]
            sz = SV[:, c] + 1j * SV[:, c + 1]
            tz = TV[:, c] + 1j * TV[:, c + 1]
        r = bt * sz - al * tz
        den = (abs(bt) * nS + abs(al) * nT) * np.abs(z).max()
        val = np.abs(r).max() / den if den > 0 else np.inf
        res[c] = val
        if k == 1:
            res[c + 1] = val
    return res


def left_residuals(S, T, U, kinds, pos, a, b, beta):
    """Relative residual of every left eigenvector u (u^H (beta S - alpha T)
    = 0, alpha = a + i b with b > 0 for a pair's columns (Re u, Im u)):
        ||u^H (beta S - alpha T)||_inf / ((|beta| ||S||_1 + |alpha| ||T||_1) ||u||_inf)
    (the 1-norms are maximum column sums, the norms of S^T and T^T)."""
    S = np.asarray(S)
    T = np.asarray(T)
    U = np.asarray(U)
    nS = np.abs(S).sum(axis=0).max()
    nT = np.abs(T).sum(axis=0).max()
    US = U.T @ S      # row c: U[:, c]^T S
    UT = U.T @ T
    res = np.zeros(len(kinds))
    for c, k in enumerate(kinds):
        if k == 2:
            continue
        p = pos[c]
        al = complex(a[p], b[p])
        bt = beta[p]
        if k == 0:
            u, us, ut = U[:, c].astype(complex), US[c].astype(complex), UT[c].astype(complex)
        else:
            u = U[:, c] + 1j * U[:, c + 1]
            us = US[c] - 1j * US[c + 1]      # u^H S = conj(u)^T S
            ut = UT[c] - 1j * UT[c + 1]
        r = bt * us - al * ut
        den = (abs(bt) * nS + abs(al) * nT) * np.abs(u).max()
        val = np.abs(r).max() / den if den > 0 else np.inf
        res[c] = val
        if k == 1:
            res[c + 1] = val
    return res


def compare_normalised(Vref, Vgot, kinds):
    """Largest componentwise |difference| after normalising ``Vgot`` at the
    index where ``Vref`` has its largest modulus (near-ties in the maximum may
    pick different indices on the two sides, so both are taken at the same
    index).  Returns (max_err, per-vector errors)."""
    ref, cols = as_complex(Vref, kinds)
    got, _ = as_complex(Vgot, kinds)
    errs = np.zeros(len(cols))
    for q, (zr, zg) in enumerate(zip(ref, got)):
        m = np.abs(zr)
        istar = int(np.argmax(m))
        d = zg[istar]
        if d == 0 or not np.isfinite(d):
            errs[q] = np.inf
            continue
        zg2 = zg / d
        zr2 = zr / zr[istar]
        errs[q] = np.abs(zg2 - zr2).max()
    return (errs.max() if errs.size else 0.0), errs


def cplx_residuals(S, T, V, alpha, beta):
    """Relative residual of every eigenvector of a complex triangular pencil:
    column c of V for (alpha_c, beta_c) = the pair of its diagonal entry
    (the columns of V follow the diagonal, ``pos`` gives the entries when a
    selection was made).  Same measure as ``residuals``."""
    S = np.asarray(S)
    T = np.asarray(T)
    V = np.asarray(V)
    nS = np.abs(S).sum(axis=1).max()
    nT = np.abs(T).sum(axis=1).max()
    SV = S @ V
    TV = T @ V
    res = np.zeros(V.shape[1])
    for c in range(V.shape[1]):
        al, bt = alpha[c], beta[c]
        r = bt * SV[:, c] - al * TV[:, c]
        den = (abs(bt) * nS + abs(al) * nT) * np.abs(V[:, c]).max()
        res[c] = np.abs(r).max() / den if den > 0 else np.inf
    return res


def compare_normalised_cplx(Vref, Vgot):
    """``compare_normalised`` for complex columns (one eigenvector each)."""
    Vref = np.asarray(Vref)
    Vgot = np.asarray(Vgot)
    errs = np.zeros(Vref.shape[1])
    for c in range(Vref.shape[1]):
        zr, zg = Vref[:, c], Vgot[:, c]
        istar = int(np.argmax(np.abs(zr)))
        d = zg[istar]
        if d == 0 or not np.isfinite(d):
            errs[c] = np.inf
            continue
        errs[c] = np.abs(zg / d - zr / zr[istar]).max()
    return (errs.max() if errs.size else 0.0), errs


def cplx_left_residuals(S, T, U, alpha, beta):
    """Relative residual of every left eigenvector u of a complex triangular
    pencil, u^H (beta S - alpha T) = 0:
        ||u^H (beta S - alpha T)||_inf / ((|beta| ||S||_1 + |alpha| ||T||_1) ||u||_inf)."""
    S = np.asarray(S)
    T = np.asarray(T)
    U = np.asarray(U)
    nS = np.abs(S).sum(axis=0).max()
    nT = np.abs(T).sum(axis=0).max()
    US = np.conj(U).T @ S
    UT = np.conj(U).T @ T
    res = np.zeros(U.shape[1])
    for c in range(U.shape[1]):
        r = beta[c] * US[c] - alpha[c] * UT[c]
        den = (abs(beta[c]) * nS + abs(alpha[c]) * nT) * np.abs(U[:, c]).max()
        res[c] = np.abs(r).max() / den if den > 0 else np.inf
    return res



def perturbation_sensitivity(S, T, Vref, kinds, evc, seed: int, eps: float = 2.0 ** -52):
    """Per eigenvector: the componentwise change of the normalised vectors
    Vref of (S, T) when every row of S and T is perturbed by eps times that
    row's largest entry (random signs, on the non-zero pattern only, so the
    Schur structure and T's diagonal 2x2 blocks stay), recomputed with evc
    (the oracle's solver).  A measured stand-in for cond * eps under
    row-normwise perturbations, the kind blocked updates make; a second
    backward-stable FP64 method may differ from the oracle by a small
    multiple of it (eps = u)."""
    rng = np.random.default_rng(seed)
    pert = []
    for A in (np.asarray(S), np.asarray(T)):
        rowmax = np.abs(A).max(axis=1, keepdims=True)
        pert.append(A + (A != 0) * rng.choice([-1.0, 1.0], A.shape) * eps * rowmax)
    st, V2, _, _ = evc(pert[0], pert[1])
    if st != 0:
        raise RuntimeError(f"perturbed pencil: status {st}")
    return compare_normalised(Vref, V2, kinds)[1]
