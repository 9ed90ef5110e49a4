"""Left eigenvectors of a real Schur pencil -- TEST INFRASTRUCTURE.

A left eigenvector u of (S, T), u^H (beta S - alpha T) = 0, is the right
eigenvector for conj(alpha) of (S^T, T^T); with J the reversal permutation,
J u is the right eigenvector of (J S^T J, J T^T J), again a real Schur pencil.
The oracle solves that pencil with its own robust substitution (oracle.evc)
and reverses the rows back; for a complex pair the imaginary column is
negated (conj(alpha) instead of alpha).  Columns follow S's diagonal, a pair as
(Re u, Im u) for the eigenvalue with positive imaginary part.

Pinned in tests/test_oracle_pins.py by the left residual (check.left_residuals,
which uses neither this module nor the flip), by exact null vectors of
(beta S - alpha T)^H over Gaussian rationals, and by a planted mistake (the
imaginary part not negated).
"""
from __future__ import annotations

import numpy as np

from . import check, eigpairs, evc


def evc_left(S, T, select=None, normalise: bool = True, nthreads: int = 1):
    """(status, U n x m, scale int32[m], m) for the left eigenvectors."""
    S = np.asarray(S, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = S.shape[0]
    Sp = np.asfortranarray(S.T[::-1, ::-1])
    Tp = np.asfortranarray(T.T[::-1, ::-1])
    selp = None if select is None else np.ascontiguousarray(np.asarray(select, dtype=np.int32)[::-1])
    st, Vp, scp, m = evc(Sp, Tp, select=selp, normalise=normalise, nthreads=nthreads)
    if st:
        return st, np.zeros((n, 0)), np.zeros(0, dtype=np.int32), 0
    _, blkp, _, _, _, _ = eigpairs(Sp, Tp)
    kinds_p, _ = check.column_kinds(blkp, selp)
    U = np.zeros((n, m), order="F")
    sc = np.zeros(m, dtype=np.int32)
    for q in range(m):
        kd = kinds_p[q]
        oc = m - 1 - q if kd == 0 else (m - 2 - q if kd == 1 else m - q)
        U[:, oc] = (-1.0 if kd == 2 else 1.0) * Vp[::-1, q]
        sc[oc] = scp[q]
    return 0, U, sc, m


def evc_left_cplx(S, T, select=None, normalise: bool = True, nthreads: int = 1):
    """Left eigenvectors of a complex triangular pencil: for every selected
    diagonal entry c, u with u^H (beta_c S - alpha_c T) = 0, (alpha_c, beta_c) =
    (S_cc, T_cc).  u^H M = 0 is M^H u = 0, and J M^H J = conj(beta) S' -
    conj(alpha) T' with (S', T') = (J S^H J, J T^H J), again upper triangular,
    whose diagonal entry n-1-c is (conj(alpha_c), conj(beta_c)).  So J u is the
    right eigenvector of (S', T') at entry n-1-c (oracle.evc_cplx); u is zero
    above c.  Returns (status, U n x m complex, scale int32[m], m) with the
    columns in the order of S's diagonal."""
    from . import evc_cplx
    S = np.asarray(S, dtype=np.complex128)
    T = np.asarray(T, dtype=np.complex128)
    n = S.shape[0]
    Sp = np.asfortranarray(np.conj(S.T)[::-1, ::-1])
    Tp = np.asfortranarray(np.conj(T.T)[::-1, ::-1])
    selp = None if select is None else np.ascontiguousarray(np.asarray(select, dtype=np.int32)[::-1])
    st, Vp, scp, m = evc_cplx(Sp, Tp, select=selp, normalise=normalise, nthreads=nthreads)
    if st:
        return st, np.zeros((n, 0), dtype=np.complex128), np.zeros(0, dtype=np.int32), 0
    return 0, np.asfortranarray(Vp[::-1, ::-1]), scp[::-1].copy(), m
