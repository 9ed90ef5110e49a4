"""Exact brute force for tiny pencils -- TEST INFRASTRUCTURE.

For a pencil whose entries are exact rationals (``pencilgen.exact_pencil``),
the eigenvector of the eigenvalue lambda = alpha/beta is the kernel of
M = beta*S - alpha*T (Section 2, the tall equation and its Lemma).  This
module computes that kernel in exact arithmetic over the Gaussian rationals
Q(i) by reduced row echelon form of the whole n x n matrix M: a general
null-space computation, not the triangular substitution the method uses.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


class GQ:
    """Gaussian rational re + i*im with Fraction parts."""
    __slots__ = ("re", "im")

    def __init__(self, re, im=0):
        self.re = Fraction(re)
        self.im = Fraction(im)

    def __add__(self, o):
        return GQ(self.re + o.re, self.im + o.im)

    def __sub__(self, o):
        return GQ(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        return GQ(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

    def __truediv__(self, o):
        d = o.re * o.re + o.im * o.im
        return GQ((self.re * o.re + self.im * o.im) / d, (self.im * o.re - self.re * o.im) / d)

    def __neg__(self):
        return GQ(-self.re, -self.im)

    def is_zero(self):
        return self.re == 0 and self.im == 0

    def abs2(self):
        return self.re * self.re + self.im * self.im

    def to_complex(self):
        return complex(float(self.re), float(self.im))


def nullspace(M):
    """Basis of the kernel of the square matrix M (list of lists of GQ)."""
    n = len(M)
    A = [row[:] for row in M]
    pivots = []
    r = 0
    for col in range(n):
        piv = None
        for i in range(r, n):
            if not A[i][col].is_zero():
                piv = i
                break
        if piv is None:
            continue
        A[r], A[piv] = A[piv], A[r]
        p = A[r][col]
        A[r] = [x / p for x in A[r]]
        for i in range(n):
            if i != r and not A[i][col].is_zero():
                f = A[i][col]
                A[i] = [x - f * y for x, y in zip(A[i], A[r])]
        pivots.append(col)
        r += 1
        if r == n:
            break
    free = [c for c in range(n) if c not in pivots]
    basis = []
    for fcol in free:
        v = [GQ(0) for _ in range(n)]
        v[fcol] = GQ(1)
        for i, pc in enumerate(pivots):
            v[pc] = -A[i][fcol]
        basis.append(v)
    return basis


def exact_eigenvectors(ep):
    """Normalised exact eigenvectors of an ``ExactPencil``.

    Returns an n x n complex array V (column c of a 1x1 block holds the real
    vector; for a 2x2 block starting at c, column c holds z for mu + i nu,
    nu > 0, and column c+1 holds its conjugate) and the kernel dimensions.
    Each vector is divided by its first entry of largest modulus.
    """
    n = len(ep.S)
    V = np.zeros((n, n), dtype=complex)
    dims = []
    c = 0
    while c < n:
        sz = 2 if ep.block[c] == 1 else 1
        if sz == 1:
            # homogeneous pair (alpha, beta) = (S_cc, T_cc): also covers beta = 0
            alpha, beta = GQ(ep.S[c][c]), GQ(ep.T[c][c])
        else:
            lr, li = ep.lam[c]
            alpha, beta = GQ(lr, li), GQ(1)
        M = [[beta * GQ(ep.S[i][j]) - alpha * GQ(ep.T[i][j]) for j in range(n)] for i in range(n)]
        basis = nullspace(M)
        dims.append(len(basis))
        v = basis[0]
        best = max(x.abs2() for x in v)
        istar = next(i for i, x in enumerate(v) if x.abs2() == best)
        d = v[istar]
        z = [x / d for x in v]
        col = np.array([x.to_complex() for x in z])
        V[:, c] = col
        if sz == 2:
            V[:, c + 1] = np.conj(col)
        c += sz
    return V, dims


def exact_left_eigenvectors(ep):
    """Normalised exact left eigenvectors of an ``ExactPencil``: u with
    u^H (beta S - alpha T) = 0, i.e. the kernel of (beta S - alpha T)^H =
    beta S^T - conj(alpha) T^T.  Layout as in exact_eigenvectors (column c of
    a 2x2 block holds u for mu + i nu, nu > 0; column c+1 its conjugate)."""
    n = len(ep.S)
    U = np.zeros((n, n), dtype=complex)
    dims = []
    c = 0
    while c < n:
        sz = 2 if ep.block[c] == 1 else 1
        if sz == 1:
            alpha, beta = GQ(ep.S[c][c]), GQ(ep.T[c][c])
        else:
            lr, li = ep.lam[c]
            alpha, beta = GQ(lr, li), GQ(1)
        calpha = GQ(alpha.re, -alpha.im)
        MH = [[beta * GQ(ep.S[j][i]) - calpha * GQ(ep.T[j][i]) for j in range(n)] for i in range(n)]
        basis = nullspace(MH)
        dims.append(len(basis))
        v = basis[0]
        best = max(x.abs2() for x in v)
        istar = next(i for i, x in enumerate(v) if x.abs2() == best)
        d = v[istar]
        z = [x / d for x in v]
        col = np.array([x.to_complex() for x in z])
        U[:, c] = col
        if sz == 2:
            U[:, c + 1] = np.conj(col)
        c += sz
    return U, dims


def exact_complex_eigenvectors(ep):
    """Normalised exact eigenvectors of a complex triangular pencil
    (``pencilgen.exact_complex_pencil``): for each diagonal entry c, the kernel
    of beta S - alpha T with (alpha, beta) = (S_cc, T_cc), by the general
    null-space computation above, divided by its first entry of largest
    modulus.  Returns the n x n complex array and the kernel dimensions."""
    n = len(ep.S)
    Sg = [[GQ(*ep.S[i][j]) for j in range(n)] for i in range(n)]
    Tg = [[GQ(*ep.T[i][j]) for j in range(n)] for i in range(n)]
    V = np.zeros((n, n), dtype=complex)
    dims = []
    for c in range(n):
        alpha, beta = Sg[c][c], Tg[c][c]
        M = [[beta * Sg[i][j] - alpha * Tg[i][j] for j in range(n)] for i in range(n)]
        basis = nullspace(M)
        dims.append(len(basis))
        v = basis[0]
        best = max(x.abs2() for x in v)
        istar = next(i for i, x in enumerate(v) if x.abs2() == best)
        d = v[istar]
        V[:, c] = np.array([(x / d).to_complex() for x in v])
    return V, dims


def exact_complex_left_eigenvectors(ep):
    """Normalised exact left eigenvectors of a complex triangular pencil: the
    kernel of (beta S - alpha T)^H = conj(beta) S^H - conj(alpha) T^H for each
    diagonal entry, by the general null-space computation."""
    n = len(ep.S)
    Sg = [[GQ(*ep.S[i][j]) for j in range(n)] for i in range(n)]
    Tg = [[GQ(*ep.T[i][j]) for j in range(n)] for i in range(n)]
    conj = lambda z: GQ(z.re, -z.im)   # noqa: E731
    U = np.zeros((n, n), dtype=complex)
    dims = []
    for c in range(n):
        ca, cb = conj(Sg[c][c]), conj(Tg[c][c])
        MH = [[cb * conj(Sg[j][i]) - ca * conj(Tg[j][i]) for j in range(n)] for i in range(n)]
        basis = nullspace(MH)
        dims.append(len(basis))
        v = basis[0]
        best = max(x.abs2() for x in v)
        istar = next(i for i, x in enumerate(v) if x.abs2() == best)
        d = v[istar]
        U[:, c] = np.array([(x / d).to_complex() for x in v])
    return U, dims

