"""Seeded synthetic pencils (S, T) in generalized real Schur form.

This module is the one input source shared by the FP64 oracle and the CUDA
path.  It draws random numbers and places them; it performs none of the
eigenvector arithmetic.

Structure of a pencil (the workloads of the paper's Section 6, which used
StarNEig's ``starneig-test`` matrices; those are not available, so these
synthetic pencils stand in for them):

* S is upper quasi-triangular with 1x1 and 2x2 diagonal blocks, T is upper
  triangular and every 2x2 diagonal block of T is diagonal (Section 2).
* Walking the diagonal, a 2x2 block starts with probability 1/3 when at least
  two rows remain, so about half of the rows sit in 2x2 blocks.
* A 1x1 block has a real eigenvalue lam ~ N(0,1), kept at least 1e-6 away from
  the eigenvalues accepted before it (the paper assumes distinct eigenvalues),
  T_cc ~ U[0.5, 2] and S_cc = lam * T_cc.
* A 2x2 block has T_jj = diag(t1, t2), t ~ U[0.5, 2], and
  S_jj = T_jj @ [[mu, nu*c], [-nu/c, mu]] with mu ~ N(0,1), nu = |N(0,1)|+0.1,
  c = exp(N(0, 0.25^2)); its eigenvalues are mu +- i*nu.
* Every other strictly upper entry of S and T is N(0,1).

The stress variant (overflow stress) multiplies T's diagonal, and with it the
diagonal blocks of S, by 2^-40, draws the eigenvalues in clusters of eight with
gaps of about 1e-8, and multiplies the off-diagonal entries of a random 5 % of
the strictly upper tiles of a fixed 64x64 grid by 1e100.

All arrays are float64 in column-major (Fortran) order.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

BASE_SEED = 20030477

# Workload table: the five configurations the library is measured and tested on.
CONFIGS = {
    0: dict(n=256, stress=False),
    1: dict(n=4000, stress=False),
    2: dict(n=10000, stress=True),
    3: dict(n=20000, stress=False),
}
BATCH_COUNT = 1024
BATCH_NMIN, BATCH_NMAX = 32, 2048


def config_seed(config: int, index: int = 0) -> int:
    """Seed of pencil ``index`` of workload ``config``."""
    return BASE_SEED + 1000 * config + index


@dataclass
class Pencil:
    S: np.ndarray
    T: np.ndarray
    block: np.ndarray            # int8[n]: 0 = 1x1, 1 = first row of a 2x2, 2 = second row
    lam_re: np.ndarray           # generated eigenvalue per row (pairs: +nu on the first row, -nu on the second)
    lam_im: np.ndarray
    stress: bool = False
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.S.shape[0]


def _block_pattern(rng: np.random.Generator, n: int) -> np.ndarray:
    block = np.zeros(n, dtype=np.int8)
    u = rng.random(n)
    i = 0
    while i < n:
        if i + 1 < n and u[i] < 1.0 / 3.0:
            block[i] = 1
            block[i + 1] = 2
            i += 2
        else:
            i += 1
    return block


def _draw_real_eigs(rng, count, stress):
    """Distinct real eigenvalues (at least 1e-6 apart, or clustered in stress)."""
    out = np.empty(count)
    if stress:
        k = 0
        while k < count:
            centre = rng.standard_normal()
            for _ in range(8):
                if k >= count:
                    break
                out[k] = centre
                centre += 1e-8 * (1.0 + 0.1 * rng.random())
                k += 1
        return out
    accepted = []
    sorted_acc = np.empty(0)
    while len(accepted) < count:
        lam = rng.standard_normal()
        if sorted_acc.size:
            pos = np.searchsorted(sorted_acc, lam)
            near = False
            for q in (pos - 1, pos):
                if 0 <= q < sorted_acc.size and abs(sorted_acc[q] - lam) < 1e-6:
                    near = True
            if near:
                continue
        accepted.append(lam)
        sorted_acc = np.insert(sorted_acc, np.searchsorted(sorted_acc, lam), lam)
    return np.asarray(accepted)


def _draw_pair_params(rng, count, stress):
    mu = np.empty(count)
    if stress:
        k = 0
        while k < count:
            centre = rng.standard_normal()
            for _ in range(8):
                if k >= count:
                    break
                mu[k] = centre
                centre += 1e-8 * (1.0 + 0.1 * rng.random())
                k += 1
    else:
        mu[:] = rng.standard_normal(count)
    nu = np.abs(rng.standard_normal(count)) + 0.1
    c = np.exp(0.25 * rng.standard_normal(count))
    return mu, nu, c


def make_pencil(n: int, seed: int, stress: bool = False, grid: int = 64,
                big_frac: float = 0.05, big: float = 1e100,
                t_scale: float = 2.0 ** -40) -> Pencil:
    """Generate one seeded pencil of order ``n``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    block = _block_pattern(rng, n)
    ones = np.flatnonzero(block == 0)
    pairs = np.flatnonzero(block == 1)
    lam = _draw_real_eigs(rng, ones.size, stress)
    mu, nu, c = _draw_pair_params(rng, pairs.size, stress)
    tdiag = rng.uniform(0.5, 2.0, n)
    if stress:
        tdiag = tdiag * t_scale

    # Off-diagonal entries, drawn as a full square in a fixed order, then the
    # lower part (and the inside of the 2x2 blocks) is overwritten.
    S = np.asfortranarray(rng.standard_normal((n, n)))
    T = np.asfortranarray(rng.standard_normal((n, n)))
    if stress and n > grid:
        g = (n + grid - 1) // grid
        pick = rng.random((g, g)) < big_frac
        for p in range(g):
            for q in range(p + 1, g):
                if pick[p, q]:
                    S[p * grid:(p + 1) * grid, q * grid:(q + 1) * grid] *= big
                    T[p * grid:(p + 1) * grid, q * grid:(q + 1) * grid] *= big
    # zero the strictly lower parts (S keeps nothing below the diagonal yet)
    for M in (S, T):
        for j in range(n - 1):
            M[j + 1:, j] = 0.0

    lam_re = np.zeros(n)
    lam_im = np.zeros(n)
    for k, i in enumerate(ones):
        S[i, i] = lam[k] * tdiag[i]
        T[i, i] = tdiag[i]
        lam_re[i] = lam[k]
    for k, i in enumerate(pairs):
        t1, t2 = tdiag[i], tdiag[i + 1]
        T[i, i] = t1
        T[i + 1, i + 1] = t2
        T[i, i + 1] = 0.0
        S[i, i] = t1 * mu[k]
        S[i, i + 1] = t1 * nu[k] * c[k]
        S[i + 1, i] = -t2 * nu[k] / c[k]
        S[i + 1, i + 1] = t2 * mu[k]
        lam_re[i] = lam_re[i + 1] = mu[k]
        lam_im[i] = nu[k]
        lam_im[i + 1] = -nu[k]
    return Pencil(S=S, T=T, block=block, lam_re=lam_re, lam_im=lam_im,
                  stress=stress, seed=seed, meta=dict(grid=grid))


def config_pencil(config: int, index: int = 0, n: int | None = None) -> Pencil:
    """Pencil ``index`` of workload ``config`` (0..3); ``n`` overrides the order."""
    cfg = CONFIGS[config]
    return make_pencil(n if n is not None else cfg["n"], config_seed(config, index),
                       stress=cfg["stress"])


def batch_orders(count: int = BATCH_COUNT, seed: int | None = None) -> np.ndarray:
    """Orders of the batched workload: n ~ round(exp(U[ln 32, ln 2048]))."""
    rng = np.random.Generator(np.random.PCG64(config_seed(4) if seed is None else seed))
    return np.rint(np.exp(rng.uniform(np.log(BATCH_NMIN), np.log(BATCH_NMAX), count))).astype(np.int64)


def batch_pencil(index: int, n: int) -> Pencil:
    """Pencil ``index`` of the batched workload; odd indices are stress pencils."""
    return make_pencil(int(n), config_seed(4, index + 1), stress=bool(index % 2))


# ---------------------------------------------------------------------------
# Exact (dyadic-rational) pencils for brute-force pins on tiny orders.
# ---------------------------------------------------------------------------

@dataclass
class ExactPencil:
    S: list                      # n x n lists of Fraction (row-major)
    T: list
    block: list
    lam: list                    # per row: (Fraction re, Fraction im)

    def as_float(self):
        n = len(self.S)
        Sf = np.zeros((n, n), order="F")
        Tf = np.zeros((n, n), order="F")
        for i in range(n):
            for j in range(n):
                Sf[i, j] = float(self.S[i][j])
                Tf[i, j] = float(self.T[i][j])
        return Sf, Tf


def exact_pencil(n: int, seed: int, two_by_two: bool = True) -> ExactPencil:
    """A pencil whose entries are dyadic rationals (exact in binary64).

    1x1 blocks: lam = k/16 distinct, T_cc = k/8 in [1/2, 2], S_cc = lam*T_cc.
    2x2 blocks: T_jj = diag(t1, t2), S_jj = T_jj @ [[mu, nu*c], [-nu/c, mu]]
    with mu, nu dyadic and c a power of two, so mu +- i*nu is exact.
    Off-diagonal entries are k/8 with |k| <= 16.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    F = Fraction
    block = [0] * n
    i = 0
    while i < n:
        if two_by_two and i + 1 < n and rng.random() < 1.0 / 3.0:
            block[i], block[i + 1] = 1, 2
            i += 2
        else:
            i += 1
    S = [[F(0)] * n for _ in range(n)]
    T = [[F(0)] * n for _ in range(n)]
    for r in range(n):
        for col in range(r + 1, n):
            S[r][col] = F(int(rng.integers(-16, 17)), 8)
            T[r][col] = F(int(rng.integers(-16, 17)), 8)
    lam = [None] * n
    used = set()
    for r in range(n):
        if block[r] == 0:
            while True:
                k = int(rng.integers(-40, 41))
                if k not in used:
                    used.add(k)
                    break
            lr = F(k, 16)
            t = F(int(rng.integers(4, 17)), 8)
            T[r][r] = t
            S[r][r] = lr * t
            lam[r] = (lr, F(0))
        elif block[r] == 1:
            t1 = F(int(rng.integers(4, 17)), 8)
            t2 = F(int(rng.integers(4, 17)), 8)
            while True:
                mu = F(int(rng.integers(-32, 33)), 16)
                nu = F(int(rng.integers(2, 33)), 16)
                if (mu, nu) not in used:
                    used.add((mu, nu))
                    break
            c = F(2) ** int(rng.integers(-1, 2))
            T[r][r], T[r + 1][r + 1], T[r][r + 1] = t1, t2, F(0)
            S[r][r] = t1 * mu
            S[r][r + 1] = t1 * nu * c
            S[r + 1][r] = -t2 * nu / c
            S[r + 1][r + 1] = t2 * mu
            lam[r] = (mu, nu)
            lam[r + 1] = (mu, -nu)
    return ExactPencil(S=S, T=T, block=block, lam=lam)


# ---------------------------------------------------------------------------
# Complex pencils in generalized (complex) Schur form.
# ---------------------------------------------------------------------------

@dataclass
class ComplexPencil:
    S: np.ndarray                # complex128, upper triangular, column-major
    T: np.ndarray
    lam: np.ndarray              # generated eigenvalue of every diagonal entry
    stress: bool = False
    seed: int = 0

    @property
    def n(self) -> int:
        return self.S.shape[0]


def _draw_complex_eigs(rng, count, stress):
    """Complex eigenvalues N(0,1) + i N(0,1), at least 1e-6 apart (or, in the
    stress variant, in clusters of eight with gaps of about 1e-8)."""
    if stress:
        out = np.empty(count, dtype=np.complex128)
        k = 0
        while k < count:
            centre = complex(rng.standard_normal(), rng.standard_normal())
            for _ in range(8):
                if k >= count:
                    break
                out[k] = centre
                centre += 1e-8 * (1.0 + 0.1 * rng.random())
                k += 1
        return out
    out = rng.standard_normal(count) + 1j * rng.standard_normal(count)
    while True:
        order = np.argsort(out.real, kind="stable")
        re, im = out.real[order], out.imag[order]
        bad = set()
        for k in range(count):
            j = k + 1
            while j < count and re[j] - re[k] < 1e-6:
                if abs(im[j] - im[k]) < 1e-6:
                    bad.add(int(order[j]))
                j += 1
        if not bad:
            return out
        for q in sorted(bad):
            out[q] = complex(rng.standard_normal(), rng.standard_normal())


def make_complex_pencil(n: int, seed: int, stress: bool = False, grid: int = 64,
                        big_frac: float = 0.05, big: float = 1e100,
                        t_scale: float = 2.0 ** -40) -> ComplexPencil:
    """A seeded complex pencil of order ``n`` in generalized Schur form.

    T's diagonal is real, T_cc ~ U[0.5, 2] (the form complex QZ returns), and
    S_cc = lam_c T_cc with lam_c ~ N(0,1) + i N(0,1).  Every strictly upper
    entry of S and T is (N(0,1) + i N(0,1)) / sqrt(2).  The stress variant
    scales T's diagonal (and with it S's) by 2^-40, clusters the eigenvalues
    and multiplies a random 5 % of the strictly upper tiles of a fixed
    64 x 64 grid by 1e100, as for real pencils.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = _draw_complex_eigs(rng, n, stress)
    tdiag = rng.uniform(0.5, 2.0, n)
    if stress:
        tdiag = tdiag * t_scale
    r = 1.0 / np.sqrt(2.0)
    S = np.asfortranarray((rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * r)
    T = np.asfortranarray((rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * r)
    if stress and n > grid:
        g = (n + grid - 1) // grid
        pick = rng.random((g, g)) < big_frac
        for p in range(g):
            for q in range(p + 1, g):
                if pick[p, q]:
                    S[p * grid:(p + 1) * grid, q * grid:(q + 1) * grid] *= big
                    T[p * grid:(p + 1) * grid, q * grid:(q + 1) * grid] *= big
    for M in (S, T):
        for j in range(n - 1):
            M[j + 1:, j] = 0.0
    idx = np.arange(n)
    T[idx, idx] = tdiag
    S[idx, idx] = lam * tdiag
    return ComplexPencil(S=S, T=T, lam=lam, stress=stress, seed=seed)


@dataclass
class ExactComplexPencil:
    S: list                      # n x n lists of (Fraction re, Fraction im), row-major
    T: list

    def as_complex(self):
        n = len(self.S)
        Sc = np.zeros((n, n), dtype=np.complex128, order="F")
        Tc = np.zeros((n, n), dtype=np.complex128, order="F")
        for i in range(n):
            for j in range(n):
                Sc[i, j] = complex(float(self.S[i][j][0]), float(self.S[i][j][1]))
                Tc[i, j] = complex(float(self.T[i][j][0]), float(self.T[i][j][1]))
        return Sc, Tc


def exact_complex_pencil(n: int, seed: int, infinite: bool = False) -> ExactComplexPencil:
    """A complex triangular pencil with dyadic-rational parts (exact in binary64).

    Diagonal: T_cc = (k1 + i k2)/8 with k1 in [4, 16], k2 in [-8, 8]; S_cc =
    lam_c T_cc with distinct lam_c = (k3 + i k4)/16.  Off-diagonal parts are
    k/8 with |k| <= 16.  With ``infinite`` the last diagonal entry of T is
    zero (an infinite eigenvalue).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    F = Fraction
    z = (F(0), F(0))
    S = [[z] * n for _ in range(n)]
    T = [[z] * n for _ in range(n)]
    for r in range(n):
        for col in range(r + 1, n):
            S[r][col] = (F(int(rng.integers(-16, 17)), 8), F(int(rng.integers(-16, 17)), 8))
            T[r][col] = (F(int(rng.integers(-16, 17)), 8), F(int(rng.integers(-16, 17)), 8))
    used = set()
    for r in range(n):
        while True:
            lr, li = int(rng.integers(-40, 41)), int(rng.integers(-40, 41))
            if (lr, li) not in used:
                used.add((lr, li))
                break
        lr, li = F(lr, 16), F(li, 16)
        tr, ti = F(int(rng.integers(4, 17)), 8), F(int(rng.integers(-8, 9)), 8)
        if infinite and r == n - 1:
            tr, ti = F(0), F(0)
            lr, li = F(int(rng.integers(4, 17)), 8), F(0)   # S_cc itself, nonzero
            S[r][r] = (lr, li)
        else:
            S[r][r] = (lr * tr - li * ti, lr * ti + li * tr)
        T[r][r] = (tr, ti)
    return ExactComplexPencil(S=S, T=T)

