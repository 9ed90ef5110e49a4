"""Back-transformation to the eigenvectors of the original pencil -- TEST INFRASTRUCTURE.

With (A, B) = (Q S Z^T, Q T Z^T), the generalized real Schur reduction of a
pencil (A, B) (Section 1 of the paper), a right eigenvector v of (S, T) gives
the right eigenvector x = Z v of (A, B) for the same eigenvalue.  The oracle
forms X = Z V with the library matrix product and scales every eigenvector (a
real column, or a complex pair (Re, Im) taken as one complex vector) so that
its entry of largest modulus -- the first one on ties -- is exactly 1; an
all-zero vector stays zero.

Pinned in tests/test_oracle_pins.py by the residual of the original pencil
(which does not use this module), by Z = I, and by a planted transposition.
"""
from __future__ import annotations

import numpy as np


def backtransform(Z, V, kinds, normalise: bool = True):
    """X = Z V (n x m) with the eigenvectors normalised; kinds[c] is 0 for a
    real eigenvector's column, 1 / 2 for the real / imaginary column of a pair."""
    X = np.asfortranarray(np.asarray(Z, dtype=np.float64) @ np.asarray(V, dtype=np.float64))
    if not normalise:
        return X
    c = 0
    while c < X.shape[1]:
        if kinds[c] == 0:
            x = X[:, c]
            i = int(np.argmax(np.abs(x)))
            if x[i] != 0.0:
                X[:, c] = x / x[i]
                X[i, c] = 1.0
            c += 1
        else:
            z = X[:, c] + 1j * X[:, c + 1]
            i = int(np.argmax(np.abs(z)))
            if z[i] != 0.0:
                z = z / z[i]
                z[i] = 1.0
            X[:, c] = z.real
            X[:, c + 1] = z.imag
            c += 2
    return X


def random_orthogonal(n: int, seed: int):
    """A seeded random orthogonal matrix (the Q factor of a Gaussian matrix)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def backtransform_cplx(Z, V, normalise: bool = True):
    """X = Z V for complex eigenvectors (the eigenvectors of (Q S Z^H, Q T Z^H)),
    each column divided by its first entry of largest modulus, which is then
    exactly 1; an all-zero column stays zero."""
    X = np.asfortranarray(np.asarray(Z, dtype=np.complex128) @ np.asarray(V, dtype=np.complex128))
    if not normalise:
        return X
    for c in range(X.shape[1]):
        i = int(np.argmax(np.abs(X[:, c])))
        d = X[i, c]
        if d != 0:
            X[:, c] = X[:, c] / d
            X[i, c] = 1.0
    return X


def random_unitary(n: int, seed: int):
    """A seeded random unitary matrix (the Q factor of a complex Gaussian matrix)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q, r = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    d = np.diag(r)
    return q * (d / np.abs(d))

