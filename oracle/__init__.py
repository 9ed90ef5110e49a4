"""FP64 CPU oracle for robust generalized eigenvectors -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the library: the two are independent restatements of
Kjelgaard Mikkelsen & Myllykoski (PPAM 2019).

``oracle.c`` holds the arithmetic (see its header for the method and the
readings of the paper), for real Schur pencils and for complex triangular
pencils; this module compiles it and wraps it with ctypes.  ``left.py`` gives
left eigenvectors through the flipped pencil, ``backtransform.py`` the
eigenvectors of the original pencil, ``check.py`` the residual and
comparison helpers and ``exact.py`` the exact-rational brute force used to
pin the oracle on tiny pencils.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

ERR_NOT_SCHUR = 1
ERR_NONFINITE = 2
ERR_INDEFINITE = 3
FLAG_NO_NORMALISE = 1
FLAG_PLAIN = 2


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (plain gcc, no FMA contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            L.orc_protect_upd.argtypes = [d, d, d]
            L.orc_protect_upd.restype = i
            L.orc_protect_div.argtypes = [d, d]
            L.orc_protect_div.restype = i
            L.orc_cdiv.argtypes = [d, d, d, d, ctypes.POINTER(d), ctypes.POINTER(d)]
            L.orc_cdiv.restype = None
            L.orc_blocks.argtypes = [i, p, i, p, i, p]
            L.orc_blocks.restype = i
            L.orc_eigpairs.argtypes = [i, p, i, p, i, p, p, p, p, p]
            L.orc_eigpairs.restype = i
            L.orc_evc.argtypes = [i, p, i, p, i, p, i, p, i, p, ctypes.POINTER(i), i]
            L.orc_evc.restype = i
            L.orc_eigpairs_cplx.argtypes = [i, p, i, p, i, p, p, p]
            L.orc_eigpairs_cplx.restype = i
            L.orc_evc_cplx.argtypes = [i, p, i, p, i, p, i, p, i, p, ctypes.POINTER(i), i]
            L.orc_evc_cplx.restype = i
            _lib = L
    return _lib


def _fortran(A):
    A = np.asarray(A, dtype=np.float64)
    return A if A.flags.f_contiguous else np.asfortranarray(A)


def protect_upd(y: float, t: float, x: float) -> int:
    """k >= 0 with 2^-k (y + t x) <= 2^1022 (ProtectUpdate, Section 4)."""
    return lib().orc_protect_upd(y, t, x)


def protect_div(b: float, t: float) -> int:
    """k >= 0 with 2^-k b <= t 2^1022 (ProtectDivision, Section 4)."""
    return lib().orc_protect_div(b, t)


def cdiv(a: complex, b: complex) -> complex:
    qr, qi = ctypes.c_double(), ctypes.c_double()
    lib().orc_cdiv(a.real, a.imag, b.real, b.imag, ctypes.byref(qr), ctypes.byref(qi))
    return complex(qr.value, qi.value)


def blocks(S, T):
    S, T = _fortran(S), _fortran(T)
    n = S.shape[0]
    blk = np.zeros(n, dtype=np.int8)
    st = lib().orc_blocks(n, S.ctypes.data, max(n, 1), T.ctypes.data, max(n, 1), blk.ctypes.data)
    return st, blk


def eigpairs(S, T):
    """(status, blk, a, b, beta, sigma): the eigenvalue (a + i b)/beta of every row."""
    S, T = _fortran(S), _fortran(T)
    n = S.shape[0]
    st, blk = blocks(S, T)
    a = np.zeros(n)
    b = np.zeros(n)
    beta = np.zeros(n)
    sigma = np.zeros(n, dtype=np.int32)
    if st == 0:
        st = lib().orc_eigpairs(n, S.ctypes.data, max(n, 1), T.ctypes.data, max(n, 1),
                                blk.ctypes.data, a.ctypes.data, b.ctypes.data, beta.ctypes.data,
                                sigma.ctypes.data)
    return st, blk, a, b, beta, sigma


def evc(S, T, select=None, normalise: bool = True, plain: bool = False, nthreads: int = 1):
    """All (or the selected) eigenvectors: returns (status, V, scale, m).

    ``V`` is n x m (column-major), ``scale`` int32[m]; with ``normalise`` each
    vector has largest-modulus entry exactly 1 and scale is the exponent of its
    growth relative to a unit tip; otherwise the represented vector is
    2^scale * V[:, c].
    """
    S, T = _fortran(S), _fortran(T)
    n = S.shape[0]
    V = np.zeros((n, max(n, 1)), order="F")
    scale = np.zeros(max(n, 1), dtype=np.int32)
    m = ctypes.c_int(0)
    sel = None
    if select is not None:
        sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32))
    flags = (0 if normalise else FLAG_NO_NORMALISE) | (FLAG_PLAIN if plain else 0)
    st = lib().orc_evc(n, S.ctypes.data, max(n, 1), T.ctypes.data, max(n, 1),
                       None if sel is None else sel.ctypes.data, flags,
                       V.ctypes.data, max(n, 1), scale.ctypes.data, ctypes.byref(m), int(nthreads))
    mm = m.value
    return st, V[:, :mm].copy(order="F"), scale[:mm].copy(), mm


def _fortran_c(A):
    A = np.asarray(A, dtype=np.complex128)
    return A if A.flags.f_contiguous else np.asfortranarray(A)


def eigpairs_cplx(S, T):
    """(status, alpha, beta, sigma) of a complex triangular pencil: the
    eigenvalue alpha/beta of every diagonal entry, pre-scaled by 2^-sigma."""
    S, T = _fortran_c(S), _fortran_c(T)
    n = S.shape[0]
    alpha = np.zeros(n, dtype=np.complex128)
    beta = np.zeros(n, dtype=np.complex128)
    sigma = np.zeros(n, dtype=np.int32)
    st = lib().orc_eigpairs_cplx(n, S.ctypes.data, max(n, 1), T.ctypes.data, max(n, 1),
                                 alpha.ctypes.data, beta.ctypes.data, sigma.ctypes.data)
    return st, alpha, beta, sigma


def evc_cplx(S, T, select=None, normalise: bool = True, plain: bool = False, nthreads: int = 1):
    """Eigenvectors of a complex pencil in generalized Schur form (S, T upper
    triangular, complex128): returns (status, V, scale, m) with V complex n x m.

    One column per selected diagonal entry, in the order of the diagonal;
    with ``normalise`` each vector has largest-modulus entry exactly 1 and
    scale is the exponent of its growth relative to a unit tip, otherwise the
    represented vector is 2^scale * V[:, c].
    """
    S, T = _fortran_c(S), _fortran_c(T)
    n = S.shape[0]
    V = np.zeros((n, max(n, 1)), dtype=np.complex128, order="F")
    scale = np.zeros(max(n, 1), dtype=np.int32)
    m = ctypes.c_int(0)
    sel = None
    if select is not None:
        sel = np.ascontiguousarray(np.asarray(select, dtype=np.int32))
    flags = (0 if normalise else FLAG_NO_NORMALISE) | (FLAG_PLAIN if plain else 0)
    st = lib().orc_evc_cplx(n, S.ctypes.data, max(n, 1), T.ctypes.data, max(n, 1),
                            None if sel is None else sel.ctypes.data, flags,
                            V.ctypes.data, max(n, 1), scale.ctypes.data, ctypes.byref(m), int(nthreads))
    mm = m.value
    return st, V[:, :mm].copy(order="F"), scale[:mm].copy(), mm
