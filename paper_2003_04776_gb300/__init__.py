"""Python binding of libpevc (robust generalized eigenvectors on GB300).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libpevc.so``; PyTorch provides device memory and streams.  The
functions ``pevc_plan``, ``pevc_solve``, ``pevc_solve_batched``,
``pevc_destroy``, ``pevc_strerror``, ``pevc_plan_info``,
``pevc_last_stats``, ``pevc_set_profile``, ``pevc_kernel_profile`` and
``pevc_solve_static`` mirror the C ABI of ``include/pevc.h`` one to one (raw
pointers and sizes); ``Plan`` wraps them for torch tensors.

There is no CPU fallback: importing this module fails loudly when the
compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpevc.so")

FP64 = 0
SPLIT_BF16X3 = 1
SPLIT_FP8X4 = 2
SPLIT_BF16X5 = 3
PRECISIONS = {"fp64": FP64, "bf16x3": SPLIT_BF16X3, "fp8x4": SPLIT_FP8X4, "bf16x5": SPLIT_BF16X5}

NO_NORMALISE = 1
NO_CORRECTION = 2
BT_EMULATED = 4      # pevc_backtransform: FP64 GEMM by fixed-point emulation
STAGE_WALK = 8       # FP64 plans: the stage walk from the host instead of the device-side scheduler
AUTOTUNE = 16        # pevc_plan: time the candidate settings and keep the fastest
DEVICE_WALK = 32     # FP64 plans: the device-side scheduler whatever the order
BT_CUBLAS = 64       # pevc_backtransform: cuBLAS FP64 GEMM instead of the library's split GEMM

SUCCESS = 0
ERR_NOT_SCHUR = 1
ERR_NONFINITE = 2
ERR_INDEFINITE = 3
ERR_TIMEOUT = 4
ERR_CUDA = 5
ERR_NOMEM = 6
ERR_UNSUPPORTED = 7
ERR_TOO_LARGE = 8

STATIC_N_MAX = 512   # largest order of pevc_solve_static

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpevc.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python paper_2003_04776_gb300/build.py")

_lib = ctypes.CDLL(LIB_PATH)
_vp, _i, _u = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
_lib.pevc_plan.argtypes = [ctypes.POINTER(_vp), _i, _i, _i, _i, _u, _vp]
_lib.pevc_plan.restype = _i
_lib.pevc_solve.argtypes = [_vp, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp, ctypes.POINTER(_i)]
_lib.pevc_solve.restype = _i
_lib.pevc_solve_batched.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.pevc_solve_batched.restype = _i
_lib.pevc_destroy.argtypes = [_vp]
_lib.pevc_destroy.restype = _i
_lib.pevc_strerror.argtypes = [_i]
_lib.pevc_strerror.restype = ctypes.c_char_p
_lib.pevc_plan_info.argtypes = [_vp, _vp]
_lib.pevc_plan_info.restype = _i
_lib.pevc_last_stats.argtypes = [_vp, _vp]
_lib.pevc_last_stats.restype = _i
_lib.pevc_set_profile.argtypes = [_vp, _i]
_lib.pevc_set_profile.restype = _i
_lib.pevc_kernel_profile.argtypes = [_vp, _vp]
_lib.pevc_kernel_profile.restype = _i
_lib.pevc_solve_static.argtypes = [_vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp, ctypes.POINTER(_i), _u, _vp]
_lib.pevc_solve_static.restype = _i
_lib.pevc_backtransform.argtypes = [_vp, _vp, _i, _i, _vp, _i, _i, _vp, _vp, _i, _u]
_lib.pevc_backtransform.restype = _i
_lib.pevc_solve_left.argtypes = [_vp, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp, ctypes.POINTER(_i)]
_lib.pevc_solve_left.restype = _i
_lib.pevc_solve_cplx.argtypes = [_vp, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp, ctypes.POINTER(_i)]
_lib.pevc_solve_cplx.restype = _i
_lib.pevc_solve_cplx_left.argtypes = [_vp, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp, ctypes.POINTER(_i)]
_lib.pevc_solve_cplx_left.restype = _i
_lib.pevc_backtransform_cplx.argtypes = [_vp, _vp, _i, _i, _vp, _i, _i, _vp, _i, _u]
_lib.pevc_backtransform_cplx.restype = _i
_lib.pevc_watchdog_selftest.argtypes = [_vp, _i, ctypes.c_longlong]
_lib.pevc_watchdog_selftest.restype = _i
_lib.pevc_scheduler_selftest.argtypes = [_vp, _i, ctypes.c_longlong]
_lib.pevc_scheduler_selftest.restype = _i
_lib.pevc_autotune_log.argtypes = [_vp, _vp, _i]
_lib.pevc_autotune_log.restype = _i
_lib.pevc_solve_host.argtypes = [_vp, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp, ctypes.POINTER(_i)]
_lib.pevc_solve_host.restype = _i
_lib.pevc_last_host_bytes.argtypes = [_vp, _vp]
_lib.pevc_last_host_bytes.restype = _i

EXPORTS = ("pevc_plan", "pevc_solve", "pevc_solve_batched", "pevc_destroy", "pevc_strerror",
           "pevc_plan_info", "pevc_last_stats", "pevc_set_profile", "pevc_kernel_profile",
           "pevc_solve_static", "pevc_backtransform", "pevc_solve_left", "pevc_solve_cplx",
           "pevc_solve_cplx_left", "pevc_backtransform_cplx", "pevc_watchdog_selftest",
           "pevc_scheduler_selftest", "pevc_autotune_log", "pevc_solve_host", "pevc_last_host_bytes")


# ----------------------------------------------------------- raw C ABI names

def pevc_plan(n_max: int, batch_max: int = 1, prec: int = FP64, tile: int = 0, flags: int = 0,
              stream: int = 0):
    """Returns (status, plan handle)."""
    h = _vp()
    st = _lib.pevc_plan(ctypes.byref(h), int(n_max), int(batch_max), int(prec), int(tile),
                        int(flags), _vp(stream) if stream else None)
    return st, h


def pevc_solve(plan, S: int, lds: int, T: int, ldt: int, n: int, select: int, V: int, ldv: int,
               scale: int):
    """Raw pointers (device addresses as ints).  Returns (status, m_out)."""
    m = _i(0)
    st = _lib.pevc_solve(plan, _vp(S), lds, _vp(T), ldt, n, _vp(select) if select else None,
                         _vp(V), ldv, _vp(scale), ctypes.byref(m))
    return st, m.value


def pevc_solve_host(plan, S: int, lds: int, T: int, ldt: int, n: int, select: int, V: int, ldv: int,
                    scale: int):
    """Raw pointers (host addresses as ints).  Returns (status, m_out)."""
    m = _i(0)
    st = _lib.pevc_solve_host(plan, _vp(S), lds, _vp(T), ldt, n, _vp(select) if select else None,
                              _vp(V), ldv, _vp(scale), ctypes.byref(m))
    return st, m.value


def pevc_last_host_bytes(plan):
    """Bytes the last pevc_solve_host copied: (status, (host to device, device to host))."""
    out = (ctypes.c_longlong * 2)()
    st = _lib.pevc_last_host_bytes(plan, out)
    return st, (int(out[0]), int(out[1]))


def pevc_solve_batched(plan, count, S, lds, T, ldt, n, select, V, ldv, scale):
    """Lists of device addresses / ints.  Returns (status, m_out list, status list)."""
    P = ctypes.c_void_p * max(count, 1)
    I = ctypes.c_int * max(count, 1)
    sel = None if select is None else P(*[_vp(x) if x else None for x in select])
    m_out = I()
    stat = I()
    st = _lib.pevc_solve_batched(plan, count, P(*[_vp(x) for x in S]), I(*lds), P(*[_vp(x) for x in T]),
                                 I(*ldt), I(*n), sel, P(*[_vp(x) for x in V]), I(*ldv),
                                 P(*[_vp(x) for x in scale]), m_out, stat)
    return st, list(m_out)[:count], list(stat)[:count]


def pevc_destroy(plan) -> int:
    return _lib.pevc_destroy(plan)


def pevc_strerror(code: int) -> str:
    return _lib.pevc_strerror(int(code)).decode()


def pevc_plan_info(plan):
    info = (ctypes.c_int * 8)()
    st = _lib.pevc_plan_info(plan, info)
    return st, list(info)


def pevc_last_stats(plan):
    stats = (ctypes.c_double * 8)()
    st = _lib.pevc_last_stats(plan, stats)
    return st, list(stats)


def pevc_set_profile(plan, on: bool) -> int:
    return _lib.pevc_set_profile(plan, 1 if on else 0)


def pevc_kernel_profile(plan):
    out = (ctypes.c_double * 12)()
    st = _lib.pevc_kernel_profile(plan, out)
    return st, list(out)


def pevc_solve_static(S: int, lds: int, T: int, ldt: int, n: int, select: int, V: int, ldv: int,
                      scale: int, flags: int = 0, stream: int = 0):
    """FP64 solve without device allocation (order <= STATIC_N_MAX; the
    workspace is a device array inside the library).  Raw pointers as in
    pevc_solve.  Returns (status, m_out)."""
    m = _i(0)
    st = _lib.pevc_solve_static(_vp(S), lds, _vp(T), ldt, n, _vp(select) if select else None, _vp(V), ldv,
                                _vp(scale), ctypes.byref(m), int(flags), _vp(stream) if stream else None)
    return st, m.value


def pevc_backtransform(plan, Z: int, ldz: int, n: int, V: int, ldv: int, m: int, kinds, X: int, ldx: int,
                       flags: int = 0):
    """X = Z V with every eigenvector normalised (raw device pointers; kinds
    a host sequence of m ints, or None for the plan's last solve).  Returns
    the status."""
    k = None
    if kinds is not None:
        k = (_i * max(len(kinds), 1))(*[int(x) for x in kinds])
    return _lib.pevc_backtransform(plan, _vp(Z), ldz, n, _vp(V), ldv, m, k, _vp(X), ldx, int(flags))


def pevc_solve_left(plan, S: int, lds: int, T: int, ldt: int, n: int, select: int, U: int, ldu: int,
                    scale: int):
    """Left eigenvectors (raw device pointers as in pevc_solve).  Returns (status, m_out)."""
    m = _i(0)
    st = _lib.pevc_solve_left(plan, _vp(S), lds, _vp(T), ldt, n, _vp(select) if select else None, _vp(U), ldu,
                              _vp(scale), ctypes.byref(m))
    return st, m.value


def pevc_solve_cplx(plan, S: int, lds: int, T: int, ldt: int, n: int, select: int, V: int, ldv: int,
                    scale: int):
    """Eigenvectors of a complex triangular pencil (raw device pointers to
    complex128 column-major arrays, leading dimensions in complex elements).
    Returns (status, m_out)."""
    m = _i(0)
    st = _lib.pevc_solve_cplx(plan, _vp(S), lds, _vp(T), ldt, n, _vp(select) if select else None, _vp(V), ldv,
                              _vp(scale), ctypes.byref(m))
    return st, m.value


def pevc_solve_cplx_left(plan, S: int, lds: int, T: int, ldt: int, n: int, select: int, U: int, ldu: int,
                         scale: int):
    """Left eigenvectors of a complex triangular pencil (raw device pointers
    as in pevc_solve_cplx).  Returns (status, m_out)."""
    m = _i(0)
    st = _lib.pevc_solve_cplx_left(plan, _vp(S), lds, _vp(T), ldt, n, _vp(select) if select else None, _vp(U),
                                   ldu, _vp(scale), ctypes.byref(m))
    return st, m.value


def pevc_backtransform_cplx(plan, Z: int, ldz: int, n: int, V: int, ldv: int, m: int, X: int, ldx: int,
                            flags: int = 0) -> int:
    """X = Z V for complex eigenvectors with every column normalised (raw
    device pointers to complex128 arrays).  Returns the status."""
    return _lib.pevc_backtransform_cplx(plan, _vp(Z), ldz, n, _vp(V), ldv, m, _vp(X), ldx, int(flags))


def pevc_watchdog_selftest(plan, withhold: int, cycles: int) -> int:
    """One bounded device wait, its arrival withheld or not.  Returns the
    status (0, or ERR_TIMEOUT when the bound ran out)."""
    return _lib.pevc_watchdog_selftest(plan, int(withhold), int(cycles))


def pevc_scheduler_selftest(plan, withhold: int, cycles: int) -> int:
    """The scheduler's bounded dependence wait (withhold=1: nothing meets the
    dependence, the wait gives up after `cycles`).  Returns the status."""
    return _lib.pevc_scheduler_selftest(plan, int(withhold), int(cycles))


def pevc_autotune_log(plan):
    """The candidates an autotuned plan timed: (count, [(tile, prec,
    stage_walk, ms), ...])."""
    cap = 64
    out = (ctypes.c_double * (4 * cap))()
    k = _lib.pevc_autotune_log(plan, out, cap)
    if k < 0:
        return k, []
    return k, [tuple(out[4 * q:4 * q + 4]) for q in range(min(k, cap))]


# ------------------------------------------------------------ torch wrapper

class PevcError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: status {code}: {pevc_strerror(code)}")


def to_device_colmajor(A, device="cuda"):
    """Column-major float64 copy of A on the device (a torch tensor whose
    storage is A in column-major order, i.e. a row-major A^T)."""
    import torch
    if isinstance(A, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T))
        return t.to(device)
    if A.dtype != torch.float64:
        A = A.double()
    return A.t().contiguous().to(device)


def to_device_colmajor_c(A, device="cuda"):
    """Column-major complex128 copy of A on the device."""
    import torch
    if isinstance(A, np.ndarray):
        return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.complex128).T)).to(device)
    if A.dtype != torch.complex128:
        A = A.to(torch.complex128)
    return A.t().contiguous().to(device)


class Plan:
    """A plan (device workspace for order <= n_max) bound to a torch stream."""

    def __init__(self, n_max: int, prec="fp64", tile: int = 0, batch_max: int = 1,
                 normalise: bool = True, correction: bool = True, stream=None,
                 autotune: bool = False, stage_walk: bool = False, device_walk: bool = False):
        import torch
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.flags = ((0 if normalise else NO_NORMALISE) | (0 if correction else NO_CORRECTION) |
                      (AUTOTUNE if autotune else 0) | (STAGE_WALK if stage_walk else 0) |
                      (DEVICE_WALK if device_walk else 0))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st, h = pevc_plan(n_max, batch_max, self.prec, tile, self.flags, self.stream.cuda_stream)
        if st:
            raise PevcError(st, "pevc_plan")
        self.h = h
        self.n_max = n_max

    def close(self):
        if getattr(self, "h", None):
            pevc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return pevc_plan_info(self.h)[1]

    @property
    def stats(self):
        return pevc_last_stats(self.h)[1]

    def profile(self, on: bool = True):
        st = pevc_set_profile(self.h, on)
        if st:
            raise PevcError(st, "pevc_set_profile")

    def kernel_profile(self):
        """Per-kind totals of the last solve (profiling on): milliseconds,
        launches and tensor-core flops of the updates, diagonal solves,
        slicing and the remaining kernels; plus the launch count."""
        out = pevc_kernel_profile(self.h)[1]
        names = ("update", "diag", "slice", "other")
        d = {}
        for k, nm in enumerate(names):
            d[f"{nm}_ms"] = out[3 * k]
            d[f"{nm}_launches"] = int(out[3 * k + 1])
            d[f"{nm}_tensor_flops"] = out[3 * k + 2]
        d["launches"] = int(self.stats[6])
        return d

    def solve_colmajor(self, St, Tt, n, V, scale, select=None, lds=None, ldt=None, ldv=None):
        """Device tensors already in column-major storage (see to_device_colmajor)."""
        st, m = pevc_solve(self.h, St.data_ptr(), lds or max(n, 1), Tt.data_ptr(), ldt or max(n, 1), n,
                           select.data_ptr() if select is not None else 0, V.data_ptr(),
                           ldv or max(n, 1), scale.data_ptr())
        return st, m

    def solve_host(self, S, T, V, scale, select=None):
        """Host arrays through pevc_solve_host (the copies stream behind the
        solve).  S, T: n x n column-major host buffers -- numpy arrays in
        Fortran order, or CPU torch tensors holding the transposes (row-major
        storage of S^T is column-major storage of S), pinned for the fastest
        copies; V: an n x n host buffer of the same kind for the output;
        scale: int32[n].  Returns (status, m_out)."""
        def ptr(x):
            if isinstance(x, np.ndarray):
                if x.ndim == 2 and not x.flags.f_contiguous:
                    raise ValueError("solve_host: numpy matrices must be in Fortran (column-major) order")
                return x.ctypes.data
            if x.is_cuda or not x.is_contiguous():
                raise ValueError("solve_host: torch tensors must be contiguous host tensors")
            return x.data_ptr()
        n = int(S.shape[0])
        sel = None
        if select is not None:
            sel = np.ascontiguousarray(select, dtype=np.int32)
        return pevc_solve_host(self.h, ptr(S), max(n, 1), ptr(T), max(n, 1), n,
                               sel.ctypes.data if sel is not None else 0, ptr(V), max(n, 1), ptr(scale))

    @property
    def host_bytes(self):
        st, b = pevc_last_host_bytes(self.h)
        if st:
            raise PevcError(st, "pevc_last_host_bytes")
        return b

    def solve_batched(self, pencils, selects=None):
        """Several pencils [(S, T), ...] in one pevc_solve_batched call (the
        plan needs batch_max >= len(pencils)).  Returns (status, [(V, scale,
        status_b), ...]) with V as n x m numpy arrays."""
        import torch
        count = len(pencils)
        keep = []
        S_p, T_p, V_p, sc_p, sel_p, n_l, ld_l = [], [], [], [], [], [], []
        for b, (S, T) in enumerate(pencils):
            n = int(S.shape[0])
            if n > 0:
                St, Tt = to_device_colmajor(S), to_device_colmajor(T)
            else:
                St = Tt = torch.zeros(1, dtype=torch.float64, device="cuda")
            V = torch.empty((max(n, 1), max(n, 1)), dtype=torch.float64, device="cuda")
            sc = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
            sel = None
            if selects is not None and selects[b] is not None:
                sel = torch.as_tensor(np.asarray(selects[b], dtype=np.int32)).to("cuda")
            keep += [St, Tt, V, sc, sel]
            S_p.append(St.data_ptr())
            T_p.append(Tt.data_ptr())
            V_p.append(V.data_ptr())
            sc_p.append(sc.data_ptr())
            sel_p.append(sel.data_ptr() if sel is not None else 0)
            n_l.append(n)
            ld_l.append(max(n, 1))
        with torch.cuda.stream(self.stream):
            st, m_out, stat = pevc_solve_batched(self.h, count, S_p, ld_l, T_p, ld_l, n_l,
                                                 sel_p if selects is not None else None, V_p, ld_l, sc_p)
        out = []
        for b in range(count):
            n, m = n_l[b], m_out[b]
            V, sc = keep[5 * b + 2], keep[5 * b + 3]
            Vh = V[:m].cpu().numpy().T if m else np.zeros((n, 0))
            out.append((np.asfortranarray(Vh[:n, :m]), sc[:m].cpu().numpy(), stat[b]))
        return st, out

    def backtransform(self, Z, V, kinds=None, normalise: bool = True, emulated: bool = False,
                      check: bool = True, cublas: bool = False):
        """X = Z V for the eigenvectors V of the plan's pencil (numpy n x m),
        each eigenvector normalised to largest-modulus entry 1 unless
        normalise is False; the library's split GEMM, or cuBLAS's FP64 GEMM
        with cublas (emulated: its fixed-point emulation).  kinds as in
        pevc_backtransform (None: the columns of the plan's last solve).
        Returns (X as numpy, status)."""
        import torch
        n, m = int(Z.shape[0]), int(V.shape[1])
        Zt = to_device_colmajor(Z)
        Vt = to_device_colmajor(V) if m else torch.zeros(1, dtype=torch.float64, device="cuda")
        X = torch.empty((max(m, 1), max(n, 1)), dtype=torch.float64, device="cuda")   # column-major storage
        flags = ((0 if normalise else NO_NORMALISE) | (BT_EMULATED if emulated else 0) |
                 (BT_CUBLAS if cublas else 0))
        with torch.cuda.stream(self.stream):
            st = pevc_backtransform(self.h, Zt.data_ptr(), max(n, 1), n, Vt.data_ptr(), max(n, 1), m,
                                    kinds, X.data_ptr(), max(n, 1), flags)
        if check and st:
            raise PevcError(st, "pevc_backtransform")
        Xh = X[:m].cpu().numpy().T if m else np.zeros((n, 0))
        return np.asfortranarray(Xh[:n, :m]), st

    def solve_left(self, S, T, select=None, check: bool = True):
        """Left eigenvectors u^H (beta S - alpha T) = 0 of (S, T) (numpy or
        torch).  Returns (U as an n x m numpy array, scale int32[m], status)."""
        import torch
        n = int(S.shape[0])
        St = to_device_colmajor(S)
        Tt = to_device_colmajor(T)
        U = torch.empty((max(n, 1), max(n, 1)), dtype=torch.float64, device="cuda")   # column-major storage
        scale = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        sel = None
        if select is not None:
            sel = torch.as_tensor(np.asarray(select, dtype=np.int32)).to("cuda")
        with torch.cuda.stream(self.stream):
            st, m = pevc_solve_left(self.h, St.data_ptr(), max(n, 1), Tt.data_ptr(), max(n, 1), n,
                                    sel.data_ptr() if sel is not None else 0, U.data_ptr(), max(n, 1),
                                    scale.data_ptr())
        if check and st:
            raise PevcError(st, "pevc_solve_left")
        Uh = U[:m].cpu().numpy().T if m else np.zeros((n, 0))
        return np.asfortranarray(Uh[:n, :m]), scale[:m].cpu().numpy(), st

    def _solve_cplx_with(self, fn, name, S, T, select, check):
        """Marshals a complex solve (right or left eigenvectors): complex128
        column-major copies of S and T on the device, the output in a torch
        tensor, the result back as an n x m complex numpy array."""
        import torch
        n = int(S.shape[0])
        St = to_device_colmajor_c(S)
        Tt = to_device_colmajor_c(T)
        V = torch.empty((max(n, 1), max(n, 1)), dtype=torch.complex128, device="cuda")   # column-major storage
        scale = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        sel = None
        if select is not None:
            sel = torch.as_tensor(np.asarray(select, dtype=np.int32)).to("cuda")
        with torch.cuda.stream(self.stream):
            st, m = fn(self.h, St.data_ptr(), max(n, 1), Tt.data_ptr(), max(n, 1), n,
                       sel.data_ptr() if sel is not None else 0, V.data_ptr(), max(n, 1), scale.data_ptr())
        if check and st:
            raise PevcError(st, name)
        Vh = V[:m].cpu().numpy().T if m else np.zeros((n, 0), dtype=complex)
        return np.asfortranarray(Vh[:n, :m]), scale[:m].cpu().numpy(), st

    def solve_cplx(self, S, T, select=None, check: bool = True):
        """Eigenvectors of a complex pencil in generalized Schur form (S, T
        upper triangular, numpy or torch, complex128).  Returns (V as an
        n x m complex numpy array, scale int32[m], status)."""
        return self._solve_cplx_with(pevc_solve_cplx, "pevc_solve_cplx", S, T, select, check)

    def solve_cplx_left(self, S, T, select=None, check: bool = True):
        """Left eigenvectors u^H (beta S - alpha T) = 0 of a complex triangular
        pencil.  Returns (U as an n x m complex numpy array, scale, status)."""
        return self._solve_cplx_with(pevc_solve_cplx_left, "pevc_solve_cplx_left", S, T, select, check)

    def backtransform_cplx(self, Z, V, normalise: bool = True, check: bool = True):
        """X = Z V for complex eigenvectors V (numpy or torch, complex128):
        the eigenvectors of (Q S Z^H, Q T Z^H).  Returns (X, status)."""
        import torch
        n, m = int(Z.shape[0]), int(V.shape[1])
        Zt = to_device_colmajor_c(Z)
        Vt = to_device_colmajor_c(V)
        X = torch.empty((max(m, 1), max(n, 1)), dtype=torch.complex128, device="cuda")   # column-major storage
        with torch.cuda.stream(self.stream):
            st = pevc_backtransform_cplx(self.h, Zt.data_ptr(), max(n, 1), n, Vt.data_ptr(), max(n, 1), m,
                                         X.data_ptr(), max(n, 1), 0 if normalise else NO_NORMALISE)
        if check and st:
            raise PevcError(st, "pevc_backtransform_cplx")
        Xh = X[:m].cpu().numpy().T if m else np.zeros((n, 0), dtype=complex)
        return np.asfortranarray(Xh[:n, :m]), st

    def solve(self, S, T, select=None, check: bool = True):
        """Eigenvectors of (S, T) given as numpy arrays or torch tensors.

        Returns (V as an n x m numpy array, scale int32[m], status)."""
        import torch
        n = int(S.shape[0])
        St = to_device_colmajor(S)
        Tt = to_device_colmajor(T)
        V = torch.empty((max(n, 1), max(n, 1)), dtype=torch.float64, device="cuda")   # column-major storage
        scale = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        sel = None
        if select is not None:
            sel = torch.as_tensor(np.asarray(select, dtype=np.int32)).to("cuda")
        with torch.cuda.stream(self.stream):
            st, m = self.solve_colmajor(St, Tt, n, V, scale, sel)
        if check and st:
            raise PevcError(st, "pevc_solve")
        Vh = V[:m].cpu().numpy().T if m else np.zeros((n, 0))
        return np.asfortranarray(Vh[:n, :m]), scale[:m].cpu().numpy(), st
