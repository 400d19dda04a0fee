"""CPU oracle for the batched 2x2 SVD of Novakovic (arXiv 2005.07403).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It wraps the plain C
in ``svd2_oracle.c`` (built with gcc, ``-ffp-contract=off``) through ctypes and
shares no code with the CUDA library.

Arrays use the split layout of Sec. 3: one 1-D array per matrix element, in the
record order of Sec. 8 -- real: (a11, a21, a12, a22); complex: (Re a11, Im a11,
Re a21, Im a21, Re a12, Im a12, Re a22, Im a22).  Here those are passed as one
2-D numpy array of shape (4, n) or (8, n), C-contiguous.

Scale exponents come back as int32 with ``ZERO_S`` (INT32_MAX) standing for the
s = DBL_MAX of the zero matrix (Eq. 2).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "svd2_oracle.c")
BODY = os.path.join(HERE, "svd2_oracle_body.h")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsvd2_oracle.so")

ZERO_S = 2**31 - 1
BACKSCALE = 1
SINE = 2          # U by Eq. 31 (sines) instead of Eq. 29 (tangents)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (x86-64 or AArch64)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(BODY))
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    libs = ["-lquadmath"] if platform.machine() in ("x86_64", "i686") else []
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, SRC] + libs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = Oracle(LIB_PATH)
    return _lib


def build_variant(src_text: str, body_text: str, out_dir: str) -> "Oracle":
    """Compile a modified copy of the oracle sources into ``out_dir`` and load
    it.  Used only by the test that plants mistakes in the oracle to show that
    the pins catch them."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "svd2_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    with open(os.path.join(out_dir, "svd2_oracle_body.h"), "w") as f:
        f.write(body_text)
    lib = os.path.join(out_dir, "libvariant.so")
    libs = ["-lquadmath"] if platform.machine() in ("x86_64", "i686") else []
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                    "-fopenmp", "-fPIC", "-shared", "-o", lib, src] + libs + ["-lm"],
                   check=True)
    return Oracle(lib)


_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def _declare(lib):
    pp = ctypes.POINTER(ctypes.c_void_p)
    for name in ("svd2o_batch_d", "svd2o_batch_s", "svd2o_batch_z", "svd2o_batch_c"):
        f = getattr(lib, name)
        f.argtypes = [_I64, pp, pp, pp, _P, _P, _P, _P, ctypes.c_uint32, ctypes.c_int]
        f.restype = None
    for name in ("svd2o_batch_s_rerun", "svd2o_batch_c_rerun", "svd2o_batch_s_tan64"):
        f = getattr(lib, name)
        f.argtypes = [_I64, pp, pp, pp, _P, _P, _P, _P, ctypes.c_int, ctypes.c_uint32,
                      ctypes.c_int]
        f.restype = _I64
    for name in ("svd2o_truth_d", "svd2o_truth_z"):
        f = getattr(lib, name)
        f.argtypes = [_I64, pp, _P, _P, _P, _P, _P]
        f.restype = None
    for name in ("svd2o_metrics_d", "svd2o_metrics_z"):
        f = getattr(lib, name)
        f.argtypes = [_I64, pp, pp, pp, _P, _P, _P, _P, _P, _P, _P]
        f.restype = None
    lib.svd2o_bwd_d.argtypes = [_I64, pp, pp, _P, _P, pp, pp, _P, _P, pp, ctypes.c_double]
    lib.svd2o_bwd_d.restype = None
    lib.svd2o_bwd_s.argtypes = [_I64, pp, pp, _P, _P, pp, pp, _P, _P, pp, ctypes.c_float]
    lib.svd2o_bwd_z.argtypes = [_I64, pp, pp, _P, _P, pp, pp, _P, _P, pp, ctypes.c_double]
    lib.svd2o_bwd_c.argtypes = [_I64, pp, pp, _P, _P, pp, pp, _P, _P, pp, ctypes.c_float]
    lib.svd2o_bwd_s.restype = None
    lib.svd2o_refgrad_d.argtypes = [_I64, pp, pp, pp, _P, _P, pp, pp, ctypes.c_double]
    lib.svd2o_refgrad_d.restype = None
    lib.svd2o_batch_q_from_d.argtypes = [_I64, pp, pp, pp, pp, pp, _P, _P, _P, _P, _P]
    lib.svd2o_batch_q_from_d.restype = None
    lib.svd2o_max_threads.restype = ctypes.c_int
    lib.svd2o_const_sqrt_dbl_max_literal.restype = ctypes.c_double
    lib.svd2o_const_sqrt_dbl_max.restype = ctypes.c_double
    lib.svd2o_const_sqrt_flt_max.restype = ctypes.c_float


def _ptrs(arr2d):
    """ctypes array of row pointers of a C-contiguous 2-D numpy array."""
    assert arr2d.flags.c_contiguous
    rows = arr2d.shape[0]
    out = (ctypes.c_void_p * rows)()
    for i in range(rows):
        out[i] = arr2d[i].ctypes.data
    return out


def _p(a):
    return None if a is None else a.ctypes.data


def _as(a, dtype, rows):
    a = np.ascontiguousarray(a, dtype=dtype)
    assert a.ndim == 2 and a.shape[0] == rows, a.shape
    return a


class Oracle:
    """One loaded build of the oracle library."""

    def __init__(self, path):
        self.lib = ctypes.CDLL(path)
        _declare(self.lib)

    def max_threads(self) -> int:
        return self.lib.svd2o_max_threads()


    def svd2(self, A, *, backscale: bool = False, sine: bool = False, nthreads: int = 0):
        """Step oracle O1 (Sec. 2 - Sec. 7, Eq. 29) over a batch.

        ``A`` has shape (4, n) (real) or (8, n) (complex), dtype float64 or float32;
        the precision of the method is the dtype's.  Returns a dict with U, V (same
        shape as A), smax, smin (scaled, Eq. 17, unless backscale), s (int32) and
        piv (uint8; bit 0 = column swap P_c, bit 1 = row swap P_r*).  ``sine``: U
        assembled by Eq. 31 from the sines sin = cos tan (Sec. 7) instead of
        the tangent form of Eq. 29.
        """
        A = np.asarray(A)
        rows = A.shape[0]
        dt = np.float64 if A.dtype == np.float64 else np.float32
        if A.dtype not in (np.float64, np.float32):
            raise TypeError("float64 or float32 input")
        A = _as(A, dt, rows)
        n = A.shape[1]
        U = np.empty_like(A)
        V = np.empty_like(A)
        smax = np.empty(n, dt)
        smin = np.empty(n, dt)
        s = np.empty(n, np.int32)
        piv = np.empty(n, np.uint8)
        lib = self.lib
        name = {(4, np.float64): "svd2o_batch_d", (4, np.float32): "svd2o_batch_s",
                (8, np.float64): "svd2o_batch_z", (8, np.float32): "svd2o_batch_c"}[(rows, dt)]
        getattr(lib, name)(n, _ptrs(A), _ptrs(U), _ptrs(V), _p(smax), _p(smin), _p(s), _p(piv),
                           (BACKSCALE if backscale else 0) | (SINE if sine else 0), nthreads)
        return dict(U=U, V=V, smax=smax, smin=smin, s=s, piv=piv)


    def svd2_rerun(self, A, tau_log2: int, *, backscale: bool = False, nthreads: int = 0):
        """FP32 form with FP64 re-run of the matrices with sigma'_min < 2^tau_log2 sigma'_max.

        ``A`` is float32 of shape (4, n) or (8, n).  Returns the dict of ``svd2``
        (float32 outputs, s on the float scale) plus ``flagged`` (uint8) and
        ``count``.
        """
        A = np.asarray(A)
        rows = A.shape[0]
        A = _as(A, np.float32, rows)
        n = A.shape[1]
        U = np.empty_like(A)
        V = np.empty_like(A)
        smax = np.empty(n, np.float32)
        smin = np.empty(n, np.float32)
        s = np.empty(n, np.int32)
        flagged = np.empty(n, np.uint8)
        lib = self.lib
        f = lib.svd2o_batch_s_rerun if rows == 4 else lib.svd2o_batch_c_rerun
        cnt = f(n, _ptrs(A), _ptrs(U), _ptrs(V), _p(smax), _p(smin), _p(s), _p(flagged),
                int(tau_log2), BACKSCALE if backscale else 0, nthreads)
        return dict(U=U, V=V, smax=smax, smin=smin, s=s, flagged=flagged, count=int(cnt))


    def svd2_tan64(self, A, tau_log2: int, *, backscale: bool = False, nthreads: int = 0):
        """FP32 form with the FP64 tangent step for the matrices with
        |r''_22| < 2^tau_log2 r11 (Eq. 6 - Eq. 7 in double, the rest in float).

        ``A`` is float32 of shape (4, n).  Returns the dict of ``svd2`` plus
        ``wide`` (uint8, 1 where the step ran in double) and ``count``.
        """
        A = _as(np.asarray(A), np.float32, 4)
        n = A.shape[1]
        U = np.empty_like(A)
        V = np.empty_like(A)
        smax = np.empty(n, np.float32)
        smin = np.empty(n, np.float32)
        s = np.empty(n, np.int32)
        wide = np.empty(n, np.uint8)
        cnt = self.lib.svd2o_batch_s_tan64(n, _ptrs(A), _ptrs(U), _ptrs(V), _p(smax), _p(smin),
                                           _p(s), _p(wide), int(tau_log2),
                                           BACKSCALE if backscale else 0, nthreads)
        return dict(U=U, V=V, smax=smax, smin=smin, s=s, wide=wide, count=int(cnt))


    def truth(self, A, s=None):
        """Closed-form singular values in binary128 (truth tier O2).

        With ``s`` (int32 per matrix, as returned by ``svd2``) the values are
        multiplied by 2^s in binary128 first, giving the truth of the scaled
        Sigma'.  Returns ``(smax_hi, smax_lo, smin_hi, smin_lo)`` float64 arrays.
        """
        A = np.asarray(A)
        rows = A.shape[0]
        A = _as(A, np.float64, rows)
        n = A.shape[1]
        out = [np.empty(n, np.float64) for _ in range(4)]
        lib = self.lib
        f = lib.svd2o_truth_d if rows == 4 else lib.svd2o_truth_z
        sp = None if s is None else np.ascontiguousarray(s, np.int32)
        f(n, _ptrs(A), _p(sp), *[_p(o) for o in out])
        return tuple(out)


    def metrics(self, A, U, V, smax, smin, s):
        """Per-matrix error metrics of Sec. 8 in binary128: rho (Eq. 33), delta
        (Eq. 34), eta (Eq. 35) and kappa (Eq. 32).  Inputs are float64 (float32
        results are widened exactly by the caller)."""
        A = np.asarray(A)
        rows = A.shape[0]
        A = _as(A, np.float64, rows)
        U = _as(U, np.float64, rows)
        V = _as(V, np.float64, rows)
        smax = np.ascontiguousarray(smax, np.float64)
        smin = np.ascontiguousarray(smin, np.float64)
        s = np.ascontiguousarray(s, np.int32)
        n = A.shape[1]
        rho, delta, eta, kappa = (np.empty(n, np.float64) for _ in range(4))
        lib = self.lib
        f = lib.svd2o_metrics_d if rows == 4 else lib.svd2o_metrics_z
        f(n, _ptrs(A), _ptrs(U), _ptrs(V), _p(smax), _p(smin), _p(s), _p(rho), _p(delta),
          _p(eta), _p(kappa))
        return dict(rho=rho, delta=delta, eta=eta, kappa=kappa)


    def bwd(self, U, V, s1, s2, gU, gV, g1, g2, rel_delta):
        """Adjoint of the 2x2 SVD (float64 or float32, by U's dtype; real with 4
        rows, complex with 8 rows of the split layout).  s1, s2 are back-scaled
        singular values.  Returns gA of U's shape."""
        U = np.asarray(U)
        dt = np.float64 if U.dtype == np.float64 else np.float32
        rows = U.shape[0]
        U = _as(U, dt, rows)
        V = _as(V, dt, rows)
        gU = _as(gU, dt, rows)
        gV = _as(gV, dt, rows)
        if rows == 8:
            s1, s2, g1, g2 = (np.ascontiguousarray(x, dt) for x in (s1, s2, g1, g2))
            gA = np.empty_like(U)
            f = self.lib.svd2o_bwd_z if dt == np.float64 else self.lib.svd2o_bwd_c
            f(U.shape[1], _ptrs(U), _ptrs(V), _p(s1), _p(s2), _ptrs(gU), _ptrs(gV),
              _p(g1), _p(g2), _ptrs(gA), float(rel_delta))
            return gA
        s1, s2, g1, g2 = (np.ascontiguousarray(x, dt) for x in (s1, s2, g1, g2))
        gA = np.empty_like(U)
        lib = self.lib
        if dt == np.float64:
            lib.svd2o_bwd_d(U.shape[1], _ptrs(U), _ptrs(V), _p(s1), _p(s2), _ptrs(gU), _ptrs(gV),
                            _p(g1), _p(g2), _ptrs(gA), float(rel_delta))
        else:
            lib.svd2o_bwd_s(U.shape[1], _ptrs(U), _ptrs(V), _p(s1), _p(s2), _ptrs(gU), _ptrs(gV),
                            _p(g1), _p(g2), _ptrs(gA), float(rel_delta))
        return gA


    def refgrad(self, A, gU, gV, g1, g2, rel_delta):
        """Binary128 reference gradient (the method in binary128, then the adjoint
        in binary128).  Returns (gA_hi, gA_lo), each (4, n) float64."""
        A = _as(A, np.float64, 4)
        gU = _as(gU, np.float64, 4)
        gV = _as(gV, np.float64, 4)
        g1 = np.ascontiguousarray(g1, np.float64)
        g2 = np.ascontiguousarray(g2, np.float64)
        hi = np.empty_like(A)
        lo = np.empty_like(A)
        self.lib.svd2o_refgrad_d(A.shape[1], _ptrs(A), _ptrs(gU), _ptrs(gV), _p(g1), _p(g2),
                                _ptrs(hi), _ptrs(lo), float(rel_delta))
        return hi, lo


    def svd2_quad(self, A):
        """The method of Sec. 2 run in binary128 on a float64 real batch; returns hi
        parts of U, V, back-scaled smax, smin, plus the pivot bits."""
        A = _as(A, np.float64, 4)
        n = A.shape[1]
        Uh, Ul, Vh, Vl = (np.empty_like(A) for _ in range(4))
        sxh, sxl, snh, snl = (np.empty(n, np.float64) for _ in range(4))
        piv = np.empty(n, np.uint8)
        self.lib.svd2o_batch_q_from_d(n, _ptrs(A), _ptrs(Uh), _ptrs(Ul), _ptrs(Vh), _ptrs(Vl),
                                     _p(sxh), _p(sxl), _p(snh), _p(snl), _p(piv))
        return dict(U=Uh, U_lo=Ul, V=Vh, V_lo=Vl, smax=sxh, smax_lo=sxl, smin=snh, smin_lo=snl,
                    piv=piv)


    def constants(self):
        lib = self.lib
        return dict(sqrt_dbl_max_literal=lib.svd2o_const_sqrt_dbl_max_literal(),
                    sqrt_dbl_max=lib.svd2o_const_sqrt_dbl_max(),
                    sqrt_flt_max=lib.svd2o_const_sqrt_flt_max())


def _default():
    return _load()


def max_threads():
    return _default().max_threads()


def svd2(A, *, backscale: bool = False, sine: bool = False, nthreads: int = 0):
    return _default().svd2(A, backscale=backscale, sine=sine, nthreads=nthreads)


def svd2_rerun(A, tau_log2: int, *, backscale: bool = False, nthreads: int = 0):
    return _default().svd2_rerun(A, tau_log2, backscale=backscale, nthreads=nthreads)


def svd2_tan64(A, tau_log2: int, *, backscale: bool = False, nthreads: int = 0):
    return _default().svd2_tan64(A, tau_log2, backscale=backscale, nthreads=nthreads)


def truth(A, s=None):
    return _default().truth(A, s)


def metrics(A, U, V, smax, smin, s):
    return _default().metrics(A, U, V, smax, smin, s)


def bwd(U, V, s1, s2, gU, gV, g1, g2, rel_delta):
    return _default().bwd(U, V, s1, s2, gU, gV, g1, g2, rel_delta)


def refgrad(A, gU, gV, g1, g2, rel_delta):
    return _default().refgrad(A, gU, gV, g1, g2, rel_delta)


def svd2_quad(A):
    return _default().svd2_quad(A)


def constants():
    return _default().constants()
