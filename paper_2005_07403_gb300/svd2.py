"""Thin Python binding of the C ABI in ``include/svd2.h`` (argument marshalling only).

Every step of the method runs in the sm_103a kernels of the shared library
built from ``csrc/``; torch only provides device memory and the current CUDA
stream.  There is no CPU fallback: if the library cannot be built or loaded,
or no CUDA device is present, the calls raise.

Arrays follow the split layout of Sec. 3: a tensor of shape (4, n) (real) or
(8, n) (complex, real and imaginary parts in separate rows) whose rows are the
element arrays in the record order of Sec. 8 -- a11, a21, a12, a22, or
Re a11, Im a11, Re a21, Im a21, Re a12, Im a12, Re a22, Im a22.  Each row must
be contiguous; rows need not be adjacent.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import torch

from . import build as _build

OK = 0
EINVAL = -1
ECUDA = -2
ENOMEM = -3
ETOOBIG = -4
NOALLOC_MAX_N = 1 << 20
S_ZERO = 2**31 - 1
BACKSCALE = 1
SINE = 2

OPS = {"d": 0, "z": 1, "s": 2, "c": 3, "s_tan64": 4}

_lock = threading.Lock()
_lib = None


class Svd2Error(RuntimeError):
    pass


KIND_D = 0
KIND_Z = 1


class BatchDesc(ctypes.Structure):
    """svd2_batch_desc of include/svd2.h."""
    _fields_ = [("kind", ctypes.c_int32), ("flags", ctypes.c_uint32), ("n", ctypes.c_int64),
                ("a", ctypes.c_void_p * 8), ("u", ctypes.c_void_p * 8), ("v", ctypes.c_void_p * 8),
                ("smax", ctypes.c_void_p), ("smin", ctypes.c_void_p), ("s", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    """svd2_tune_result of include/svd2.h."""
    _fields_ = [("block", ctypes.c_int), ("mpt", ctypes.c_int), ("unroll", ctypes.c_int),
                ("waves", ctypes.c_int), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"block": self.block, "mpt": self.mpt, "unroll": self.unroll,
                "waves": self.waves, "ms": self.ms}


def lib():
    """Load (building first if sources changed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    P = ctypes.c_void_p
    PP = ctypes.POINTER(ctypes.c_void_p)
    for name in ("svd2_batch_d", "svd2_batch_z", "svd2_batch_s", "svd2_batch_c"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_int64, PP, PP, PP, P, P, P, ctypes.c_uint32, P]
        f.restype = ctypes.c_int
    for name in ("svd2_values_d", "svd2_values_z", "svd2_values_s", "svd2_values_c"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_int64, PP, P, P, P, ctypes.c_uint32, P]
        f.restype = ctypes.c_int
    for name in ("svd2_batch_interleaved_d", "svd2_batch_interleaved_z",
                 "svd2_batch_interleaved_s", "svd2_batch_interleaved_c"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_int64, P, P, P, P, P, P, ctypes.c_uint32, P]
        f.restype = ctypes.c_int
    L.svd2_kog_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int64]
    L.svd2_kog_workspace_bytes.restype = ctypes.c_size_t
    for name in ("svd2_kog_step_d", "svd2_kog_step_z", "svd2_kog_step_s", "svd2_kog_step_c"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int64, P, P, ctypes.c_size_t, P]
        f.restype = ctypes.c_int
    L.svd2_kog_skipped.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    L.svd2_kog_skipped.restype = ctypes.c_int
    for name in ("svd2_batch_s_rerun", "svd2_batch_c_rerun"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_int64, PP, PP, PP, P, P, P, ctypes.c_int, ctypes.c_uint32, P,
                      ctypes.c_size_t, P]
        f.restype = ctypes.c_int
    L.svd2_batch_s_tan64.argtypes = [ctypes.c_int64, PP, PP, PP, P, P, P, ctypes.c_int,
                                     ctypes.c_uint32, P, P]
    L.svd2_batch_s_tan64.restype = ctypes.c_int
    L.svd2_batch_s_rerun_noalloc.argtypes = [ctypes.c_int64, PP, PP, PP, P, P, P, ctypes.c_int,
                                             ctypes.c_uint32, P]
    L.svd2_batch_s_rerun_noalloc.restype = ctypes.c_int
    L.svd2_rerun_workspace_bytes.argtypes = [ctypes.c_int64]
    L.svd2_rerun_workspace_bytes.restype = ctypes.c_size_t
    L.svd2_rerun_count.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    L.svd2_rerun_count.restype = ctypes.c_int
    L.svd2_multi_plan_bytes.argtypes = [ctypes.c_int32]
    L.svd2_multi_plan_bytes.restype = ctypes.c_size_t
    L.svd2_multi_prepare.argtypes = [ctypes.POINTER(BatchDesc), ctypes.c_int32, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_int64)]
    L.svd2_multi_prepare.restype = ctypes.c_int
    L.svd2_multi_run.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    L.svd2_multi_run.restype = ctypes.c_int
    L.svd2_multi_graph_create.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    L.svd2_multi_graph_create.restype = ctypes.c_int
    L.svd2_graph_launch.argtypes = [P, P]
    L.svd2_graph_launch.restype = ctypes.c_int
    L.svd2_graph_destroy.argtypes = [P]
    L.svd2_graph_destroy.restype = ctypes.c_int
    L.svd2_autotune_fwd.argtypes = [ctypes.c_int, ctypes.c_int64, PP, PP, PP, P, P, P,
                                    ctypes.c_int, ctypes.POINTER(TuneResult), P]
    L.svd2_autotune_fwd.restype = ctypes.c_int
    L.svd2_multi_autotune.argtypes = [ctypes.POINTER(BatchDesc), ctypes.c_int32, P,
                                      ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(TuneResult), P]
    L.svd2_multi_autotune.restype = ctypes.c_int
    L.svd2_bwd_d.argtypes = [ctypes.c_int64, PP, PP, P, P, PP, PP, P, P, PP, ctypes.c_double, P]
    L.svd2_bwd_d.restype = ctypes.c_int
    L.svd2_bwd_s.argtypes = [ctypes.c_int64, PP, PP, P, P, PP, PP, P, P, PP, ctypes.c_float, P]
    L.svd2_bwd_s.restype = ctypes.c_int
    L.svd2_bwd_z.argtypes = [ctypes.c_int64, PP, PP, P, P, PP, PP, P, P, PP, ctypes.c_double, P]
    L.svd2_bwd_z.restype = ctypes.c_int
    L.svd2_bwd_c.argtypes = [ctypes.c_int64, PP, PP, P, P, PP, PP, P, P, PP, ctypes.c_float, P]
    L.svd2_bwd_c.restype = ctypes.c_int
    L.svd2_batch_host.argtypes = [ctypes.c_int, ctypes.c_int64, PP, PP, PP, P, P, P,
                                  ctypes.c_uint32, ctypes.c_int64, P]
    L.svd2_batch_host.restype = ctypes.c_int
    L.svd2_arith_check.argtypes = [ctypes.c_int, ctypes.c_int64, P, P, P, P, P]
    L.svd2_arith_check.restype = ctypes.c_int
    L.svd2_fp32_selfcheck.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, P, P]
    L.svd2_fp32_selfcheck.restype = ctypes.c_int
    L.svd2_set_launch.argtypes = [ctypes.c_int] * 5
    L.svd2_set_launch.restype = ctypes.c_int
    L.svd2_get_launch.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4
    L.svd2_get_launch.restype = ctypes.c_int
    L.svd2_last_cuda_error.restype = ctypes.c_int
    L.svd2_version.restype = ctypes.c_char_p


def check(rc: int, what: str):
    if rc != OK:
        err = lib().svd2_last_cuda_error()
        raise Svd2Error(f"{what} failed with code {rc} (cudaError {err})")


def ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


def current_stream_handle(device=None) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _kind(rows: int, dtype: torch.dtype) -> str:
    if dtype == torch.float64:
        return {4: "d", 8: "z"}[rows]
    if dtype == torch.float32:
        return {4: "s", 8: "c"}[rows]
    raise TypeError(f"unsupported dtype {dtype}")


@dataclass
class Svd2Result:
    U: torch.Tensor      # (rows, n), element order of A
    V: torch.Tensor      # (rows, n)
    smax: torch.Tensor   # (n,) sigma'_max (or sigma_max with backscale)
    smin: torch.Tensor   # (n,)
    s: torch.Tensor      # (n,) int32 scale exponents (Eq. 2); S_ZERO for A = 0


def _rows(t: torch.Tensor, what: str):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.dim() != 2 or t.shape[0] not in (4, 8):
        raise ValueError(f"{what} must have shape (4, n) or (8, n)")
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError(f"{what}: each row must be contiguous")
    return [t[i].data_ptr() for i in range(t.shape[0])]


def empty_result(rows: int, n: int, dtype, device) -> Svd2Result:
    return Svd2Result(
        U=torch.empty((rows, n), dtype=dtype, device=device),
        V=torch.empty((rows, n), dtype=dtype, device=device),
        smax=torch.empty(n, dtype=dtype, device=device),
        smin=torch.empty(n, dtype=dtype, device=device),
        s=torch.empty(n, dtype=torch.int32, device=device))


def svd2(A: torch.Tensor, *, backscale: bool = False, out: Svd2Result | None = None,
         stream: int | None = None, sine: bool = False) -> Svd2Result:
    """Batched 2x2 SVD of the split-layout batch ``A`` (shape (4, n) or (8, n),
    float64 or float32, on a CUDA device).  ``sine``: U assembled by Eq. 31
    (sines and cosines) instead of Eq. 29.  Asynchronous on ``stream``
    (default: torch's current stream)."""
    rows, n = A.shape
    kind = _kind(rows, A.dtype)
    a_ptrs = _rows(A, "A")
    if out is None:
        out = empty_result(rows, n, A.dtype, A.device)
    u_ptrs = _rows(out.U, "U")
    v_ptrs = _rows(out.V, "V")
    h = current_stream_handle(A.device) if stream is None else stream
    f = getattr(lib(), "svd2_batch_" + kind)
    rc = f(n, ptr_array(a_ptrs), ptr_array(u_ptrs), ptr_array(v_ptrs), out.smax.data_ptr(),
           out.smin.data_ptr(), out.s.data_ptr(),
           (BACKSCALE if backscale else 0) | (SINE if sine else 0), h)
    check(rc, "svd2_batch_" + kind)
    return out


@dataclass
class Svd2Values:
    smax: torch.Tensor
    smin: torch.Tensor
    s: torch.Tensor


def svd2_values(A: torch.Tensor, *, backscale: bool = False, out: Svd2Values | None = None,
                stream: int | None = None) -> Svd2Values:
    """Singular values only (svd2_values_*): the split-layout batch ``A`` as in
    svd2(); returns sigma'_max, sigma'_min and s (sigma with s = 0 when
    ``backscale``), the same values svd2() stores."""
    rows, n = A.shape
    kind = _kind(rows, A.dtype)
    a_ptrs = _rows(A, "A")
    if out is None:
        out = Svd2Values(smax=torch.empty(n, dtype=A.dtype, device=A.device),
                         smin=torch.empty(n, dtype=A.dtype, device=A.device),
                         s=torch.empty(n, dtype=torch.int32, device=A.device))
    h = current_stream_handle(A.device) if stream is None else stream
    rc = getattr(lib(), "svd2_values_" + kind)(
        n, ptr_array(a_ptrs), out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr(),
        BACKSCALE if backscale else 0, h)
    check(rc, "svd2_values_" + kind)
    return out


_INTERLEAVED_KIND = {torch.float64: "d", torch.complex128: "z", torch.float32: "s",
                     torch.complex64: "c"}


def svd2_interleaved(A: torch.Tensor, *, values_only: bool = False, backscale: bool = False,
                     stream: int | None = None) -> Svd2Result:
    """The interleaved layout (svd2_batch_interleaved_*): ``A`` of shape (n, 2, 2),
    float64, float32, complex128 or complex64, contiguous, on a CUDA device.
    Returns U, V of A's shape and dtype (None with ``values_only``), and
    sigma'_max, sigma'_min (the real dtype) and s, so that
    A = U diag(2^-s sigma') V^H; with ``backscale`` sigma and s = 0."""
    if A.dim() != 3 or tuple(A.shape[1:]) != (2, 2) or not A.is_contiguous() or not A.is_cuda:
        raise ValueError("A must be a contiguous CUDA tensor of shape (n, 2, 2)")
    kind = _INTERLEAVED_KIND.get(A.dtype)
    if kind is None:
        raise TypeError(f"unsupported dtype {A.dtype}")
    n = A.shape[0]
    rdt = torch.float64 if kind in "dz" else torch.float32
    out = Svd2Result(U=None if values_only else torch.empty_like(A),
                     V=None if values_only else torch.empty_like(A),
                     smax=torch.empty(n, dtype=rdt, device=A.device),
                     smin=torch.empty(n, dtype=rdt, device=A.device),
                     s=torch.empty(n, dtype=torch.int32, device=A.device))
    h = current_stream_handle(A.device) if stream is None else stream
    rc = getattr(lib(), "svd2_batch_interleaved_" + kind)(
        n, A.data_ptr(), None if values_only else out.U.data_ptr(),
        None if values_only else out.V.data_ptr(), out.smax.data_ptr(), out.smin.data_ptr(),
        out.s.data_ptr(), BACKSCALE if backscale else 0, h)
    check(rc, "svd2_batch_interleaved_" + kind)
    return out


def kog_workspace(G: torch.Tensor) -> torch.Tensor:
    """Workspace of svd2_kog_step_* for the m x m matrix G (a uint8 device tensor)."""
    kind = _INTERLEAVED_KIND[G.dtype]
    nbytes = lib().svd2_kog_workspace_bytes(OPS[kind], G.shape[0])
    return torch.empty(nbytes + 256, dtype=torch.uint8, device=G.device)


def _aligned256(ws: torch.Tensor) -> int:
    return (ws.data_ptr() + 255) // 256 * 256


def kog_step(G: torch.Tensor, pairs: torch.Tensor, *, workspace: torch.Tensor | None = None,
             stream: int | None = None) -> torch.Tensor:
    """One parallel Kogbetliantz step (svd2_kog_step_*) in place on the square
    CUDA tensor ``G`` (float64, float32, complex128 or complex64; row-major or
    column-major, i.e. G or G.T contiguous up to the leading dimension) with the
    pivot pairs ``pairs`` (int32 CUDA tensor of m entries p_0, q_0, p_1, ...).
    Returns G."""
    if G.dim() != 2 or G.shape[0] != G.shape[1] or not G.is_cuda:
        raise ValueError("G must be a square CUDA matrix")
    kind = _INTERLEAVED_KIND.get(G.dtype)
    if kind is None:
        raise TypeError(f"unsupported dtype {G.dtype}")
    if pairs.dtype != torch.int32 or not pairs.is_cuda or pairs.numel() != G.shape[0]:
        raise ValueError("pairs must be an int32 CUDA tensor with one entry per row of G")
    rs, cs = G.stride()
    ws = kog_workspace(G) if workspace is None else workspace
    h = current_stream_handle(G.device) if stream is None else stream
    rc = getattr(lib(), "svd2_kog_step_" + kind)(
        G.shape[0], G.data_ptr(), rs, cs, pairs.contiguous().data_ptr(), _aligned256(ws),
        ws.numel() - 256, h)
    check(rc, "svd2_kog_step_" + kind)
    return G


def kog_skipped(workspace: torch.Tensor) -> int:
    c = ctypes.c_int64()
    check(lib().svd2_kog_skipped(_aligned256(workspace), ctypes.byref(c)), "svd2_kog_skipped")
    return c.value


def _host_rows(t: torch.Tensor, what: str):
    if t.is_cuda or t.dim() != 2 or t.shape[0] not in (4, 8):
        raise ValueError(f"{what} must be a host tensor of shape (4, n) or (8, n)")
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError(f"{what}: each row must be contiguous")
    return [t[i].data_ptr() for i in range(t.shape[0])]


def empty_host_result(rows: int, n: int, dtype, pin: bool = True) -> Svd2Result:
    mk = (lambda *a, **k: torch.empty(*a, **k).pin_memory()) if pin else torch.empty
    return Svd2Result(U=mk((rows, n), dtype=dtype), V=mk((rows, n), dtype=dtype),
                      smax=mk(n, dtype=dtype), smin=mk(n, dtype=dtype), s=mk(n, dtype=torch.int32))


def svd2_host(A: torch.Tensor, *, backscale: bool = False, out: Svd2Result | None = None,
              chunk: int = 0, device=None, stream: int | None = None,
              tan64: bool = False) -> Svd2Result:
    """Forward form on a batch in host memory (svd2_batch_host): A is a CPU
    tensor (pinned for overlap) of shape (4, n) or (8, n); outputs are host
    tensors.  ``tan64``: the real FP32 form with the FP64 tangent step at the
    default threshold.  Asynchronous on the device's current stream (or
    ``stream``): synchronise before reading the outputs."""
    rows, n = A.shape
    kind = _kind(rows, A.dtype)
    if tan64 and kind != "s":
        raise TypeError("the FP64 tangent step form takes real float32 input")
    if out is None:
        out = empty_host_result(rows, n, A.dtype)
    dev = torch.device("cuda") if device is None else torch.device(device)
    h = current_stream_handle(dev) if stream is None else stream
    rc = lib().svd2_batch_host(HOST_OP_S_TAN64 if tan64 else OPS[kind], n, ptr_array(_host_rows(A, "A")),
                               ptr_array(_host_rows(out.U, "U")), ptr_array(_host_rows(out.V, "V")),
                               out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr(),
                               BACKSCALE if backscale else 0, int(chunk), h)
    check(rc, "svd2_batch_host")
    return out


RERUN_TAU_LOG2 = -8
TAN64_TAU_LOG2 = -3
HOST_OP_S_TAN64 = 4


def svd2_tan64(A: torch.Tensor, *, tau_log2: int = TAN64_TAU_LOG2, backscale: bool = False,
               out: Svd2Result | None = None, count: torch.Tensor | None = None,
               stream: int | None = None) -> Svd2Result:
    """Real FP32 form with the FP64 tangent step (svd2_batch_s_tan64) for the
    matrices with |r''_22| < 2^tau_log2 r11.  ``A`` is float32 of shape (4, n).
    ``count``: optional one-element int64 CUDA tensor to which the call adds
    the number of matrices that took the step."""
    rows, n = A.shape
    if A.dtype != torch.float32 or rows != 4:
        raise TypeError("svd2_tan64 takes real float32 input of shape (4, n)")
    a_ptrs = _rows(A, "A")
    if out is None:
        out = empty_result(rows, n, A.dtype, A.device)
    h = current_stream_handle(A.device) if stream is None else stream
    cp = None
    if count is not None:
        if count.dtype != torch.int64 or count.numel() != 1 or not count.is_cuda:
            raise TypeError("count must be a one-element int64 CUDA tensor")
        cp = count.data_ptr()
    rc = lib().svd2_batch_s_tan64(n, ptr_array(a_ptrs), ptr_array(_rows(out.U, "U")),
                                  ptr_array(_rows(out.V, "V")), out.smax.data_ptr(),
                                  out.smin.data_ptr(), out.s.data_ptr(), int(tau_log2),
                                  BACKSCALE if backscale else 0, cp, h)
    check(rc, "svd2_batch_s_tan64")
    return out


def rerun_workspace(n: int, device="cuda") -> torch.Tensor:
    """Device workspace for svd2_rerun (bytes as a uint8 tensor)."""
    return torch.empty(int(lib().svd2_rerun_workspace_bytes(n)), dtype=torch.uint8, device=device)


def svd2_rerun(A: torch.Tensor, *, tau_log2: int = RERUN_TAU_LOG2, backscale: bool = False,
               out: Svd2Result | None = None, workspace: torch.Tensor | None = None,
               stream: int | None = None) -> Svd2Result:
    """FP32 form with FP64 re-run of the matrices with sigma'_min < 2^tau_log2 sigma'_max.
    ``A`` is float32 of shape (4, n) or (8, n)."""
    rows, n = A.shape
    if A.dtype != torch.float32:
        raise TypeError("svd2_rerun takes float32 input")
    kind = _kind(rows, A.dtype)
    a_ptrs = _rows(A, "A")
    if out is None:
        out = empty_result(rows, n, A.dtype, A.device)
    if workspace is None:
        workspace = rerun_workspace(n, A.device)
    h = current_stream_handle(A.device) if stream is None else stream
    f = getattr(lib(), f"svd2_batch_{kind}_rerun")
    rc = f(n, ptr_array(a_ptrs), ptr_array(_rows(out.U, "U")), ptr_array(_rows(out.V, "V")),
           out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr(), int(tau_log2),
           BACKSCALE if backscale else 0, workspace.data_ptr(), workspace.numel(), h)
    check(rc, f"svd2_batch_{kind}_rerun")
    out.workspace = workspace
    return out


def rerun_count(workspace: torch.Tensor) -> int:
    """Matrices re-run by the last completed call that used ``workspace``."""
    c = ctypes.c_int64()
    check(lib().svd2_rerun_count(workspace.data_ptr(), ctypes.byref(c)), "svd2_rerun_count")
    return c.value


def arith_check(op: str, x: torch.Tensor, y: torch.Tensor | None = None):
    """The library's double division ("div"), square root ("sqrt"), rounding to
    float ("d2f", results widened exactly), widening of the float in the low
    32 bits of each element ("f2d") or double quotient of two floats completed
    from their float quotient ("div_ff": x, y rounded to float first; NaN
    where the operands are outside its domain) next to the hardware
    instruction, on float64 CUDA tensors; returns (lib, hw)."""
    lib_out = torch.empty_like(x)
    hw_out = torch.empty_like(x)
    code = {"div": 0, "sqrt": 1, "d2f": 2, "f2d": 3, "div_ff": 4}[op]
    rc = lib().svd2_arith_check(code, x.numel(), x.data_ptr(),
                                None if y is None else y.data_ptr(), lib_out.data_ptr(),
                                hw_out.data_ptr(), current_stream_handle(x.device))
    check(rc, "svd2_arith_check")
    return lib_out, hw_out


def fp32_selfcheck(op: str, begin: int, count: int, device="cuda") -> dict:
    """The branch-free single-precision "rcp", "sqrt", "div_sig" (significand
    pairs) or "div_rand" (random operands on the stated domain) against the
    hardware's correctly rounded sequences over indices [begin, begin + count)
    (svd2_fp32_selfcheck); returns mismatches, first mismatching index, cases
    checked."""
    res = torch.tensor([0, -1, 0], dtype=torch.int64, device=device)   # -1: UINT64_MAX
    code = {"rcp": 0, "sqrt": 1, "div_sig": 2, "div_rand": 3}[op]
    rc = lib().svd2_fp32_selfcheck(code, int(begin), int(count), res.data_ptr(),
                                   current_stream_handle(res.device))
    check(rc, "svd2_fp32_selfcheck")
    v = res.cpu().tolist()
    return {"mismatches": v[0], "first": v[1] & (2**64 - 1), "checked": v[2]}


def default_rel_delta(dtype) -> float:
    """Relative singular-value gap below which the adjoint's rotation term is
    damped: 64 units of roundoff of the dtype."""
    return 64 * torch.finfo(dtype).eps


def _opt_rows(t, n, what):
    if t is None:
        return None
    return ptr_array(_rows(t, what))


def svd2_bwd(U, V, s1, s2, gU=None, gV=None, g1=None, g2=None, rel_delta=None,
             out: torch.Tensor | None = None, stream: int | None = None) -> torch.Tensor:
    """Adjoint of the 2x2 SVD (svd2_bwd_{d,s,z,c}): gA of U's shape from U, V
    ((4, n) real or (8, n) complex split layout), the singular values s1, s2
    (n,) and the upstream gradients (None = zero); for complex data the rows
    of a gradient are dL/dRe and dL/dIm of the corresponding rows."""
    rows, n = U.shape
    if rows not in (4, 8) or U.dtype not in (torch.float64, torch.float32):
        raise ValueError("svd2_bwd takes (4, n) or (8, n) float64/float32 factors")
    if rel_delta is None:
        rel_delta = default_rel_delta(U.dtype)
    if out is None:
        out = torch.empty_like(U)
    f = getattr(lib(), "svd2_bwd_" + _kind(rows, U.dtype))
    h = current_stream_handle(U.device) if stream is None else stream
    p = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    rc = f(n, ptr_array(_rows(U, "U")), ptr_array(_rows(V, "V")), s1.data_ptr(), s2.data_ptr(),
           _opt_rows(gU, n, "gU"), _opt_rows(gV, n, "gV"), p(g1), p(g2),
           ptr_array(_rows(out, "gA")), float(rel_delta), h)
    check(rc, "svd2_bwd")
    return out


def autotune_fwd(A: torch.Tensor, out: Svd2Result | None = None, reps: int = 5,
                 form: str = "plain") -> dict:
    """Time every launch shape of A's form on A (svd2_autotune_fwd) and keep the
    fastest as that form's launch shape.  ``form``: "plain", or "tan64" for the
    real FP32 form with the FP64 tangent step.  Returns the winning shape."""
    rows, n = A.shape
    kind = _kind(rows, A.dtype)
    if form == "tan64":
        if kind != "s":
            raise TypeError("the FP64 tangent step form takes real float32 input")
        kind = "s_tan64"
    if out is None:
        out = empty_result(rows, n, A.dtype, A.device)
    res = TuneResult()
    rc = lib().svd2_autotune_fwd(OPS[kind], n, ptr_array(_rows(A, "A")),
                                 ptr_array(_rows(out.U, "U")), ptr_array(_rows(out.V, "V")),
                                 out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr(),
                                 reps, ctypes.byref(res), current_stream_handle(A.device))
    check(rc, "svd2_autotune_fwd")
    return res.as_dict()


class MultiBatch:
    """Several FP64 batches (real (4, n_i) and complex (8, n_i) float64 CUDA
    tensors) decomposed by one persistent launch (svd2_multi_*).  Outputs are
    allocated here, one Svd2Result per batch; the input tensors may be
    overwritten between runs (a Kogbetliantz step updates them in place)."""

    def __init__(self, batches, block: int = 256, mpt: int = 1, unroll: int = 1,
                 backscale: bool = False):
        self.inputs = list(batches)
        self.outputs = []
        descs = (BatchDesc * max(1, len(self.inputs)))()
        for i, A in enumerate(self.inputs):
            rows, n = A.shape
            if A.dtype != torch.float64 or rows not in (4, 8):
                raise ValueError("MultiBatch takes float64 (4, n) or (8, n) batches")
            out = empty_result(rows, n, A.dtype, A.device)
            self.outputs.append(out)
            d = descs[i]
            d.kind = KIND_Z if rows == 8 else KIND_D
            d.flags = BACKSCALE if backscale else 0
            d.n = n
            for e, p in enumerate(_rows(A, "A")):
                d.a[e] = p
            for e, p in enumerate(_rows(out.U, "U")):
                d.u[e] = p
            for e, p in enumerate(_rows(out.V, "V")):
                d.v[e] = p
            d.smax, d.smin, d.s = out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr()
        self.descs = descs
        self.nbatch = len(self.inputs)
        dev = self.inputs[0].device if self.inputs else torch.device("cuda")
        self.plan = torch.empty(int(lib().svd2_multi_plan_bytes(self.nbatch)), dtype=torch.uint8,
                                device=dev)
        self.prepare(block, mpt, unroll)

    def prepare(self, block, mpt, unroll):
        tiles = ctypes.c_int64()
        check(lib().svd2_multi_prepare(self.descs, self.nbatch, block, mpt, unroll,
                                       self.plan.data_ptr(), self.plan.numel(),
                                       ctypes.byref(tiles)), "svd2_multi_prepare")
        self.shape = (block, mpt, unroll)
        self.tiles = tiles.value

    def run(self, stream: int | None = None, grid: int = 0):
        h = current_stream_handle(self.plan.device) if stream is None else stream
        check(lib().svd2_multi_run(self.plan.data_ptr(), *self.shape, grid, h), "svd2_multi_run")

    def autotune(self, reps: int = 5) -> dict:
        res = TuneResult()
        check(lib().svd2_multi_autotune(self.descs, self.nbatch, self.plan.data_ptr(),
                                        self.plan.numel(), reps, ctypes.byref(res),
                                        current_stream_handle(self.plan.device)),
              "svd2_multi_autotune")
        self.shape = (res.block, res.mpt, res.unroll)
        return res.as_dict()

    def graph(self) -> "Graph":
        h = ctypes.c_void_p()
        check(lib().svd2_multi_graph_create(self.plan.data_ptr(), *self.shape, 0, ctypes.byref(h)),
              "svd2_multi_graph_create")
        return Graph(h, self)


class Graph:
    """An executable CUDA graph of one persistent multi-batch launch."""

    def __init__(self, handle, owner):
        self.handle = handle
        self.owner = owner   # keeps the plan and the batch tensors alive

    def launch(self, stream: int | None = None):
        h = current_stream_handle(self.owner.plan.device) if stream is None else stream
        check(lib().svd2_graph_launch(self.handle, h), "svd2_graph_launch")

    def close(self):
        if self.handle:
            check(lib().svd2_graph_destroy(self.handle), "svd2_graph_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_launch(kind: str, block: int, mpt: int, unroll: int, waves: int = 0):
    check(lib().svd2_set_launch(OPS[kind], block, mpt, unroll, waves), "svd2_set_launch")


def get_launch(kind: str):
    vals = [ctypes.c_int() for _ in range(4)]
    check(lib().svd2_get_launch(OPS[kind], *[ctypes.byref(v) for v in vals]), "svd2_get_launch")
    return tuple(v.value for v in vals)


def version() -> str:
    return lib().svd2_version().decode()
