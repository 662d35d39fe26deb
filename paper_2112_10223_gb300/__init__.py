"""GB300 SpKAdd: B = A_1 + ... + A_k for k same-shape CSC sparse matrices.

Thin ctypes binding of ``libspkadd.so`` (declared in ``include/spkadd.h``).
It marshals arguments only: every step of the computation runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.

Entry points carry the C names:

    h = spkadd_plan(A, m, dtype=torch.float64, stream=None, options=None)
    nnz = spkadd_symbolic(h)
    spkadd_numeric(h, B_col_ptr, B_row_idx, B_val)
    spkadd_destroy(h)

``A`` is a list of k CSC matrices given as ``(col_ptr int32[n+1],
row_idx int32[nnz], val float32|float64[nnz])`` CUDA tensors.  ``spkadd(A, m)``
runs the three phases and returns ``(col_ptr int64, row_idx int32, val)``.

If the library has not been built, every call raises ``SpkaddError``; there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import torch

from ._build import LIB_PATH, build  # noqa: F401  (build is re-exported)

__all__ = [
    "SpkaddError", "Options", "Info", "library", "default_options", "spkadd_plan", "spkadd_symbolic",
    "spkadd_numeric", "spkadd_destroy", "spkadd_get_info", "spkadd_status_string", "spkadd", "Handle",
    "STATUS", "spkadd_scan_counts_noalloc", "SCAN_NOALLOC_MAX_N",
]

SCAN_NOALLOC_MAX_N = 4096 * 4096

STATUS = {
    0: "SPKADD_OK", 1: "SPKADD_ERR_INVALID_ARG", 2: "SPKADD_ERR_SHAPE_MISMATCH", 3: "SPKADD_ERR_UNSORTED",
    4: "SPKADD_ERR_INDEX_RANGE", 5: "SPKADD_ERR_OVERFLOW", 6: "SPKADD_ERR_NOMEM", 7: "SPKADD_ERR_CUDA",
    8: "SPKADD_ERR_TIMEOUT", 9: "SPKADD_ERR_STATE", 10: "SPKADD_ERR_UNSUPPORTED", 11: "SPKADD_ERR_INTERNAL",
}


class SpkaddError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{what}: {self.name}" if what else self.name)


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class CSC(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("validate", ctypes.c_int32), ("warp_max", ctypes.c_int32), ("cta_max", ctypes.c_int32),
                ("window_max", ctypes.c_int32), ("sort_mode", ctypes.c_int32), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "k", "m", "n", "nnz_in", "nnz_out", "cols_warp", "cols_cta", "cols_heavy", "windows", "windows_split",
        "cols_unique", "workspace_bytes", "kernel_launches")]


_lib = None


def library():
    """The loaded libspkadd.so (raises SpkaddError when it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SpkaddError(-1, f"CUDA library missing at {LIB_PATH}; run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        lib.spkadd_default_options.argtypes = [ctypes.POINTER(Options)]
        lib.spkadd_default_options.restype = None
        lib.spkadd_plan.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(CSC), ctypes.c_int, P,
                                    ctypes.POINTER(Options)]
        lib.spkadd_plan.restype = ctypes.c_int
        lib.spkadd_symbolic.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        lib.spkadd_symbolic.restype = ctypes.c_int
        lib.spkadd_numeric.argtypes = [P, P, P, P]
        lib.spkadd_numeric.restype = ctypes.c_int
        lib.spkadd_get_info.argtypes = [P, ctypes.POINTER(Info)]
        lib.spkadd_get_info.restype = ctypes.c_int
        lib.spkadd_destroy.argtypes = [P]
        lib.spkadd_destroy.restype = ctypes.c_int
        lib.spkadd_status_string.argtypes = [ctypes.c_int]
        lib.spkadd_status_string.restype = ctypes.c_char_p
        lib.spkadd_version.argtypes = []
        lib.spkadd_version.restype = ctypes.c_int
        lib.spkadd_scan_counts_noalloc.argtypes = [P, ctypes.c_int64, P, P]
        lib.spkadd_scan_counts_noalloc.restype = ctypes.c_int
        _lib = lib
    return _lib


def spkadd_status_string(status: int) -> str:
    return library().spkadd_status_string(status).decode()


def _check(status: int, what: str):
    if status != 0:
        raise SpkaddError(status, what)


def default_options(**overrides) -> Options:
    o = Options()
    library().spkadd_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


_DTYPE = {torch.float32: 0, torch.float64: 1}


class Handle:
    """Owns a spkadd_handle*; keeps the borrowed input tensors alive."""

    def __init__(self, ptr, inputs, n, dtype, stream):
        self.ptr = ptr
        self.inputs = inputs
        self.n = n
        self.dtype = dtype
        self.stream = stream
        self.nnz = None

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                library().spkadd_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream, ctypes.c_void_p(stream.cuda_stream)


def spkadd_plan(A, m: int, dtype=None, stream=None, options: Options | None = None) -> Handle:
    """spkadd_plan: check the inputs, allocate the workspace, bin the columns."""
    lib = library()
    k = len(A)
    if k == 0:
        _check(1, "spkadd_plan")
    dtype = dtype or A[0][2].dtype
    if dtype not in _DTYPE:
        raise TypeError("values must be float32 or float64")
    arr = (CSC * k)()
    keep = []
    for i, (cp, ri, va) in enumerate(A):
        for t, dt in ((cp, torch.int32), (ri, torch.int32), (va, dtype)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise TypeError(f"input {i}: expected contiguous CUDA tensors (int32, int32, {dtype})")
        arr[i].m = int(m)
        arr[i].n = cp.numel() - 1
        arr[i].nnz = ri.numel()
        arr[i].col_ptr = cp.data_ptr()
        arr[i].row_idx = ri.data_ptr() if ri.numel() else None
        arr[i].val = va.data_ptr() if va.numel() else None
        keep.append((cp, ri, va))
    stream, sp = _stream_ptr(stream)
    h = ctypes.c_void_p()
    _check(lib.spkadd_plan(ctypes.byref(h), k, arr, _DTYPE[dtype], sp,
                           ctypes.byref(options) if options is not None else None), "spkadd_plan")
    return Handle(h, keep, A[0][0].numel() - 1, dtype, stream)


def spkadd_symbolic(h: Handle) -> int:
    """spkadd_symbolic: nnz(B(:,j)) per column, their scan, and nnz(B) (blocks once)."""
    nnz = ctypes.c_int64()
    _check(library().spkadd_symbolic(h.ptr, ctypes.byref(nnz)), "spkadd_symbolic")
    h.nnz = int(nnz.value)
    return h.nnz


def spkadd_numeric(h: Handle, col_ptr: torch.Tensor, row_idx: torch.Tensor, val: torch.Tensor) -> None:
    """spkadd_numeric: write B into caller-allocated device tensors."""
    if col_ptr.dtype != torch.int64 or row_idx.dtype != torch.int32 or val.dtype != h.dtype:
        raise TypeError("B buffers must be int64 col_ptr, int32 row_idx and values of the plan's dtype")
    if col_ptr.numel() != h.n + 1 or (h.nnz is not None and (row_idx.numel() < h.nnz or val.numel() < h.nnz)):
        raise ValueError("B buffers too small")
    _check(library().spkadd_numeric(h.ptr, col_ptr.data_ptr(), row_idx.data_ptr() if row_idx.numel() else None,
                                    val.data_ptr() if val.numel() else None), "spkadd_numeric")


def spkadd_get_info(h: Handle) -> dict:
    info = Info()
    st = library().spkadd_get_info(h.ptr, ctypes.byref(info))
    d = {name: int(getattr(info, name)) for name, _ in Info._fields_}
    d["status"] = STATUS.get(st, st)
    return d


def spkadd_destroy(h: Handle) -> None:
    if h.ptr:
        ptr, h.ptr = h.ptr, None
        _check(library().spkadd_destroy(ptr), "spkadd_destroy")


def spkadd(A, m: int, dtype=None, stream=None, options: Options | None = None, info: bool = False):
    """B = sum of the inputs; returns (col_ptr int64, row_idx int32, val) CUDA tensors."""
    h = spkadd_plan(A, m, dtype=dtype, stream=stream, options=options)
    try:
        nnz = spkadd_symbolic(h)
        dev = A[0][0].device
        col_ptr = torch.empty(h.n + 1, dtype=torch.int64, device=dev)
        row_idx = torch.empty(nnz, dtype=torch.int32, device=dev)
        val = torch.empty(nnz, dtype=h.dtype, device=dev)
        spkadd_numeric(h, col_ptr, row_idx, val)
        stats = spkadd_get_info(h) if info else None
    finally:
        spkadd_destroy(h)
    return (col_ptr, row_idx, val, stats) if info else (col_ptr, row_idx, val)


def spkadd_scan_counts_noalloc(counts: torch.Tensor, col_ptr: torch.Tensor, stream=None) -> None:
    """col_ptr = exclusive scan of counts (int32 -> int64) without any device allocation.

    For callers that must not allocate device memory inside a call (memory
    handed to their own arena up front, or no room for cudaMalloc's implicit
    synchronisation).  The library keeps a fixed 32 KB scratch array per GPU;
    calls that can overlap on the GPU race on it.  The first call on a device
    should come before any stream capture.
    """
    if counts.dtype != torch.int32 or not counts.is_cuda or not counts.is_contiguous():
        raise TypeError("counts must be a contiguous int32 CUDA tensor")
    if col_ptr.dtype != torch.int64 or not col_ptr.is_cuda or col_ptr.numel() != counts.numel() + 1:
        raise TypeError("col_ptr must be an int64 CUDA tensor with len(counts) + 1 elements")
    _, sp = _stream_ptr(stream)
    _check(library().spkadd_scan_counts_noalloc(counts.data_ptr() if counts.numel() else None, counts.numel(),
                                                col_ptr.data_ptr(), sp), "spkadd_scan_counts_noalloc")
