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

Batches of independent problems (each with its own k, shape and dtype) run
as one set of launches:

    h = spkadd_batch_plan(problems)          # problems: [(A, m), ...]
    nnz = spkadd_batch_symbolic(h)           # list, one per problem
    spkadd_batch_numeric(h, outs)            # outs: [(col_ptr, row_idx, val), ...]
    spkadd_destroy(h)

``spkadd_batch_plan_raw`` takes the descriptors as flat integer arrays
instead of tensors (device addresses), for callers that hold many problems
in packed buffers.

If the library has not been built, every call raises ``SpkaddError``; there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from ._build import LIB_PATH, build  # noqa: F401  (build is re-exported)

__all__ = [
    "SpkaddError", "Options", "Info", "library", "default_options", "spkadd_plan", "spkadd_symbolic",
    "spkadd_numeric", "spkadd_onepass", "spkadd_destroy", "spkadd_get_info", "spkadd_status_string", "spkadd", "Handle",
    "STATUS", "spkadd_scan_counts_noalloc", "SCAN_NOALLOC_MAX_N", "spkadd_batch_plan", "spkadd_batch_plan_raw",
    "spkadd_batch_symbolic", "spkadd_batch_numeric", "spkadd_batch_numeric_raw", "spkadd_batch", "BatchHandle",
    "SpkaddStream",
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
                ("window_max", ctypes.c_int32), ("sort_mode", ctypes.c_int32), ("input_order", ctypes.c_int32),
                ("block_accumulator", ctypes.c_int32),
                ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("wait_timeout_ms", ctypes.c_int32), ("test_stall", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "k", "m", "n", "nnz_in", "nnz_out", "cols_warp", "cols_cta", "cols_heavy", "windows", "windows_split",
        "cols_unique", "workspace_bytes", "kernel_launches", "problems", "onepass")]


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
        lib.spkadd_onepass.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        lib.spkadd_onepass.restype = ctypes.c_int
        lib.spkadd_get_info.argtypes = [P, ctypes.POINTER(Info)]
        lib.spkadd_get_info.restype = ctypes.c_int
        lib.spkadd_destroy.argtypes = [P]
        lib.spkadd_destroy.restype = ctypes.c_int
        lib.spkadd_status_string.argtypes = [ctypes.c_int]
        lib.spkadd_status_string.restype = ctypes.c_char_p
        lib.spkadd_version.argtypes = []
        lib.spkadd_version.restype = ctypes.c_int
        lib.spkadd_batch_plan.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, P, P, P, ctypes.POINTER(Options)]
        lib.spkadd_batch_plan.restype = ctypes.c_int
        lib.spkadd_batch_symbolic.argtypes = [P, P]
        lib.spkadd_batch_symbolic.restype = ctypes.c_int
        lib.spkadd_batch_numeric.argtypes = [P, P, P, P]
        lib.spkadd_batch_numeric.restype = ctypes.c_int
        lib.spkadd_scan_counts_noalloc.argtypes = [P, ctypes.c_int64, P, P]
        lib.spkadd_scan_counts_noalloc.restype = ctypes.c_int
        I64P = ctypes.POINTER(ctypes.c_int64)
        lib.spkadd_stream_create.argtypes = [ctypes.POINTER(P), ctypes.c_int64, ctypes.c_int64, ctypes.c_int, P,
                                             ctypes.POINTER(Options)]
        lib.spkadd_stream_add.argtypes = [P, ctypes.c_int, ctypes.POINTER(CSC)]
        lib.spkadd_stream_query.argtypes = [P, I64P, I64P, I64P]
        lib.spkadd_stream_view.argtypes = [P, ctypes.POINTER(CSC)]
        lib.spkadd_stream_result.argtypes = [P, P, P, P]
        lib.spkadd_stream_destroy.argtypes = [P]
        for f in ("create", "add", "query", "view", "result", "destroy"):
            getattr(lib, "spkadd_stream_" + f).restype = ctypes.c_int
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
    """Owns a spkadd_handle*; keeps the borrowed input tensors alive.

    Every library call on the handle runs with the handle's device current
    (the C side launches on the current device).
    """

    def __init__(self, ptr, inputs, n, dtype, stream, device=None):
        self.ptr = ptr
        self.inputs = inputs
        self.n = n
        self.dtype = dtype
        self.stream = stream
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nnz = None

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                with torch.cuda.device(self.device):
                    library().spkadd_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream, ctypes.c_void_p(stream.cuda_stream)


def _csc_array(A, m: int, dtype):
    """spkadd_csc descriptors of the inputs (and the tensors to keep alive)."""
    arr = (CSC * len(A))()
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
    return arr, keep


def spkadd_plan(A, m: int, dtype=None, stream=None, options: Options | None = None) -> Handle:
    """spkadd_plan: check the inputs, allocate the workspace, bin the columns."""
    lib = library()
    k = len(A)
    if k == 0:
        _check(1, "spkadd_plan")
    dtype = dtype or A[0][2].dtype
    if dtype not in _DTYPE:
        raise TypeError("values must be float32 or float64")
    arr, keep = _csc_array(A, m, dtype)
    dev = A[0][0].device
    if any(t.device != dev for a in A for t in a):
        raise TypeError("all inputs must be on one device")
    with torch.cuda.device(dev):
        stream, sp = _stream_ptr(stream)
        h = ctypes.c_void_p()
        _check(lib.spkadd_plan(ctypes.byref(h), k, arr, _DTYPE[dtype], sp,
                               ctypes.byref(options) if options is not None else None), "spkadd_plan")
    return Handle(h, keep, A[0][0].numel() - 1, dtype, stream, dev)


def spkadd_symbolic(h: Handle) -> int:
    """spkadd_symbolic: nnz(B(:,j)) per column, their scan, and nnz(B) (blocks once)."""
    nnz = ctypes.c_int64()
    with torch.cuda.device(h.device):
        _check(library().spkadd_symbolic(h.ptr, ctypes.byref(nnz)), "spkadd_symbolic")
    h.nnz = int(nnz.value)
    return h.nnz


def spkadd_numeric(h: Handle, col_ptr: torch.Tensor, row_idx: torch.Tensor, val: torch.Tensor) -> None:
    """spkadd_numeric: write B into caller-allocated device tensors."""
    dev = h.inputs[0][0].device if h.inputs else None
    _out_tensor(col_ptr, torch.int64, "col_ptr", dev)
    _out_tensor(row_idx, torch.int32, "row_idx", dev)
    _out_tensor(val, h.dtype, "val", dev)
    if col_ptr.numel() != h.n + 1 or (h.nnz is not None and (row_idx.numel() < h.nnz or val.numel() < h.nnz)):
        raise ValueError("B buffers too small")
    with torch.cuda.device(h.device):
        _check(library().spkadd_numeric(h.ptr, col_ptr.data_ptr(), row_idx.data_ptr() if row_idx.numel() else None,
                                        val.data_ptr() if val.numel() else None), "spkadd_numeric")


def _out_tensor(t: torch.Tensor, dtype, what: str, device) -> None:
    """Output buffers are written as n consecutive elements: require exactly that."""
    if t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous {dtype} CUDA tensor")
    if device is not None and t.device != device:
        raise TypeError(f"{what} must be on {device}")


def spkadd_onepass(h: Handle, col_ptr: torch.Tensor, row_idx: torch.Tensor, val: torch.Tensor) -> int:
    """spkadd_onepass: B in one pass over the inputs into buffers of at least sum nnz(A_i) entries.

    Returns nnz(B); the first nnz(B) entries of row_idx / val are B's.
    """
    dev = h.inputs[0][0].device if h.inputs else None
    _out_tensor(col_ptr, torch.int64, "col_ptr", dev)
    _out_tensor(row_idx, torch.int32, "row_idx", dev)
    _out_tensor(val, h.dtype, "val", dev)
    if col_ptr.numel() != h.n + 1:
        raise ValueError("col_ptr must hold n + 1 entries")
    cap = min(row_idx.numel(), val.numel())
    nnz = ctypes.c_int64()
    with torch.cuda.device(h.device):
        _check(library().spkadd_onepass(h.ptr, col_ptr.data_ptr(), row_idx.data_ptr() if row_idx.numel() else None,
                                        val.data_ptr() if val.numel() else None, cap, ctypes.byref(nnz)),
               "spkadd_onepass")
    h.nnz = int(nnz.value)
    return h.nnz


def spkadd_get_info(h: Handle) -> dict:
    info = Info()
    with torch.cuda.device(h.device):
        st = library().spkadd_get_info(h.ptr, ctypes.byref(info))
    d = {name: int(getattr(info, name)) for name, _ in Info._fields_}
    d["status"] = STATUS.get(st, st)
    return d


def spkadd_destroy(h: Handle) -> None:
    if h.ptr:
        ptr, h.ptr = h.ptr, None
        with torch.cuda.device(h.device):
            _check(library().spkadd_destroy(ptr), "spkadd_destroy")


def spkadd(A, m: int, dtype=None, stream=None, options: Options | None = None, info: bool = False,
           method: str = "twopass"):
    """B = sum of the inputs; returns (col_ptr int64, row_idx int32, val) CUDA tensors.

    method "onepass": spkadd_onepass into buffers of sum nnz(A_i) entries
    (row_idx / val are views of their first nnz(B) entries); "twopass":
    spkadd_symbolic, then exact-size buffers and spkadd_numeric.
    """
    if method not in ("onepass", "twopass"):
        raise ValueError("method must be 'onepass' or 'twopass'")
    h = spkadd_plan(A, m, dtype=dtype, stream=stream, options=options)
    try:
        dev = A[0][0].device
        col_ptr = torch.empty(h.n + 1, dtype=torch.int64, device=dev)
        if method == "onepass":
            cap = sum(a[1].numel() for a in A)
            row_idx = torch.empty(cap, dtype=torch.int32, device=dev)
            val = torch.empty(cap, dtype=h.dtype, device=dev)
            nnz = spkadd_onepass(h, col_ptr, row_idx, val)
            row_idx, val = row_idx[:nnz], val[:nnz]
        else:
            nnz = spkadd_symbolic(h)
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
    _out_tensor(col_ptr, torch.int64, "col_ptr", counts.device)
    if col_ptr.numel() != counts.numel() + 1:
        raise TypeError("col_ptr must be an int64 CUDA tensor with len(counts) + 1 elements")
    with torch.cuda.device(counts.device):
        _, sp = _stream_ptr(stream)
        _check(library().spkadd_scan_counts_noalloc(counts.data_ptr() if counts.numel() else None, counts.numel(),
                                                    col_ptr.data_ptr(), sp), "spkadd_scan_counts_noalloc")


# ---------------------------------------------------------------------------
# Batches.
# ---------------------------------------------------------------------------
_CSC_NP = np.dtype([("m", np.int64), ("n", np.int64), ("nnz", np.int64), ("col_ptr", np.uint64),
                    ("row_idx", np.uint64), ("val", np.uint64)])
assert _CSC_NP.itemsize == ctypes.sizeof(CSC)


class BatchHandle(Handle):
    """A spkadd_handle* of a batch; n and dtype are per-problem lists."""

    def __init__(self, ptr, inputs, ns, dtypes, stream, device=None):
        super().__init__(ptr, inputs, ns, dtypes, stream, device)


def spkadd_batch_plan_raw(k, m, n, nnz, col_ptr, row_idx, val, dtypes, stream=None,
                          options: Options | None = None, keep=None, device=None) -> BatchHandle:
    """spkadd_batch_plan from flat descriptor arrays.

    k: per-problem input counts (count entries); m, n: per-problem shapes
    (count entries); nnz, col_ptr, row_idx, val: per-input nnz and device
    addresses (sum(k) entries, problem by problem); dtypes: per-problem
    torch.float32 / torch.float64.  `keep` is held by the handle so that the
    buffers behind the addresses outlive it.  The addresses must be memory
    of `device` (default: the current device).
    """
    lib = library()
    k = np.ascontiguousarray(k, dtype=np.int32)
    count = int(k.size)
    if count == 0:
        _check(1, "spkadd_batch_plan")
    tk = int(k.sum())
    desc = np.zeros(tk, dtype=_CSC_NP)
    rep = np.repeat(np.arange(count), k)
    desc["m"] = np.asarray(m, dtype=np.int64)[rep]
    desc["n"] = np.asarray(n, dtype=np.int64)[rep]
    desc["nnz"] = np.asarray(nnz, dtype=np.int64)
    desc["col_ptr"] = np.asarray(col_ptr, dtype=np.uint64)
    desc["row_idx"] = np.asarray(row_idx, dtype=np.uint64)
    desc["val"] = np.asarray(val, dtype=np.uint64)
    starts = np.concatenate([[0], np.cumsum(k)[:-1]]).astype(np.uint64)
    ptrs = (np.uint64(desc.ctypes.data) + starts * np.uint64(_CSC_NP.itemsize)).astype(np.uint64)
    codes = np.asarray([_DTYPE[d] for d in dtypes], dtype=np.int32)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        stream, sp = _stream_ptr(stream)
        h = ctypes.c_void_p()
        _check(lib.spkadd_batch_plan(ctypes.byref(h), count, k.ctypes.data, ptrs.ctypes.data, codes.ctypes.data, sp,
                                     ctypes.byref(options) if options is not None else None), "spkadd_batch_plan")
    return BatchHandle(h, keep, [int(x) for x in n], list(dtypes), stream, dev)


def spkadd_batch_plan(problems, stream=None, options: Options | None = None) -> BatchHandle:
    """spkadd_batch_plan over [(A, m), ...], each A a list of (col_ptr, row_idx, val) CUDA tensors."""
    ks, ms, ns, nnz, cps, ris, vas, dts, keep = [], [], [], [], [], [], [], [], []
    for q, (A, m) in enumerate(problems):
        if len(A) == 0:
            _check(1, "spkadd_batch_plan")
        dtype = A[0][2].dtype
        if dtype not in _DTYPE:
            raise TypeError("values must be float32 or float64")
        ks.append(len(A))
        ms.append(int(m))
        ns.append(A[0][0].numel() - 1)
        dts.append(dtype)
        for i, (cp, ri, va) in enumerate(A):
            for t, dt in ((cp, torch.int32), (ri, torch.int32), (va, dtype)):
                if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                    raise TypeError(f"problem {q} input {i}: expected contiguous CUDA tensors (int32, int32, {dtype})")
            if cp.numel() - 1 != ns[-1]:
                _check(2, "spkadd_batch_plan")
            nnz.append(ri.numel())
            cps.append(cp.data_ptr())
            ris.append(ri.data_ptr() if ri.numel() else 0)
            vas.append(va.data_ptr() if va.numel() else 0)
        keep.append(A)
    dev = problems[0][0][0][0].device
    if any(t.device != dev for A, _ in problems for a in A for t in a):
        raise TypeError("all problems must be on one device")
    return spkadd_batch_plan_raw(ks, ms, ns, nnz, cps, ris, vas, dts, stream=stream, options=options, keep=keep,
                                 device=dev)


def spkadd_batch_symbolic(h: BatchHandle) -> list:
    """spkadd_batch_symbolic: nnz(B_q) for every problem (blocks once)."""
    count = len(h.n)
    out = np.zeros(count, dtype=np.int64)
    with torch.cuda.device(h.device):
        _check(library().spkadd_batch_symbolic(h.ptr, out.ctypes.data), "spkadd_batch_symbolic")
    h.nnz = [int(x) for x in out]
    return h.nnz


def spkadd_batch_numeric(h: BatchHandle, outs) -> None:
    """spkadd_batch_numeric: outs[q] = (col_ptr int64[n_q+1], row_idx int32, val) device tensors."""
    count = len(h.n)
    if len(outs) != count:
        raise ValueError("one output triple per problem")
    cp = np.zeros(count, dtype=np.uint64)
    ri = np.zeros(count, dtype=np.uint64)
    va = np.zeros(count, dtype=np.uint64)
    for q, (c, r, v) in enumerate(outs):
        _out_tensor(c, torch.int64, f"problem {q} col_ptr", h.device)
        _out_tensor(r, torch.int32, f"problem {q} row_idx", h.device)
        _out_tensor(v, h.dtype[q], f"problem {q} val", h.device)
        if c.numel() != h.n[q] + 1 or (h.nnz is not None and (r.numel() < h.nnz[q] or v.numel() < h.nnz[q])):
            raise ValueError(f"problem {q}: B buffers too small")
        cp[q] = c.data_ptr()
        ri[q] = r.data_ptr() if r.numel() else 0
        va[q] = v.data_ptr() if v.numel() else 0
    with torch.cuda.device(h.device):
        _check(library().spkadd_batch_numeric(h.ptr, cp.ctypes.data, ri.ctypes.data, va.ctypes.data),
               "spkadd_batch_numeric")


def spkadd_batch_numeric_raw(h: BatchHandle, col_ptr, row_idx, val) -> None:
    """spkadd_batch_numeric from flat arrays of device addresses (count entries each).

    The caller guarantees the sizes (n_q + 1 int64, nnz_q int32, nnz_q values
    of problem q's dtype); nothing is checked here beyond the count.
    """
    count = len(h.n)
    cp = np.ascontiguousarray(col_ptr, dtype=np.uint64)
    ri = np.ascontiguousarray(row_idx, dtype=np.uint64)
    va = np.ascontiguousarray(val, dtype=np.uint64)
    if not (cp.size == ri.size == va.size == count):
        raise ValueError("one address per problem in each array")
    with torch.cuda.device(h.device):
        _check(library().spkadd_batch_numeric(h.ptr, cp.ctypes.data, ri.ctypes.data, va.ctypes.data),
               "spkadd_batch_numeric")


def spkadd_batch(problems, stream=None, options: Options | None = None, info: bool = False):
    """B_q for every problem [(A, m), ...]; returns a list of (col_ptr, row_idx, val)."""
    h = spkadd_batch_plan(problems, stream=stream, options=options)
    try:
        nnz = spkadd_batch_symbolic(h)
        outs = []
        for q, (A, _) in enumerate(problems):
            dev = A[0][0].device
            outs.append((torch.empty(h.n[q] + 1, dtype=torch.int64, device=dev),
                         torch.empty(nnz[q], dtype=torch.int32, device=dev),
                         torch.empty(nnz[q], dtype=h.dtype[q], device=dev)))
        spkadd_batch_numeric(h, outs)
        stats = spkadd_get_info(h) if info else None
    finally:
        spkadd_destroy(h)
    return (outs, stats) if info else outs


class SpkaddStream:
    """spkadd_stream_*: a running sum B on the device, B <- B + (a batch of inputs) per add.

    Each add is one (k+1)-way SpKAdd with B as input 0, so only the current
    batch of inputs need be resident.  The inputs of an add are kept alive
    until the next add (their numeric work may still be running).
    """

    def __init__(self, m: int, n: int, dtype=torch.float64, stream=None, options: Options | None = None,
                 device=None):
        if dtype not in _DTYPE:
            raise TypeError("values must be float32 or float64")
        self.m, self.n, self.dtype = int(m), int(n), dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.ptr = ctypes.c_void_p()
        self._keep = None
        with torch.cuda.device(self.device):
            self.stream, sp = _stream_ptr(stream)
            _check(library().spkadd_stream_create(ctypes.byref(self.ptr), self.m, self.n, _DTYPE[dtype], sp,
                                                  ctypes.byref(options) if options is not None else None),
                   "spkadd_stream_create")

    def add(self, A) -> int:
        """B <- B + sum(A); returns nnz(B)."""
        if len(A) == 0:
            _check(1, "spkadd_stream_add")
        arr, keep = _csc_array(A, self.m, self.dtype)
        if any(t.device != self.device for a in A for t in a):
            raise TypeError(f"inputs must be on {self.device}")
        with torch.cuda.device(self.device):
            _check(library().spkadd_stream_add(self.ptr, len(A), arr), "spkadd_stream_add")
        self._keep = keep
        return self.nnz

    def query(self) -> dict:
        nnz, adds, launches = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(library().spkadd_stream_query(self.ptr, ctypes.byref(nnz), ctypes.byref(adds), ctypes.byref(launches)),
               "spkadd_stream_query")
        return {"nnz": int(nnz.value), "adds": int(adds.value), "kernel_launches": int(launches.value)}

    @property
    def nnz(self) -> int:
        return self.query()["nnz"]

    def result(self):
        """B as (col_ptr int64, row_idx int32, val) CUDA tensors (copies)."""
        nnz = self.nnz
        dev = self.device
        with torch.cuda.device(dev), torch.cuda.stream(self.stream):
            cp = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
            ri = torch.empty(nnz, dtype=torch.int32, device=dev)
            va = torch.empty(nnz, dtype=self.dtype, device=dev)
            _check(library().spkadd_stream_result(self.ptr, cp.data_ptr(), ri.data_ptr() if nnz else None,
                                                  va.data_ptr() if nnz else None), "spkadd_stream_result")
        return cp, ri, va

    def close(self) -> None:
        if getattr(self, "ptr", None):
            ptr, self.ptr = self.ptr, None
            with torch.cuda.device(self.device):
                _check(library().spkadd_stream_destroy(ptr), "spkadd_stream_destroy")
        self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
