"""CPU oracle for SpKAdd -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and its ``--impl reference`` arm) may import this
package.  The GPU library (``paper_2112_10223_gb300``) shares no code with it
and never imports it.

The oracle is ``spk_oracle.c``: the definition of SpKAdd (Sec. II-A,
B = A_1 + ... + A_k) written out per column as gather / sort by (row, input) /
compensated fp64 sum of each run of equal rows (Alg. 2's column-by-column
template).  Output columns are sorted by row and keep structural zeros.  This
module compiles it with gcc (plain C + OpenMP) and calls it through ctypes.

Inputs are lists of CSC triples ``(col_ptr int32[n+1], row_idx int32[nnz],
val float32|float64[nnz])`` as numpy arrays or CPU torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libspk_oracle.so")
_lock = threading.Lock()
_lib = None

PLANTS = ("OFF_BY_ONE_COLUMN", "SIGN_FLIP", "DROP_LAST_TERM", "DROP_ZEROS",
          "REVERSE_ORDER")


def build(plant: str | None = None, out: str | None = None) -> str:
    """Compile the oracle with gcc; returns the path of the shared library.

    ``plant`` names one SPK_ORACLE_PLANT_* mutation (tests only: they check
    that the pins fail on a deliberately wrong oracle).
    """
    os.makedirs(_BUILD, exist_ok=True)
    if out is None:
        out = _LIB if plant is None else os.path.join(_BUILD, f"libspk_oracle_{plant}.so")
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", out + ".tmp", "-lm"]
    if plant is not None:
        if plant not in PLANTS:
            raise ValueError(f"unknown plant {plant}")
        cmd.insert(1, f"-DSPK_ORACLE_PLANT_{plant}")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.spk_oracle_union_sizes.argtypes = [ctypes.c_int, i64, P, P, i64, P, P, ctypes.c_int]
    lib.spk_oracle_union_sizes.restype = ctypes.c_int
    lib.spk_oracle_columns.argtypes = [ctypes.c_int, i64, P, P, P, ctypes.c_int, i64, P, P, P, P, P, P,
                                       ctypes.c_int]
    lib.spk_oracle_columns.restype = ctypes.c_int
    lib.spk_oracle_threads.argtypes = [ctypes.c_int]
    lib.spk_oracle_threads.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(path)
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
                build()
            _lib = _bind(_LIB)
    return _lib


def _np(x, dtype=None):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    x = np.ascontiguousarray(x)
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {x.dtype}")
    return x


class _Inputs:
    """Keeps the numpy copies alive and the pointer arrays the C side reads."""

    def __init__(self, A):
        self.k = len(A)
        if self.k < 1:
            raise ValueError("need at least one input")
        self.cp = [_np(a[0], np.int32) for a in A]
        self.ri = [_np(a[1], np.int32) for a in A]
        self.va = [_np(a[2]) for a in A]
        dts = {v.dtype for v in self.va}
        if len(dts) != 1 or next(iter(dts)) not in (np.float32, np.float64):
            raise TypeError("values must all be float32 or all float64")
        self.is_f64 = int(next(iter(dts)) == np.float64)
        self.n = len(self.cp[0]) - 1
        if any(len(c) - 1 != self.n for c in self.cp):
            raise ValueError("inputs disagree on n")
        ptr = lambda arrs: (ctypes.c_void_p * self.k)(*[a.ctypes.data for a in arrs])
        self.p_cp, self.p_ri, self.p_va = ptr(self.cp), ptr(self.ri), ptr(self.va)


def union_sizes(A, cols=None, threads: int = 0, lib=None) -> np.ndarray:
    """nnz(B(:,j)) for the listed columns (all columns when cols is None)."""
    lib = lib or load()
    X = _Inputs(A)
    c = None if cols is None else _np(np.asarray(cols, dtype=np.int64), np.int64)
    nc = X.n if c is None else len(c)
    u = np.empty(nc, dtype=np.int32)
    rc = lib.spk_oracle_union_sizes(X.k, X.n, X.p_cp, X.p_ri, nc, None if c is None else c.ctypes.data,
                                    u.ctypes.data, threads)
    if rc != 0:
        raise MemoryError("oracle ran out of host memory")
    return u


def add(A, cols=None, threads: int = 0, lib=None) -> dict:
    """B = sum_i A_i restricted to the listed columns (all when cols is None).

    Returns a dict of numpy arrays: ``col_ptr`` (int64, len(cols)+1), ``row_idx``
    (int32), ``val`` (float64), ``abs_sum`` (float64, sum of |terms|) and
    ``terms`` (int32, number of inputs holding the entry).
    """
    lib = lib or load()
    X = _Inputs(A)
    c = None if cols is None else _np(np.asarray(cols, dtype=np.int64), np.int64)
    nc = X.n if c is None else len(c)
    cptr = None if c is None else c.ctypes.data
    u = np.empty(nc, dtype=np.int32)
    rc = lib.spk_oracle_union_sizes(X.k, X.n, X.p_cp, X.p_ri, nc, cptr, u.ctypes.data, threads)
    if rc != 0:
        raise MemoryError("oracle ran out of host memory")
    col_ptr = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(u, out=col_ptr[1:])
    nnz = int(col_ptr[-1])
    row = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    abs_sum = np.empty(nnz, dtype=np.float64)
    terms = np.empty(nnz, dtype=np.int32)
    rc = lib.spk_oracle_columns(X.k, X.n, X.p_cp, X.p_ri, X.p_va, X.is_f64, nc, cptr, col_ptr.ctypes.data,
                                row.ctypes.data, val.ctypes.data, abs_sum.ctypes.data, terms.ctypes.data,
                                threads)
    if rc == -1:
        raise MemoryError("oracle ran out of host memory")
    if rc == -2:
        raise RuntimeError("oracle column sizes disagree between its two passes")
    return {"col_ptr": col_ptr, "row_idx": row, "val": val, "abs_sum": abs_sum, "terms": terms}


def threads_used(threads: int = 0) -> int:
    return int(load().spk_oracle_threads(threads))
