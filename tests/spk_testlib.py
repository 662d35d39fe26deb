"""Helpers shared by the GPU parity tests: run the CUDA path, run the oracle on
the same inputs, compare.

Comparison rule (see the module docstring of test_gpu_parity.py):
  col_ptr and row_idx bit-exact;
  values bit-exact when exact=True (small-integer fp64 inputs), otherwise
  |gpu - oracle| <= tol * sum|terms| per entry, tol = 1e-12 (fp64), 1e-5 (fp32).
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2112_10223_gb300 as spk

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def to_np(A):
    return [tuple(t.detach().cpu().numpy() for t in a) for a in A]


def run_gpu(A, m, dtype=None, options=None, info=False, method="onepass"):
    dev = torch.device("cuda:0")
    Ad = [tuple(t.to(dev) for t in a) for a in A]
    out = spk.spkadd(Ad, m, dtype=dtype, options=options, info=info, method=method)
    torch.cuda.synchronize()
    return out


def compare(gpu, want, dtype, exact=False, cols=None):
    """gpu = (col_ptr, row_idx, val) numpy for the listed columns (or all)."""
    cp, ri, va = gpu
    assert np.array_equal(cp, want["col_ptr"]), "col_ptr differs"
    assert np.array_equal(ri, want["row_idx"]), "row_idx differs"
    if exact:
        assert np.array_equal(va.astype(np.float64), want["val"]), "values differ (exact)"
        return 0.0
    err = np.abs(va.astype(np.float64) - want["val"])
    bound = TOL[dtype] * want["abs_sum"]
    bad = np.flatnonzero(err > bound)
    assert bad.size == 0, f"{bad.size} values outside tolerance; first at {bad[0]}: err {err[bad[0]]} bound {bound[bad[0]]}"
    return float((err / np.maximum(want["abs_sum"], 1e-300)).max(initial=0.0))


def check_full(A, m, dtype, exact=False, options=None):
    """Whole-matrix parity against the oracle; returns (info, max relative error)."""
    cp, ri, va, info = run_gpu(A, m, dtype=dtype, options=options, info=True)
    want = oracle.add(to_np(A))
    rel = compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), want, dtype, exact=exact)
    return info, rel


def gather_columns(A, cols: torch.Tensor):
    """Sub-inputs holding only the listed columns (in order), gathered on the inputs' device."""
    out = []
    for cp, ri, va in A:
        cpl = cp.to(torch.int64)
        st, en = cpl[cols], cpl[cols + 1]
        ln = en - st
        sub_cp = torch.zeros(cols.numel() + 1, dtype=torch.int64, device=cp.device)
        sub_cp[1:] = torch.cumsum(ln, 0)
        tot = int(sub_cp[-1])
        if tot:
            seg = torch.repeat_interleave(torch.arange(cols.numel(), device=cp.device), ln)
            idx = st[seg] + torch.arange(tot, device=cp.device) - sub_cp[:-1][seg]
        else:
            idx = torch.zeros(0, dtype=torch.int64, device=cp.device)
        out.append((sub_cp.to(torch.int32), ri[idx], va[idx]))
    return out


def gather_output_columns(B, cols: torch.Tensor):
    cp, ri, va = B
    st, en = cp[cols], cp[cols + 1]
    ln = en - st
    sub_cp = torch.zeros(cols.numel() + 1, dtype=torch.int64, device=cp.device)
    sub_cp[1:] = torch.cumsum(ln, 0)
    tot = int(sub_cp[-1])
    if tot:
        seg = torch.repeat_interleave(torch.arange(cols.numel(), device=cp.device), ln)
        idx = st[seg] + torch.arange(tot, device=cp.device) - sub_cp[:-1][seg]
    else:
        idx = torch.zeros(0, dtype=torch.int64, device=cp.device)
    return sub_cp, ri[idx], va[idx]


def sample_columns(A, count: int, heavy: int, seed: int = 0):
    """Column sample: the `heavy` columns with the largest summed input count, plus `count` random ones."""
    n = A[0][0].numel() - 1
    dev = A[0][0].device
    s = torch.zeros(n, dtype=torch.int64, device=dev)
    for cp, _, _ in A:
        s += (cp[1:] - cp[:-1]).to(torch.int64)
    top = torch.topk(s, min(heavy, n)).indices
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    rnd = torch.randint(0, n, (count,), generator=g).to(dev)
    edge = torch.tensor([0, n - 1], device=dev)
    return torch.unique(torch.cat([top, rnd, edge])), s


def check_sampled(A, B, m, cols, dtype, exact=False):
    sub = gather_columns(A, cols)
    want = oracle.add(to_np(sub))
    got = gather_output_columns(B, cols)
    return compare(tuple(t.cpu().numpy() for t in got), want, dtype, exact=exact)


def check_global_invariants(A, B, m):
    """Properties that hold at any size, checked with plain torch ops on the device."""
    cp, ri, va = B
    n = cp.numel() - 1
    nnz_in = sum(a[1].numel() for a in A)
    nnz = int(cp[-1])
    assert int(cp[0]) == 0 and nnz <= nnz_in, "nnz(B) must not exceed sum nnz(A_i)"
    assert bool((cp[1:] >= cp[:-1]).all()), "col_ptr not monotone"
    assert ri.numel() >= nnz
    ri = ri[:nnz]
    assert bool(((ri >= 0) & (ri < m)).all()), "row out of range"
    if nnz > 1:
        starts = torch.zeros(nnz, dtype=torch.bool, device=ri.device)
        ne = cp[:-1][cp[:-1] < cp[1:]]
        starts[ne] = True
        ok = (ri[1:] > ri[:-1]) | starts[1:]
        assert bool(ok.all()), "rows not strictly increasing inside a column"
    # per-column counts: at least the largest input column, at most the sum
    s = torch.zeros(n, dtype=torch.int64, device=cp.device)
    mx = torch.zeros(n, dtype=torch.int64, device=cp.device)
    for a in A:
        ln = (a[0][1:] - a[0][:-1]).to(torch.int64)
        s += ln
        mx = torch.maximum(mx, ln)
    u = cp[1:] - cp[:-1]
    assert bool((u <= s).all() and (u >= mx).all()), "per-column nnz outside [max_i nnz, sum_i nnz]"
    tot_in = sum(float(a[2].to(torch.float64).sum()) for a in A)
    tot_out = float(va[:nnz].to(torch.float64).sum())
    scale = sum(float(a[2].to(torch.float64).abs().sum()) for a in A)
    assert abs(tot_in - tot_out) <= 1e-6 * max(scale, 1.0), "sum of values not preserved"
