"""Seeded synthetic SpKAdd inputs.

This module only draws inputs; it holds none of SpKAdd's arithmetic.  The GPU
path's tests and benchmark and the CPU oracle's tests all take their inputs
from here, so both sides see the same matrices.

Every generator returns a list of k CSC matrices, each a tuple
``(col_ptr int32[n+1], row_idx int32[nnz], val float32|float64[nnz])`` of torch
tensors on ``device``, with rows strictly increasing inside every column.
Randomness comes from one ``torch.Generator`` seeded with ``seed`` on
``device``; the CPU and CUDA generators give different streams, so a workload
is "generator X on device D with seed s".  Parity tests copy inputs between
devices instead of regenerating them.

Input families (the paper's workloads, Sec. IV-A):
  * ``er``         -- Erdos-Renyi columns: exactly d distinct uniform rows per
                      column of every input.
  * ``rmat``       -- R-MAT graphs (Chakrabarti et al.) with quadrant
                      probabilities a, b, c, d; in-matrix duplicate edges are
                      summed.  The paper generates both its ER (a=b=c=d=.25)
                      and its RMAT (a=.57, b=c=.19, d=.05) inputs this way.
  * ``spgemm_like``-- partial products of an SpGEMM: every column j has a
                      candidate row set of size 4*L_j and each input draws L_j
                      distinct rows from it, so patterns overlap heavily
                      (the SUMMA stage sums of Sec. IV-E).
  * ``random_csc`` -- small irregular matrices for edge-case tests (empty
                      columns, empty matrices, ragged lengths).
"""
from __future__ import annotations

import math

import torch

__all__ = ["er", "rmat", "spgemm_like", "random_csc", "values", "to_device", "batch_instance_params", "take_columns",
           "instance", "instance_nnz_estimate"]


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def values(g: torch.Generator, count: int, dtype: torch.dtype, kind: str, device) -> torch.Tensor:
    """Value draws.

    ``int8``: integers uniform in {-8..-1, 1..8} (exact in any float type).
    ``uniform``: uniform on [-1, 1] on an exact grid -- x * 2^-52 - 1 for
    float64 (x integer in [0, 2^53]) and x * 2^-23 - 1 for float32
    (x in [0, 2^24]), so every value is representable without rounding.
    """
    if kind == "int8":
        x = torch.randint(0, 16, (count,), generator=g, device=device, dtype=torch.int64)
        x = torch.where(x < 8, x - 8, x - 7)
        return x.to(dtype)
    if kind == "uniform":
        if dtype == torch.float64:
            x = torch.randint(0, (1 << 53) + 1, (count,), generator=g, device=device, dtype=torch.int64)
            return x.to(torch.float64) * (2.0 ** -52) - 1.0
        if dtype == torch.float32:
            x = torch.randint(0, (1 << 24) + 1, (count,), generator=g, device=device, dtype=torch.int64)
            return (x.to(torch.float64) * (2.0 ** -23) - 1.0).to(torch.float32)
    raise ValueError(f"unsupported value kind/dtype {kind}/{dtype}")


def _distinct_sorted_rows(g, n: int, d: int, m: int, device) -> torch.Tensor:
    """(n, d) int64: each row of the result holds d distinct values of [0, m), ascending."""
    if d > m:
        raise ValueError("d > m")
    if d == 0 or n == 0:
        return torch.empty((n, d), dtype=torch.int64, device=device)
    rows = torch.randint(0, m, (n, d), generator=g, device=device, dtype=torch.int64).sort(dim=1).values
    while True:
        bad = (rows[:, 1:] == rows[:, :-1]).any(dim=1)
        idx = bad.nonzero().squeeze(1)
        nb = int(idx.numel())
        if nb == 0:
            return rows
        rows[idx] = torch.randint(0, m, (nb, d), generator=g, device=device, dtype=torch.int64).sort(dim=1).values


def er(k: int, m: int, n: int, d: int, seed: int = 0, dtype=torch.float64, value_kind: str = "uniform",
       device="cpu"):
    """k Erdos-Renyi m x n matrices, exactly d distinct uniform rows in every column."""
    g = _gen(seed, device)
    out = []
    for _ in range(k):
        rows = _distinct_sorted_rows(g, n, d, m, device).reshape(-1).to(torch.int32)
        col_ptr = (torch.arange(n + 1, device=device, dtype=torch.int64) * d).to(torch.int32)
        out.append((col_ptr, rows, values(g, n * d, dtype, value_kind, device)))
    return out


def _csc_from_keys(keys: torch.Tensor, vals: torch.Tensor, m: int, n: int):
    """Sort (col*m+row) keys, sum equal keys exactly in fp64, build CSC."""
    uk, inv = torch.unique(keys, sorted=True, return_inverse=True)
    acc = torch.zeros(uk.numel(), dtype=torch.float64, device=keys.device)
    acc.index_add_(0, inv, vals.to(torch.float64))
    cols = torch.div(uk, m, rounding_mode="floor")
    rows = (uk - cols * m).to(torch.int32)
    counts = torch.bincount(cols, minlength=n)
    col_ptr = torch.zeros(n + 1, dtype=torch.int64, device=keys.device)
    col_ptr[1:] = torch.cumsum(counts, 0)
    if int(col_ptr[-1]) >= 2 ** 31:
        raise ValueError("matrix too large for int32 col_ptr")
    return col_ptr.to(torch.int32), rows, acc.to(vals.dtype)


def rmat(k: int, scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, dtype=torch.float32, value_kind: str = "uniform", device="cpu", chunk: int = 1 << 24):
    """k independent R-MAT matrices of 2^scale x 2^scale with edge_factor * 2^scale edges each.

    Each edge picks, at every one of ``scale`` levels, quadrant a = (row bit 0,
    col bit 0), b = (0, 1), c = (1, 0) or d = (1, 1); no noise, no
    permutation, self loops kept.  Values are uniform on [-1, 1]; duplicate
    edges inside one matrix are summed.  Values are multiples of 2^-23 with
    magnitude <= 1, so the fp64 sums of duplicates are exact (independent of
    order) and are then rounded once to ``dtype``.
    """
    g = _gen(seed, device)
    m = n = 1 << scale
    E = edge_factor << scale
    out = []
    for _ in range(k):
        keys_parts, vals_parts = [], []
        for s0 in range(0, E, chunk):
            e = min(chunk, E - s0)
            rows = torch.zeros(e, dtype=torch.int64, device=device)
            cols = torch.zeros(e, dtype=torch.int64, device=device)
            for lvl in range(scale):
                u = torch.rand(e, generator=g, device=device, dtype=torch.float64)
                rbit = (u >= a + b).to(torch.int64)
                cbit = (((u >= a) & (u < a + b)) | (u >= a + b + c)).to(torch.int64)
                sh = scale - 1 - lvl
                rows |= rbit << sh
                cols |= cbit << sh
            keys_parts.append(cols * m + rows)
            vals_parts.append(values(g, e, dtype, value_kind, device))
        out.append(_csc_from_keys(torch.cat(keys_parts), torch.cat(vals_parts), m, n))
    return out


def spgemm_like(k: int, m: int, n: int, L, seed: int = 0, dtype=torch.float64, value_kind: str = "uniform",
                device="cpu"):
    """Partial-product-shaped inputs.

    ``L`` is an int or an int tensor of length n (entries per column in every
    input).  Column j gets a candidate set of min(4*L_j, m) distinct uniform
    rows; every input draws L_j distinct rows from it (so patterns overlap and
    nnz(B(:,j)) <= 4*L_j however large k is).
    """
    g = _gen(seed, device)
    if isinstance(L, int):
        L = torch.full((n,), L, dtype=torch.int64, device=device)
    L = L.to(device=device, dtype=torch.int64)
    C = torch.clamp(4 * L, max=m)
    out_rows = [[] for _ in range(k)]
    # group columns by (L, C) so every group is one rectangular draw
    pairs = torch.stack([L, C], 1)
    uniq, inv = torch.unique(pairs, dim=0, return_inverse=True)
    order_cols = []
    per_group = []
    for gi in range(uniq.shape[0]):
        lj, cj = int(uniq[gi, 0]), int(uniq[gi, 1])
        cols = (inv == gi).nonzero().squeeze(1)
        cand = _distinct_sorted_rows(g, cols.numel(), cj, m, device)  # (nc, cj)
        picks = []
        for _ in range(k):
            # lj distinct positions of [0, cj): argsort of uniform keys, first lj, sorted
            r = torch.rand((cols.numel(), cj), generator=g, device=device)
            pos = r.argsort(dim=1)[:, :lj].sort(dim=1).values
            picks.append(torch.gather(cand, 1, pos))
        per_group.append((cols, lj, picks))
        order_cols.append(cols)
    res = []
    for i in range(k):
        col_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
        col_ptr[1:] = torch.cumsum(L, 0)
        rows = torch.empty(int(col_ptr[-1]), dtype=torch.int32, device=device)
        for cols, lj, picks in per_group:
            if lj == 0:
                continue
            starts = col_ptr[cols]
            idx = starts[:, None] + torch.arange(lj, device=device)[None, :]
            rows[idx.reshape(-1)] = picks[i].reshape(-1).to(torch.int32)
        res.append((col_ptr.to(torch.int32), rows, values(g, rows.numel(), dtype, value_kind, device)))
    return res


def random_csc(k: int, m: int, n: int, density: float = 0.1, seed: int = 0, dtype=torch.float64,
               value_kind: str = "uniform", device="cpu", empty_col_frac: float = 0.2, empty_matrix_frac: float = 0.0):
    """Irregular small inputs: per-input, per-column random lengths, some empty columns/matrices."""
    g = _gen(seed, device)
    out = []
    for _ in range(k):
        if empty_matrix_frac > 0 and float(torch.rand((), generator=g, device=device)) < empty_matrix_frac:
            out.append((torch.zeros(n + 1, dtype=torch.int32, device=device),
                        torch.empty(0, dtype=torch.int32, device=device),
                        torch.empty(0, dtype=dtype, device=device)))
            continue
        mask = torch.rand((n, m), generator=g, device=device) < density
        empty = torch.rand((n,), generator=g, device=device) < empty_col_frac
        mask &= ~empty[:, None]
        cols, rows = mask.nonzero(as_tuple=True)  # row-major over (col, row): sorted by col then row
        counts = torch.bincount(cols, minlength=n)
        col_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
        col_ptr[1:] = torch.cumsum(counts, 0)
        out.append((col_ptr.to(torch.int32), rows.to(torch.int32),
                    values(g, rows.numel(), dtype, value_kind, device)))
    return out


def to_device(A, device):
    return [tuple(t.to(device) for t in a) for a in A]


def batch_instance_params(count: int, seed: int = 0, k_range=(2, 256), mn_range=(1 << 10, 1 << 16),
                          L_range=(4, 64)):
    """Descriptors of a batch of independent SpKAdd instances (CPU, deterministic).

    k and m = n log-uniform over their ranges, the per-column length range
    [L_lo, L_hi], half ER and half SpGEMM-like, dtype fp64 or fp32 with
    probability 1/2 each.  Returns a list of dicts.
    """
    g = _gen(seed, "cpu")
    u = torch.rand((count, 4), generator=g, dtype=torch.float64)
    out = []
    for q in range(count):
        lk = math.log(k_range[0]) + float(u[q, 0]) * (math.log(k_range[1]) - math.log(k_range[0]))
        lm = math.log(mn_range[0]) + float(u[q, 1]) * (math.log(mn_range[1]) - math.log(mn_range[0]))
        out.append({
            "k": max(k_range[0], min(k_range[1], int(round(math.exp(lk))))),
            "m": max(mn_range[0], min(mn_range[1], int(round(math.exp(lm))))),
            "family": "er" if float(u[q, 2]) < 0.5 else "spgemm_like",
            "dtype": torch.float64 if float(u[q, 3]) < 0.5 else torch.float32,
            "L_range": L_range,
            "seed": int(seed) * 1000003 + q,
        })
    return out


def take_columns(A, cols: torch.Tensor):
    """Sub-inputs holding only the listed columns, in the listed order (pure data movement)."""
    out = []
    for cp, ri, va in A:
        cols_d = cols.to(cp.device)
        cpl = cp.to(torch.int64)
        st, en = cpl[cols_d], cpl[cols_d + 1]
        ln = en - st
        sub_cp = torch.zeros(cols_d.numel() + 1, dtype=torch.int64, device=cp.device)
        sub_cp[1:] = torch.cumsum(ln, 0)
        tot = int(sub_cp[-1])
        if tot:
            seg = torch.repeat_interleave(torch.arange(cols_d.numel(), device=cp.device), ln)
            idx = st[seg] + torch.arange(tot, device=cp.device) - sub_cp[:-1][seg]
        else:
            idx = torch.zeros(0, dtype=torch.int64, device=cp.device)
        out.append((sub_cp.to(torch.int32), ri[idx], va[idx]))
    return out


# ---------------------------------------------------------------------------
# Batch instances: every column j of an instance has one length L_j, shared by
# the instance's k inputs (so the inputs share one col_ptr array).
# ---------------------------------------------------------------------------
def _distinct_rows_var(g, L: torch.Tensor, m: int, reps: int, device, max_elems: int = 1 << 26) -> torch.Tensor:
    """(reps, sum(L)) int32: for every rep and column j, L_j distinct uniform rows of [0, m), ascending.

    Draw L_j uniform rows; while a value repeats, redraw the repeats.  The
    result is the set of the first L_j distinct values of an iid uniform
    sequence, i.e. a uniform L_j-subset of [0, m).  Columns with L_j = m take
    every row.
    """
    n = L.numel()
    total = int(L.sum())
    out = torch.empty((reps, total), dtype=torch.int32, device=device)
    if n == 0 or total == 0 or reps == 0:
        return out
    Lmax = int(L.max())
    if Lmax > m:
        raise ValueError("L_j > m")
    valid = torch.arange(Lmax, device=device)[None, :] < L[:, None]  # (n, Lmax)
    full = (L == m)[None, :, None]
    every = torch.arange(Lmax, device=device, dtype=torch.int64)[None, None, :]
    chunk = max(1, max_elems // (n * Lmax))
    for r0 in range(0, reps, chunk):
        c = min(chunk, reps - r0)
        x = torch.randint(0, m, (c, n, Lmax), generator=g, device=device, dtype=torch.int64)
        x = torch.where(full, every, x)
        x = torch.where(valid[None], x, m).sort(dim=-1).values
        bad = ((x[..., 1:] == x[..., :-1]) & valid[None, :, 1:]).any(dim=-1).nonzero()  # (nb, 2)
        while bad.shape[0]:
            y = x[bad[:, 0], bad[:, 1]]  # (nb, Lmax), sorted, padding m at the end
            rep = torch.zeros_like(y, dtype=torch.bool)
            rep[:, 1:] = y[:, 1:] == y[:, :-1]
            rep &= y < m
            fresh = torch.randint(0, m, y.shape, generator=g, device=device, dtype=torch.int64)
            y = torch.where(rep, fresh, y).sort(dim=-1).values
            x[bad[:, 0], bad[:, 1]] = y
            still = ((y[:, 1:] == y[:, :-1]) & (y[:, 1:] < m)).any(dim=-1)
            bad = bad[still]
        out[r0:r0 + c] = x[:, valid].to(torch.int32)
    return out


def instance(params: dict, device="cpu"):
    """The inputs of one batch instance drawn by batch_instance_params.

    Returns (A, m): A is a list of k CSC tuples sharing one col_ptr.  Column
    lengths L_j are uniform on params["L_range"] (inclusive).  "er": every
    input draws L_j distinct uniform rows of column j.  "spgemm_like": column
    j has a candidate set of min(4 L_j, m) distinct uniform rows and every
    input draws L_j distinct rows of it (partial products of an SpGEMM).
    Values are uniform on [-1, 1] on the exact grid of ``values``.
    """
    g = _gen(params["seed"], device)
    k, m = params["k"], params["m"]
    n = params.get("n", m)
    dtype = params["dtype"]
    lo, hi = params["L_range"]
    L = torch.randint(lo, hi + 1, (n,), generator=g, device=device, dtype=torch.int64)
    L = torch.clamp(L, max=m)
    col_ptr64 = torch.zeros(n + 1, dtype=torch.int64, device=device)
    col_ptr64[1:] = torch.cumsum(L, 0)
    tot = int(col_ptr64[-1])
    if tot >= 2 ** 31:
        raise ValueError("instance input too large for int32 col_ptr")
    col_ptr = col_ptr64.to(torch.int32)
    if params["family"] == "er":
        rows = _distinct_rows_var(g, L, m, k, device)
    else:
        C = torch.clamp(4 * L, max=m)
        cand = _distinct_rows_var(g, C, m, 1, device)[0]  # (sum C,)
        Cmax = int(C.max())
        cptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
        cptr[1:] = torch.cumsum(C, 0)
        cvalid = torch.arange(Cmax, device=device)[None, :] < C[:, None]
        cand_pad = torch.zeros((n, Cmax), dtype=torch.int32, device=device)
        cand_pad[cvalid] = cand
        Lmax = int(L.max())
        lvalid = torch.arange(Lmax, device=device)[None, :] < L[:, None]
        rows = torch.empty((k, tot), dtype=torch.int32, device=device)
        chunk = max(1, (1 << 26) // (n * Cmax))
        for i0 in range(0, k, chunk):
            c = min(chunk, k - i0)
            key = torch.rand((c, n, Cmax), generator=g, device=device)
            key = torch.where(cvalid[None], key, 2.0)
            pos = key.argsort(dim=-1)[..., :Lmax]
            pos = torch.where(lvalid[None], pos, Cmax).sort(dim=-1).values.clamp_(max=Cmax - 1)
            picked = torch.gather(cand_pad[None].expand(c, n, Cmax), 2, pos)
            rows[i0:i0 + c] = picked[:, lvalid]
    vals = values(g, k * tot, dtype, "uniform", device).reshape(k, tot)
    return [(col_ptr, rows[i], vals[i]) for i in range(k)], m


def instance_nnz_estimate(params: dict) -> int:
    """Expected input nnz of an instance (k * n * mean L), for memory planning."""
    lo, hi = params["L_range"]
    return int(params["k"] * params.get("n", params["m"]) * min((lo + hi) / 2.0, params["m"]))
