"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Bar: col_ptr and row_idx bit-exact; values bit-exact for small-integer fp64
inputs, otherwise per entry |gpu - oracle| <= 1e-12 * sum|terms| (fp64) or
1e-5 * sum|terms| (fp32).  Small cases compare every entry; the full-size
workloads compare sampled columns (the heaviest ones and a random set) with
the oracle and check size-independent invariants on every column.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2112_10223_gb300 as spk
import synth
from spk_testlib import (check_full, check_global_invariants, check_sampled, compare, run_gpu, sample_columns,
                         to_np)

pytestmark = pytest.mark.gpu

F64, F32 = torch.float64, torch.float32


@pytest.fixture(scope="module", autouse=True)
def _built():
    spk.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_er_k4_1024_small_integers_bit_exact():
    """k = 4 ER 1024 x 1024, 8 distinct rows per column, fp64 integers in [-8, 8] \\ {0}, seed 0."""
    A = synth.er(4, 1024, 1024, 8, seed=0, dtype=F64, value_kind="int8")
    info, _ = check_full(A, 1024, F64, exact=True)
    assert info["cols_warp"] == 1024
    u = oracle.union_sizes(to_np(A))
    s = sum((a[0][1:] - a[0][:-1]).numpy() for a in A)
    assert info["cols_unique"] == int((u == s).sum())


@pytest.mark.parametrize("sort_mode", [0, 1])
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("seed", range(3))
def test_irregular_small(seed, dtype, sort_mode):
    A = synth.random_csc(7, 300, 257, density=0.05, seed=seed, dtype=dtype, empty_matrix_frac=0.1)
    check_full(A, 300, dtype, options=spk.default_options(sort_mode=sort_mode))


@pytest.mark.parametrize("dtype", [F64, F32])
def test_classes_forced_small_thresholds(dtype):
    """Tiny thresholds push ordinary columns through the CTA and heavy-bitmap paths."""
    A = synth.random_csc(9, 500, 200, density=0.08, seed=4, dtype=dtype)
    opt = spk.default_options(warp_max=250, cta_max=320)
    info, _ = check_full(A, 500, dtype, options=opt)
    assert info["cols_warp"] > 0 and info["cols_cta"] > 0 and info["cols_heavy"] > 0, info


@pytest.mark.parametrize("dtype", [F32, F64])
def test_rmat_split_windows(dtype):
    """R-MAT scale 14: heavy columns with more distinct rows than one window holds."""
    A = synth.rmat(32, 14, 16, seed=1, dtype=dtype)
    opt = spk.default_options(warp_max=32, cta_max=64, window_max=1024)
    info, _ = check_full(A, 1 << 14, dtype, options=opt)
    # columns cut into more than 3 windows use per-input binary searches, the
    # others let each window read its whole column: both kinds occur here
    assert info["windows_split"] > 0, info
    assert info["windows"] - info["windows_split"] > info["cols_cta"], info


def test_rmat_default_thresholds():
    A = synth.rmat(16, 13, 16, seed=2, dtype=F32)
    info, _ = check_full(A, 1 << 13, F32)
    assert info["cols_heavy"] > 0


def test_heavy_columns_span_two_row_slabs():
    """m > 2^20: the heavy symbolic pass runs its bitmap over two row slabs."""
    m = (1 << 20) + 4099
    A = synth.er(6, m, 5, 1500, seed=3, dtype=F64, value_kind="int8")
    info, _ = check_full(A, m, F64, exact=True, options=spk.default_options(window_max=1024))
    assert info["cols_heavy"] == 5 and info["windows_split"] > 0


def test_spgemm_like_overlapping_patterns():
    A = synth.spgemm_like(40, 2000, 300, 24, seed=5, dtype=F64)
    info, _ = check_full(A, 2000, F64)
    assert info["nnz_out"] <= 300 * 96


def test_k1_identity():
    A = synth.random_csc(1, 200, 150, density=0.1, seed=6, dtype=F64)
    cp, ri, va = run_gpu(A, 200)
    assert np.array_equal(cp.cpu().numpy(), A[0][0].numpy().astype(np.int64))
    assert np.array_equal(ri.cpu().numpy(), A[0][1].numpy())
    assert np.array_equal(va.cpu().numpy(), A[0][2].numpy())


def test_all_empty_and_zero_columns():
    A = [(torch.zeros(51, dtype=torch.int32), torch.zeros(0, dtype=torch.int32), torch.zeros(0, dtype=F64))
         for _ in range(3)]
    cp, ri, va = run_gpu(A, 10)
    assert cp.cpu().tolist() == [0] * 51 and ri.numel() == 0 and va.numel() == 0


def test_single_row_matrices():
    A = synth.random_csc(5, 1, 400, density=0.5, seed=7, dtype=F64, value_kind="int8")
    check_full(A, 1, F64, exact=True)


def test_full_dense_column_and_last_row():
    m, k = 3000, 6
    rows = torch.arange(m, dtype=torch.int32)
    A = []
    for i in range(k):
        cp = torch.tensor([0, 0, m, m + 1], dtype=torch.int32)  # col 0 empty, col 1 full, col 2 = last row
        ri = torch.cat([rows, torch.tensor([m - 1], dtype=torch.int32)])
        A.append((cp, ri, synth.values(torch.Generator().manual_seed(i), m + 1, F64, "int8", "cpu")))
    check_full(A, m, F64, exact=True)


def test_identical_inputs_compression_k():
    A1 = synth.er(1, 5000, 400, 40, seed=8, dtype=F64, value_kind="int8")
    A = A1 * 24  # cf = 24
    info, _ = check_full(A, 5000, F64, exact=True)
    assert info["nnz_out"] == 400 * 40


@pytest.mark.parametrize("s", [511, 512, 513, 4095, 4096, 4097])
def test_class_boundaries(s):
    """Columns whose summed input count sits on each side of the class limits."""
    k = 8
    m = 20000
    per = [s // k + (1 if i < s % k else 0) for i in range(k)]
    g = torch.Generator().manual_seed(s)
    A = []
    for i in range(k):
        rows = torch.randperm(m, generator=g)[:per[i]].sort().values.to(torch.int32)
        A.append((torch.tensor([0, per[i]], dtype=torch.int32), rows, synth.values(g, per[i], F64, "int8", "cpu")))
    check_full(A, m, F64, exact=True)


def test_cancellation_keeps_positive_zero():
    A = synth.random_csc(1, 400, 300, density=0.05, seed=9, dtype=F64)
    A = A + [(A[0][0], A[0][1], -A[0][2])]
    cp, ri, va = run_gpu(A, 400)
    v = va.cpu().numpy()
    assert len(v) == A[0][1].numel() and (v == 0).all() and not np.signbit(v).any()


def test_many_inputs_span_several_chunks():
    A = synth.random_csc(300, 900, 60, density=0.01, seed=10, dtype=F32)
    check_full(A, 900, F32)


def test_permutation_invariance_indices_bit_identical():
    A = synth.random_csc(12, 700, 300, density=0.03, seed=11, dtype=F64)
    B1 = run_gpu(A, 700)
    perm = torch.randperm(12, generator=torch.Generator().manual_seed(0)).tolist()
    B2 = run_gpu([A[p] for p in perm], 700)
    assert torch.equal(B1[0], B2[0]) and torch.equal(B1[1], B2[1])
    np.testing.assert_allclose(B1[2].cpu().numpy(), B2[2].cpu().numpy(), rtol=0, atol=1e-13)


def test_repeated_runs_indices_bit_identical():
    A = synth.rmat(8, 12, 8, seed=12, dtype=F32)
    outs = [run_gpu(A, 1 << 12) for _ in range(3)]
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1])


# ---------------------------------------------------------------- error paths
def _plan(A, m, **opts):
    Ad = [tuple(t.cuda() for t in a) for a in A]
    return spk.spkadd_plan(Ad, m, options=spk.default_options(**opts))


def test_validate_accepts_valid_input():
    A = synth.random_csc(3, 50, 40, density=0.2, seed=13, dtype=F64)
    h = _plan(A, 50, validate=1)
    spk.spkadd_destroy(h)


def test_validate_rejects_unsorted_rows():
    cp = torch.tensor([0, 3], dtype=torch.int32)
    A = [(cp, torch.tensor([1, 5, 3], dtype=torch.int32), torch.ones(3, dtype=F64))]
    with pytest.raises(spk.SpkaddError) as e:
        _plan(A, 10, validate=1)
    assert e.value.status == 3


def test_validate_rejects_duplicate_rows():
    cp = torch.tensor([0, 2], dtype=torch.int32)
    A = [(cp, torch.tensor([4, 4], dtype=torch.int32), torch.ones(2, dtype=F64))]
    with pytest.raises(spk.SpkaddError) as e:
        _plan(A, 10, validate=1)
    assert e.value.status == 3


def test_validate_rejects_row_out_of_range():
    cp = torch.tensor([0, 2], dtype=torch.int32)
    A = [(cp, torch.tensor([4, 10], dtype=torch.int32), torch.ones(2, dtype=F64))]
    with pytest.raises(spk.SpkaddError) as e:
        _plan(A, 10, validate=1)
    assert e.value.status == 4


@pytest.mark.parametrize("bad_row", [10, 4096, -5, 2**31 - 1])
@pytest.mark.parametrize("batch", [False, True])
def test_row_out_of_range_in_warp_column_reported_without_validation(bad_row, batch):
    """validate = 0: a warp-class column holding a row outside [0, m) is caught
    by the symbolic pass (its bucket passes index shared counters by row and
    must not run on it); spkadd_symbolic reports SPKADD_ERR_INDEX_RANGE."""
    cp = torch.tensor([0, 3, 5], dtype=torch.int32)
    A = [(cp, torch.tensor([1, 4, 7, 2, 3], dtype=torch.int32), torch.ones(5, dtype=F64)),
         (cp, torch.tensor([0, 4, bad_row, 5, 9], dtype=torch.int32), torch.ones(5, dtype=F64))]
    Ad = [tuple(t.to("cuda:0") for t in a) for a in A]
    with pytest.raises(spk.SpkaddError) as e:
        if batch:
            spk.spkadd_batch([(Ad, 10)])
        else:
            spk.spkadd(Ad, 10)
    assert e.value.name == "SPKADD_ERR_INDEX_RANGE"


def test_validate_rejects_bad_col_ptr():
    cp = torch.tensor([0, 3, 2], dtype=torch.int32)
    A = [(cp, torch.tensor([1, 2], dtype=torch.int32), torch.ones(2, dtype=F64))]
    with pytest.raises(spk.SpkaddError) as e:
        _plan(A, 10, validate=1)
    assert e.value.status == 4


def test_numeric_before_symbolic_is_a_state_error():
    A = synth.random_csc(2, 30, 20, density=0.2, seed=14, dtype=F64)
    h = _plan(A, 30)
    cp = torch.empty(21, dtype=torch.int64, device="cuda")
    with pytest.raises(spk.SpkaddError) as e:
        spk.spkadd_numeric(h, cp, torch.empty(100, dtype=torch.int32, device="cuda"),
                           torch.empty(100, dtype=F64, device="cuda"))
    assert e.value.status == 9
    spk.spkadd_destroy(h)


def test_user_allocator_and_allocation_failure():
    A = synth.random_csc(4, 100, 80, density=0.1, seed=15, dtype=F64)
    Ad = [tuple(t.cuda() for t in a) for a in A]
    live = {}

    @spk.ALLOC_FN
    def alloc(nbytes, stream, ctx):
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @spk.FREE_FN
    def free(ptr, stream, ctx):
        live.pop(ptr, None)

    o = spk.default_options()
    o.alloc, o.free = alloc, free
    cp, ri, va = spk.spkadd(Ad, 100, options=o)
    torch.cuda.synchronize()
    want = oracle.add(to_np(A))
    compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), want, F64)

    @spk.ALLOC_FN
    def failing(nbytes, stream, ctx):
        return None

    o2 = spk.default_options()
    o2.alloc, o2.free = failing, free
    with pytest.raises(spk.SpkaddError) as e:
        spk.spkadd_plan(Ad, 100, options=o2)
    assert e.value.status == 6


# ---------------------------------------------------------- full-size workloads
def _full_size_every_column(A, m, dtype, methods):
    """Whole-matrix parity at full size: every column against the oracle (OpenMP over the host's cores)."""
    want = oracle.add(to_np(A))
    infos = {}
    for method in methods:
        cp, ri, va, info = spk.spkadd(A, m, info=True, method=method)
        torch.cuda.synchronize()
        check_global_invariants(A, (cp, ri, va), m)
        compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), want, dtype)
        infos[method] = info
        del cp, ri, va
    return infos


def test_er_k32_2pow20_d16_fp64_every_column():
    """k = 32 ER 2^20 x 2^20, 16 distinct rows per column, fp64 uniform [-1, 1]: every column vs the oracle,
    through the one-pass kernel and through the symbolic + numeric kernels."""
    dev = torch.device("cuda:0")
    A = synth.er(32, 1 << 20, 1 << 20, 16, seed=0, dtype=F64, device=dev)
    infos = _full_size_every_column(A, 1 << 20, F64, ("onepass", "twopass"))
    assert infos["onepass"]["onepass"] == 1 and infos["twopass"]["cols_warp"] == 1 << 20


def test_rmat_k64_scale20_fp32_every_column():
    """k = 64 independent R-MAT scale 20, edge factor 16, (.57, .19, .19, .05), fp32: every column vs the oracle."""
    dev = torch.device("cuda:0")
    A = synth.rmat(64, 20, 16, seed=0, dtype=F32, device=dev)
    infos = _full_size_every_column(A, 1 << 20, F32, ("twopass",))
    info = infos["twopass"]
    assert info["cols_heavy"] > 0 and info["windows_split"] > 0


@pytest.mark.parametrize("dtype,kind", [(F64, "int8"), (F64, "uniform"), (F32, "uniform")])
def test_register_path_equal_short_segments(dtype, kind):
    """k = 32 inputs of 16 rows per column (16-byte aligned segments): the register-resident warp path."""
    A = synth.er(32, 4096, 1500, 16, seed=11, dtype=dtype, value_kind=kind)
    info, _ = check_full(A, 4096, dtype, exact=(kind == "int8"))
    assert info["cols_warp"] == 1500


def _cap_columns(A, cap):
    """Keep the first `cap` rows of every column (pure data movement)."""
    out = []
    for cp, ri, va in A:
        cpl = cp.to(torch.int64)
        ln = torch.clamp(cpl[1:] - cpl[:-1], max=cap)
        keep = torch.zeros(ri.numel(), dtype=torch.bool)
        for j in range(cp.numel() - 1):
            keep[int(cpl[j]):int(cpl[j]) + int(ln[j])] = True
        ncp = torch.zeros_like(cpl)
        ncp[1:] = torch.cumsum(ln, 0)
        out.append((ncp.to(torch.int32), ri[keep], va[keep]))
    return out


@pytest.mark.parametrize("sort_mode", [0, 1])
@pytest.mark.parametrize("dtype", [F64, F32])
def test_register_path_ragged_unaligned_segments(dtype, sort_mode):
    """k = 32 inputs, lengths 0..16 varying per input and column (unaligned starts: scalar loads)."""
    A = _cap_columns(synth.random_csc(32, 256, 500, density=0.04, seed=12, dtype=dtype, empty_col_frac=0.05), 16)
    lens = torch.stack([a[0][1:] - a[0][:-1] for a in A])
    assert int(lens.max()) == 16 and int(lens.min()) == 0
    check_full(A, 256, dtype, options=spk.default_options(sort_mode=sort_mode))


def _filter_hash(r):
    return ((r * 0x9E3779B1) & 0xFFFFFFFF) >> 17


@pytest.mark.parametrize("seed", range(3))
def test_symbolic_filter_collisions_and_repeats(seed):
    """Warp columns built from rows that collide in the symbolic filter's hash,
    mixed with true repeats across inputs in every arrangement."""
    g = torch.Generator().manual_seed(seed)
    m = 1 << 20
    # collision classes: several distinct rows with one hash value
    by_hash = {}
    while True:
        r = int(torch.randint(0, m, (1,), generator=g))
        by_hash.setdefault(_filter_hash(r), set()).add(r)
        classes = [sorted(v) for v in by_hash.values() if len(v) >= 3]
        if len(classes) >= 40:
            break
    k, n = 12, 300
    cols = [[set() for _ in range(n)] for _ in range(k)]
    for j in range(n):
        cls = classes[j % len(classes)]
        extra = torch.randint(0, m, (6,), generator=g).tolist()
        pool = cls + extra
        for i in range(k):
            pick = torch.rand(len(pool), generator=g) < 0.45
            cols[i][j] = {pool[t] for t in range(len(pool)) if pick[t]}
    A = []
    for i in range(k):
        cp = [0]
        rows = []
        for j in range(n):
            rr = sorted(cols[i][j])
            rows += rr
            cp.append(len(rows))
        vals = synth.values(g, len(rows), F64, "int8", "cpu")
        A.append((torch.tensor(cp, dtype=torch.int32), torch.tensor(rows, dtype=torch.int32), vals))
    info, _ = check_full(A, m, F64, exact=True)
    assert info["cols_warp"] == n


# ---------------------------------------------------------------------------
# Maximum sizes.
# ---------------------------------------------------------------------------
def test_output_over_2pow31_nonzeros_int64_col_ptr():
    """nnz(B) > 2^31 (int64 col_ptr_B): k = 2 ER inputs of 2^20 columns with 1030 rows each
    (CTA class), generated on the device; sampled columns against the oracle plus invariants."""
    dev = torch.device("cuda:0")
    m = n = 1 << 20
    A = synth.er(2, m, n, 1030, seed=21, dtype=F32, device=dev)
    cp, ri, va, info = spk.spkadd(A, m, info=True)
    torch.cuda.synchronize()
    assert int(cp[-1]) > 2 ** 31 and info["cols_cta"] == n
    check_global_invariants(A, (cp, ri, va), m)
    cols, _ = sample_columns(A, 64, 8, seed=1)
    last = torch.tensor([n - 3, n - 2, n - 1], device=dev)  # columns whose entries sit past 2^31
    check_sampled(A, (cp, ri, va), m, torch.unique(torch.cat([cols, last])), F32)
    del A, cp, ri, va
    torch.cuda.empty_cache()


def test_max_k_inputs():
    """k = SPKADD_MAX_K = 65536 inputs (one entry each in a few columns): chunk loops over 2048
    groups of 32 inputs, heavy columns with per-input window searches."""
    k, m, n = 65536, 3000, 3
    g = torch.Generator().manual_seed(5)
    rows = torch.randint(0, m, (k,), generator=g)
    colsel = torch.randint(0, n, (k,), generator=g)
    A = []
    for i in range(k):
        cp = torch.zeros(n + 1, dtype=torch.int32)
        cp[int(colsel[i]) + 1:] = 1
        A.append((cp, rows[i:i + 1].to(torch.int32), torch.tensor([float((i % 15) - 7)], dtype=F64)))
    info, _ = check_full(A, m, F64, exact=True, options=spk.default_options(window_max=1024))
    assert info["k"] == k and info["cols_heavy"] == n


def test_rows_near_int32_max():
    """m = 2^31 - 2: rows at the top of the int32 range in warp, CTA and heavy columns."""
    m = 2 ** 31 - 2
    top = [m - 1, m - 2, m - 3, m - 1000, 2 ** 30, 0, 1, 2 ** 31 - 65]
    g = torch.Generator().manual_seed(6)
    k, n = 6, 3
    A = []
    for i in range(k):
        cols = []
        for j in range(n):
            cnt = [8, 600, 5000][j]  # warp (s = 48), CTA (3,600) and heavy (30,000) columns
            r = torch.unique(torch.cat([torch.tensor(top), torch.randint(m - 2 ** 22, m, (cnt,), generator=g)]))
            cols.append(r[torch.randperm(r.numel(), generator=g)[:cnt]].sort().values)
        cp = torch.zeros(n + 1, dtype=torch.int32)
        cp[1:] = torch.cumsum(torch.tensor([c.numel() for c in cols]), 0)
        rr = torch.cat(cols).to(torch.int32)
        A.append((cp, rr, synth.values(g, rr.numel(), F64, "int8", "cpu")))
    info, _ = check_full(A, m, F64, exact=True, options=spk.default_options(window_max=1024))
    assert info["cols_warp"] == 1 and info["cols_cta"] == 1 and info["cols_heavy"] == 1


# ---------------------------------------------------------------------------
# Unordered input columns (option input_order = 1).
# ---------------------------------------------------------------------------
def _shuffle_within_columns(A, seed):
    """Permute each input column's (row, value) pairs (pure data movement)."""
    g = torch.Generator().manual_seed(seed)
    out = []
    for cp, ri, va in A:
        cpl = cp.to(torch.int64)
        n = cp.numel() - 1
        col = torch.repeat_interleave(torch.arange(n), cpl[1:] - cpl[:-1])
        key = col.to(torch.float64) + torch.rand(ri.numel(), generator=g, dtype=torch.float64) * 0.5
        perm = torch.argsort(key)
        out.append((cp, ri[perm], va[perm]))
    return out


UNORDERED = dict(input_order=1)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_unordered_inputs_all_classes(dtype):
    A = _shuffle_within_columns(synth.random_csc(9, 500, 200, density=0.08, seed=31, dtype=dtype,
                                                 value_kind="int8"), 1)
    assert any(bool((a[1][1:] < a[1][:-1]).any()) for a in A)  # really unordered
    opt = spk.default_options(warp_max=250, cta_max=320, **UNORDERED)
    info, _ = check_full(A, 500, dtype, exact=True, options=opt)
    assert info["cols_warp"] > 0 and info["cols_cta"] > 0 and info["cols_heavy"] > 0, info


def test_unordered_inputs_rmat_windows_read_whole_columns():
    """Split heavy windows without per-input binary searches: every window reads its whole column."""
    A = _shuffle_within_columns(synth.rmat(16, 13, 16, seed=32, dtype=F32), 2)
    opt = spk.default_options(warp_max=32, cta_max=64, window_max=1024, **UNORDERED)
    info, _ = check_full(A, 1 << 13, F32, options=opt)
    assert info["windows"] > info["cols_cta"] + info["cols_heavy"] and info["windows_split"] == 0, info


def test_unordered_inputs_two_row_slabs():
    m = (1 << 20) + 4099
    A = _shuffle_within_columns(synth.er(6, m, 5, 1500, seed=33, dtype=F64, value_kind="int8"), 3)
    info, _ = check_full(A, m, F64, exact=True, options=spk.default_options(window_max=1024, **UNORDERED))
    assert info["cols_heavy"] == 5


def test_unordered_inputs_repeated_row_inside_one_input_is_summed():
    """With unordered inputs a row may repeat inside one input column; it is summed like any term."""
    cp = torch.tensor([0, 4, 7], dtype=torch.int32)
    A = [(cp, torch.tensor([5, 2, 5, 9, 1, 1, 3], dtype=torch.int32),
          torch.tensor([1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0], dtype=F64)),
         (torch.tensor([0, 1, 2], dtype=torch.int32), torch.tensor([5, 3], dtype=torch.int32),
          torch.tensor([128.0, 256.0], dtype=F64))]
    cp_b, ri_b, va_b = run_gpu(A, 10, options=spk.default_options(**UNORDERED))
    assert cp_b.tolist() == [0, 3, 5]
    assert ri_b.tolist() == [2, 5, 9, 1, 3]
    assert va_b.tolist() == [2.0, 133.0, 8.0, 48.0, 320.0]
    want = oracle.add(to_np(A))
    assert np.array_equal(ri_b.cpu().numpy(), want["row_idx"]) and np.array_equal(va_b.cpu().numpy(), want["val"])


def test_validate_with_unordered_inputs():
    A = _shuffle_within_columns(synth.er(3, 400, 50, 9, seed=34, dtype=F64), 4)
    run_gpu(A, 400, options=spk.default_options(validate=1, **UNORDERED))  # accepted
    with pytest.raises(spk.SpkaddError) as e:  # ordered mode rejects the same inputs
        run_gpu(A, 400, options=spk.default_options(validate=1))
    assert e.value.name == "SPKADD_ERR_UNSORTED"
    bad = [A[0], A[1], (A[2][0], torch.where(A[2][1] == A[2][1][0], 400, A[2][1]), A[2][2])]
    with pytest.raises(spk.SpkaddError) as e:
        run_gpu(bad, 400, options=spk.default_options(validate=1, **UNORDERED))
    assert e.value.name == "SPKADD_ERR_INDEX_RANGE"


# ---------------------------------------------------------------------------
# Unsorted output (sort_mode = 2).
# ---------------------------------------------------------------------------
def _sorted_columns(cp, ri, va):
    """Each column's (row, value) pairs sorted by row (host numpy)."""
    cp, ri, va = cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()
    order = np.concatenate([cp[j] + np.argsort(ri[cp[j]:cp[j + 1]], kind="stable") for j in range(len(cp) - 1)]
                           or [np.zeros(0, dtype=np.int64)]).astype(np.int64)
    return cp, ri[order], va[order]


@pytest.mark.parametrize("dtype,kind", [(F64, "int8"), (F32, "uniform")])
def test_unsorted_output_same_pairs(dtype, kind):
    # m = 2^20: most columns have no repeated row, so they skip the sort
    A = synth.er(32, 1 << 20, 700, 16, seed=41, dtype=dtype, value_kind=kind)
    # sort_mode 2 is a mode of the numeric kernel (the one-pass kernel sorts every column)
    cp, ri, va = run_gpu(A, 1 << 20, options=spk.default_options(sort_mode=2), method="twopass")
    unsorted = any(bool((ri[int(cp[j]) + 1:int(cp[j + 1])] < ri[int(cp[j]):int(cp[j + 1]) - 1]).any())
                   for j in range(700))
    assert unsorted  # the mode really leaves some columns unsorted
    want = oracle.add(to_np(A))
    compare(_sorted_columns(cp, ri, va), want, dtype, exact=(kind == "int8"))


def test_unsorted_output_with_repeats_and_all_classes():
    A = synth.random_csc(9, 300, 200, density=0.1, seed=42, dtype=F64, value_kind="int8")
    opt = spk.default_options(sort_mode=2, warp_max=200, cta_max=300)
    cp, ri, va = run_gpu(A, 300, options=opt)
    compare(_sorted_columns(cp, ri, va), oracle.add(to_np(A)), F64, exact=True)


# ---------------------------------------------------------------------------
# Thread-block accumulators (option block_accumulator): the flat row bitmap
# (1) and the compact word table (2) on the same inputs.
# ---------------------------------------------------------------------------
ACCS = [1, 2]


@pytest.mark.parametrize("acc", ACCS)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_accumulators_all_classes(acc, dtype):
    A = synth.random_csc(9, 500, 200, density=0.08, seed=4, dtype=dtype)
    opt = spk.default_options(warp_max=250, cta_max=320, block_accumulator=acc)
    info, _ = check_full(A, 500, dtype, options=opt)
    assert info["cols_cta"] > 0 and info["cols_heavy"] > 0, info


@pytest.mark.parametrize("acc", ACCS)
@pytest.mark.parametrize("dtype", [F32, F64])
def test_accumulators_rmat_split_windows(acc, dtype):
    """Skewed windows: dense near row 0 (full 32-row words), sparse in the tail."""
    A = synth.rmat(32, 14, 16, seed=1, dtype=dtype)
    opt = spk.default_options(warp_max=32, cta_max=64, window_max=1024, block_accumulator=acc)
    info, _ = check_full(A, 1 << 14, dtype, options=opt)
    assert info["windows_split"] > 0, info


@pytest.mark.parametrize("acc", ACCS)
def test_accumulators_two_row_slabs(acc):
    """m > 2^20: items spanning two slabs run the accumulator once per slab."""
    m = (1 << 20) + 4099
    A = synth.er(6, m, 5, 1500, seed=3, dtype=F64, value_kind="int8")
    info, _ = check_full(A, m, F64, exact=True, options=spk.default_options(window_max=1024, block_accumulator=acc))
    assert info["cols_heavy"] == 5


@pytest.mark.parametrize("acc", ACCS)
def test_accumulators_unordered_two_row_slabs(acc):
    m = (1 << 20) + 4099
    A = _shuffle_within_columns(synth.er(6, m, 5, 1500, seed=33, dtype=F64, value_kind="int8"), 3)
    opt = spk.default_options(window_max=1024, block_accumulator=acc, **UNORDERED)
    check_full(A, m, F64, exact=True, options=opt)


@pytest.mark.parametrize("acc", ACCS)
def test_accumulators_dense_column(acc):
    """A full column: every 32-row word of the item is full."""
    m, k = 3000, 6
    rows = torch.arange(m, dtype=torch.int32)
    A = []
    for i in range(k):
        cp = torch.tensor([0, 0, m, m + 1], dtype=torch.int32)
        ri = torch.cat([rows, torch.tensor([m - 1], dtype=torch.int32)])
        A.append((cp, ri, synth.values(torch.Generator().manual_seed(i), m + 1, F64, "int8", "cpu")))
    check_full(A, m, F64, exact=True, options=spk.default_options(block_accumulator=acc))


@pytest.mark.parametrize("acc", ACCS)
@pytest.mark.parametrize("dtype", [F64, F32])
def test_accumulators_one_row_per_word_at_table_capacity(acc, dtype):
    """4096 distinct rows, each alone in its 32-row word, over m = 2^20: the
    compact table holds exactly window_max words (its capacity)."""
    k, m, n = 4, 1 << 20, 6
    g = torch.Generator().manual_seed(77)
    words = [torch.randperm(m // 32, generator=g)[:4096].sort().values for _ in range(n)]
    A = []
    for i in range(k):
        cps, ris = [0], []
        for j in range(n):
            mine = words[j][i::k] * 32 + torch.randint(0, 32, (1024,), generator=g)  # disjoint across inputs
            ris.append(mine.to(torch.int32))
            cps.append(cps[-1] + 1024)
        ri = torch.cat(ris)
        A.append((torch.tensor(cps, dtype=torch.int32), ri, synth.values(g, ri.numel(), dtype, "uniform", "cpu")))
    info, _ = check_full(A, m, dtype, options=spk.default_options(block_accumulator=acc))
    assert info["cols_cta"] == n and info["nnz_out"] == 4096 * n, info


@pytest.mark.parametrize("acc", ACCS)
def test_accumulators_mixed_dtype_batch(acc):
    problems_cpu = [(synth.rmat(8, 12, 16, seed=90 + q, dtype=F64 if q % 2 else F32), 1 << 12) for q in range(4)]
    problems_cpu.append((synth.er(5, (1 << 20) + 17, 4, 900, seed=95, dtype=F32), (1 << 20) + 17))
    problems = [([tuple(t.to("cuda:0") for t in a) for a in A], m) for A, m in problems_cpu]
    opt = spk.default_options(warp_max=64, cta_max=128, window_max=1024, block_accumulator=acc)
    outs, info = spk.spkadd_batch(problems, options=opt, info=True)
    torch.cuda.synchronize()
    assert info["cols_cta"] > 0 and info["cols_heavy"] > 0, info
    for (A, m), (cp, ri, va) in zip(problems_cpu, outs):
        compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), oracle.add(to_np(A)), A[0][2].dtype)


@pytest.mark.parametrize("acc", ACCS)
@pytest.mark.parametrize("order", ["sorted", "unordered"])
def test_accumulators_heavy_column_many_subranges(acc, order):
    """A heavy column with ~32K distinct rows over 2^20 rows (its compact
    symbolic form cuts the slab into several sub-ranges) next to a dense one
    (every row of [0, 40000): full 32-row words, one sub-range)."""
    k, m = 8, 1 << 20
    g = torch.Generator().manual_seed(78)
    A = []
    for i in range(k):
        sparse = torch.randperm(m, generator=g)[:4000].sort().values
        dense = torch.arange(i * 5000, i * 5000 + 5000)  # rows [0, 40000) over the 8 inputs
        ri = torch.cat([sparse, dense]).to(torch.int32)
        cp = torch.tensor([0, 4000, 9000], dtype=torch.int32)
        A.append((cp, ri, synth.values(g, ri.numel(), F64, "int8", "cpu")))
    if order == "unordered":
        A = _shuffle_within_columns(A, 5)
    opt = spk.default_options(window_max=1024, block_accumulator=acc, input_order=1 if order == "unordered" else 0)
    info, _ = check_full(A, m, F64, exact=True, options=opt)
    assert info["cols_heavy"] == 2 and info["windows"] > 60, info


# ---------------------------------------------------------------------------
# fp32 with many terms per output entry: past 167 inputs the thread-block
# accumulators sum in float phases of 128 inputs (double past k = 4992), and
# warp columns always sum a row's run in double, so the 1e-5 * sum|terms| bar
# holds for any k.
# ---------------------------------------------------------------------------
def test_fp32_k300_every_class_within_bound():
    """k = 300 SpGEMM-like fp32 inputs (each row in about a quarter of the inputs): warp, CTA and heavy items."""
    A = synth.spgemm_like(300, 512, 120, 4, seed=12, dtype=F32)
    opt = spk.default_options(warp_max=256, cta_max=1024, window_max=1024)
    for method in ("twopass", "onepass"):
        cp, ri, va, info = run_gpu(A, 512, options=opt, info=True, method=method)
        compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), oracle.add(to_np(A)), F32)
    assert info["cols_cta"] + info["cols_heavy"] > 0


def test_fp32_many_terms_per_entry():
    """k = 1024 SpGEMM-like fp32 inputs of 8 rows per column drawn from 32 candidates: an output entry collects
    about 256 terms (well past 167, and past the k <= 512 of the served workload)."""
    A = synth.spgemm_like(1024, 1 << 12, 16, 8, seed=13, dtype=F32)
    want = oracle.add(to_np(A))
    assert want["terms"].max() > 167
    cp, ri, va = run_gpu(A, 1 << 12)
    compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), want, F32)
