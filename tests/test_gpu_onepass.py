"""The one-pass path (spkadd_onepass: symbolic count, look-back scan and numeric
sum in one kernel) against the CPU oracle, element by element, through the C
ABI; the same cases through the two-pass path (spkadd_symbolic +
spkadd_numeric) for comparison; its fallback, argument checks and bounded
waits.

Bar: col_ptr and row_idx bit-exact; values bit-exact for small-integer fp64
inputs, otherwise |gpu - oracle| <= 1e-12 * sum|terms| (fp64) or
1e-5 * sum|terms| (fp32) per entry.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2112_10223_gb300 as spk
import synth
from spk_testlib import compare, to_np

pytestmark = pytest.mark.gpu

F64, F32 = torch.float64, torch.float32
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    spk.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(A, m, method, options=None, dtype=None):
    Ad = synth.to_device(A, torch.device(DEV))
    cp, ri, va, info = spk.spkadd(Ad, m, dtype=dtype, options=options, info=True, method=method)
    torch.cuda.synchronize()
    return (cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), info


def check(A, m, dtype, exact=False, options=None, expect_onepass=True):
    want = oracle.add(to_np(A))
    got1, info1 = run(A, m, "onepass", options)
    assert info1["onepass"] == (1 if expect_onepass else 0), info1
    compare(got1, want, dtype, exact=exact)
    got2, info2 = run(A, m, "twopass", options)
    assert info2["onepass"] == 0
    compare(got2, want, dtype, exact=exact)
    return info1


def test_config1_er_k4_1024_bit_exact():
    """k = 4 ER 1024 x 1024, 8 distinct rows per column, fp64 integers in [-8, 8] \\ {0}, seed 0."""
    A = synth.er(4, 1024, 1024, 8, seed=0, dtype=F64, value_kind="int8")
    info = check(A, 1024, F64, exact=True)
    u = oracle.union_sizes(to_np(A))
    s = sum((a[0][1:] - a[0][:-1]).numpy() for a in A)
    assert info["cols_unique"] == int((u == s).sum())


@pytest.mark.parametrize("k", [1, 2, 5, 16, 31, 32])
@pytest.mark.parametrize("dtype", [F64, F32])
def test_er_many_k(k, dtype):
    """Equal-length segments (the one-multiply position map), n not a multiple of the tile width."""
    d = max(1, 512 // (k * 2))
    A = synth.er(k, 1 << 14, 1003, d, seed=k, dtype=dtype)
    check(A, 1 << 14, dtype)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("dtype", [F64, F32])
def test_irregular_ragged(seed, dtype):
    """Ragged segments, empty columns and empty matrices (the shuffle search path)."""
    A = synth.random_csc(7, 300, 257, density=0.05, seed=seed, dtype=dtype, empty_matrix_frac=0.1)
    check(A, 300, dtype)


def test_full_light_columns_and_repeats():
    """s_j = 512 exactly, every input identical (each row repeated k times: cf = k)."""
    one = synth.er(1, 4096, 777, 16, seed=3, dtype=F64, value_kind="int8")[0]
    A = [tuple(t.clone() for t in one) for _ in range(32)]
    info = check(A, 4096, F64, exact=True)
    assert info["cols_unique"] == 0


def test_heavy_overlap_spgemm_like():
    """SpGEMM-partial-product-like columns: rows drawn from a shared candidate set (many repeats)."""
    A = synth.spgemm_like(24, 1 << 12, 3000, 16, seed=5, dtype=F32)
    check(A, 1 << 12, F32)


@pytest.mark.parametrize("m", [1, 2, 63, 64, 65, (1 << 31) - 2])
def test_row_extremes(m):
    """Tiny m (buckets wider than the row range), and rows next to 2^31."""
    rng = np.random.default_rng(m % 1000)
    n, k = 100, 6
    A = []
    for i in range(k):
        cps, rows = [0], []
        for j in range(n):
            c = int(rng.integers(0, min(m, 40) + 1))
            r = np.sort(rng.choice(min(m, 1 << 20), size=c, replace=False)) + (m - min(m, 1 << 20))
            rows.append(r)
            cps.append(cps[-1] + c)
        ri = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
        va = rng.integers(-8, 9, size=ri.size).astype(np.float64)
        A.append((torch.tensor(cps, dtype=torch.int32), torch.from_numpy(ri), torch.from_numpy(va)))
    check(A, m, F64, exact=True)


def test_many_tiles_lookback_chain():
    """2^17 columns: 16384 tiles, so each tile's offset comes from a long look-back chain."""
    A = synth.er(8, 1 << 18, 1 << 17, 8, seed=9, dtype=F64, value_kind="int8")
    check(A, 1 << 18, F64, exact=True)


def test_single_column_and_single_entry():
    A = [(torch.tensor([0, 1], dtype=torch.int32), torch.tensor([5], dtype=torch.int32),
          torch.tensor([2.0], dtype=F64))]
    check(A, 10, F64, exact=True)
    A2 = [(torch.tensor([0, 0], dtype=torch.int32), torch.zeros(0, dtype=torch.int32), torch.zeros(0, dtype=F64))
          for _ in range(3)]
    got, info = run(A2, 10, "onepass")
    assert list(got[0]) == [0, 0] and got[1].size == 0


def test_force_dedup_and_unordered_inputs():
    """sort_mode 1 (always the duplicate-merging write) and rows in any order inside input columns."""
    A = synth.er(12, 2048, 600, 20, seed=4, dtype=F64, value_kind="int8")
    check(A, 2048, F64, exact=True, options=spk.default_options(sort_mode=1))
    rng = np.random.default_rng(0)
    U = []
    for cp, ri, va in A:
        ri2, va2 = ri.clone(), va.clone()
        cpn = cp.numpy()
        for j in range(cpn.size - 1):
            p = rng.permutation(cpn[j + 1] - cpn[j]) + cpn[j]
            ri2[cpn[j]:cpn[j + 1]] = ri[p]
            va2[cpn[j]:cpn[j + 1]] = va[p]
        U.append((cp, ri2, va2))
    check(U, 2048, F64, exact=True, options=spk.default_options(input_order=1))


def test_many_inputs_and_fallback():
    """k > 32 (chunks of 32 inputs) runs one pass; columns above warp_max take the two-pass kernels (onepass = 0)."""
    A = synth.er(40, 4096, 300, 4, seed=2, dtype=F64, value_kind="int8")
    check(A, 4096, F64, exact=True)
    B = synth.er(300, 1 << 14, 200, 1, seed=3, dtype=F32)
    check(B, 1 << 14, F32)
    R = synth.rmat(8, 12, 16, seed=1, dtype=F64, value_kind="int8")
    check(R, 1 << 12, F64, exact=True, expect_onepass=False)


def test_capacity_and_output_checks():
    A = synth.to_device(synth.er(4, 1024, 64, 8, seed=0, dtype=F64), torch.device(DEV))
    h = spk.spkadd_plan(A, 1024)
    cp = torch.empty(65, dtype=torch.int64, device=DEV)
    small = sum(a[1].numel() for a in A) - 1
    with pytest.raises(spk.SpkaddError) as e:
        spk.spkadd_onepass(h, cp, torch.empty(small, dtype=torch.int32, device=DEV),
                           torch.empty(small, dtype=F64, device=DEV))
    assert e.value.status == 1
    big = small + 1
    with pytest.raises(TypeError):  # a strided view would be written past its storage
        spk.spkadd_onepass(h, torch.zeros(1, dtype=torch.int64, device=DEV).expand(65),
                           torch.empty(big, dtype=torch.int32, device=DEV), torch.empty(big, dtype=F64, device=DEV))
    with pytest.raises(TypeError):  # host memory handed to a kernel
        spk.spkadd_onepass(h, torch.empty(65, dtype=torch.int64), torch.empty(big, dtype=torch.int32, device=DEV),
                           torch.empty(big, dtype=F64, device=DEV))
    nnz = spk.spkadd_onepass(h, cp, torch.empty(big, dtype=torch.int32, device=DEV),
                             torch.empty(big, dtype=F64, device=DEV))
    assert nnz == int(cp[-1].item())
    spk.spkadd_destroy(h)


def test_row_out_of_range_is_reported():
    A = synth.er(4, 1024, 64, 8, seed=0, dtype=F64)
    A[2][1][17] = 5000  # a row outside [0, m)
    Ad = synth.to_device(A, torch.device(DEV))
    with pytest.raises(spk.SpkaddError) as e:
        spk.spkadd(Ad, 1024, method="onepass")
    assert e.value.status == 4


def test_bounded_wait_returns_timeout_and_the_device_stays_usable():
    """The tile producer never fills a stage: the consumers' bounded wait runs out, the call returns
    SPKADD_ERR_TIMEOUT (nothing hangs or traps), and the next call on the device succeeds."""
    A = synth.er(4, 1024, 256, 8, seed=0, dtype=F64, value_kind="int8")
    Ad = synth.to_device(A, torch.device(DEV))
    with pytest.raises(spk.SpkaddError) as e:
        spk.spkadd(Ad, 1024, method="onepass", options=spk.default_options(test_stall=1, wait_timeout_ms=20))
    assert e.value.status == 8
    torch.cuda.synchronize()
    want = oracle.add(to_np(A))
    got, info = run(A, 1024, "onepass")
    assert info["onepass"] == 1
    compare(got, want, F64, exact=True)


def test_repeat_calls_same_handle():
    """spkadd_onepass twice on one handle, then spkadd_numeric's path on a fresh one: identical B."""
    A = synth.to_device(synth.er(16, 1 << 16, 5000, 16, seed=7, dtype=F32), torch.device(DEV))
    cap = sum(a[1].numel() for a in A)
    h = spk.spkadd_plan(A, 1 << 16)
    outs = []
    for _ in range(2):
        cp = torch.empty(5001, dtype=torch.int64, device=DEV)
        ri = torch.empty(cap, dtype=torch.int32, device=DEV)
        va = torch.empty(cap, dtype=F32, device=DEV)
        nnz = spk.spkadd_onepass(h, cp, ri, va)
        outs.append((cp, ri[:nnz], va[:nnz]))
    spk.spkadd_destroy(h)
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    two = spk.spkadd(A, 1 << 16, method="twopass")
    assert torch.equal(outs[0][0], two[0]) and torch.equal(outs[0][1], two[1])
    assert torch.allclose(outs[0][2], two[2], rtol=0, atol=1e-5 * 16)
