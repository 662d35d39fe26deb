"""The allocation-free column-pointer scan (spkadd_scan_counts_noalloc).

Some callers cannot allocate device memory during a call: serving runtimes
that give the GPU's whole memory to their own arena up front, and
latency-critical code that cannot take cudaMalloc's implicit device-wide
synchronisation.  For them the library offers this one entry point, which
keeps its scratch in a fixed array inside the library.  These tests call it
through the C ABI and check that it gives exactly the column pointers the
ordinary path (spkadd_plan / spkadd_symbolic / spkadd_numeric) produces, on
two calls in a row (the scratch array keeps the previous call's contents).
The file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import pytest
import torch

import paper_2112_10223_gb300 as spk
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    spk.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("shape", [(6, 700, 300), (3, 5000, 20000)])
def test_noalloc_scan_matches_spkadd_col_ptr_twice(shape):
    k, m, n = shape
    A = synth.to_device(synth.random_csc(k, m, n, density=0.01, seed=n, dtype=torch.float64), "cuda")
    col_ptr, _, _ = spk.spkadd(A, m)
    counts = (col_ptr[1:] - col_ptr[:-1]).to(torch.int32)
    for _ in range(2):
        out = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
        spk.spkadd_scan_counts_noalloc(counts, out)
        torch.cuda.synchronize()
        assert torch.equal(out, col_ptr)


def test_noalloc_scan_many_tiles_twice():
    n = 3 * 4096 * 17 + 5
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    counts = torch.randint(0, 1000, (n,), generator=g, device="cuda", dtype=torch.int32)
    want = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    want[1:] = torch.cumsum(counts.to(torch.int64), 0)
    for _ in range(2):
        out = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        spk.spkadd_scan_counts_noalloc(counts, out)
        torch.cuda.synchronize()
        assert torch.equal(out, want)


def test_noalloc_scan_rejects_too_many_columns():
    counts = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    lib = spk.library()
    st = lib.spkadd_scan_counts_noalloc(counts.data_ptr(), spk.SCAN_NOALLOC_MAX_N + 1, out.data_ptr(), None)
    assert st == 10  # SPKADD_ERR_UNSUPPORTED, nothing launched
    assert lib.spkadd_scan_counts_noalloc(counts.data_ptr(), -1, out.data_ptr(), None) == 1


def test_noalloc_scan_at_the_size_limit_and_empty():
    """n = SPKADD_SCAN_NOALLOC_MAX_N fills every tile slot of the scratch array (the last holds the total);
    n = 0 writes the single column pointer 0."""
    n = spk.SCAN_NOALLOC_MAX_N
    g = torch.Generator(device="cuda")
    g.manual_seed(2)
    counts = torch.randint(0, 64, (n,), generator=g, device="cuda", dtype=torch.int32)
    want = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    want[1:] = torch.cumsum(counts.to(torch.int64), 0)
    for _ in range(2):
        out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
        spk.spkadd_scan_counts_noalloc(counts, out)
        torch.cuda.synchronize()
        assert torch.equal(out, want)
    del counts, want, out
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    one = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    spk.spkadd_scan_counts_noalloc(empty, one)
    torch.cuda.synchronize()
    assert int(one.item()) == 0


def test_noalloc_scan_takes_no_device_memory_after_the_first_call():
    """After a first call on the device, a further call leaves the device's free memory unchanged."""
    n = 4096 * 40 + 3
    counts = torch.ones(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    spk.spkadd_scan_counts_noalloc(counts, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    spk.spkadd_scan_counts_noalloc(counts, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert int(out[-1].item()) == n
