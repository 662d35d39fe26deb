"""Parity of streaming accumulation (spkadd_stream_*) against the CPU oracle.

A stream adds batches of inputs into a running sum B kept on the device (each
add is one (k+1)-way SpKAdd with B as input 0).  After any sequence of adds B
must equal the oracle's sum of every input added: col_ptr and row_idx
bit-exact, values bit-exact for small-integer fp64 inputs, otherwise within
1e-12 (fp64) / 1e-5 (fp32) of sum|terms| per entry (each addition of a
streamed sum rounds once, as in a one-shot sum, so the bound is the same).
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


def _dev(A):
    return [tuple(t.to(DEV) for t in a) for a in A]


def _stream(A, m, groups, dtype, options=None):
    s = spk.SpkaddStream(m, A[0][0].numel() - 1, dtype=dtype, options=options)
    i = 0
    for g in groups:
        s.add(_dev(A[i:i + g]))
        i += g
    assert i == len(A)
    out = s.result()
    torch.cuda.synchronize()
    info = s.query()
    s.close()
    return tuple(t.cpu().numpy() for t in out), info


@pytest.mark.parametrize("groups", [[24], [5, 1, 8, 10], [1] * 24])
def test_stream_groups_equal_oracle_exact(groups):
    """SpGEMM-like partial products (overlapping patterns), fp64 integers: any grouping is bit-exact."""
    A = synth.spgemm_like(24, 3000, 400, 20, seed=11, dtype=F64, value_kind="int8")
    got, info = _stream(A, 3000, groups, F64)
    compare(got, oracle.add(to_np(A)), F64, exact=True)
    assert info["adds"] == len(groups)


@pytest.mark.parametrize("dtype", [F32, F64])
def test_stream_all_classes_rmat(dtype):
    """R-MAT scale 12 in four batches with small class limits: warp, CTA and heavy columns every add."""
    A = synth.rmat(16, 12, 16, seed=12, dtype=dtype)
    opt = spk.default_options(warp_max=64, cta_max=256, window_max=1024)
    got, _ = _stream(A, 1 << 12, [4, 4, 4, 4], dtype, options=opt)
    compare(got, oracle.add(to_np(A)), dtype)


def test_stream_matches_one_shot_indices():
    A = synth.er(12, 20000, 3000, 40, seed=13, dtype=F32)
    got, _ = _stream(A, 20000, [3, 3, 3, 3], F32)
    cp, ri, va = spk.spkadd(_dev(A), 20000)
    assert np.array_equal(got[0], cp.cpu().numpy()) and np.array_equal(got[1], ri.cpu().numpy())
    compare(got, oracle.add(to_np(A)), F32)


def test_stream_unordered_inputs():
    g = torch.Generator().manual_seed(14)
    A = synth.random_csc(9, 500, 200, density=0.08, seed=14, dtype=F64, value_kind="int8")
    out = []
    for cp, ri, va in A:  # shuffle (row, value) pairs inside every column
        cpl = cp.to(torch.int64)
        col = torch.repeat_interleave(torch.arange(cp.numel() - 1), cpl[1:] - cpl[:-1])
        perm = torch.argsort(col.to(torch.float64) + torch.rand(ri.numel(), generator=g, dtype=torch.float64) * 0.5)
        out.append((cp, ri[perm], va[perm]))
    opt = spk.default_options(warp_max=250, cta_max=320, input_order=1)
    got, _ = _stream(out, 500, [2, 3, 4], F64, options=opt)
    compare(got, oracle.add(to_np(A)), F64, exact=True)


def test_stream_empty_before_any_add_and_empty_inputs():
    s = spk.SpkaddStream(50, 7, dtype=F64)
    cp, ri, va = s.result()
    torch.cuda.synchronize()
    assert cp.cpu().tolist() == [0] * 8 and ri.numel() == 0 and va.numel() == 0
    empty = [(torch.zeros(8, dtype=torch.int32), torch.zeros(0, dtype=torch.int32), torch.zeros(0, dtype=F64))] * 2
    assert s.add(_dev(empty)) == 0
    A = synth.random_csc(3, 50, 7, density=0.2, seed=15, dtype=F64, value_kind="int8")
    s.add(_dev(A))
    got = tuple(t.cpu().numpy() for t in s.result())
    s.close()
    compare(got, oracle.add(to_np(A)), F64, exact=True)


def test_stream_errors_leave_the_sum_unchanged():
    A = synth.random_csc(4, 60, 9, density=0.2, seed=16, dtype=F64, value_kind="int8")
    s = spk.SpkaddStream(60, 9, dtype=F64)
    s.add(_dev(A[:2]))
    before = tuple(t.cpu().numpy() for t in s.result())
    wrong = synth.random_csc(1, 60, 10, density=0.2, seed=17, dtype=F64)  # n = 10, not 9
    with pytest.raises(spk.SpkaddError) as e:
        s.add(_dev(wrong))
    assert e.value.name == "SPKADD_ERR_SHAPE_MISMATCH"
    after = tuple(t.cpu().numpy() for t in s.result())
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    s.add(_dev(A[2:]))
    got = tuple(t.cpu().numpy() for t in s.result())
    s.close()
    compare(got, oracle.add(to_np(A)), F64, exact=True)


def test_stream_user_allocator_holds_the_sum_and_releases_everything():
    """With options.alloc / free, the running sum and every add's workspace come
    from the caller's allocator; after close every allocation is returned, and
    a failing allocator leaves the sum unchanged."""
    A = synth.random_csc(6, 200, 40, density=0.1, seed=18, dtype=F64, value_kind="int8")
    live, count, failing = {}, [0], [False]

    @spk.ALLOC_FN
    def alloc(nbytes, stream, ctx):
        if failing[0]:
            return None
        t = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
        live[t.data_ptr()] = t
        count[0] += 1
        return t.data_ptr()

    @spk.FREE_FN
    def free(ptr, stream, ctx):
        live.pop(ptr, None)

    o = spk.default_options()
    o.alloc, o.free = alloc, free
    s = spk.SpkaddStream(200, 40, dtype=F64, options=o)
    s.add(_dev(A[:3]))
    before = tuple(t.cpu().numpy() for t in s.result())
    failing[0] = True
    with pytest.raises(spk.SpkaddError) as e:
        s.add(_dev(A[3:]))
    assert e.value.name == "SPKADD_ERR_NOMEM"
    failing[0] = False
    assert all(np.array_equal(x, y) for x, y in zip(before, (t.cpu().numpy() for t in s.result())))
    s.add(_dev(A[3:]))
    got = tuple(t.cpu().numpy() for t in s.result())
    torch.cuda.synchronize()
    assert len(live) == 3 and count[0] > 3  # the sum's col_ptr, rows and values remain
    s.close()
    torch.cuda.synchronize()
    assert len(live) == 0
    compare(got, oracle.add(to_np(A)), F64, exact=True)
