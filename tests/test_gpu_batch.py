"""Parity of the batched CUDA path (spkadd_batch_*) against the CPU oracle.

A batch runs many independent problems -- each with its own k, shape and
dtype -- through one set of launches.  Every problem's result must meet the
single-problem bar: col_ptr and row_idx bit-exact, values bit-exact for
small-integer inputs and otherwise within 1e-12 (fp64) / 1e-5 (fp32) of
sum|terms| per entry.
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


def _check_batch(problems_cpu, options=None, exact=()):
    """Run the batch on the GPU; compare every problem with the oracle."""
    problems = [(_dev(A), m) for A, m in problems_cpu]
    outs, info = spk.spkadd_batch(problems, options=options, info=True)
    torch.cuda.synchronize()
    for q, ((A, m), (cp, ri, va)) in enumerate(zip(problems_cpu, outs)):
        want = oracle.add(to_np(A))
        dtype = A[0][2].dtype
        try:
            compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), want, dtype, exact=q in exact)
        except AssertionError as e:
            raise AssertionError(f"problem {q}: {e}") from None
    return outs, info


def test_mixed_batch_of_instances():
    """24 instances drawn like the batched workload (ER and SpGEMM-like, mixed dtypes), small sizes."""
    params = synth.batch_instance_params(24, seed=0, k_range=(2, 40), mn_range=(256, 4096), L_range=(4, 64))
    problems = [synth.instance(p) for p in params]
    assert len({p["dtype"] for p in params}) == 2 and len({p["family"] for p in params}) == 2
    _, info = _check_batch(problems)
    assert info["problems"] == 24
    assert info["k"] == sum(p["k"] for p in params)
    assert info["n"] == sum(p["m"] for p in params)


@pytest.mark.parametrize("dtype", [F64, F32])
def test_batch_with_every_class_and_degenerate_problems(dtype):
    """Warp, CTA and heavy (split-window) columns, plus empty problems, in one batch of one dtype."""
    problems = [
        (synth.rmat(12, 12, 16, seed=5, dtype=dtype), 1 << 12),
        (synth.random_csc(5, 300, 120, density=0.06, seed=6, dtype=dtype, empty_matrix_frac=0.2), 300),
        (synth.er(3, 50, 0, 0, seed=7, dtype=dtype), 50),                   # n = 0
        (synth.random_csc(2, 40, 30, density=0.0, seed=8, dtype=dtype), 40),  # all columns empty
        (synth.er(40, 6000, 9, 100, seed=9, dtype=dtype), 6000),             # s_j = 4000: CTA class
        (synth.er(1, 1, 1, 1, seed=10, dtype=dtype), 1),                     # 1 x 1
    ]
    opt = spk.default_options(window_max=1024)
    _, info = _check_batch(problems, options=opt)
    assert info["cols_warp"] > 0 and info["cols_cta"] > 0 and info["cols_heavy"] > 0, info
    assert info["windows"] > info["cols_cta"] + info["cols_heavy"], info  # some heavy columns cut into windows


def test_mixed_dtypes_with_forced_classes():
    """Mixed fp32/fp64 problems whose columns land in all three classes (small thresholds)."""
    problems = []
    for q in range(10):
        dtype = F64 if q % 2 else F32
        problems.append((synth.random_csc(3 + q, 400 + 37 * q, 90 + q, density=0.1, seed=20 + q, dtype=dtype), 400 + 37 * q))
    problems.append((synth.rmat(8, 11, 16, seed=31, dtype=F64), 1 << 11))
    problems.append((synth.rmat(8, 11, 16, seed=32, dtype=F32), 1 << 11))
    opt = spk.default_options(warp_max=64, cta_max=128, window_max=1024)
    _, info = _check_batch(problems, options=opt)
    assert info["cols_warp"] > 0 and info["cols_cta"] > 0 and info["cols_heavy"] > 0, info


def test_small_integer_batch_bit_exact():
    """fp64 small-integer inputs: every problem bit-exact (sums are exact in any order)."""
    problems = [(synth.er(2 + q, 512 + 64 * q, 200 + q, 8 + q, seed=40 + q, dtype=F64, value_kind="int8"), 512 + 64 * q)
                for q in range(12)]
    _check_batch(problems, exact=set(range(12)))


def test_batch_matches_single_problem_calls():
    """Indices of a batch equal those of one spkadd call per problem; values agree within tolerance."""
    params = synth.batch_instance_params(6, seed=3, k_range=(2, 20), mn_range=(512, 2048), L_range=(4, 64))
    problems = [(_dev(A), m) for A, m in (synth.instance(p) for p in params)]
    outs = spk.spkadd_batch(problems)
    for (A, m), (cp, ri, va) in zip(problems, outs):
        cp1, ri1, va1 = spk.spkadd(A, m)
        assert torch.equal(cp, cp1) and torch.equal(ri, ri1)
        tol = 1e-12 if va.dtype == F64 else 1e-5
        scale = sum(a[2].abs().to(F64).sum() for a in A)
        assert float((va.to(F64) - va1.to(F64)).abs().max()) <= tol * float(scale)


def test_batch_of_one_equals_spkadd():
    A = synth.er(5, 3000, 700, 20, seed=50, dtype=F64, value_kind="int8")
    Ad = _dev(A)
    (cp, ri, va), = spk.spkadd_batch([(Ad, 3000)])
    cp1, ri1, va1 = spk.spkadd(Ad, 3000)
    assert torch.equal(cp, cp1) and torch.equal(ri, ri1) and torch.equal(va, va1)


def test_batch_numeric_twice_and_nnz_per_problem():
    """nnz per problem from the batch symbolic pass; numeric may run again into fresh buffers."""
    problems_cpu = [(synth.er(3, 800, 100 + q, 12, seed=60 + q, dtype=F32), 800) for q in range(5)]
    problems = [(_dev(A), m) for A, m in problems_cpu]
    h = spk.spkadd_batch_plan(problems)
    try:
        nnz = spk.spkadd_batch_symbolic(h)
        want = [oracle.add(to_np(A)) for A, _ in problems_cpu]
        assert nnz == [int(w["col_ptr"][-1]) for w in want]
        for _ in range(2):
            outs = [(torch.empty(h.n[q] + 1, dtype=torch.int64, device=DEV),
                     torch.full((nnz[q],), -7, dtype=torch.int32, device=DEV),
                     torch.empty(nnz[q], dtype=F32, device=DEV)) for q in range(5)]
            spk.spkadd_batch_numeric(h, outs)
            torch.cuda.synchronize()
            for (cp, ri, va), w in zip(outs, want):
                compare((cp.cpu().numpy(), ri.cpu().numpy(), va.cpu().numpy()), w, F32)
    finally:
        spk.spkadd_destroy(h)


def test_batch_state_and_argument_errors():
    problems = [(_dev(synth.er(2, 100, 10, 3, seed=70, dtype=F64)), 100)]
    h = spk.spkadd_batch_plan(problems)
    try:
        outs = [(torch.empty(11, dtype=torch.int64, device=DEV), torch.empty(30, dtype=torch.int32, device=DEV),
                 torch.empty(30, dtype=F64, device=DEV))]
        with pytest.raises(spk.SpkaddError) as e:
            spk.spkadd_batch_numeric(h, outs)
        assert e.value.name == "SPKADD_ERR_STATE"
        with pytest.raises(spk.SpkaddError) as e:  # single-problem calls reject a batch handle
            spk.spkadd_symbolic(h)
        assert e.value.name == "SPKADD_ERR_INVALID_ARG"
    finally:
        spk.spkadd_destroy(h)


def test_validate_reports_a_bad_problem_in_a_batch():
    good = synth.er(2, 100, 10, 3, seed=71, dtype=F64)
    bad = synth.er(2, 100, 10, 3, seed=72, dtype=F64)
    ri = bad[1][1].clone()
    ri[4] = 100  # row outside [0, m)
    bad[1] = (bad[1][0], ri, bad[1][2])
    with pytest.raises(spk.SpkaddError) as e:
        spk.spkadd_batch([(_dev(good), 100), (_dev(bad), 100)], options=spk.default_options(validate=1))
    assert e.value.name == "SPKADD_ERR_INDEX_RANGE"


def test_batch_launch_count_does_not_grow_with_problems():
    """The launch count of a batch is a constant: it does not depend on the number of problems."""
    counts = []
    for count in (4, 64):
        problems = [(_dev(synth.er(3, 256, 64, 8, seed=80 + q, dtype=F32)), 256) for q in range(count)]
        _, info = spk.spkadd_batch(problems, info=True)
        counts.append(info["kernel_launches"])
    assert counts[0] == counts[1], counts
    assert counts[0] <= 12, counts


def test_autotuned_options_give_the_same_batch(tmp_path):
    """The library's autotuner times candidate options on a batch, caches its choice, and the chosen options
    give the oracle's result."""
    from paper_2112_10223_gb300 import autotune

    params = synth.batch_instance_params(12, seed=3, k_range=(2, 64), mn_range=(256, 2048), L_range=(4, 64))
    problems_cpu = [synth.instance(p) for p in params]
    problems = [(_dev(A), m) for A, m in problems_cpu]
    ks, ms, ns, nnz, cps, ris, vas, dts = [], [], [], [], [], [], [], []
    for A, m in problems:
        ks.append(len(A))
        ms.append(m)
        ns.append(A[0][0].numel() - 1)
        dts.append(A[0][2].dtype)
        for cp, ri, va in A:
            nnz.append(ri.numel())
            cps.append(cp.data_ptr())
            ris.append(ri.data_ptr() if ri.numel() else 0)
            vas.append(va.data_ptr() if va.numel() else 0)
    desc = dict(k=np.asarray(ks, dtype=np.int32), m=np.asarray(ms), n=np.asarray(ns), nnz=np.asarray(nnz),
                cp=np.asarray(cps, dtype=np.uint64), ri=np.asarray(ris, dtype=np.uint64),
                va=np.asarray(vas, dtype=np.uint64), dtypes=dts)
    tuner = autotune.Autotuner(cache_path=str(tmp_path / "tune.json"))
    opt = autotune.tune_batch(desc, device=DEV, tuner=tuner, repeats=1)
    assert not tuner.last["cached"] and tuner.last["timed"] > 1
    again = autotune.tune_batch(desc, device=DEV, tuner=autotune.Autotuner(cache_path=str(tmp_path / "tune.json")))
    assert all(getattr(opt, f) == getattr(again, f) for f in autotune.DEFAULTS)
    _check_batch(problems_cpu, options=opt)


def test_float_sums_in_phases_and_in_double_in_one_batch():
    """One batch holding fp32 problems with k <= 167 (float sums), 167 < k <= 4992 (float sums in phases of
    128 inputs, including a ragged last phase) and k > 4992 (double sums), plus an fp64 problem: four launches
    of the thread-block kernels, one per kind, each problem within the fp32 bound of 1e-5 * sum|terms| per
    entry."""
    problems = [
        (synth.spgemm_like(40, 512, 24, 16, seed=90, dtype=F32), 512),     # float, one phase
        (synth.spgemm_like(168, 512, 24, 16, seed=91, dtype=F32), 512),    # two phases: 128 + 40
        (synth.spgemm_like(300, 256, 20, 8, seed=92, dtype=F32), 256),     # three phases, the last 44 inputs
        (synth.spgemm_like(6920, 64, 3, 1, seed=93, dtype=F32), 64),       # double accumulators
        (synth.spgemm_like(200, 512, 24, 16, seed=94, dtype=F64), 512),
    ]
    opt = spk.default_options(warp_max=128, cta_max=1024, window_max=1024)
    outs, info = _check_batch(problems, options=opt)
    assert info["cols_cta"] + info["cols_heavy"] > 0, info
    for (A, m) in problems[1:4]:
        assert oracle.add(to_np(A))["terms"].max() > 48  # entries collect many terms, from several phases
