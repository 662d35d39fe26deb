"""Pins for the CPU oracle (oracle/spk_oracle.c), all on CPU.

Each check ties the oracle to something other than itself:
  * a hand-computed example (tests/golden/fig1_handworked.json, Sec. II-A,
    shaped after the Fig. 1 caption);
  * dense brute-force addition on tiny inputs (the definition B = sum A_i,
    Sec. II-A) with the union-of-patterns rule for structure;
  * scipy's 2-matrix "+" for k = 2 (Sec. II-A names it as the k = 2 case);
  * exact rational sums (fractions.Fraction) for the value error bound;
  * invariants the paper states or implies: nnz(B) <= sum nnz(A_i) (Sec.
    II-A), k = 1 is the identity, input order does not matter, the sum of
    all values is preserved, disjoint inputs give single-term entries,
    cancellation keeps an explicit zero;
  * the Erdos-Renyi closed form E[nnz(B(:,j))] = m (1 - (1 - d/m)^k);
  * a global sort-and-merge of all (row, col, val) triples.
The last test builds deliberately broken copies of the oracle and checks that
these pins catch every one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _np_inputs(A):
    return [(a[0].numpy(), a[1].numpy(), a[2].numpy()) for a in A]


def _dense(a, m, n):
    cp, ri, va = a
    D = np.zeros((m, n), dtype=np.float64)
    P = np.zeros((m, n), dtype=bool)
    for j in range(n):
        for e in range(cp[j], cp[j + 1]):
            D[ri[e], j] += float(va[e])
            P[ri[e], j] = True
    return D, P


def brute_force(A, m, n):
    """Dense definition: pattern = OR of patterns, value = dense sum at those positions."""
    S = np.zeros((m, n), dtype=np.float64)
    P = np.zeros((m, n), dtype=bool)
    T = np.zeros((m, n), dtype=np.int32)
    for a in A:
        D, Q = _dense(a, m, n)
        S += D
        P |= Q
        T += Q
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    rows, vals, terms = [], [], []
    for j in range(n):
        r = np.nonzero(P[:, j])[0]
        rows.append(r)
        vals.append(S[r, j])
        terms.append(T[r, j])
        col_ptr[j + 1] = col_ptr[j] + len(r)
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return col_ptr, cat(rows, np.int32), cat(vals, np.float64), cat(terms, np.int32)


def check_against_brute_force(A, m, n, lib=None, exact=True):
    B = oracle.add(A, lib=lib)
    cp, r, v, t = brute_force(A, m, n)
    assert np.array_equal(B["col_ptr"], cp)
    assert np.array_equal(B["row_idx"], r)
    assert np.array_equal(B["terms"], t)
    if exact:
        assert np.array_equal(B["val"], v)
    else:
        np.testing.assert_allclose(B["val"], v, rtol=0, atol=1e-13 * max(1.0, float(np.abs(v).max(initial=0))))
    return B


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        G = json.load(f)
    A = [(np.array(x["col_ptr"], np.int32), np.array(x["row_idx"], np.int32), np.array(x["val"], np.float64))
         for x in G["inputs"]]
    return G, A


def check_golden(lib=None):
    G, A = load_golden("fig1_handworked.json")
    B = oracle.add(A, lib=lib)
    E = G["expected"]
    assert B["col_ptr"].tolist() == E["col_ptr"]
    assert B["row_idx"].tolist() == E["row_idx"]
    assert B["val"].tolist() == E["val"]
    assert B["abs_sum"].tolist() == E["abs_sum"]
    assert B["terms"].tolist() == E["terms"]
    assert not np.signbit(B["val"][-1])  # the cancelled entry is +0.0


def test_golden_fig1():
    check_golden()


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 17, 9), (5, 40, 23), (8, 64, 64), (2, 1, 30)])
def test_dense_brute_force_integers(seed, shape):
    k, m, n = shape
    A = _np_inputs(synth.random_csc(k, m, n, density=0.3, seed=seed, value_kind="int8",
                                    empty_matrix_frac=0.15))
    check_against_brute_force(A, m, n, exact=True)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("seed", range(4))
def test_dense_brute_force_floats(seed, dtype):
    A = _np_inputs(synth.random_csc(6, 48, 33, density=0.25, seed=100 + seed, dtype=dtype))
    check_against_brute_force(A, 48, 33, exact=False)


@pytest.mark.parametrize("seed", range(4))
def test_k2_equals_scipy_plus(seed):
    sp = pytest.importorskip("scipy.sparse")
    m, n = 37, 29
    A = _np_inputs(synth.random_csc(2, m, n, density=0.2, seed=seed, value_kind="int8"))
    S = [sp.csc_matrix((a[2], a[1], a[0]), shape=(m, n)) for a in A]
    want = (S[0] + S[1]).toarray()
    B = oracle.add(A)
    got = sp.csc_matrix((B["val"], B["row_idx"], B["col_ptr"]), shape=(m, n)).toarray()
    assert np.array_equal(got, want)


def test_value_error_within_bound_of_exact_sum():
    """Neumaier summation: |oracle - exact| <= 2 eps |exact| + 4 t eps^2 sum|terms|."""
    rng = np.random.default_rng(7)
    k, m, n = 12, 6, 40
    A = []
    for _ in range(k):
        cp = np.arange(n + 1, dtype=np.int32) * m
        ri = np.tile(np.arange(m, dtype=np.int32), n)
        va = rng.standard_normal(n * m) * 10.0 ** rng.integers(-8, 9, n * m)
        A.append((cp, ri, va))
    B = oracle.add(A)
    eps = 2.0 ** -53
    for j in range(n):
        for r in range(m):
            exact = sum((Fraction(float(a[2][j * m + r])) for a in A), Fraction(0))
            got = B["val"][B["col_ptr"][j] + r]
            bound = 2 * eps * abs(float(exact)) + 4 * k * eps * eps * float(B["abs_sum"][B["col_ptr"][j] + r])
            assert abs(Fraction(got) - exact) <= Fraction(bound) + Fraction(1, 10 ** 300)


def test_compensation_recovers_small_term():
    cp = np.array([0, 1], np.int32)
    ri = np.array([0], np.int32)
    A = [(cp, ri, np.array([v])) for v in (1e16, 1.0, -1e16)]
    assert oracle.add(A)["val"].tolist() == [1.0]


def test_k1_is_identity():
    A = _np_inputs(synth.random_csc(1, 50, 40, density=0.2, seed=3))
    B = oracle.add(A)
    assert np.array_equal(B["col_ptr"], A[0][0].astype(np.int64))
    assert np.array_equal(B["row_idx"], A[0][1])
    assert np.array_equal(B["val"], A[0][2])


@pytest.mark.parametrize("seed", range(3))
def test_permutation_invariance(seed):
    A = _np_inputs(synth.random_csc(7, 60, 30, density=0.3, seed=seed))
    B1 = oracle.add(A)
    perm = np.random.default_rng(seed).permutation(len(A))
    B2 = oracle.add([A[p] for p in perm])
    assert np.array_equal(B1["col_ptr"], B2["col_ptr"])
    assert np.array_equal(B1["row_idx"], B2["row_idx"])
    np.testing.assert_allclose(B1["val"], B2["val"], rtol=0, atol=1e-14)
    Ai = _np_inputs(synth.random_csc(7, 60, 30, density=0.3, seed=seed, value_kind="int8"))
    C1, C2 = oracle.add(Ai), oracle.add([Ai[p] for p in perm])
    assert np.array_equal(C1["val"], C2["val"])


def test_value_sum_preserved_and_nnz_bound():
    A = _np_inputs(synth.random_csc(9, 80, 70, density=0.2, seed=11, value_kind="int8"))
    B = oracle.add(A)
    assert B["val"].sum() == sum(float(a[2].sum()) for a in A)
    assert len(B["row_idx"]) <= sum(len(a[1]) for a in A)
    assert B["terms"].sum() == sum(len(a[1]) for a in A)


def test_pattern_is_union():
    m, n = 45, 38
    A = _np_inputs(synth.random_csc(5, m, n, density=0.2, seed=5))
    B = oracle.add(A)
    for j in range(n):
        want = set()
        for a in A:
            want |= set(a[1][a[0][j]:a[0][j + 1]].tolist())
        got = B["row_idx"][B["col_ptr"][j]:B["col_ptr"][j + 1]].tolist()
        assert got == sorted(want)


def test_disjoint_inputs_are_bit_exact():
    m, n, k = 64, 20, 4
    rng = np.random.default_rng(1)
    A = []
    for i in range(k):
        rows = np.arange(i, m, k, dtype=np.int32)  # input i owns rows = i mod k
        cp = np.arange(n + 1, dtype=np.int32) * len(rows)
        A.append((cp, np.tile(rows, n), rng.standard_normal(n * len(rows))))
    B = oracle.add(A)
    assert (B["terms"] == 1).all()
    for j in range(n):
        for i, a in enumerate(A):
            seg = slice(B["col_ptr"][j], B["col_ptr"][j + 1])
            sel = B["row_idx"][seg] % k == i
            assert np.array_equal(B["val"][seg][sel], a[2][a[0][j]:a[0][j + 1]])


def test_cancellation_keeps_explicit_positive_zero():
    A = _np_inputs(synth.random_csc(1, 30, 25, density=0.3, seed=2))
    neg = [(A[0][0], A[0][1], -A[0][2])]
    B = oracle.add(A + neg)
    assert len(B["row_idx"]) == len(A[0][1])
    assert (B["val"] == 0).all() and not np.signbit(B["val"]).any()


def test_er_union_size_closed_form():
    k, m, n, d = 4, 1024, 1024, 8
    A = _np_inputs(synth.er(k, m, n, d, seed=0, value_kind="int8"))
    u = oracle.union_sizes(A)
    expect = m * (1 - (1 - d / m) ** k)
    # per-column variance is below 1; the mean of n columns is within 0.1 with overwhelming probability
    assert abs(u.mean() - expect) < 0.1
    assert u.min() >= d and u.max() <= k * d


def test_global_triple_sort_and_merge_agrees():
    """Same result from one global lexsort of all (col, row) triples with reduceat."""
    k, m, n = 8, 3000, 2500
    A = _np_inputs(synth.random_csc(k, m, n, density=0.002, seed=9, value_kind="int8"))
    B = oracle.add(A)
    cols = np.concatenate([np.repeat(np.arange(n), np.diff(a[0])) for a in A])
    rows = np.concatenate([a[1] for a in A])
    vals = np.concatenate([a[2] for a in A]).astype(np.float64)
    o = np.lexsort((rows, cols))
    key = cols[o].astype(np.int64) * m + rows[o]
    starts = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
    sums = np.add.reduceat(vals[o], starts)
    assert np.array_equal(B["row_idx"], rows[o][starts])
    assert np.array_equal(B["val"], sums)
    assert np.array_equal(np.diff(B["col_ptr"]), np.bincount(cols[o][starts], minlength=n))


def test_union_sizes_and_listed_columns():
    A = _np_inputs(synth.random_csc(5, 90, 60, density=0.15, seed=4))
    full = oracle.add(A)
    u = oracle.union_sizes(A)
    assert np.array_equal(np.diff(full["col_ptr"]), u)
    cols = np.array([59, 0, 17, 17, 3])
    part = oracle.add(A, cols=cols)
    for q, j in enumerate(cols):
        a, b = full["col_ptr"][j], full["col_ptr"][j + 1]
        c, d = part["col_ptr"][q], part["col_ptr"][q + 1]
        assert np.array_equal(part["row_idx"][c:d], full["row_idx"][a:b])
        assert np.array_equal(part["val"][c:d], full["val"][a:b])


@pytest.mark.parametrize("groups", [[2, 3, 1], [1, 1, 1, 1, 1, 1], [6]])
def test_sum_taken_batch_by_batch_equals_one_shot(groups):
    """Streaming reading (Sec. V: inputs added batch by batch): feeding each
    partial sum back as an input gives the one-shot sum -- the same pattern
    (a union of unions is the union) and, for small integers, the same values
    exactly (integer sums are exact in any grouping)."""
    A = _np_inputs(synth.random_csc(6, 40, 25, density=0.25, seed=9, value_kind="int8"))
    want = oracle.add(A)
    run = None
    i = 0
    for g in groups:
        batch = A[i:i + g]
        i += g
        if run is not None:
            batch = [(run["col_ptr"].astype(np.int32), run["row_idx"], run["val"])] + batch
        run = oracle.add(batch)
    assert np.array_equal(run["col_ptr"], want["col_ptr"])
    assert np.array_equal(run["row_idx"], want["row_idx"])
    assert np.array_equal(run["val"], want["val"])
    cp, r, v, _ = brute_force(A, 40, 25)
    assert np.array_equal(run["row_idx"], r) and np.array_equal(run["val"], v)


def test_unordered_columns_and_repeats_inside_one_input():
    """Table I: the hash method needs no sorted input.  Permuting the entries
    inside every input column leaves the sum unchanged, and a row repeated
    inside one input column is summed like any other term (dense brute force,
    which adds every entry)."""
    rng = np.random.default_rng(21)
    A = _np_inputs(synth.random_csc(4, 30, 12, density=0.3, seed=21, value_kind="int8"))
    want = oracle.add(A)
    shuffled = []
    for cp, ri, va in A:
        ri2, va2 = ri.copy(), va.copy()
        for j in range(len(cp) - 1):
            perm = rng.permutation(cp[j + 1] - cp[j]) + cp[j]
            ri2[cp[j]:cp[j + 1]], va2[cp[j]:cp[j + 1]] = ri[perm], va[perm]
        shuffled.append((cp, ri2, va2))
    got = oracle.add(shuffled)
    for key in ("col_ptr", "row_idx", "val"):
        assert np.array_equal(got[key], want[key])
    # one input column holding row 5 three times and row 2 once, next to another input
    rep = [(np.array([0, 4], np.int32), np.array([5, 2, 5, 5], np.int32), np.array([1.0, 2.0, 4.0, 8.0])),
           (np.array([0, 2], np.int32), np.array([5, 7], np.int32), np.array([16.0, 32.0]))]
    B = oracle.add(rep)
    cp, r, v, _ = brute_force(rep, 10, 1)
    assert np.array_equal(B["row_idx"], r) and B["row_idx"].tolist() == [2, 5, 7]
    assert np.array_equal(B["val"], v) and B["val"].tolist() == [2.0, 29.0, 32.0]


def test_output_columns_sorted_strictly():
    A = _np_inputs(synth.rmat(6, 8, 8, seed=1))
    B = oracle.add(A)
    for j in range(len(B["col_ptr"]) - 1):
        seg = B["row_idx"][B["col_ptr"][j]:B["col_ptr"][j + 1]]
        assert (np.diff(seg) > 0).all()


def _pins_pass(lib):
    try:
        check_golden(lib)
        for seed in range(3):
            A = _np_inputs(synth.random_csc(4, 20, 15, density=0.3, seed=seed, value_kind="int8"))
            check_against_brute_force(A, 20, 15, lib=lib, exact=True)
        A = _np_inputs(synth.random_csc(1, 30, 25, density=0.3, seed=2))
        B = oracle.add(A + [(A[0][0], A[0][1], -A[0][2])], lib=lib)
        assert len(B["row_idx"]) == len(A[0][1])
    except (AssertionError, RuntimeError):
        return False
    return True


def test_pins_pass_on_the_oracle():
    assert _pins_pass(oracle.load())


@pytest.mark.parametrize("plant", oracle.PLANTS)
def test_pins_catch_planted_mistakes(plant):
    lib = oracle.load(oracle.build(plant=plant))
    assert not _pins_pass(lib), f"pins missed planted mistake {plant}"
