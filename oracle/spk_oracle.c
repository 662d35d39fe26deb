/*
 * spk_oracle.c -- CPU oracle for SpKAdd.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and
 * its reference arm) may build, load or call this file.  The GPU library
 * shares no code with it and never links it.
 *
 * What it computes (Sec. II-A of the paper): B = A_1 + ... + A_k for k sparse
 * matrices of one shape m x n in CSC form.  Column j of B holds every row r
 * that occurs in at least one A_i(:,j), and B(r,j) is the sum of those
 * A_i(r,j).  The paper's generic k-way template (Alg. 2) computes columns
 * independently; so does this file.
 *
 * Readings of the paper that this file fixes:
 *   - Structural zeros are kept.  An entry whose terms cancel stays in B with
 *     value 0: the hash accumulator (Alg. 5) never removes an entry and the
 *     symbolic phase (Alg. 6, Sec. II-D) counts rows without looking at
 *     values.
 *   - Output columns are sorted by row (the optional sort of Alg. 4 and 5,
 *     taken as required).
 *   - If an input column repeats a row (invalid when inputs are declared
 *     sorted, allowed when they are declared unordered) every copy is still
 *     one term of the sum.
 *
 * Method: the definition written out, nothing more.  For each requested
 * column, gather the triples (r, i, v) of all k inputs, sort them by
 * (r, i, position), and add each run of equal r in that order.  Sums are
 * fp64 with Neumaier's compensated summation; fp32 inputs are widened to
 * fp64 first.  Each output entry also reports sum |v| over its terms and the
 * number of terms, which the parity tests use for their error bound.
 *
 * The mutation hooks (SPK_ORACLE_PLANT_*) exist so that a CPU test can build
 * deliberately wrong copies of this file and check that the pins catch them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t r;    /* row index                         */
    int32_t i;    /* which input matrix                */
    int64_t e;    /* position inside that input        */
    double v;     /* value, widened to fp64            */
} spk_triple;

static int cmp_triple(const void* pa, const void* pb) {
    const spk_triple* a = (const spk_triple*)pa;
    const spk_triple* b = (const spk_triple*)pb;
    if (a->r != b->r) return a->r < b->r ? -1 : 1;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    if (a->e != b->e) return a->e < b->e ? -1 : 1;
    return 0;
}

/* Gather column j of all inputs into t (capacity >= sum of lengths).
 * Returns the number of triples. */
static int64_t gather_column(int k, int64_t j, const int32_t* const* cp,
                             const int32_t* const* ri, const void* const* vals,
                             int is_f64, spk_triple* t) {
    int64_t c = 0;
    for (int i = 0; i < k; ++i) {
#ifdef SPK_ORACLE_PLANT_OFF_BY_ONE_COLUMN
        int64_t beg = cp[i][j + 1] > cp[i][j] ? cp[i][j] + 1 : cp[i][j];
#else
        int64_t beg = cp[i][j];
#endif
        int64_t end = cp[i][j + 1];
        for (int64_t e = beg; e < end; ++e) {
            t[c].r = ri[i][e];
            t[c].i = i;
            t[c].e = e;
            if (vals == NULL) t[c].v = 0.0;
            else if (is_f64) t[c].v = ((const double*)vals[i])[e];
            else t[c].v = (double)((const float*)vals[i])[e];
#ifdef SPK_ORACLE_PLANT_SIGN_FLIP
            if (i == 1) t[c].v = -t[c].v;
#endif
            ++c;
        }
    }
    return c;
}

static int64_t column_length(int k, int64_t j, const int32_t* const* cp) {
    int64_t s = 0;
    for (int i = 0; i < k; ++i) s += (int64_t)cp[i][j + 1] - cp[i][j];
    return s;
}

/* Thread-private growing buffer. */
typedef struct { spk_triple* p; int64_t cap; } spk_buf;

static int buf_reserve(spk_buf* b, int64_t need) {
    if (need <= b->cap) return 0;
    int64_t cap = b->cap ? b->cap : 1024;
    while (cap < need) cap *= 2;
    spk_triple* np = (spk_triple*)realloc(b->p, (size_t)cap * sizeof(spk_triple));
    if (!np) return -1;
    b->p = np;
    b->cap = cap;
    return 0;
}

int spk_oracle_threads(int requested) {
#ifdef _OPENMP
    return requested > 0 ? requested : omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

/*
 * Number of distinct rows nnz(B(:,j)) for each listed column (Sec. II-D).
 * cols == NULL means all n columns, in order.  Returns 0, or -1 when out of
 * host memory.
 */
int spk_oracle_union_sizes(int k, int64_t n, const int32_t* const* cp,
                           const int32_t* const* ri, int64_t ncols,
                           const int64_t* cols, int32_t* u_out, int threads) {
    int failed = 0;
    if (cols == NULL) ncols = n;
#pragma omp parallel num_threads(spk_oracle_threads(threads)) reduction(| : failed)
    {
        spk_buf b = {NULL, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < ncols; ++q) {
            int64_t j = cols ? cols[q] : q;
            int64_t s = column_length(k, j, cp);
            if (buf_reserve(&b, s + 1)) { failed = 1; u_out[q] = -1; continue; }
            int64_t c = gather_column(k, j, cp, ri, NULL, 0, b.p);
            qsort(b.p, (size_t)c, sizeof(spk_triple), cmp_triple);
            int32_t u = 0;
            for (int64_t x = 0; x < c; ++x)
                if (x == 0 || b.p[x].r != b.p[x - 1].r) ++u;
            u_out[q] = u;
        }
        free(b.p);
    }
    return failed ? -1 : 0;
}

/*
 * Values of the listed columns.  out_ptr[q]..out_ptr[q+1] is the slot range
 * of listed column q (the caller builds it from spk_oracle_union_sizes).
 * Writes rows (ascending), fp64 values, sum |terms| and term counts.
 * vals[i] points at fp64 data when is_f64 != 0, else at fp32 data.
 * Returns 0, -1 when out of host memory, -2 when a column does not have the
 * size out_ptr promises.
 */
int spk_oracle_columns(int k, int64_t n, const int32_t* const* cp,
                       const int32_t* const* ri, const void* const* vals,
                       int is_f64, int64_t ncols, const int64_t* cols,
                       const int64_t* out_ptr, int32_t* out_r, double* out_v,
                       double* out_abs, int32_t* out_terms, int threads) {
    int failed = 0;
    if (cols == NULL) ncols = n;
#pragma omp parallel num_threads(spk_oracle_threads(threads)) reduction(| : failed)
    {
        spk_buf b = {NULL, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < ncols; ++q) {
            int64_t j = cols ? cols[q] : q;
            int64_t s = column_length(k, j, cp);
            if (buf_reserve(&b, s + 1)) { failed |= 1; continue; }
            int64_t c = gather_column(k, j, cp, ri, vals, is_f64, b.p);
            qsort(b.p, (size_t)c, sizeof(spk_triple), cmp_triple);
            int64_t o = out_ptr[q];
            int64_t x = 0;
            while (x < c) {
                int64_t y = x;
                while (y < c && b.p[y].r == b.p[x].r) ++y;
#ifdef SPK_ORACLE_PLANT_DROP_LAST_TERM
                if (y - x > 1) --y;
#endif
                /* Neumaier compensated summation over the run, ascending i. */
                double sum = 0.0, comp = 0.0, abs_sum = 0.0;
                for (int64_t z = x; z < y; ++z) {
                    double t = b.p[z].v;
                    double nsum = sum + t;
                    if (fabs(sum) >= fabs(t)) comp += (sum - nsum) + t;
                    else comp += (t - nsum) + sum;
                    sum = nsum;
                    abs_sum += fabs(t);
                }
#ifdef SPK_ORACLE_PLANT_DROP_LAST_TERM
                while (y < c && b.p[y].r == b.p[x].r) ++y;
#endif
                double value = sum + comp;
#ifdef SPK_ORACLE_PLANT_DROP_ZEROS
                if (value == 0.0) { x = y; continue; }
#endif
                if (o >= out_ptr[q + 1]) { failed |= 2; break; }
                out_r[o] = b.p[x].r;
                out_v[o] = value;
                if (out_abs) out_abs[o] = abs_sum;
                if (out_terms) out_terms[o] = (int32_t)(y - x);
                ++o;
                x = y;
            }
            if (o != out_ptr[q + 1]) failed |= 2;
#ifdef SPK_ORACLE_PLANT_REVERSE_ORDER
            for (int64_t lo = out_ptr[q], hi = o - 1; lo < hi; ++lo, --hi) {
                int32_t tr = out_r[lo]; out_r[lo] = out_r[hi]; out_r[hi] = tr;
                double tv = out_v[lo]; out_v[lo] = out_v[hi]; out_v[hi] = tv;
                if (out_abs) { tv = out_abs[lo]; out_abs[lo] = out_abs[hi]; out_abs[hi] = tv; }
                if (out_terms) { tr = out_terms[lo]; out_terms[lo] = out_terms[hi]; out_terms[hi] = tr; }
            }
#endif
        }
        free(b.p);
    }
    if (failed & 1) return -1;
    if (failed & 2) return -2;
    return 0;
}
