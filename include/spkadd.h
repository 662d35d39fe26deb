/*
 * spkadd.h -- C ABI of the GB300 SpKAdd library (libspkadd.so).
 *
 * SpKAdd (Sec. II-A of "Parallel Algorithms for Adding a Collection of Sparse
 * Matrices"): B = A_1 + A_2 + ... + A_k for k sparse matrices of one shape
 * m x n, all in CSC form; B is CSC with rows sorted ascending in every column.
 * An output entry exists wherever at least one input has an entry (the union
 * of the input patterns, Sec. II-A / Alg. 5); entries whose terms cancel are
 * kept with value 0.  nnz(B) <= sum_i nnz(A_i) (Sec. II-A).
 *
 * Values: an entry's terms are summed in an unspecified order.  Double
 * values are summed in double.  Float values are summed so that every entry
 * is within 1e-5 * sum|terms| of the exact sum for any k: in float while no
 * entry can collect more than 167 terms (the float error bound
 * (t - 1) 2^-24 sum|terms| then holds), in float phases of 128 inputs whose
 * partial sums are added in float for k up to 4992, in double beyond;
 * runs of repeated rows in the one-warp columns are summed in double.
 *
 * The computation runs in phases, as the paper's k-way algorithms do:
 *   spkadd_plan      -- per-column input counts and load-balancing classes
 *                       (Sec. III-A: "in the symbolic phase we use total input
 *                       non-zeros per column ... to balance loads").
 *   spkadd_symbolic  -- nnz(B(:,j)) for every column (Alg. 6 HashSymbolic,
 *                       Alg. 7 SlHashSymbolic for heavy columns, Sec. II-D),
 *                       the exclusive scan into B's column pointers, and the
 *                       total nnz(B), returned to the host so the caller can
 *                       allocate B (Sec. II-D: "pre-allocate necessary memory").
 *   spkadd_numeric   -- the values (Alg. 5 HashAdd, Alg. 8 SlHashAdd for heavy
 *                       columns) and the per-column sort (Alg. 5, last step).
 *   spkadd_destroy   -- releases the handle and its device workspace.
 *
 * Conventions for every entry point:
 *   - Pointers documented "device" must point to memory of the current CUDA
 *     device; "host" pointers to ordinary host memory.
 *   - All device work of a handle is ordered on the stream given to
 *     spkadd_plan (a cudaStream_t passed as void*; NULL = legacy default
 *     stream).  spkadd_symbolic synchronises that stream once to read nnz(B),
 *     spkadd_onepass twice; no other computing call blocks the host.
 *   - Every call returns a status; nothing aborts, throws or traps.  A failed
 *     kernel launch returns SPKADD_ERR_CUDA; errors raised asynchronously by
 *     the device surface at the next call on the handle.
 *   - Calls out of order (numeric before symbolic) return SPKADD_ERR_STATE.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef SPKADD_H
#define SPKADD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spkadd_status {
    SPKADD_OK = 0,
    SPKADD_ERR_INVALID_ARG = 1,     /* null pointer, k < 1, negative size, bad option */
    SPKADD_ERR_SHAPE_MISMATCH = 2,  /* inputs disagree on m or n */
    SPKADD_ERR_UNSORTED = 3,        /* validate mode: a column's rows are not strictly increasing */
    SPKADD_ERR_INDEX_RANGE = 4,     /* validate mode: row outside [0, m) or col_ptr not monotone / not ending at nnz */
    SPKADD_ERR_OVERFLOW = 5,        /* m or n >= 2^31, or a column's input count >= 2^31 */
    SPKADD_ERR_NOMEM = 6,           /* the workspace allocation failed */
    SPKADD_ERR_CUDA = 7,            /* a CUDA runtime call or kernel launch failed */
    SPKADD_ERR_TIMEOUT = 8,         /* a bounded device wait gave up */
    SPKADD_ERR_STATE = 9,           /* call out of order */
    SPKADD_ERR_UNSUPPORTED = 10,    /* valid request this library does not handle (e.g. k > SPKADD_MAX_K) */
    SPKADD_ERR_INTERNAL = 11        /* a device-side size invariant failed; the result is not valid */
} spkadd_status;

typedef enum spkadd_dtype {
    SPKADD_F32 = 0,   /* float values  (8 bytes per (row, value) pair, Sec. III-B's b = 8) */
    SPKADD_F64 = 1    /* double values (12 bytes per pair, the Sec. IV-B example)        */
} spkadd_dtype;

/* Largest k one handle accepts. */
#define SPKADD_MAX_K 65536

/*
 * One input matrix A_i in CSC form (Sec. II-A: a column is a list of
 * (rowid, val) tuples).  All three arrays are device memory, borrowed: they
 * must stay valid and unmodified until spkadd_numeric's work on the stream is
 * done (or the handle is destroyed).
 *   col_ptr[n+1]  int32, col_ptr[0] = 0, non-decreasing, col_ptr[n] = nnz
 *   row_idx[nnz]  int32, in [0, m), strictly increasing inside each column
 *   val[nnz]      float or double, as the plan's dtype says
 * nnz may be 0 (row_idx and val may then be NULL).
 */
typedef struct spkadd_csc {
    int64_t m;
    int64_t n;
    int64_t nnz;
    const int32_t* col_ptr;
    const int32_t* row_idx;
    const void* val;
} spkadd_csc;

/*
 * Tuning and behaviour knobs.  Fill with spkadd_default_options() and
 * override fields; pass NULL to spkadd_plan for the defaults.
 */
typedef struct spkadd_options {
    /* Nonzero: spkadd_plan checks every input on the device (one extra read
     * of all row indices, then one stream synchronisation) and returns
     * SPKADD_ERR_UNSORTED / SPKADD_ERR_INDEX_RANGE on bad input.  Zero: the
     * inputs are trusted.  Then a row outside [0, m) in a column with
     * s_j <= warp_max is still caught (spkadd_symbolic returns
     * SPKADD_ERR_INDEX_RANGE); one in a larger column, or rows out of order,
     * give an unspecified B (shared-memory accesses stay in bounds); col_ptr
     * values outside [0, nnz] make the kernels read outside row_idx/val. */
    int32_t validate;
    /* Columns whose summed input count s_j = sum_i nnz(A_i(:,j)) is at most
     * warp_max run one warp per column (range 1..512). */
    int32_t warp_max;
    /* Columns with warp_max < s_j <= cta_max run one thread block per column
     * (range warp_max..4096).  Larger columns are "heavy": the symbolic pass
     * uses a shared-memory row bitmap and the numeric pass splits them into
     * row windows (Sec. III-B, sliding hash). */
    int32_t cta_max;
    /* Maximum distinct rows per numeric row window of a heavy column
     * (range 1024..4096). */
    int32_t window_max;
    /* 0 = default: every column of B sorted by row.
     * 1 = as 0, but warp-class columns always take the duplicate-merging
     *     path of the numeric pass, even when the symbolic pass found no
     *     repeated row (a test and diagnosis switch; results are the same).
     * 2 = rows of a column of B may come in any order (Alg. 5 sorts only
     *     when sorted output is wanted): warp-class columns without repeated
     *     rows skip their final sort; col_ptr and each column's set of
     *     (row, value) pairs are the same as with 0. */
    int32_t sort_mode;
    /* 0 = rows are strictly increasing inside every input column (the
     * default; heavy columns are split into row windows by binary search,
     * Sec. III-B).  1 = rows may come in any order inside a column (Table I:
     * the hash method needs no sorted input): windows then read their whole
     * column and keep the rows in range, validation checks ranges only, and
     * a row repeated inside one input column is summed like a repeat across
     * inputs.  B is sorted either way. */
    int32_t input_order;
    /* Layout of Sec. II-D's dense accumulator in the thread-block kernels
     * (numeric CTA-class columns and heavy-column windows; heavy-column
     * symbolic count); the result is the same.  1 = a flat row bitmap
     * over a slab of up to 2^20 rows.  2 = a compact table: a summary bit
     * per 32-row word plus a table of only the non-empty words, so shared
     * memory follows window_max (numeric) or a fixed table size
     * (symbolic: the slab is cut into sub-ranges that fit), not m.
     * 0 = automatic: numeric items take the layout with more resident
     * blocks per SM; the heavy symbolic count takes the flat bitmap. */
    int32_t block_accumulator;
    /* Workspace allocator.  NULL alloc: cudaMallocAsync / cudaFreeAsync on
     * the plan's stream.  Otherwise alloc(bytes, stream, ctx) must return
     * device memory usable on `stream` (or NULL on failure) and
     * free(ptr, stream, ctx) releases it. */
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* alloc_ctx;
    /* Longest time, in milliseconds, that any device-side wait of the
     * one-pass kernel (spkadd_onepass: a predecessor tile's published sum)
     * may last before the kernel gives up
     * and the call returns SPKADD_ERR_TIMEOUT (range 1..600000). */
    int32_t wait_timeout_ms;
    /* Test switch, 0 in normal use.  1: in the one-pass kernel the second
     * column tile's look-back also waits for a word that nothing writes, so
     * its bounded wait runs out (the call returns SPKADD_ERR_TIMEOUT; nothing
     * hangs and the device stays usable). */
    int32_t test_stall;
} spkadd_options;

/* Planning statistics (host copy), for tests and benchmarks.  For a batch
 * handle k is the total input count, m the largest m and n the total column
 * count of all problems; the class and window counts cover all problems. */
typedef struct spkadd_info {
    int64_t k, m, n;
    int64_t nnz_in;         /* sum_i nnz(A_i) */
    int64_t nnz_out;        /* nnz(B); -1 before spkadd_symbolic */
    int64_t cols_warp;      /* columns per class (valid after spkadd_symbolic) */
    int64_t cols_cta;
    int64_t cols_heavy;
    int64_t windows;        /* numeric thread-block work items (CTA columns + heavy windows) */
    int64_t windows_split;  /* of those, row windows that needed per-input binary searches */
    int64_t cols_unique;    /* warp columns in which no row repeats across the inputs */
    int64_t workspace_bytes;
    int64_t kernel_launches; /* kernels this handle has launched so far */
    int64_t problems;       /* problems of the handle (1 unless made by spkadd_batch_plan) */
    int64_t onepass;        /* 1 when B was last computed by the one-pass kernel (spkadd_onepass) */
} spkadd_info;

typedef struct spkadd_handle spkadd_handle;

/* Fills *opt with the defaults (validate 0, warp_max 512, cta_max 4096,
 * window_max 4096, sort_mode 0, input_order 0, cudaMallocAsync,
 * wait_timeout_ms 2000, test_stall 0).  No CUDA call. */
void spkadd_default_options(spkadd_options* opt);

/*
 * Plans B = A[0] + ... + A[k-1].
 *   h       host out: the new handle (set to NULL on failure)
 *   k       number of inputs, 1 <= k <= SPKADD_MAX_K
 *   A       host array of k descriptors (copied; the arrays they point to
 *           are borrowed device memory, see spkadd_csc)
 *   dtype   value type of every input and of B
 *   stream  cudaStream_t (as void*) all work is ordered on
 *   opt     NULL for defaults
 * Host-side checks first (null pointers, k, shapes, sizes: no CUDA call is
 * made when they fail); then the workspace is allocated and the column
 * binning kernel is enqueued.  Does not block unless opt->validate is set.
 */
spkadd_status spkadd_plan(spkadd_handle** h, int k, const spkadd_csc* A, spkadd_dtype dtype, void* stream,
                          const spkadd_options* opt);

/*
 * Symbolic phase: counts nnz(B(:,j)) for every column, scans them into B's
 * column pointers (kept in the workspace) and writes the total nnz(B) to
 * *nnz_B (host).  Blocks until the stream reaches that point.
 */
spkadd_status spkadd_symbolic(spkadd_handle* h, int64_t* nnz_B);

/*
 * Numeric phase: writes B.  All three are device memory the caller
 * allocated from nnz_B:
 *   B_col_ptr[n+1]   int64 (nnz(B) may exceed 2^31)
 *   B_row_idx[nnz_B] int32, sorted ascending inside every column
 *   B_val[nnz_B]     float or double per the plan's dtype
 * Enqueued on the plan's stream; returns without blocking.  May be called
 * again (with the same or other output buffers) to recompute B.
 */
spkadd_status spkadd_numeric(spkadd_handle* h, int64_t* B_col_ptr, int32_t* B_row_idx, void* B_val);

/*
 * One-pass SpKAdd: the symbolic count (Alg. 6), the scan of Sec. II-D and the
 * numeric sum with the per-column sort (Alg. 5) in a single pass over the
 * inputs.  Sec. II-D needs the symbolic phase so that B can be allocated
 * first; here B goes into buffers sized by the bound nnz(B) <= sum_i
 * nnz(A_i) of Sec. II-A, and each column's offset in B comes from a
 * decoupled look-back over column tiles, so every input entry is read once.
 *   h           a handle of spkadd_plan (a batch handle: SPKADD_ERR_INVALID_ARG)
 *   B_col_ptr   device, n+1 int64 (written)
 *   B_row_idx   device, `capacity` int32; the first nnz(B) are B's rows
 *   B_val       device, `capacity` values of the plan's dtype
 *   capacity    entries B_row_idx / B_val hold; must be >= sum_i nnz(A_i)
 *               (spkadd_info.nnz_in), else SPKADD_ERR_INVALID_ARG.  Entries
 *               past nnz(B) are left unspecified.
 *   nnz_B       host out: nnz(B)
 * The one-pass kernel runs when every column has s_j <= warp_max (any k);
 * otherwise the call runs the kernels of spkadd_symbolic and spkadd_numeric
 * into the same buffers, with the same result (spkadd_info.onepass says
 * which ran).
 * Blocks the host twice (class counts after the plan, nnz(B) at the end).
 * Its device waits are bounded by opt.wait_timeout_ms: when one runs out the
 * call returns SPKADD_ERR_TIMEOUT and B is not valid.  May be called again;
 * afterwards the handle is in the state spkadd_numeric leaves it in.
 */
spkadd_status spkadd_onepass(spkadd_handle* h, int64_t* B_col_ptr, int32_t* B_row_idx, void* B_val,
                             int64_t capacity, int64_t* nnz_B);

/*
 * Batches.  Many independent SpKAdd problems B_q = A_q,1 + ... + A_q,k_q
 * (q = 0..count-1, each with its own k, shape and dtype) run as one: every
 * phase is one set of kernel launches over the columns of all problems,
 * so the launch count and the host synchronisations do not grow with count.
 * The paper has no batch interface; its per-column independence (Sec. III:
 * columns are added independently and in parallel) is what makes one.
 * Semantics per problem are those of spkadd_plan / spkadd_symbolic /
 * spkadd_numeric.  Release with spkadd_destroy; spkadd_get_info works too.
 * spkadd_symbolic and spkadd_numeric reject a batch handle
 * (SPKADD_ERR_INVALID_ARG); the batch calls accept a handle of spkadd_plan
 * as a batch of one.
 *
 * spkadd_batch_plan
 *   h       host out: the new handle
 *   count   number of problems, >= 1
 *   k       host array of count input counts (1 <= k[q] <= SPKADD_MAX_K)
 *   A       host array of count pointers; A[q] is a host array of k[q]
 *           descriptors of problem q (same rules as spkadd_plan's A)
 *   dtype   host array of count value types
 *   stream, opt  as for spkadd_plan (the options apply to every problem)
 * The total input count and the total column count must stay below 2^31
 * (SPKADD_ERR_OVERFLOW otherwise).  Host checks fail with the first bad
 * problem's status before any CUDA call.
 *
 * spkadd_batch_symbolic
 *   nnz_B   host out, count entries: nnz(B_q).  Blocks once for the batch.
 *
 * spkadd_batch_numeric
 *   B_col_ptr, B_row_idx, B_val  host arrays of count device pointers:
 *           problem q's outputs as in spkadd_numeric (B_col_ptr[q] has
 *           n_q + 1 int64; B_row_idx[q] / B_val[q] may be NULL when
 *           nnz(B_q) = 0).  The pointer arrays are copied before the call
 *           returns; the call does not block.
 */
spkadd_status spkadd_batch_plan(spkadd_handle** h, int count, const int* k, const spkadd_csc* const* A,
                                const spkadd_dtype* dtype, void* stream, const spkadd_options* opt);
spkadd_status spkadd_batch_symbolic(spkadd_handle* h, int64_t* nnz_B);
spkadd_status spkadd_batch_numeric(spkadd_handle* h, int64_t* const* B_col_ptr, int32_t* const* B_row_idx,
                                   void* const* B_val);

/* Statistics of the handle (host out).  May synchronise the stream. */
spkadd_status spkadd_get_info(spkadd_handle* h, spkadd_info* info);

/* Frees the workspace (stream-ordered) and the handle.  NULL is accepted. */
spkadd_status spkadd_destroy(spkadd_handle* h);

/*
 * Exclusive scan of per-column counts into CSC column pointers, allocating
 * nothing: col_ptr[0] = 0 and col_ptr[j+1] = col_ptr[j] + counts[j] -- the
 * scan spkadd_symbolic runs on nnz(B(:,j)).  The paper has no counterpart of
 * this entry point.  It exists for callers that must not allocate device
 * memory inside a call: services that hand all of a GPU's memory to their own
 * arena up front (so a cudaMalloc would fail or break their accounting), and
 * latency-critical code for which cudaMalloc's implicit device-wide
 * synchronisation is not acceptable.
 *   counts   device, n int32 counts, each >= 0
 *   n        0 <= n <= SPKADD_SCAN_NOALLOC_MAX_N; a larger n returns
 *            SPKADD_ERR_UNSUPPORTED and launches nothing
 *   col_ptr  device, n+1 int64, caller-allocated (written)
 *   stream   cudaStream_t (as void*); enqueued, does not block
 * Scratch: one fixed array of SPKADD_SCAN_NOALLOC_MAX_N / 4096 + 1 int64
 * (32 KB) defined inside the library; every GPU that loads the library holds
 * it until the process exits.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current)
 * and loads the scan kernels' code onto the device; CUDA loads a module's
 * code lazily and that load takes device memory, so make the first call on
 * each device at set-up: before the caller's arena claims the device's
 * memory, and before any stream capture.  Later calls load nothing.  All calls share the array
 * and it keeps the last call's contents; nothing needs to start at zero
 * (every element a call reads, that call wrote first).  Calls that can
 * overlap on the GPU -- on different streams without ordering between them,
 * or from several host threads -- race on the array and give wrong results.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define SPKADD_SCAN_NOALLOC_MAX_N (4096 * 4096)
spkadd_status spkadd_scan_counts_noalloc(const int32_t* counts, int64_t n, int64_t* col_ptr, void* stream);

/*
 * Streaming accumulation.  Sec. IV (distributed SpGEMM) adds the stage
 * results of sparse SUMMA; Sec. V notes that inputs arriving in batches, or
 * too many to fit in memory together, can be arranged in batches with SpKAdd
 * applied per batch.  A stream keeps the running sum B on the device; each
 * spkadd_stream_add of k inputs is one (k+1)-way SpKAdd (the phases above)
 * with B as input 0, so only the current batch of inputs need be resident.
 * B stays the union of all inputs added so far, rows sorted in every column.
 *
 * spkadd_stream_create: B = the empty m x n matrix of `dtype`.  All device
 *   work of the stream is ordered on `stream` (cudaStream_t as void*, NULL =
 *   legacy default stream).  `opt` as for spkadd_plan (NULL = defaults); its
 *   allocator, if any, also holds B.  Errors: INVALID_ARG (null s, negative
 *   size, bad dtype or option), OVERFLOW (m or n >= 2^31), NOMEM, CUDA.
 * spkadd_stream_add: B <- B + A[0] + ... + A[k-1] (1 <= k < SPKADD_MAX_K;
 *   A as spkadd_plan takes them, shapes equal to the stream's).  Blocks once
 *   (the symbolic phase); the numeric work runs on the stream afterwards, so
 *   the inputs must stay valid until it is done.  nnz(B) must stay below
 *   2^31 (B is the next add's input): otherwise OVERFLOW and B is unchanged.
 *   Every error leaves B unchanged.
 * spkadd_stream_query: nnz(B); optionally the number of adds and of kernel
 *   launches so far.
 * spkadd_stream_view: B as an spkadd_csc (int32 col_ptr; device memory owned
 *   by the stream, valid until the next add or destroy).
 * spkadd_stream_result: copies B into caller buffers (device): int64
 *   col_ptr[n+1], row_idx[nnz], val[nnz]; asynchronous on the stream.
 * spkadd_stream_destroy: releases B (stream-ordered); NULL is allowed.
 * Like a handle, a stream is not thread-safe; distinct streams are
 * independent.
 */
typedef struct spkadd_stream spkadd_stream;
spkadd_status spkadd_stream_create(spkadd_stream** s, int64_t m, int64_t n, spkadd_dtype dtype, void* stream,
                                   const spkadd_options* opt);
spkadd_status spkadd_stream_add(spkadd_stream* s, int k, const spkadd_csc* A);
spkadd_status spkadd_stream_query(spkadd_stream* s, int64_t* nnz_B, int64_t* adds, int64_t* kernel_launches);
spkadd_status spkadd_stream_view(spkadd_stream* s, spkadd_csc* B);
spkadd_status spkadd_stream_result(spkadd_stream* s, int64_t* B_col_ptr, int32_t* B_row_idx, void* B_val);
spkadd_status spkadd_stream_destroy(spkadd_stream* s);

/* Static, human-readable name of a status code. */
const char* spkadd_status_string(spkadd_status s);

/* Library version as major*10000 + minor*100 + patch. */
int spkadd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPKADD_H */
