// spk_common.cuh -- device helpers shared by the SpKAdd kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define SPK_FULL 0xffffffffu

namespace spk {

// ---------------------------------------------------------------------------
// Work classes (Sec. III-A: columns are balanced by their summed input count).
// ---------------------------------------------------------------------------
enum : int32_t { CLS_EMPTY = 0, CLS_WARP = 1, CLS_CTA = 2, CLS_HEAVY = 3 };

// Error bits in Counters::err (device side; the host maps them to statuses).
enum : int32_t {
  ERR_OVERFLOW = 1,      // a column's input count does not fit int32
  ERR_UNSORTED = 2,      // validate: rows not strictly increasing in a column
  ERR_RANGE = 4,         // validate: row outside [0, m) or bad col_ptr
  ERR_WINDOW_CAP = 8,    // more row windows than the workspace holds
  ERR_INTERNAL = 16,     // a size invariant failed (bug guard; work skipped)
  ERR_TIMEOUT = 32,      // a bounded device-side wait gave up
};

// One thread-block work item of the numeric pass: a whole CTA-class column
// or one row window of a heavy column (Alg. 8's B(r1:r2, j)).
struct Window {
  int32_t col;
  int32_t r_lo, r_hi;   // rows [r_lo, r_hi)
  int32_t u;            // distinct rows in the range (symbolic result)
  int32_t out_off;      // first output slot of the range inside column col
  int32_t search;       // -1: whole column; else row of the per-input offset table
};

struct Counters {
  int32_t n_warp, n_cta, n_heavy;
  int32_t n_windows;    // Window records appended
  int32_t n_search;     // of those, split windows needing per-input offsets
  int32_t n_unique;     // warp columns whose input rows are all distinct (u_j == s_j)
  int32_t err;
  int32_t n_big;        // heavy columns with s_j > BIG_S (listed apart, counted in n_heavy too)
  int32_t heavy_next;   // work counter of the heavy-column symbolic kernels
  int32_t kind_n[4];    // batches of several problem kinds: thread-block items per kind
  int32_t kind_fill[4]; //   and their placement counters
  int32_t pad[3];
};

// Float sums.  A float sum of t terms, in any order, errs by at most
// (t - 1) 2^-24 sum|terms| (first order), within 1e-5 sum|terms| for
// t <= FP32_ACC_TERMS.  Thread-block accumulators of problems with k <= 167
// sum in float, and so do those slabs of larger problems whose entries
// leave no row more than 167 terms (a row's terms number at most
// s - u + 1 for s entries on u distinct rows).  Other slabs of problems
// with k <= FP32_PHASED_MAX_K sum in phases of FP32_PHASE_INPUTS inputs:
// each phase in float, its partial sums then added in float into B's
// values, so an entry collects at most 128 terms in a phase and at most
// ceil(k / 128) phase sums, and its error stays below
// (127 + ceil(k / 128) - 1) 2^-24 sum|terms| <= 166 * 2^-24 sum|terms|.
// Beyond FP32_PHASED_MAX_K the accumulators are double.  Warp columns
// always sum a row's run in double.
constexpr int FP32_ACC_TERMS = 167;
constexpr int FP32_PHASE_INPUTS = 128;  // whole 32-input chunks, one per warp group of a 256-thread block
constexpr int FP32_PHASED_MAX_K = 4992;
static_assert((FP32_PHASE_INPUTS - 1) + (FP32_PHASED_MAX_K / FP32_PHASE_INPUTS - 1) <= FP32_ACC_TERMS - 1,
              "phased float sums must stay within the float error bound");
static_assert(FP32_PHASE_INPUTS % 32 == 0, "phases are whole 32-input chunks");


// Heavy columns above this summed input count are listed apart and handed out
// first (largest work first keeps one huge R-MAT column from finishing last).
constexpr int32_t BIG_S = 1 << 18;

// One SpKAdd problem of a batch, as the kernels see it.  A single call is a
// batch of one.  Columns of all problems are numbered in one global column
// space: problem q owns global columns [colbase, colbase + n), and B's entries
// of problem q sit at global col_ptr_B positions minus col_ptr_B[colbase].
struct Inst {
  int32_t k, m, n, dtype;   // dtype: 0 = float, 1 = double
  int32_t colbase;          // first global column
  int32_t ptr_off;          // first (problem, input) entry of the pointer tables
  uint32_t bucket_mul[16];  // floor(2^32 * 2^q / m), clamped below 2^32, q = 0..15
};

struct Inputs {
  const Inst* inst;
  const int32_t* col_inst;  // global column -> problem (nullptr for a batch of one)
  const int32_t* const* cp; // pointer tables, one entry per (problem, input)
  const int32_t* const* ri;
  const void* const* val;
  int32_t ninst;
  int32_t ncols;            // total columns of all problems
  int32_t kmax;
  int32_t mmax;
  int32_t sorted;           // rows strictly increasing inside every input column
};

__device__ __forceinline__ int inst_of(const Inputs& in, int g) { return in.col_inst ? __ldg(in.col_inst + g) : 0; }

// Where B goes: the caller's buffers, through per-problem pointer tables
// (rows/vals/cps, a batch) or directly (row0/val0/cp0: a single problem, and
// problem 0 of any batch, so a batch of one may use either).  Row/value positions inside a problem's
// buffers are global col_ptr_B values minus col_ptr_B[colbase].
struct Outs {
  int32_t* row0;
  void* val0;
  int64_t* cp0;
  int32_t* const* rows;
  void* const* vals;
  int64_t* const* cps;
};
__device__ __forceinline__ int32_t* out_row_of(const Outs& o, int q) { return o.rows ? o.rows[q] : o.row0; }
__device__ __forceinline__ void* out_val_of(const Outs& o, int q) { return o.vals ? o.vals[q] : o.val0; }
__device__ __forceinline__ int64_t* out_cp_of(const Outs& o, int q) { return o.cps ? o.cps[q] : o.cp0; }

// ---------------------------------------------------------------------------
// Hash functions.  The paper hashes with (a * r) & (2^q - 1), a prime
// (Sec. II-C).  The low q bits of a*r depend only on the low q bits of r, so
// structured row sets (R-MAT) collide; we keep the prime multiplier and take
// the high q bits of the 32-bit product instead (multiplicative hashing).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hash_scrambled(int32_t r, int q) {
  return (static_cast<uint32_t>(r) * 0x9E3779B1u) >> (32 - q);
}

__device__ __forceinline__ int ceil_log2(int x) {  // x >= 1
  return x <= 1 ? 0 : 32 - __clz(x - 1);
}

// ---------------------------------------------------------------------------
// Warp-level helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(SPK_FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

__device__ __forceinline__ int warp_sum(int x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(SPK_FULL, x, o);
  return x;
}

__device__ __forceinline__ int warp_max(int x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(SPK_FULL, x, o));
  return x;
}

// ---------------------------------------------------------------------------
// Segment walker.  A warp walks the concatenation of up to 32 segments (one
// per lane: input `base + lane`, elements [beg, beg + len) of that input).
// Flattened position e (0 <= e < total) belongs to segment
// find(e) = max{ l : P_l <= e } where P is the exclusive prefix of lengths;
// empty segments are skipped automatically.  The element's index inside its
// input is e + delta(seg).  Consecutive positions of a warp round are
// consecutive memory inside each segment, so loads stay coalesced.
// ---------------------------------------------------------------------------
struct SegWalk {
  int P;      // this lane's segment start in the flattened order
  int delta;  // beg - P
  int total;  // sum of the 32 lengths

  __device__ __forceinline__ void init(int beg, int len, int lane) {
    int inc = warp_incl_scan(len, lane);
    total = __shfl_sync(SPK_FULL, inc, 31);
    P = inc - len;
    delta = beg - P;
  }
  // Every lane of the warp must call this (it shuffles).
  __device__ __forceinline__ int find(int e) const {
    int idx = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      int w = __shfl_sync(SPK_FULL, P, idx + step);
      if (w <= e) idx += step;
    }
    return idx;
  }
  __device__ __forceinline__ int index_in_input(int e, int seg) const {
    return e + __shfl_sync(SPK_FULL, delta, seg);
  }
};

// ---------------------------------------------------------------------------
// Chunk map: the segment walker plus a fast path for chunks whose segments all
// have one length L (Erdos-Renyi and partial-product inputs give every input
// the same count per column).  Then position e lies in segment e / L, found
// with one multiply-high instead of five shuffles.  `nvalid` is the number of
// real inputs in the chunk (lanes at or beyond it carry empty segments).
// ---------------------------------------------------------------------------
struct ChunkMap {
  SegWalk w;
  int beg;          // this lane's segment begin (fast path)
  int total;
  int L;
  int shift;        // log2(L) when L is a power of two, else -1
  uint32_t magic32; // floor((2^32 - 1) / L) + 1: e / L == umulhi(e, magic32) for e < 2^16, 2 <= L < 2^16
  bool equal;

  __device__ __forceinline__ void init(int beg_, int len, int lane, int nvalid) {
    beg = beg_;
    const int L0 = __shfl_sync(SPK_FULL, len, 0);
    equal = __all_sync(SPK_FULL, lane >= nvalid || len == L0) && L0 >= 2 && L0 < 65536 &&
            (int64_t)L0 * nvalid < 65536;
    if (equal) {
      L = L0;
      total = L0 * nvalid;
      shift = (L0 & (L0 - 1)) == 0 ? __ffs(L0) - 1 : -1;
      magic32 = 0xFFFFFFFFu / (uint32_t)L0 + 1u;  // a 32-bit division (a 64-bit one costs far more)
    } else {
      w.init(beg_, len, lane);
      total = w.total;
    }
  }
  // Segment of flattened position e and the position's offset inside that
  // segment.  Every lane must call it (it may shuffle).
  __device__ __forceinline__ int seg_off(int e, int* off) const {
    if (equal) {
      const int sg = shift >= 0 ? (e >> shift) : (int)__umulhi((uint32_t)e, magic32);
      *off = e - sg * L;
      return sg;
    }
    const int sg = w.find(e);
    *off = e - __shfl_sync(SPK_FULL, w.P, sg);
    return sg;
  }
  // Element index (inside its input) of flattened position e; *seg = segment.
  // Every lane must call it (it shuffles).
  __device__ __forceinline__ int locate(int e, int* seg) const {
    if (equal) {
      const int sg = (int)__umulhi((uint32_t)e, magic32);
      const int b = __shfl_sync(SPK_FULL, beg, sg & 31);
      *seg = sg;
      return b + (e - sg * L);
    }
    const int sg = w.find(e);
    *seg = sg;
    return w.index_in_input(e, sg);
  }
};

// ---------------------------------------------------------------------------
// Block-level exclusive scan of one int per thread (BLOCK threads).
// `tmp` must hold BLOCK/32 ints.  Returns the exclusive prefix; *total gets
// the block sum.  Contains __syncthreads().
// ---------------------------------------------------------------------------
template <int BLOCK>
__device__ __forceinline__ int block_excl_scan(int x, int* tmp, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = warp_incl_scan(x, lane);
  if (lane == 31) tmp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int v = lane < BLOCK / 32 ? tmp[lane] : 0;
    int vi = warp_incl_scan(v, lane);
    if (lane < BLOCK / 32) tmp[lane] = vi - v;
    if (lane == 31) tmp[BLOCK / 32] = vi;  // needs BLOCK/32 + 1 slots
  }
  __syncthreads();
  int r = tmp[wid] + inc - x;
  *total = tmp[BLOCK / 32];
  __syncthreads();
  return r;
}

// Lower bound: first position p in [lo, hi) with a[p] >= key (hi if none).
__device__ __forceinline__ int lower_bound_i32(const int32_t* __restrict__ a, int lo, int hi, int32_t key) {
  while (lo < hi) {
    int mid = lo + ((hi - lo) >> 1);
    if (__ldg(a + mid) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Order-preserving bucket of a row: floor(r * mul / 2^32), mul = floor(2^32 * NB / m)
// (clamped below 2^32), so buckets are monotone in r and < NB for r < m.
__device__ __forceinline__ uint32_t bucket_hi(int32_t r, uint32_t mul) {
  return __umulhi(static_cast<uint32_t>(r), mul);
}

// Sets bit rr of a 64-bit-word bitmap with a 32-bit atomic on the word's
// half that holds it.  Returns true when that half was empty before (then the
// 64-bit word may have been empty: the caller marks it in its summary; a
// word can be marked twice, which is harmless).
__device__ __forceinline__ bool set_row_bit(unsigned long long* bm, uint32_t rr) {
  uint32_t* half = reinterpret_cast<uint32_t*>(bm) + (rr >> 5);  // little-endian: bits 0-31 first
  return atomicOr(half, 1u << (rr & 31)) == 0u;
}

// ---------------------------------------------------------------------------
// Thread-block entry walk (thread-block items of the symbolic and numeric
// passes).
// ---------------------------------------------------------------------------
// Runs every entry of input segments [beg_i, beg_i + len_i) of the item's
// inputs, 32 inputs per chunk; the warps of the block split each chunk's
// flattened entries.  Equal-length chunks use the one-multiply map.  Lane i
// holds input i's row (and value) pointer; an entry takes its segment's
// pointer by shuffle.  Per-entry work is fpre(row, value) -> token, issued for
// a round's U entries before any fpost(token, row, value), so the round's
// shared atomics are in flight together.
__device__ __forceinline__ const int32_t* shfl_iptr(const int32_t* p, int src) {
  return reinterpret_cast<const int32_t*>(__shfl_sync(SPK_FULL, reinterpret_cast<unsigned long long>(p), src));
}
template <typename V>
__device__ __forceinline__ const V* shfl_vptr(const V* p, int src) {
  return reinterpret_cast<const V*>(__shfl_sync(SPK_FULL, reinterpret_cast<unsigned long long>(p), src));
}

// Starts moving [p, p + bytes) toward L2 (128-byte lines) without waiting:
// used for a value segment one pass ahead of the pass that reads it.
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p) & ~static_cast<uintptr_t>(127);
  const uintptr_t a1 = reinterpret_cast<uintptr_t>(p) + bytes;
  for (uintptr_t a = a0; a < a1; a += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Ragged chunks whose segments average at least this many entries are walked
// segment by segment instead of in flattened order.
constexpr int SEG_MAJOR_MIN = 24;

// A lane's segment bounds, kept from pass A for pass B when its warp walks a
// single chunk (k <= 32 * warp groups): pass B then skips the reload.
struct SegCache {
  int beg, len;
  bool valid;
};

// Inputs [k_lo, k) of the item (k_lo a multiple of 32).  PREF (a pass that
// reads rows only, ahead of one that also reads values): each lane first
// starts moving its value segment into L2.
template <bool VALS, typename V, int BLOCK, int U, typename SegF, typename FPre, typename FPost, bool PREF = false>
__device__ __forceinline__ void block_for_each_entry(const Inputs& in, int k_lo, int k, int off, SegF& seg,
                                                     FPre& fpre, FPost& fpost, SegCache& sc) {
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // The chunks of 32 inputs run side by side: `groups` of `per` warps, group
  // g taking chunks g, g + groups, ... (all chunks' loads are in flight at once).
  const int nch = (k - k_lo + 31) >> 5;
  const int groups = min(nch, NW);
  const int per = NW / groups;
  const int gid = wid / per, lw = wid - gid * per;
  if (gid >= groups) return;  // (warp-uniform) spare warps
  for (int cb = k_lo + gid * 32; cb < k; cb += groups * 32) {
    const int i = cb + lane;
    int beg = 0, len = 0;
    const int32_t* rp = nullptr;
    const V* vp = nullptr;
    if (i < k) {
      if (sc.valid) {
        beg = sc.beg;
        len = sc.len;
      } else {
        seg(i, &beg, &len);
      }
      rp = in.ri[off + i] + beg;
      if constexpr (VALS) vp = static_cast<const V*>(in.val[off + i]) + beg;
      if constexpr (PREF)
        if (lw == 0 && len > 0)  // one warp of the group per chunk
          l2_prefetch(static_cast<const V*>(in.val[off + i]) + beg, (size_t)len * sizeof(V));
    }
    if (nch <= groups) {  // this warp's only chunk: remember its bounds for the next pass
      sc.beg = beg;
      sc.len = len;
      sc.valid = true;
    }
    ChunkMap cm;
    const int nvalid = min(32, k - cb);
    cm.init(beg, len, lane, nvalid);
    if (!cm.equal && cm.total >= SEG_MAJOR_MIN * nvalid) {
      // Ragged segments long enough to fill warp rounds: each warp walks
      // whole segments (inputs lw, lw + per, ...), so an entry's segment is
      // known without the per-entry search of the flattened order.
      for (int sgi = lw; sgi < nvalid; sgi += per) {
        const int ls = __shfl_sync(SPK_FULL, len, sgi);
        const int32_t* p = shfl_iptr(rp, sgi);
        const V* q = nullptr;
        if constexpr (VALS) q = shfl_vptr(vp, sgi);
        for (int e0 = 0; e0 < ls; e0 += 32 * U) {
          int32_t r[U];
          V v[U];
#pragma unroll
          for (int t = 0; t < U; ++t) {
            r[t] = -1;
            v[t] = V(0);
            const int o = e0 + t * 32 + lane;
            if (e0 + t * 32 < ls && o < ls) {  // (the first test is warp-uniform)
              r[t] = __ldg(p + o);
              if constexpr (VALS) v[t] = __ldg(q + o);
            }
          }
          uint32_t tok[U];
#pragma unroll
          for (int t = 0; t < U; ++t) tok[t] = r[t] >= 0 ? fpre(r[t], v[t]) : 0u;
#pragma unroll
          for (int t = 0; t < U; ++t)
            if (r[t] >= 0) fpost(tok[t], r[t], v[t]);
        }
      }
      continue;
    }
    if (lw * 32 * U >= cm.total) continue;  // (warp-uniform) this warp has no entries in the chunk
    for (int e0 = lw * 32 * U; e0 < cm.total; e0 += per * 32 * U) {
      int32_t r[U];
      V v[U];
#pragma unroll
      for (int t = 0; t < U; ++t) {
        r[t] = -1;
        v[t] = V(0);
        if (e0 + t * 32 >= cm.total) continue;  // (warp-uniform) slot wholly past the chunk's end
        const int e = e0 + t * 32 + lane;
        int off_in;
        const int sg = cm.seg_off(e, &off_in);
        const int32_t* p = shfl_iptr(rp, sg & 31);
        const V* q = nullptr;
        if constexpr (VALS) q = shfl_vptr(vp, sg & 31);
        if (e < cm.total) {
          r[t] = __ldg(p + off_in);
          if constexpr (VALS) v[t] = __ldg(q + off_in);
        }
      }
      uint32_t tok[U];
#pragma unroll
      for (int t = 0; t < U; ++t) tok[t] = r[t] >= 0 ? fpre(r[t], v[t]) : 0u;
#pragma unroll
      for (int t = 0; t < U; ++t)
        if (r[t] >= 0) fpost(tok[t], r[t], v[t]);
    }
  }
}

template <bool VALS, typename V, int BLOCK, int U, typename SegF, typename FPre, typename FPost, bool PREF = false>
__device__ __forceinline__ void block_for_each_entry(const Inputs& in, int k, int off, SegF& seg, FPre& fpre,
                                                     FPost& fpost, SegCache& sc) {
  block_for_each_entry<VALS, V, BLOCK, U, SegF, FPre, FPost, PREF>(in, 0, k, off, seg, fpre, fpost, sc);
}

}  // namespace spk
