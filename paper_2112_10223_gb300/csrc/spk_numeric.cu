// spk_numeric.cu -- a4/a5 of the hot path for thread-block work items: the
// CTA-class columns and the row windows of heavy columns.  Accumulate the
// values and write each item's output rows sorted.
//
// Alg. 5 (HashAdd) keeps an insert-or-add table keyed by row and sorts it at
// the end; Sec. II-D allows a dense accumulator in place of the hash.  Here the
// table is indexed by the exact output rank of the row, taken from a bitmap of
// the item's rows (the symbolic pass's structure, rebuilt in shared memory):
//
//   pass A   every entry sets bit (r - lo) of a 64-bit-word row bitmap; the
//            first bit set in a word also sets the word's bit in a summary
//            bitmap (one bit per word)
//   rank     the non-empty words (found through the summary) get the
//            exclusive popcount prefix of the words before them, and are
//            listed in row order
//   pass B   every entry adds its value at acc[rank(r)], rank(r) =
//            prefix(word) + popcount(word & bits below r)
//   write    the listed words are expanded to rows in rank order (one thread
//            per word) and rows and acc[rank] are written out coalesced,
//            already in row order; the touched words are cleared for the next
//            item.
//
// The bitmap covers a slab of 2^slab_log2 rows (at most 2^20): an item whose
// rows span more is processed slab by slab, with per-input binary searches
// for each slab's entries.
//
// A second layout, the compact word table (k_num_compact, below), keeps only
// a summary bit per 32-row word and a table of the item's non-empty words, so
// its shared memory follows window_max instead of the slab; the launcher runs
// whichever layout has more blocks resident per SM.
#include <mutex>
#include <type_traits>

#include "spk_common.cuh"
#include "spk_launch.h"

namespace spk {

constexpr int NUM_SLAB_LOG2_MAX = 20;  // 2^20 rows: 128 KB of bitmap

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(SPK_FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of one 64-bit value per thread; `tmp` holds
// BLOCK/32 + 1 entries.  Contains __syncthreads().
template <int BLOCK>
__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long x, unsigned long long* tmp,
                                                                  unsigned long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long inc = warp_incl_scan_u64(x, lane);
  if (lane == 31) tmp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const unsigned long long v = lane < BLOCK / 32 ? tmp[lane] : 0ull;
    const unsigned long long vi = warp_incl_scan_u64(v, lane);
    if (lane < BLOCK / 32) tmp[lane] = vi - v;
    if (lane == 31) tmp[BLOCK / 32] = vi;
  }
  __syncthreads();
  const unsigned long long r = tmp[wid] + inc - x;
  *total = tmp[BLOCK / 32];
  __syncthreads();
  return r;
}

// Shared-memory layout of the bitmap kernel.
struct BitmapSmem {
  unsigned long long* bm;  // W64 words: row bitmap of the slab (kept zero between slabs)
  uint16_t* wpre;          // W64: exclusive popcount prefix of each non-empty word
  uint32_t* summ;          // NSW = max(1, W64/32): one bit per bitmap word (kept zero between slabs)
  uint16_t* nel;           // umax: the non-empty words in row order
  int32_t* rows;           // umax: output rows of the slab in rank order
  unsigned char* acc;      // umax values
  unsigned long long* red; // BLOCK/32 + 1 scan slots
  int W64, NSW, umax;
};

// Bitmap words per thread for `nwords` words: a power of two <= 32, so a
// thread's run of words sits inside one summary word.
template <int BLOCK>
__device__ __forceinline__ int words_per_thread(int nwords) {
  int per = 1;
  while (per * BLOCK < nwords && per < 32) per <<= 1;
  return per;
}

// The summary bits of words [w0, w0 + per) (per a power of two <= 32, w0 a multiple of per).
__device__ __forceinline__ uint32_t own_word_mask(const uint32_t* summ, int w0, int per, int nwords) {
  if (w0 >= nwords) return 0u;
  const uint32_t all = summ[w0 >> 5] >> (w0 & 31);
  return per == 32 ? all : (all & ((1u << per) - 1u));
}

// Item filter of a launch over one problem kind (a check: the records it is
// given are grouped by kind, so it keeps them all): 0 float, 1 double, 2
// float with k <= FP32_ACC_TERMS, 3 float with FP32_ACC_TERMS < k <=
// FP32_PHASED_MAX_K, 4 float with larger k; -1 (a batch of one kind) keeps
// every item.
__device__ __forceinline__ bool item_selected(int sel, const Inst* I) {
  if (sel == 1) return I->dtype == 1;
  if (I->dtype != 0) return false;
  if (sel == 2) return I->k <= FP32_ACC_TERMS;
  if (sel == 3) return I->k > FP32_ACC_TERMS && I->k <= FP32_PHASED_MAX_K;
  if (sel == 4) return I->k > FP32_PHASED_MAX_K;
  return true;
}

// Problem kinds of the thread-block numeric launches, one launch per kind
// present: 0 float with k <= FP32_ACC_TERMS, 1 float with
// FP32_ACC_TERMS < k <= FP32_PHASED_MAX_K (sums in phases), 2 float with
// larger k (double accumulators), 3 double.
__device__ __forceinline__ int item_kind(const Inst* I) {
  if (I->dtype == 1) return 3;
  return I->k <= FP32_ACC_TERMS ? 0 : (I->k <= FP32_PHASED_MAX_K ? 1 : 2);
}

// Pass B of an item's slab: every entry's value added at its rank.  Without
// phases the sums stay in acc for the caller's write (returns false).
// PHASED (float sums of problems with k > FP32_ACC_TERMS): a slab whose
// s_ent entries on slab_u rows can give a row more than FP32_ACC_TERMS
// terms runs its inputs in phases of FP32_PHASE_INPUTS; after each phase the
// slab's first `lim` partial sums are added into B's values (the first phase
// stores them) and acc is zeroed (returns true: the values are written).
template <typename V, typename A, bool PHASED, int BLOCK, int U, typename SegF, typename FAdd>
__device__ __forceinline__ bool add_values(const Inputs& in, int k, int off, SegF& seg, FAdd& add, SegCache& sc,
                                           A* acc, V* oval, int slab_u, int lim, int s_ent) {
  auto none = [](uint32_t, int32_t, V) {};
  if (!PHASED || s_ent - slab_u < FP32_ACC_TERMS) {
    block_for_each_entry<true, V, BLOCK, U>(in, 0, k, off, seg, add, none, sc);
    return false;
  }
  for (int p0 = 0; p0 < k; p0 += FP32_PHASE_INPUTS) {
    SegCache fresh{0, 0, false};  // a phase's chunks differ from pass A's
    block_for_each_entry<true, V, BLOCK, U>(in, p0, min(k, p0 + FP32_PHASE_INPUTS), off, seg, add, none, fresh);
    __syncthreads();
    for (int q = threadIdx.x; q < slab_u; q += BLOCK) {
      if (q < lim) oval[q] = p0 == 0 ? (V)acc[q] : oval[q] + (V)acc[q];
      acc[q] = A(0);
    }
    __syncthreads();
  }
  return true;
}

// One item (a CTA-class column or a heavy column's row window [r_lo, r_hi),
// Alg. 8: B(r1:r2, j) <- HashAdd(A_1(r1:r2, j), ..., A_k(r1:r2, j))).
template <typename V, typename A, bool PHASED, int BLOCK, int U>
__device__ __forceinline__ void bitmap_item(const Inputs& in, const Window& W, const Inst* I, const int32_t* offs,
                                            int32_t* __restrict__ out_row, V* __restrict__ out_val,
                                            const BitmapSmem& sm, int slab_log2, Counters* ctr_w) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int k = I->k, off = I->ptr_off, j = W.col - I->colbase;
  A* acc = reinterpret_cast<A*>(sm.acc);
  const int64_t S = (int64_t)1 << slab_log2;
  const int64_t span = (int64_t)W.r_hi - W.r_lo;
  const int nsl = span <= 0 ? 0 : (int)((span + S - 1) >> slab_log2);
  int u_done = 0;
  bool bad = false;
  for (int t = 0; t < nsl; ++t) {
    const int lo = W.r_lo + (int)(t * S);
    const int hi = (int)min((int64_t)W.r_hi, (int64_t)lo + S);
    const uint32_t width = (uint32_t)(hi - lo);
    // The item's entries of input i that fall in [lo, hi).
    auto seg = [&](int i, int* beg, int* len) {
      int b, e;
      if (W.search < 0) {
        const int32_t* cp = in.cp[off + i];
        b = __ldg(cp + j);
        e = __ldg(cp + j + 1);
      } else {
        const int32_t* o = offs + ((int64_t)W.search * in.kmax + i) * 2;
        b = o[0];
        e = o[1];
      }
      if (nsl > 1 && in.sorted) {  // unordered inputs: the whole segment, rows outside the slab skipped
        const int32_t* ri = in.ri[off + i];
        b = lower_bound_i32(ri, b, e, lo);
        e = lower_bound_i32(ri, b, e, hi);
      }
      *beg = b;
      *len = e - b;
    };
    // Pass A: row bits (rows outside the slab are ignored: they cannot occur
    // for valid inputs, and shared-memory accesses stay in bounds).
    int n_ent = 0;  // PHASED: entries this thread met in the slab
    auto setbit = [&](int32_t r, V) -> uint32_t {
      const uint32_t rr = (uint32_t)(r - lo);
      if constexpr (PHASED) n_ent += rr < width;
      return (rr < width && set_row_bit(sm.bm, rr)) ? 1u : 0u;
    };
    auto mark_word = [&](uint32_t fresh, int32_t r, V) {
      if (fresh) {
        const uint32_t w = (uint32_t)(r - lo) >> 6;
        atomicOr(&sm.summ[w >> 5], 1u << (w & 31));
      }
    };
    SegCache sc{0, 0, false};
    block_for_each_entry<false, V, BLOCK, U, decltype(seg), decltype(setbit), decltype(mark_word), true>(
        in, k, off, seg, setbit, mark_word, sc);
    __syncthreads();
    int s_ent = 0;
    if constexpr (PHASED) block_excl_scan<BLOCK>(n_ent, reinterpret_cast<int*>(sm.red), &s_ent);
    // Rank prefix: thread t owns bitmap words [t*per, t*per + per); their
    // non-empty ones are the set bits of `mine` (kept for the clear below).
    const int nwords = (int)((width + 63) >> 6);
    const int per = words_per_thread<BLOCK>(nwords);
    if (per * BLOCK < nwords) {  // the host sizes blocks so this cannot happen; never skip words silently
      if (threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);
      bad = true;
    }
    const int w0 = threadIdx.x * per;
    const uint32_t mine = own_word_mask(sm.summ, w0, per, nwords);
    unsigned long long loc = (unsigned long long)__popc(mine) << 32;  // (non-empty words << 32) | rows
    for (uint32_t bits = mine; bits; bits &= bits - 1) loc += (unsigned long long)__popcll(sm.bm[w0 + __ffs(bits) - 1]);
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan_u64<BLOCK>(loc, sm.red, &tot);
    const int slab_u = (int)(tot & 0xffffffffull);
    const int slab_ne = (int)(tot >> 32);
    const bool fits = u_done + slab_u <= sm.umax && !bad;
    if (fits) {
      int rank = (int)(ex & 0xffffffffull), pos = (int)(ex >> 32);
      for (uint32_t bits = mine; bits; bits &= bits - 1) {
        const int w = w0 + __ffs(bits) - 1;
        sm.wpre[w] = (uint16_t)rank;
        sm.nel[pos++] = (uint16_t)w;
        rank += __popcll(sm.bm[w]);
      }
      for (int q = threadIdx.x; q < slab_u; q += BLOCK) acc[q] = A(0);
    } else {
      bad = true;
    }
    __syncthreads();
    if (fits) {
      // Pass B: values at their rank.
      auto add = [&](int32_t r, V v) -> uint32_t {
        const uint32_t rr = (uint32_t)(r - lo);
        if (rr < width) {
          const uint32_t w = rr >> 6;
          const unsigned long long bits = sm.bm[w];
          const uint32_t below = rr & 63;
          const int q = (int)sm.wpre[w] + __popcll(below ? (bits << (64 - below)) : 0ull);
          if (bits && q < slab_u) atomicAdd(&acc[q], (A)v);
        }
        return 0u;
      };
      // Ranks past the symbolic count are never written (B holds W.u rows
      // here); they can only arise if the inputs changed between the passes.
      const bool written = add_values<V, A, PHASED, BLOCK, U>(in, k, off, seg, add, sc, acc, out_val + u_done, slab_u,
                                                              min(slab_u, W.u - u_done), s_ent);
      // Rows in rank order: one thread per non-empty word.
      for (int p = threadIdx.x; p < slab_ne; p += BLOCK) {
        const int w = sm.nel[p];
        int q = sm.wpre[w];
        const int rbase = lo + (w << 6);
        for (unsigned long long bits = sm.bm[w]; bits; bits &= bits - 1) sm.rows[q++] = rbase + __ffsll(bits) - 1;
      }
      __syncthreads();
      // Coalesced write of the slab's rows and values.
      const int lim = min(slab_u, W.u - u_done);
      int32_t* orow = out_row + u_done;
      V* oval = out_val + u_done;
      for (int q = threadIdx.x; q < lim; q += BLOCK) {
        orow[q] = sm.rows[q];
        if (!written) oval[q] = (V)acc[q];
      }
      u_done += slab_u;
    }
    // Clear this thread's words; then the summary.
    for (uint32_t bits = mine; bits; bits &= bits - 1) sm.bm[w0 + __ffs(bits) - 1] = 0ull;
    __syncthreads();
    for (int x = threadIdx.x; x < ((nwords + 31) >> 5); x += BLOCK) sm.summ[x] = 0u;
    __syncthreads();
  }
  if (threadIdx.x == 0 && (bad || u_done != W.u)) atomicOr(&ctr_w->err, ERR_INTERNAL);
}

// ---------------------------------------------------------------------------
// Compact word table: the same exact-rank accumulator for items whose rows
// span a large slab but are few (at most umax distinct rows).  The flat
// bitmap's size follows the slab (128 KB at 2^20 rows); here only the
// summary follows the slab (one bit per 32-row word: 4 KB at 2^20) and the
// row bits live in a table of the non-empty words, which has at most umax
// entries.  Shared memory drops to about a quarter, so several items are in
// flight per SM instead of one.  One more pass over the item's entries:
//
//   pass A1  every entry sets its word's summary bit
//   rank 1   popcount prefix over the summary: word w gets the compact
//            index c(w) = prefix(w / 32) + popcount(summary bits below w);
//            nel[c] = w lists the non-empty words in row order
//   pass A2  every entry sets its bit in cw[c(w)]
//   rank 2   popcount prefix over cw: wpre[c]
//   pass B   acc[wpre[c] + popcount(cw[c] & bits below r)] += value
//   write    words expanded to rows in rank order, values copied out
// ---------------------------------------------------------------------------
struct CompactSmem {
  uint32_t* summ;  // NSW: one bit per 32-row word of the slab (kept zero between slabs)
  uint16_t* spre;  // NSW: exclusive popcount prefix of the summary words
  uint32_t* cw;    // umax: row bits of the non-empty words, in row order (kept zero)
  uint16_t* wpre;  // umax: exclusive popcount prefix of cw
  uint16_t* nel;   // umax: word index of each compact word
  unsigned char* acc;
  int* red;        // BLOCK/32 + 1 scan slots
  int NSW, umax;
};

// Compact index of the non-empty 32-row word w.
__device__ __forceinline__ int compact_index(const CompactSmem& sm, uint32_t w) {
  const uint32_t x = w >> 5;
  return (int)sm.spre[x] + __popc(sm.summ[x] & ((1u << (w & 31)) - 1u));
}

template <typename V, typename A, bool PHASED, int BLOCK, int U>
__device__ __forceinline__ void compact_item(const Inputs& in, const Window& W, const Inst* I, const int32_t* offs,
                                             int32_t* __restrict__ out_row, V* __restrict__ out_val,
                                             const CompactSmem& sm, int slab_log2, Counters* ctr_w) {
  const int k = I->k, off = I->ptr_off, j = W.col - I->colbase;
  A* acc = reinterpret_cast<A*>(sm.acc);
  const int64_t S = (int64_t)1 << slab_log2;
  const int64_t span = (int64_t)W.r_hi - W.r_lo;
  const int nsl = span <= 0 ? 0 : (int)((span + S - 1) >> slab_log2);
  int u_done = 0;
  bool bad = false;
  for (int t = 0; t < nsl; ++t) {
    const int lo = W.r_lo + (int)(t * S);
    const int hi = (int)min((int64_t)W.r_hi, (int64_t)lo + S);
    const uint32_t width = (uint32_t)(hi - lo);
    auto seg = [&](int i, int* beg, int* len) {
      int b, e;
      if (W.search < 0) {
        const int32_t* cp = in.cp[off + i];
        b = __ldg(cp + j);
        e = __ldg(cp + j + 1);
      } else {
        const int32_t* o = offs + ((int64_t)W.search * in.kmax + i) * 2;
        b = o[0];
        e = o[1];
      }
      if (nsl > 1 && in.sorted) {
        const int32_t* ri = in.ri[off + i];
        b = lower_bound_i32(ri, b, e, lo);
        e = lower_bound_i32(ri, b, e, hi);
      }
      *beg = b;
      *len = e - b;
    };
    auto none = [](uint32_t, int32_t, V) {};
    // Pass A1: summary bits (a read first: dense items hit few words often).
    int n_ent = 0;  // PHASED: entries this thread met in the slab
    auto mark = [&](int32_t r, V) -> uint32_t {
      const uint32_t rr = (uint32_t)(r - lo);
      if (rr < width) {
        if constexpr (PHASED) ++n_ent;
        const uint32_t w = rr >> 5, bit = 1u << (w & 31);
        if (!(sm.summ[w >> 5] & bit)) atomicOr(&sm.summ[w >> 5], bit);
      }
      return 0u;
    };
    SegCache sc{0, 0, false};
    block_for_each_entry<false, V, BLOCK, U, decltype(seg), decltype(mark), decltype(none), true>(in, k, off, seg,
                                                                                                  mark, none, sc);
    __syncthreads();
    int s_ent = 0;
    if constexpr (PHASED) block_excl_scan<BLOCK>(n_ent, sm.red, &s_ent);
    // Rank 1: thread t owns summary words [t*ps, t*ps + ps).
    const int nwords = (int)((width + 31) >> 5);
    const int nsw = (nwords + 31) >> 5;
    const int ps = (nsw + BLOCK - 1) / BLOCK;
    const int x0 = min(nsw, (int)threadIdx.x * ps), x1 = min(nsw, x0 + ps);
    int loc = 0;
    for (int x = x0; x < x1; ++x) loc += __popc(sm.summ[x]);
    int ne;
    int c = block_excl_scan<BLOCK>(loc, sm.red, &ne);
    const bool ne_fits = ne <= sm.umax && !bad;
    if (ne_fits) {
      for (int x = x0; x < x1; ++x) {
        sm.spre[x] = (uint16_t)c;
        for (uint32_t bits = sm.summ[x]; bits; bits &= bits - 1) sm.nel[c++] = (uint16_t)(x * 32 + __ffs(bits) - 1);
      }
    } else {
      bad = true;
    }
    __syncthreads();
    int slab_u = 0;
    bool fits = false;
    if (ne_fits) {
      // Pass A2: row bits of the compact words.
      auto setbit = [&](int32_t r, V) -> uint32_t {
        const uint32_t rr = (uint32_t)(r - lo);
        if (rr < width) {
          const int cc = compact_index(sm, rr >> 5);
          const uint32_t bit = 1u << (rr & 31);
          if (cc < ne && !(sm.cw[cc] & bit)) atomicOr(&sm.cw[cc], bit);
        }
        return 0u;
      };
      block_for_each_entry<false, V, BLOCK, U>(in, k, off, seg, setbit, none, sc);
      __syncthreads();
      // Rank 2: thread t owns compact words [t*pc, t*pc + pc).
      const int pc = (ne + BLOCK - 1) / BLOCK;
      const int c0 = min(ne, (int)threadIdx.x * pc), c1 = min(ne, c0 + pc);
      int rl = 0;
      for (int cc = c0; cc < c1; ++cc) rl += __popc(sm.cw[cc]);
      int rank = block_excl_scan<BLOCK>(rl, sm.red, &slab_u);
      fits = u_done + slab_u <= sm.umax;
      if (fits) {
        for (int cc = c0; cc < c1; ++cc) {
          sm.wpre[cc] = (uint16_t)rank;
          rank += __popc(sm.cw[cc]);
        }
        for (int q = threadIdx.x; q < slab_u; q += BLOCK) acc[q] = A(0);
      } else {
        bad = true;
      }
      __syncthreads();
    }
    if (fits) {
      // Pass B: values at their rank.
      auto add = [&](int32_t r, V v) -> uint32_t {
        const uint32_t rr = (uint32_t)(r - lo);
        if (rr < width) {
          const int cc = compact_index(sm, rr >> 5);
          if (cc < ne) {
            const uint32_t bits = sm.cw[cc], b = rr & 31;
            const int q = (int)sm.wpre[cc] + __popc(bits & ((1u << b) - 1u));
            if (((bits >> b) & 1u) && q < slab_u) atomicAdd(&acc[q], (A)v);
          }
        }
        return 0u;
      };
      // Ranks past the symbolic count are never written (B holds W.u rows here).
      const bool written = add_values<V, A, PHASED, BLOCK, U>(in, k, off, seg, add, sc, acc, out_val + u_done, slab_u,
                                                              min(slab_u, W.u - u_done), s_ent);
      __syncthreads();
      // Values copied out first; then the rows, expanded from the words into
      // the accumulator's slots (free once the values are out; a word's rows
      // go to consecutive ranks), so that both are written coalesced.
      const int lim = min(slab_u, W.u - u_done);
      int32_t* orow = out_row + u_done;
      V* oval = out_val + u_done;
      if (!written)
        for (int q = threadIdx.x; q < lim; q += BLOCK) oval[q] = (V)acc[q];
      __syncthreads();
      int32_t* rows = reinterpret_cast<int32_t*>(acc);  // slab_u <= umax slots of at least 4 bytes
      for (int cc = threadIdx.x; cc < ne; cc += BLOCK) {
        int q = sm.wpre[cc];
        const int rbase = lo + ((int)sm.nel[cc] << 5);
        for (uint32_t bits = sm.cw[cc]; bits; bits &= bits - 1) rows[q++] = rbase + __ffs(bits) - 1;
      }
      __syncthreads();
      for (int q = threadIdx.x; q < lim; q += BLOCK) orow[q] = rows[q];
      u_done += slab_u;
      __syncthreads();
    }
    // Clear the compact words, then this thread's summary words.
    if (ne_fits)
      for (int cc = threadIdx.x; cc < ne; cc += BLOCK) sm.cw[cc] = 0u;
    for (int x = x0; x < x1; ++x) sm.summ[x] = 0u;
    __syncthreads();
  }
  if (threadIdx.x == 0 && (bad || u_done != W.u)) atomicOr(&ctr_w->err, ERR_INTERNAL);
}

template <int DT, int ACC, int BLOCK, int U>
__global__ void __launch_bounds__(BLOCK, (DT == 0 && ACC == 0) ? 0 : 3) k_num_compact(Inputs in, const Window* __restrict__ win, int nwin,
                                                       const int32_t* __restrict__ offs,
                                                       const int64_t* __restrict__ col_ptr, Outs o, int slab_log2,
                                                       int umax, int only_dtype, Counters* ctr_w) {
  using V = typename std::conditional<DT == 1, double, float>::type;
  using A = typename std::conditional<DT == 1 || ACC == 2, double, float>::type;  // accumulator
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int red[BLOCK / 32 + 1];
  CompactSmem sm;
  sm.NSW = 1 << (slab_log2 - 10);
  sm.umax = umax;
  sm.acc = sm_raw;
  sm.summ = reinterpret_cast<uint32_t*>(sm.acc + (size_t)umax * sizeof(A));
  sm.cw = sm.summ + sm.NSW;
  sm.spre = reinterpret_cast<uint16_t*>(sm.cw + umax);
  sm.wpre = sm.spre + sm.NSW;
  sm.nel = sm.wpre + umax;
  sm.red = red;
  for (int x = threadIdx.x; x < sm.NSW; x += BLOCK) sm.summ[x] = 0u;
  for (int x = threadIdx.x; x < umax; x += BLOCK) sm.cw[x] = 0u;
  __syncthreads();
  Window Wn{};
  if (blockIdx.x < nwin) Wn = win[blockIdx.x];
  for (int wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
    const Window W = Wn;
    if (wi + (int)gridDim.x < nwin) Wn = win[wi + gridDim.x];
    const int q = inst_of(in, W.col);
    const Inst* I = in.inst + q;
    if (only_dtype >= 0 && !item_selected(only_dtype, I)) continue;
    const int64_t out = col_ptr[W.col] - (in.col_inst ? col_ptr[I->colbase] : 0) + W.out_off;
    compact_item<V, A, ACC == 1, BLOCK, U>(in, W, I, offs, out_row_of(o, q) + out, static_cast<V*>(out_val_of(o, q)) + out, sm,
                              slab_log2, ctr_w);
  }
}

// DT: 0 = float values, 1 = double values; ACC: 0 sums in the value type, 1
// float sums in phases, 2 float values summed in double.  A batch of several
// problem kinds runs the kernel once per kind over that kind's records
// (only_dtype: the item filter above).
template <int DT, int ACC, int BLOCK, int U>
__global__ void __launch_bounds__(BLOCK) k_num_bitmap(Inputs in, const Window* __restrict__ win, int nwin,
                                                      const int32_t* __restrict__ offs,
                                                      const int64_t* __restrict__ col_ptr, Outs o, int slab_log2,
                                                      int umax, int only_dtype, Counters* ctr_w) {
  using V = typename std::conditional<DT == 1, double, float>::type;
  using A = typename std::conditional<DT == 1 || ACC == 2, double, float>::type;  // accumulator
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ unsigned long long red[BLOCK / 32 + 1];
  BitmapSmem sm;
  sm.W64 = 1 << (slab_log2 - 6);
  sm.NSW = (sm.W64 + 31) >> 5;
  sm.umax = umax;
  sm.bm = reinterpret_cast<unsigned long long*>(sm_raw);
  sm.acc = reinterpret_cast<unsigned char*>(sm.bm + sm.W64);
  sm.wpre = reinterpret_cast<uint16_t*>(sm.acc + (size_t)umax * sizeof(A));
  sm.summ = reinterpret_cast<uint32_t*>(sm.wpre + ((sm.W64 + 1) & ~1));
  sm.rows = reinterpret_cast<int32_t*>(sm.summ + sm.NSW);
  sm.nel = reinterpret_cast<uint16_t*>(sm.rows + umax);
  sm.red = red;
  for (int x = threadIdx.x; x < sm.W64; x += BLOCK) sm.bm[x] = 0ull;
  for (int x = threadIdx.x; x < sm.NSW; x += BLOCK) sm.summ[x] = 0u;
  __syncthreads();
  // The next item's window record is fetched while the current item runs.
  Window Wn{};
  if (blockIdx.x < nwin) Wn = win[blockIdx.x];
  for (int wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
    const Window W = Wn;
    if (wi + (int)gridDim.x < nwin) Wn = win[wi + gridDim.x];
    const int q = inst_of(in, W.col);
    const Inst* I = in.inst + q;
    if (only_dtype >= 0 && !item_selected(only_dtype, I)) continue;
    const int64_t out = col_ptr[W.col] - (in.col_inst ? col_ptr[I->colbase] : 0) + W.out_off;
    bitmap_item<V, A, ACC == 1, BLOCK, U>(in, W, I, offs, out_row_of(o, q) + out, static_cast<V*>(out_val_of(o, q)) + out, sm,
                             slab_log2, ctr_w);
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
// Resident blocks per SM of a kernel at a block size and dynamic shared
// memory size (registers, shared memory and threads all counted), or 0 on
// error.  Cached: the query is not free.  The launch sets the kernel's
// shared-memory limit itself (another size may have been set since).
int resident_blocks(const void* fn, int block, size_t smem) {
  struct Entry {
    const void* fn;
    int block;
    size_t smem;
    int blocks;
  };
  static std::mutex mu;
  static Entry cache[64];
  static int ncache = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < ncache; ++i)
    if (cache[i].fn == fn && cache[i].block == block && cache[i].smem == smem) return cache[i].blocks;
  int b = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, block, smem) != cudaSuccess) {
    (void)cudaGetLastError();  // not sticky: leave no stale error for the next check
    return 0;
  }
  if (b > 0 && ncache < 64) cache[ncache++] = Entry{fn, block, smem, b};
  return b;
}

// Shared bytes of the flat-bitmap kernel for a slab of 2^slab_log2 rows, umax ranks.
static size_t bitmap_smem_bytes(int slab_log2, int umax, size_t vsize) {
  const size_t w64 = (size_t)1 << (slab_log2 - 6);
  const size_t nsw = (w64 + 31) / 32;
  return w64 * 8 + (size_t)umax * vsize + ((w64 + 1) & ~(size_t)1) * 2 + nsw * 4 + (size_t)umax * 4 +
         (size_t)umax * 2 + 16;
}

// Shared bytes of the compact-table kernel.
static size_t compact_smem_bytes(int slab_log2, int umax, size_t vsize) {
  const size_t nsw = (size_t)1 << (slab_log2 - 10);
  return (size_t)umax * vsize + nsw * 4 + (size_t)umax * 4 + nsw * 2 + (size_t)umax * 4 + 16;
}

template <typename K>
static cudaError_t launch_items(K kern, int block, int blocks_per_sm, const Inputs& in, const Window* win, int n_win,
                                const int32_t* offs, const int64_t* col_ptr, const Outs& out, int slab_log2, int umax,
                                size_t smem, int only_dtype, Counters* ctr_w, const DeviceInfo& dev, cudaStream_t st) {
  if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = dev.sms * blocks_per_sm;
  if (grid > n_win) grid = n_win;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, block, smem, st>>>(in, win, n_win, offs, col_ptr, out, slab_log2, umax, only_dtype, ctr_w);
  return cudaGetLastError();
}

// accumulator: 0 = automatic, 1 = flat bitmap, 2 = compact word table.
// Automatic takes the compact table when more of its blocks are resident per
// SM (the flat bitmap's size follows the slab, the table's follows umax):
// items are latency chains, so items in flight per SM decide the rate.
template <int DT, int ACC>
static cudaError_t launch_num_cta_t(const Inputs& in, const Window* win, int n_win, const int32_t* offs,
                                    const int64_t* col_ptr, const Outs& out, int umax, int accumulator,
                                    int only_dtype, Counters* ctr_w, const DeviceInfo& dev, cudaStream_t st) {
  constexpr size_t VS = (DT == 1 || ACC == 2) ? 8 : 4;  // accumulator bytes
  int slab_log2 = 10;
  while (slab_log2 < NUM_SLAB_LOG2_MAX && ((int64_t)1 << slab_log2) < (int64_t)in.mmax) ++slab_log2;
  const size_t sf = bitmap_smem_bytes(slab_log2, umax, VS), sc = compact_smem_bytes(slab_log2, umax, VS);
  // Small bitmaps leave room for several blocks per SM: 256 threads each
  // (measured best, with 8 entries per lane and round); a bitmap that fills
  // the SM gets one 1024-thread block.
  const bool small = sf <= (size_t)dev.smem_per_sm / 2 - 2048;
  const void* kf = small ? (const void*)k_num_bitmap<DT, ACC, 256, 8> : (const void*)k_num_bitmap<DT, ACC, 1024, 4>;
  const void* kc = (const void*)k_num_compact<DT, ACC, 256, 8>;
  int bf = 0, bc = 0;
  if (accumulator != 2 && sf <= (size_t)dev.smem_optin) bf = resident_blocks(kf, small ? 256 : 1024, sf);
  if (accumulator != 1 && sc <= (size_t)dev.smem_optin) bc = resident_blocks(kc, 256, sc);
  const bool compact = accumulator == 2 || (accumulator == 0 && bc > bf);
  if (compact)
    return launch_items(k_num_compact<DT, ACC, 256, 8>, 256, bc, in, win, n_win, offs, col_ptr, out, slab_log2, umax, sc,
                        only_dtype, ctr_w, dev, st);
  if (small)
    return launch_items(k_num_bitmap<DT, ACC, 256, 8>, 256, bf, in, win, n_win, offs, col_ptr, out, slab_log2, umax, sf,
                        only_dtype, ctr_w, dev, st);
  return launch_items(k_num_bitmap<DT, ACC, 1024, 4>, 1024, bf, in, win, n_win, offs, col_ptr, out, slab_log2, umax, sf,
                      only_dtype, ctr_w, dev, st);
}

// Batches of several problem kinds: after the symbolic phase the
// thread-block items' records are copied, grouped by kind (count, then place
// with warp-aggregated appends; order inside a kind is arbitrary), so that
// each kind's numeric launch reads only its own items.  The windows counted
// by the symbolic kernels are read from the counters (at most `cap`).
__global__ void k_kind_count(Inputs in, const Window* __restrict__ win, int cap, Counters* ctr_w) {
  const int nwin = min(ctr_w->n_windows, cap);
  int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  for (int wi = blockIdx.x * blockDim.x + threadIdx.x; wi < nwin; wi += gridDim.x * blockDim.x) {
    const int kd = item_kind(in.inst + inst_of(in, win[wi].col));
    c0 += kd == 0;
    c1 += kd == 1;
    c2 += kd == 2;
    c3 += kd == 3;
  }
  c0 = warp_sum(c0);
  c1 = warp_sum(c1);
  c2 = warp_sum(c2);
  c3 = warp_sum(c3);
  if ((threadIdx.x & 31) == 0) {
    if (c0) atomicAdd(&ctr_w->kind_n[0], c0);
    if (c1) atomicAdd(&ctr_w->kind_n[1], c1);
    if (c2) atomicAdd(&ctr_w->kind_n[2], c2);
    if (c3) atomicAdd(&ctr_w->kind_n[3], c3);
  }
}

__global__ void k_kind_place(Inputs in, const Window* __restrict__ win, int cap, Window* __restrict__ wsort,
                             Counters* ctr_w) {
  __shared__ int base[4];
  if (threadIdx.x == 0) {
    int b = 0;
    for (int q = 0; q < 4; ++q) {
      base[q] = b;
      b += ctr_w->kind_n[q];
    }
  }
  __syncthreads();
  const int nwin = min(ctr_w->n_windows, cap);
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int w0 = blockIdx.x * blockDim.x; w0 < nwin; w0 += stride) {  // (block-uniform)
    const int wi = w0 + (int)threadIdx.x;
    Window W{};
    int kd = -1;
    if (wi < nwin) {
      W = win[wi];
      kd = item_kind(in.inst + inst_of(in, W.col));
    }
    for (int q = 0; q < 4; ++q) {
      const unsigned m = __ballot_sync(SPK_FULL, kd == q);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      int pos = 0;
      if (lane == leader) pos = atomicAdd(&ctr_w->kind_fill[q], __popc(m));
      pos = __shfl_sync(SPK_FULL, pos, leader);
      if (kd == q) wsort[base[q] + pos + __popc(m & ((1u << lane) - 1u))] = W;
    }
  }
}

int num_cta_kinds(int dt, int f32_kinds) { return (dt != 1 ? (f32_kinds & 7) : 0) | (dt != 0 ? 8 : 0); }

cudaError_t launch_kind_sort(const Inputs& in, const Window* win, int cap, Window* wsort, Counters* ctr_w,
                             const DeviceInfo& dev, cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(&ctr_w->kind_n[0], 0, 8 * sizeof(int32_t), st);  // kind_n, kind_fill
  if (e != cudaSuccess) return e;
  int blocks = (cap + 255) / 256;
  if (blocks > dev.sms * 8) blocks = dev.sms * 8;
  k_kind_count<<<blocks, 256, 0, st>>>(in, win, cap, ctr_w);
  k_kind_place<<<blocks, 256, 0, st>>>(in, win, cap, wsort, ctr_w);
  return cudaGetLastError();
}

cudaError_t launch_num_cta(const Inputs& in, int dt, int f32_kinds, const Window* win, int n_win,
                           const Window* wsort, const int32_t* kind_n, const int32_t* offs, const int64_t* col_ptr,
                           const Outs& out, int window_max, int accumulator, Counters* ctr_w, const DeviceInfo& dev,
                           cudaStream_t st, int* launches) {
  *launches = 0;
  if (n_win <= 0) return cudaSuccess;
  // Float problems: k <= FP32_ACC_TERMS sum in float, up to
  // FP32_PHASED_MAX_K in float by phases, beyond in double; each kind that
  // the batch holds gets its own launch, over its own group of the records
  // (the item filter of kind q, sel[q], only checks that).
  const int kinds = num_cta_kinds(dt, f32_kinds);
  const bool alone = __builtin_popcount(kinds) == 1;
  constexpr int sel[4] = {2, 3, 4, 1};
  int base = 0;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
    if (!((kinds >> q) & 1)) continue;
    const Window* w = alone ? win : wsort + base;
    const int n = alone ? n_win : kind_n[q];
    base += alone ? 0 : kind_n[q];
    if (n <= 0) continue;
    ++*launches;
    const int f = alone ? -1 : sel[q];
    switch (q) {
      case 0: e = launch_num_cta_t<0, 0>(in, w, n, offs, col_ptr, out, window_max, accumulator, f, ctr_w, dev, st); break;
      case 1: e = launch_num_cta_t<0, 1>(in, w, n, offs, col_ptr, out, window_max, accumulator, f, ctr_w, dev, st); break;
      case 2: e = launch_num_cta_t<0, 2>(in, w, n, offs, col_ptr, out, window_max, accumulator, f, ctr_w, dev, st); break;
      default: e = launch_num_cta_t<1, 0>(in, w, n, offs, col_ptr, out, window_max, accumulator, f, ctr_w, dev, st);
    }
  }
  return e;
}

}  // namespace spk
