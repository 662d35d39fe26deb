// spk_symbolic.cu -- a2 of the hot path: nnz(B(:,j)) per column.
//
// Warp class (s_j <= warp_max): see spk_warp.cu.
// CTA class (s_j <= cta_max): one thread block per column, same table with the
//   scrambled (multiplicative) hash.  Emits one numeric work item per column.
// Heavy class: one thread block per column with a shared-memory bitmap of a
//   slab of up to 2^20 rows (the dense-accumulator form of the symbolic step,
//   which Sec. II-D allows in place of the hash).  Popcounts give nnz(B(:,j))
//   and cut the column into row windows of fewer than window_max distinct rows
//   each (Alg. 7/8's sliding windows, sized to shared memory and balanced by
//   count rather than by equal row ranges).  An optional compact form
//   (k_sym_heavy_compact) does the same from a summary bit per 32-row word
//   and a bounded table of non-empty words.
#include "spk_common.cuh"
#include "spk_launch.h"

namespace spk {

template <int BLOCK, int U>
__global__ void __launch_bounds__(BLOCK) k_sym_cta(Inputs in, const int32_t* __restrict__ list,
                                                   const int32_t* __restrict__ s_arr, const Counters* __restrict__ ctr,
                                                   int32_t* __restrict__ u_out, Window* __restrict__ win,
                                                   int64_t win_cap, int tmax, Counters* ctr_w) {
  extern __shared__ int32_t keys[];
  __shared__ int red[BLOCK / 32 + 1];
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ncols = ctr->n_cta;
  for (int c = blockIdx.x; c < ncols; c += gridDim.x) {
    const int g = list[c];
    const Inst* I = in.inst + inst_of(in, g);
    const int k = I->k, off = I->ptr_off, j = g - I->colbase;
    const int s = s_arr[g];
    const int q = max(6, ceil_log2(2 * s));
    const int T = 1 << q;
    if (T > tmax) {
      if (threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);
      continue;
    }
    for (int p = threadIdx.x; p < T; p += BLOCK) keys[p] = -1;
    __syncthreads();
    int newc = 0;
    const int nch = (k + 31) >> 5;
    const int groups = min(nch, NW);
    const int per = NW / groups;
    const int gid = wid / per, lw = wid - gid * per;
    for (int cb = gid * 32; gid < groups && cb < k; cb += groups * 32) {
      const int i = cb + lane;
      int beg = 0, len = 0;
      if (i < k) {
        const int32_t* cp = in.cp[off + i];
        beg = __ldg(cp + j);
        len = __ldg(cp + j + 1) - beg;
      }
      SegWalk w;
      w.init(beg, len, lane);
      for (int e0 = lw * 32 * U; e0 < w.total; e0 += per * 32 * U) {
        int32_t r[U];
#pragma unroll
        for (int t = 0; t < U; ++t) {
          r[t] = -1;
          if (e0 + t * 32 >= w.total) continue;  // (warp-uniform) slot wholly past the chunk's end
          const int e = e0 + t * 32 + lane;
          const int seg = w.find(e);
          const int idx = w.index_in_input(e, seg);
          if (e < w.total) r[t] = __ldg(in.ri[off + cb + seg] + idx);
        }
#pragma unroll
        for (int t = 0; t < U; ++t) {
          if (r[t] < 0) continue;
          uint32_t h = hash_scrambled(r[t], q);
          for (int probes = 0; probes < T; ++probes) {  // T > s_j keys: an empty slot is always found
            const int old = atomicCAS(&keys[h], -1, r[t]);
            if (old == -1) {
              ++newc;
              break;
            }
            if (old == r[t]) break;
            h = (h + 1) & (T - 1);
          }
        }
      }
    }
    int total;
    block_excl_scan<BLOCK>(newc, red, &total);
    if (threadIdx.x == 0) {
      u_out[g] = total;
      const int wi = atomicAdd(&ctr_w->n_windows, 1);
      if (wi < win_cap) {
        Window w;
        w.col = g;
        w.r_lo = 0;
        w.r_hi = I->m;
        w.u = total;
        w.out_off = 0;
        w.search = -1;
        win[wi] = w;
      } else {
        atomicOr(&ctr_w->err, ERR_WINDOW_CAP);
      }
    }
    __syncthreads();
  }
}

constexpr int HEAVY_BLOCK = 1024;
constexpr int MAX_SLAB_WINDOWS = 1100;  // 2^20 rows / (1024 - 64) + 2
constexpr int FILTER_WINDOWS = 3;       // see the window records below
constexpr int FILTER_SEG = 64;

// Heavy columns: one thread block per column (from a work counter, columns
// with s_j > BIG_S first).  Rows of one slab of 2^20 rows
// at a time go into a 64-bit-word bitmap plus a summary bitmap (one bit per
// non-empty word), both kept zero between slabs, so the work per slab grows
// with the rows present, not with the slab.  The popcount prefix over the
// non-empty words gives nnz(B(:,j)) and cuts the column into windows of at
// most win_target + 63 distinct rows (boundaries on 64-row words).
template <int BLOCK, int U>
__global__ void __launch_bounds__(BLOCK, BLOCK >= 1024 ? 1 : 4) k_sym_heavy(Inputs in, const int32_t* __restrict__ list,
                                                     const int32_t* __restrict__ s_arr,
                                                     const Counters* __restrict__ ctr, int32_t* __restrict__ u_out,
                                                     Window* __restrict__ win, int32_t* __restrict__ search_list,
                                                     int64_t win_cap, int win_target, int slab_log2,
                                                     Counters* ctr_w) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int red[BLOCK / 32 + 1];
  __shared__ int bnd[MAX_SLAB_WINDOWS + 1];
  __shared__ int cval[MAX_SLAB_WINDOWS + 1];
  __shared__ int s_col_u, s_wbase, s_sbase;
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int W64 = 1 << (slab_log2 - 6);
  const int NSW = (W64 + 31) >> 5;
  unsigned long long* bm = reinterpret_cast<unsigned long long*>(sm_raw);
  uint32_t* summ = reinterpret_cast<uint32_t*>(bm + W64);
  for (int x = threadIdx.x; x < W64; x += BLOCK) bm[x] = 0ull;
  for (int x = threadIdx.x; x < NSW; x += BLOCK) summ[x] = 0u;
  __syncthreads();
  const int n_big = ctr->n_big;
  const int ncols = n_big + ctr->n_heavy;
  const int slab_rows = 1 << slab_log2;
  // Columns are handed out by a work counter, the largest list first; the
  // next column's ticket is taken while the current one runs.
  __shared__ int s_tk[2];
  if (threadIdx.x == 0) s_tk[0] = atomicAdd(&ctr_w->heavy_next, 1);
  __syncthreads();
  for (int it = 0;; ++it) {
    const int c = s_tk[it & 1];
    if (c >= ncols) break;
    if (threadIdx.x == 0) s_tk[(it + 1) & 1] = atomicAdd(&ctr_w->heavy_next, 1);
    const int g = c < n_big ? list[in.ncols + c] : list[c - n_big];
    const Inst* I = in.inst + inst_of(in, g);
    const int k = I->k, off = I->ptr_off, m = I->m, j = g - I->colbase;
    const int nslabs = (int)(((int64_t)m + slab_rows - 1) / slab_rows);
    if (threadIdx.x == 0) s_col_u = 0;
    for (int slab = 0; slab < nslabs; ++slab) {
      const int lo = slab * slab_rows;
      const int hi = (int)min((int64_t)m, (int64_t)lo + slab_rows);
      const uint32_t width = (uint32_t)(hi - lo);
      // Chunks of 32 inputs side by side: `groups` of `wpg` warps.
      const int nch = (k + 31) >> 5;
      const int groups = min(nch, NW);
      const int wpg = NW / groups;
      const int gid = wid / wpg, lw = wid - gid * wpg;
      for (int cb = gid * 32; gid < groups && cb < k; cb += groups * 32) {
        const int i = cb + lane;
        int beg = 0, len = 0;
        const int32_t* rp = nullptr;  // this lane's input segment (its rows from beg)
        if (i < k) {
          const int32_t* cp = in.cp[off + i];
          const int32_t* ri = in.ri[off + i];
          int b = __ldg(cp + j), e = __ldg(cp + j + 1);
          if (nslabs > 1 && in.sorted) {  // unordered inputs: the whole column, rows outside the slab skipped
            b = lower_bound_i32(ri, b, e, lo);
            e = lower_bound_i32(ri, b, e, hi);
          }
          beg = b;
          len = e - b;
          rp = ri + b;
        }
        ChunkMap cm;
        const int nvalid = min(32, k - cb);
        cm.init(beg, len, lane, nvalid);
        // Sets the row bits of U rows (r < 0: none), then the summary marks they call for.
        auto set_rows = [&](const int32_t (&r)[U]) {
          bool fresh[U];
#pragma unroll
          for (int t = 0; t < U; ++t) {
            const uint32_t rr = (uint32_t)(r[t] - lo);
            fresh[t] = r[t] >= 0 && rr < width && set_row_bit(bm, rr);
          }
#pragma unroll
          for (int t = 0; t < U; ++t)
            if (fresh[t]) {
              const uint32_t w = (uint32_t)(r[t] - lo) >> 6;
              atomicOr(&summ[w >> 5], 1u << (w & 31));
            }
        };
        if (!cm.equal && cm.total >= SEG_MAJOR_MIN * nvalid) {
          // Long ragged segments: each warp walks whole segments (no per-entry search).
          for (int sgi = lw; sgi < nvalid; sgi += wpg) {
            const int ls = __shfl_sync(SPK_FULL, len, sgi);
            const int32_t* p = reinterpret_cast<const int32_t*>(
                __shfl_sync(SPK_FULL, reinterpret_cast<unsigned long long>(rp), sgi));
            for (int e0 = 0; e0 < ls; e0 += 32 * U) {
              int32_t r[U];
#pragma unroll
              for (int t = 0; t < U; ++t) {
                const int o = e0 + t * 32 + lane;
                r[t] = (e0 + t * 32 < ls && o < ls) ? __ldg(p + o) : -1;
              }
              set_rows(r);
            }
          }
          continue;
        }
        if (lw * 32 * U >= cm.total) continue;  // (warp-uniform) no entries for this warp
        for (int e0 = lw * 32 * U; e0 < cm.total; e0 += wpg * 32 * U) {
          int32_t r[U];
#pragma unroll
          for (int t = 0; t < U; ++t) {
            r[t] = -1;
            if (e0 + t * 32 >= cm.total) continue;  // (warp-uniform) slot wholly past the chunk's end
            const int e = e0 + t * 32 + lane;
            int o;
            const int sg = cm.seg_off(e, &o);
            const int32_t* p = reinterpret_cast<const int32_t*>(
                __shfl_sync(SPK_FULL, reinterpret_cast<unsigned long long>(rp), sg & 31));
            if (e < cm.total) r[t] = __ldg(p + o);
          }
          // All bit sets of the round first, then the summary marks they call for.
          set_rows(r);
        }
      }
      __syncthreads();
      // Popcount prefix over the non-empty words: thread t owns bitmap words
      // [t*per, t*per + per) (a power of two <= 32, inside one summary word);
      // `mine` holds which of them are non-empty.
      const int nwords = (int)((width + 63) >> 6);
      int per = 1;
      while (per * BLOCK < nwords && per < 32) per <<= 1;
      if (per * BLOCK < nwords && threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);  // host sizing prevents it
      const int w0 = threadIdx.x * per;
      uint32_t mine = 0u;
      if (w0 < nwords) {
        mine = summ[w0 >> 5] >> (w0 & 31);
        if (per < 32) mine &= (1u << per) - 1u;
      }
      int loc = 0;
      for (uint32_t bits = mine; bits; bits &= bits - 1) loc += __popcll(bm[w0 + __ffs(bits) - 1]);
      int slab_u;
      const int ex = block_excl_scan<BLOCK>(loc, red, &slab_u);
      const int P = slab_u == 0 ? 0 : (slab_u + win_target - 1) / win_target;
      const bool whole = (nslabs == 1 && P == 1);
      // Windows read per-input offsets found by binary search when the inputs
      // are sorted, except in a column of one slab cut into at most
      // FILTER_WINDOWS windows whose input segments are short (s_j <=
      // FILTER_SEG * k): there every window reads the whole column and keeps
      // its rows, since a few extra passes over short segments cost less
      // than k binary searches per window.  Unordered inputs always do so.
      const bool searched = !whole && in.sorted &&
                            (nslabs > 1 || P > FILTER_WINDOWS || (int64_t)s_arr[g] > (int64_t)FILTER_SEG * k);
      if (P > MAX_SLAB_WINDOWS) {  // win_target is validated on the host; guard anyway
        if (threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);
      } else if (P > 0) {
        if (threadIdx.x == 0) {
          bnd[0] = 0;
          cval[0] = 0;
          bnd[P] = nwords;
          cval[P] = slab_u;
          s_wbase = atomicAdd(&ctr_w->n_windows, P);
          s_sbase = searched ? atomicAdd(&ctr_w->n_search, P) : -1;
        }
        // Window p starts after the word in which the running count first
        // reaches p * win_target.
        if (P > 1) {
          int run = ex;
          for (uint32_t bits = mine; bits; bits &= bits - 1) {
            const int wd = w0 + __ffs(bits) - 1;
            const int before = run;
            run += __popcll(bm[wd]);
            const int pb = before / win_target, pa = run / win_target;
            if (pa > pb && pa >= 1 && pa <= P - 1) {
              bnd[pa] = wd + 1;
              cval[pa] = run;
            }
          }
        }
        __syncthreads();
        const int col_u = s_col_u;
        for (int p = threadIdx.x; p < P; p += BLOCK) {
          const int wi = s_wbase + p;
          if (wi < win_cap && (!searched || s_sbase + p < win_cap)) {
            Window w;
            w.col = g;
            w.r_lo = whole ? 0 : lo + 64 * bnd[p];
            w.r_hi = whole ? m : (int)min((int64_t)hi, (int64_t)lo + 64 * (int64_t)bnd[p + 1]);
            w.u = cval[p + 1] - cval[p];
            w.out_off = col_u + cval[p];
            w.search = searched ? s_sbase + p : -1;
            win[wi] = w;
            if (searched) search_list[s_sbase + p] = wi;
          } else {
            atomicOr(&ctr_w->err, ERR_WINDOW_CAP);
          }
        }
      }
      // Clear this thread's words, then the summary, for the next slab or column.
      for (uint32_t bits = mine; bits; bits &= bits - 1) bm[w0 + __ffs(bits) - 1] = 0ull;
      __syncthreads();
      for (int x = threadIdx.x; x < ((nwords + 31) >> 5); x += BLOCK) summ[x] = 0u;
      if (threadIdx.x == 0) s_col_u += slab_u;
      __syncthreads();
    }
    if (threadIdx.x == 0) u_out[g] = s_col_u;
    __syncthreads();
  }
}

// Heavy columns, compact form: the same count and window cuts from a summary
// bit per 32-row word and a table of at most `cap` non-empty words, instead of
// a bitmap over the whole slab (128 KB at 2^20 rows), so that several columns
// are in flight per SM.  Per slab:
//
//   pass A1  every entry sets its word's summary bit
//   rank 1   popcount prefix over the summary words; the slab is cut into
//            sub-ranges of whole summary words holding at most `cap`
//            non-empty words each (one sub-range unless the column is huge)
//   per sub-range:
//     pass A2  every entry of the sub-range sets its row bit in the table
//              (sorted inputs: the sub-range's slice found by binary search)
//     rank 2   popcount prefix over the table: distinct rows, and the window
//              cuts where the running count reaches multiples of win_target
//              (on 32-row words: a window holds at most win_target + 31 rows)
template <int BLOCK, int U>
__global__ void __launch_bounds__(BLOCK) k_sym_heavy_compact(Inputs in, const int32_t* __restrict__ list,
                                                             const int32_t* __restrict__ s_arr,
                                                             const Counters* __restrict__ ctr,
                                                             int32_t* __restrict__ u_out, Window* __restrict__ win,
                                                             int32_t* __restrict__ search_list, int64_t win_cap,
                                                             int win_target, int slab_log2, int cap,
                                                             Counters* ctr_w) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int red[BLOCK / 32 + 1];
  __shared__ int bnd[MAX_SLAB_WINDOWS + 1];
  __shared__ int cval[MAX_SLAB_WINDOWS + 1];
  __shared__ int s_col_u, s_wbase, s_sbase;
  const int NSW = 1 << (slab_log2 - 10);
  uint32_t* summ = reinterpret_cast<uint32_t*>(sm_raw);     // NSW: one bit per 32-row word (kept zero)
  uint32_t* cw = summ + NSW;                                // cap: row bits of non-empty words (kept zero)
  int32_t* spre = reinterpret_cast<int32_t*>(cw + cap);     // NSW: exclusive prefix of non-empty words
  int32_t* srs = spre + NSW;                                // NSW: first summary word of each sub-range
  for (int x = threadIdx.x; x < NSW; x += BLOCK) summ[x] = 0u;
  for (int x = threadIdx.x; x < cap; x += BLOCK) cw[x] = 0u;
  __syncthreads();
  const int n_big = ctr->n_big;
  const int ncols = n_big + ctr->n_heavy;
  const int slab_rows = 1 << slab_log2;
  const int capw = cap - 32;  // a sub-range starts below capw words: it ends below cap
  // Columns are handed out by a work counter, the largest list first; the
  // next column's ticket is taken while the current one runs.
  __shared__ int s_tk[2];
  if (threadIdx.x == 0) s_tk[0] = atomicAdd(&ctr_w->heavy_next, 1);
  __syncthreads();
  for (int it = 0;; ++it) {
    const int c = s_tk[it & 1];
    if (c >= ncols) break;
    if (threadIdx.x == 0) s_tk[(it + 1) & 1] = atomicAdd(&ctr_w->heavy_next, 1);
    const int g = c < n_big ? list[in.ncols + c] : list[c - n_big];
    const Inst* I = in.inst + inst_of(in, g);
    const int k = I->k, off = I->ptr_off, m = I->m, j = g - I->colbase;
    const int nslabs = (int)(((int64_t)m + slab_rows - 1) / slab_rows);
    if (threadIdx.x == 0) s_col_u = 0;
    for (int slab = 0; slab < nslabs; ++slab) {
      const int lo = slab * slab_rows;
      const int hi = (int)min((int64_t)m, (int64_t)lo + slab_rows);
      const uint32_t width = (uint32_t)(hi - lo);
      // The column's entries of input i in rows [a, b) of this slab.
      auto seg_rows = [&](int i, int a, int b, int* beg, int* len) {
        const int32_t* cp = in.cp[off + i];
        int x = __ldg(cp + j), y = __ldg(cp + j + 1);
        if (in.sorted && (a > 0 || b < m)) {  // unordered inputs: all entries, rows outside skipped
          const int32_t* ri = in.ri[off + i];
          x = lower_bound_i32(ri, x, y, a);
          y = lower_bound_i32(ri, x, y, b);
        }
        *beg = x;
        *len = y - x;
      };
      auto seg_slab = [&](int i, int* beg, int* len) { seg_rows(i, nslabs > 1 ? lo : 0, nslabs > 1 ? hi : m, beg, len); };
      auto none = [](uint32_t, int32_t, float) {};
      auto mark = [&](int32_t r, float) -> uint32_t {
        const uint32_t rr = (uint32_t)(r - lo);
        if (rr < width) {
          const uint32_t w = rr >> 5, bit = 1u << (w & 31);
          if (!(summ[w >> 5] & bit)) atomicOr(&summ[w >> 5], bit);
        }
        return 0u;
      };
      SegCache sc{0, 0, false};
      block_for_each_entry<false, float, BLOCK, U>(in, k, off, seg_slab, mark, none, sc);
      __syncthreads();
      // Rank 1: thread t owns summary words [x0, x1).
      const int nwords = (int)((width + 31) >> 5);
      const int nsw = (nwords + 31) >> 5;
      const int ps = (nsw + BLOCK - 1) / BLOCK;
      const int x0 = min(nsw, (int)threadIdx.x * ps), x1 = min(nsw, x0 + ps);
      int loc = 0;
      for (int x = x0; x < x1; ++x) loc += __popc(summ[x]);
      int ne;
      int run = block_excl_scan<BLOCK>(loc, red, &ne);
      {
        int prev_sub = x0 > 0 ? (run - __popc(summ[x0 - 1])) / capw : -1;  // sub-range of word x0 - 1
        for (int x = x0; x < x1; ++x) {
          const int sub = run / capw;
          if (sub != prev_sub) srs[sub] = x;  // the prefix grows by <= 32 <= capw per word: no sub-range skipped
          prev_sub = sub;
          spre[x] = run;
          run += __popc(summ[x]);
        }
      }
      __syncthreads();
      const int R = spre[nsw - 1] / capw + 1;
      int slab_run = 0;
      for (int sub = 0; sub < R; ++sub) {
        const int xa = srs[sub], xb = sub + 1 < R ? srs[sub + 1] : nsw;
        const int cbase = spre[xa];
        const int nsub = (xb < nsw ? spre[xb] : ne) - cbase;
        if (nsub > cap) {  // cannot happen (see capw); never index past the table
          if (threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);
          continue;
        }
        // Pass A2: row bits of the sub-range's non-empty words.
        auto setbit = [&](int32_t r, float) -> uint32_t {
          const uint32_t rr = (uint32_t)(r - lo);
          if (rr < width) {
            const uint32_t w = rr >> 5;
            const int x = (int)(w >> 5);
            if (x >= xa && x < xb) {
              const int cc = spre[x] + __popc(summ[x] & ((1u << (w & 31)) - 1u)) - cbase;
              const uint32_t bit = 1u << (rr & 31);
              if (cc < nsub && !(cw[cc] & bit)) atomicOr(&cw[cc], bit);  // cc < nsub: pass A1 set w's bit
            }
          }
          return 0u;
        };
        if (R == 1) {
          block_for_each_entry<false, float, BLOCK, U>(in, k, off, seg_slab, setbit, none, sc);
        } else {
          const int ra = lo + xa * 1024, rb = (int)min((int64_t)hi, (int64_t)lo + (int64_t)xb * 1024);
          auto seg_sub = [&](int i, int* beg, int* len) { seg_rows(i, ra, rb, beg, len); };
          SegCache sc2{0, 0, false};
          block_for_each_entry<false, float, BLOCK, U>(in, k, off, seg_sub, setbit, none, sc2);
        }
        __syncthreads();
        // Rank 2, by summary word: thread t owns summary words [y0, y1) of the sub-range.
        const int nx = xb - xa;
        const int ps2 = (nx + BLOCK - 1) / BLOCK;
        const int y0 = xa + min(nx, (int)threadIdx.x * ps2), y1 = xa + min(nx, (int)threadIdx.x * ps2 + ps2);
        int l2 = 0;
        for (int x = y0; x < y1; ++x) {
          int cc = spre[x] - cbase;
          for (int t = __popc(summ[x]); t > 0; --t) l2 += __popc(cw[cc++]);
        }
        int sub_u;
        int run2 = slab_run + block_excl_scan<BLOCK>(l2, red, &sub_u);
        // Window p starts after the word in which the running count first reaches p * win_target.
        for (int x = y0; x < y1; ++x) {
          int cc = spre[x] - cbase;
          for (uint32_t bits = summ[x]; bits; bits &= bits - 1) {
            const int wd = x * 32 + __ffs(bits) - 1;
            const int before = run2;
            run2 += __popc(cw[cc++]);
            const int pb = before / win_target, pa = run2 / win_target;
            if (pa > pb && pa >= 1 && pa <= MAX_SLAB_WINDOWS - 1) {
              bnd[pa] = wd + 1;
              cval[pa] = run2;
            }
          }
        }
        __syncthreads();
        for (int cc = threadIdx.x; cc < nsub; cc += BLOCK) cw[cc] = 0u;
        slab_run += sub_u;
        __syncthreads();
      }
      const int slab_u = slab_run;
      const int P = slab_u == 0 ? 0 : (slab_u + win_target - 1) / win_target;
      const bool whole = (nslabs == 1 && P == 1);
      // As in the bitmap form: split windows of sorted inputs are searched
      // unless the column has one slab, at most FILTER_WINDOWS windows and
      // short segments.
      const bool searched = !whole && in.sorted &&
                            (nslabs > 1 || P > FILTER_WINDOWS || (int64_t)s_arr[g] > (int64_t)FILTER_SEG * k);
      if (P > MAX_SLAB_WINDOWS) {
        if (threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);
      } else if (P > 0) {
        if (threadIdx.x == 0) {
          bnd[0] = 0;
          cval[0] = 0;
          bnd[P] = nwords;
          cval[P] = slab_u;
          s_wbase = atomicAdd(&ctr_w->n_windows, P);
          s_sbase = searched ? atomicAdd(&ctr_w->n_search, P) : -1;
        }
        __syncthreads();
        const int col_u = s_col_u;
        for (int p = threadIdx.x; p < P; p += BLOCK) {
          const int wi = s_wbase + p;
          if (wi < win_cap && (!searched || s_sbase + p < win_cap)) {
            Window w;
            w.col = g;
            w.r_lo = whole ? 0 : lo + 32 * bnd[p];
            w.r_hi = whole ? m : (int)min((int64_t)hi, (int64_t)lo + 32 * (int64_t)bnd[p + 1]);
            w.u = cval[p + 1] - cval[p];
            w.out_off = col_u + cval[p];
            w.search = searched ? s_sbase + p : -1;
            win[wi] = w;
            if (searched) search_list[s_sbase + p] = wi;
          } else {
            atomicOr(&ctr_w->err, ERR_WINDOW_CAP);
          }
        }
      }
      for (int x = x0; x < x1; ++x) summ[x] = 0u;
      __syncthreads();
      if (threadIdx.x == 0) s_col_u += slab_u;
      __syncthreads();
    }
    if (threadIdx.x == 0) u_out[g] = s_col_u;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
static int blocks_per_sm(const DeviceInfo& dev, size_t smem_per_block, int threads_per_block) {
  const size_t reserve = 1024;  // per-block system shared memory
  int b = (int)(dev.smem_per_sm / (smem_per_block + reserve));
  int bt = 2048 / threads_per_block;
  if (b > bt) b = bt;
  if (b > 32) b = 32;
  return b < 1 ? 1 : b;
}

static int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

cudaError_t launch_sym_cta(const Inputs& in, const int32_t* list, const int32_t* s, const Counters* ctr, int32_t* u,
                           Window* win, int64_t win_cap, Counters* ctr_w, int cta_max, const DeviceInfo& dev,
                           cudaStream_t st) {
  constexpr int BLOCK = 512;
  const int tmax = pow2_at_least(2 * cta_max);
  const size_t smem = (size_t)tmax * sizeof(int32_t);
  auto kern = k_sym_cta<BLOCK, 4>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = dev.sms * blocks_per_sm(dev, smem, BLOCK);
  kern<<<grid, BLOCK, smem, st>>>(in, list, s, ctr, u, win, win_cap, tmax, ctr_w);
  return cudaGetLastError();
}

constexpr int HEAVY_CAP = 4096;  // non-empty 32-row words per sub-range of the compact form

// accumulator: 0 or 1 = slab bitmap, 2 = compact table.  Unlike the numeric
// items, the automatic choice keeps the slab bitmap even when it holds the
// SM: a heavy column has thousands of entries or more, enough for a
// 1024-thread block, and the largest R-MAT columns (10^5 distinct rows and
// more) need dozens of compact sub-ranges, each with 2k binary searches on
// the one block that owns the column (measured: R-MAT k=64 scale 20, heavy
// symbolic 7.2 ms as a bitmap, about 13 ms compact).
cudaError_t launch_sym_heavy(const Inputs& in, const int32_t* list, const int32_t* s, const Counters* ctr, int32_t* u,
                             Window* win, int32_t* search_list, int64_t win_cap, Counters* ctr_w, int window_max,
                             int accumulator, const DeviceInfo& dev, cudaStream_t st) {
  int slab_log2 = 10;
  while (slab_log2 < SLAB_BITS && ((int64_t)1 << slab_log2) < (int64_t)in.mmax) ++slab_log2;
  const size_t w64 = (size_t)1 << (slab_log2 - 6);
  const size_t smem = w64 * 8 + ((w64 + 31) / 32) * 4 + 16;
  const size_t nsw = (size_t)1 << (slab_log2 - 10);
  const size_t smem_c = nsw * 4 + (size_t)HEAVY_CAP * 4 + nsw * 8 + 16;
  // Small slabs: 256-thread blocks, several columns in flight per SM; a slab
  // bitmap that fills the SM: one 1024-thread block.
  const bool small = smem * 2 + 4096 <= (size_t)dev.smem_per_sm / 2;
  auto kern = small ? k_sym_heavy<256, 8> : k_sym_heavy<HEAVY_BLOCK, 8>;
  auto kern_c = k_sym_heavy_compact<256, 8>;
  const int block = small ? 256 : HEAVY_BLOCK;
  int bf = 0, bc = 0;
  if (accumulator != 2 && smem <= (size_t)dev.smem_optin) bf = resident_blocks((const void*)kern, block, smem);
  if (accumulator == 2) bc = resident_blocks((const void*)kern_c, 256, smem_c);
  if (accumulator == 2) {
    if (bc < 1) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(kern_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
    if (e != cudaSuccess) return e;
    // Windows end on 32-row words: a window holds at most win_target + 31 rows.
    kern_c<<<dev.sms * bc, 256, smem_c, st>>>(in, list, s, ctr, u, win, search_list, win_cap, window_max - 64,
                                             slab_log2, HEAVY_CAP, ctr_w);
    return cudaGetLastError();
  }
  if (bf < 1) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // Windows end on 64-row words: a window holds at most win_target + 63 rows.
  kern<<<dev.sms * bf, block, smem, st>>>(in, list, s, ctr, u, win, search_list, win_cap, window_max - 64, slab_log2,
                                          ctr_w);
  return cudaGetLastError();
}

}  // namespace spk
