// spk_symbolic.cu -- a2 of the hot path: nnz(B(:,j)) per column.
//
// Warp class (s_j <= warp_max): see spk_warp.cu.
// CTA class (s_j <= cta_max): one thread block per column, same table with the
//   scrambled (multiplicative) hash.  Emits one numeric work item per column.
// Heavy class: one thread block per column with a shared-memory bitmap of a
//   2^20-row slab (the dense-accumulator form of the symbolic step, which
//   Sec. II-D allows in place of the hash).  Popcounts give nnz(B(:,j)) and
//   cut the column into row windows of at most window_max distinct rows each
//   (Alg. 7/8's sliding windows, sized to shared memory and balanced by count
//   rather than by equal row ranges).
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
    for (int cb = 0; cb < k; cb += 32) {
      const int i = cb + lane;
      int beg = 0, len = 0;
      if (i < k) {
        const int32_t* cp = in.cp[off + i];
        beg = __ldg(cp + j);
        len = __ldg(cp + j + 1) - beg;
      }
      SegWalk w;
      w.init(beg, len, lane);
      for (int e0 = wid * 32 * U; e0 < w.total; e0 += NW * 32 * U) {
        int32_t r[U];
#pragma unroll
        for (int t = 0; t < U; ++t) {
          const int e = e0 + t * 32 + lane;
          const int seg = w.find(e);
          const int idx = w.index_in_input(e, seg);
          r[t] = -1;
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

// The bitmap keeps one pad word after every 32: a thread that scans 32
// consecutive words then starts on its own bank.
__device__ __forceinline__ int bm_pad(int w) { return w + (w >> 5); }
constexpr int MAX_SLAB_WINDOWS = 1100;  // (2^20 rows / 32 bits per word) / (1024 - 32) + 2

template <int BLOCK, int U>
__global__ void __launch_bounds__(BLOCK) k_sym_heavy(Inputs in, const int32_t* __restrict__ list,
                                                     const Counters* __restrict__ ctr, int32_t* __restrict__ u_out,
                                                     Window* __restrict__ win, int32_t* __restrict__ search_list,
                                                     int64_t win_cap, int win_target, int slab_words,
                                                     Counters* ctr_w) {
  extern __shared__ uint32_t bm[];
  __shared__ int red[BLOCK / 32 + 1];
  __shared__ int bnd[MAX_SLAB_WINDOWS + 1];
  __shared__ int cval[MAX_SLAB_WINDOWS + 1];
  __shared__ int s_col_u, s_wbase, s_sbase;
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ncols = ctr->n_heavy;
  const int slab_rows = slab_words * 32;
  for (int c = blockIdx.x; c < ncols; c += gridDim.x) {
    const int g = list[c];
    const Inst* I = in.inst + inst_of(in, g);
    const int k = I->k, off = I->ptr_off, m = I->m, j = g - I->colbase;
    const int nslabs = (int)(((int64_t)m + slab_rows - 1) / slab_rows);
    if (threadIdx.x == 0) s_col_u = 0;
    for (int slab = 0; slab < nslabs; ++slab) {
      const int lo = slab * slab_rows;
      const int hi = (int)min((int64_t)m, (int64_t)lo + slab_rows);
      const int words = (hi - lo + 31) >> 5;
      {
        uint4* bm4 = reinterpret_cast<uint4*>(bm);
        const int w4 = (bm_pad(words) + 3) >> 2;  // the bitmap buffer is rounded up to whole uint4
        for (int p = threadIdx.x; p < w4; p += BLOCK) bm4[p] = make_uint4(0u, 0u, 0u, 0u);
      }
      __syncthreads();
      for (int cb = 0; cb < k; cb += 32) {
        const int i = cb + lane;
        int beg = 0, len = 0;
        if (i < k) {
          const int32_t* cp = in.cp[off + i];
          int b = __ldg(cp + j), e = __ldg(cp + j + 1);
          if (nslabs > 1) {
            const int32_t* ri = in.ri[off + i];
            b = lower_bound_i32(ri, b, e, lo);
            e = lower_bound_i32(ri, b, e, hi);
          }
          beg = b;
          len = e - b;
        }
        SegWalk w;
        w.init(beg, len, lane);
        for (int e0 = wid * 32 * U; e0 < w.total; e0 += NW * 32 * U) {
          int32_t r[U];
#pragma unroll
          for (int t = 0; t < U; ++t) {
            const int e = e0 + t * 32 + lane;
            const int seg = w.find(e);
            const int idx = w.index_in_input(e, seg);
            r[t] = -1;
            if (e < w.total) r[t] = __ldg(in.ri[off + cb + seg] + idx);
          }
#pragma unroll
          for (int t = 0; t < U; ++t) {
            const int rr = r[t] - lo;
            if (r[t] >= 0 && rr < hi - lo) atomicOr(&bm[bm_pad(rr >> 5)], 1u << (rr & 31));
          }
        }
      }
      __syncthreads();
      // Popcount prefix over the slab's words (thread t owns a contiguous run).
      const int per = (words + BLOCK - 1) / BLOCK;
      const int w0 = threadIdx.x * per;
      int loc = 0;
      for (int t = 0; t < per; ++t)
        if (w0 + t < words) loc += __popc(bm[bm_pad(w0 + t)]);
      int slab_u;
      const int ex = block_excl_scan<BLOCK>(loc, red, &slab_u);
      const int P = slab_u == 0 ? 0 : (slab_u + win_target - 1) / win_target;
      const bool whole = (nslabs == 1 && P == 1);
      if (P > MAX_SLAB_WINDOWS) {  // win_target is validated on the host; guard anyway
        if (threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);
      } else if (P > 0) {
        if (threadIdx.x == 0) {
          bnd[0] = 0;
          cval[0] = 0;
          bnd[P] = words;
          cval[P] = slab_u;
          s_wbase = atomicAdd(&ctr_w->n_windows, P);
          s_sbase = whole ? -1 : atomicAdd(&ctr_w->n_search, P);
        }
        int run = ex;
        for (int t = 0; t < per; ++t) {
          const int wd = w0 + t;
          if (wd >= words) break;
          const int before = run;
          run += __popc(bm[bm_pad(wd)]);
          const int pb = before / win_target, pa = run / win_target;
          if (pa > pb && pa >= 1 && pa <= P - 1) {
            bnd[pa] = wd + 1;
            cval[pa] = run;
          }
        }
        __syncthreads();
        const int col_u = s_col_u;
        for (int p = threadIdx.x; p < P; p += BLOCK) {
          const int wi = s_wbase + p;
          if (wi < win_cap && (whole || s_sbase + p < win_cap)) {
            Window w;
            w.col = g;
            w.r_lo = whole ? 0 : lo + 32 * bnd[p];
            w.r_hi = whole ? m : (int)min((int64_t)hi, (int64_t)lo + 32 * (int64_t)bnd[p + 1]);
            w.u = cval[p + 1] - cval[p];
            w.out_off = col_u + cval[p];
            w.search = whole ? -1 : s_sbase + p;
            win[wi] = w;
            if (!whole) search_list[s_sbase + p] = wi;
          } else {
            atomicOr(&ctr_w->err, ERR_WINDOW_CAP);
          }
        }
      }
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

cudaError_t launch_sym_heavy(const Inputs& in, const int32_t* list, const Counters* ctr, int32_t* u, Window* win,
                             int32_t* search_list, int64_t win_cap, Counters* ctr_w, int window_max,
                             const DeviceInfo& dev, cudaStream_t st) {
  const int slab_rows = (int)(in.mmax < (1 << SLAB_BITS) ? in.mmax : (1 << SLAB_BITS));
  const int slab_words = (slab_rows + 31) / 32 > 0 ? (slab_rows + 31) / 32 : 1;
  const int padded = slab_words + slab_words / 32 + 1;
  const size_t smem = (size_t)((padded + 3) / 4 * 4) * sizeof(uint32_t);
  auto kern = k_sym_heavy<HEAVY_BLOCK, 4>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const size_t static_smem = sizeof(int) * (2 * (MAX_SLAB_WINDOWS + 1) + HEAVY_BLOCK / 32 + 4);
  const int grid = dev.sms * blocks_per_sm(dev, smem + static_smem, HEAVY_BLOCK);
  kern<<<grid, HEAVY_BLOCK, smem, st>>>(in, list, ctr, u, win, search_list, win_cap, window_max - 32, slab_words,
                                        ctr_w);
  return cudaGetLastError();
}

}  // namespace spk
