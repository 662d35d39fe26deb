// spk_numeric.cu -- a4/a5 of the hot path: accumulate values and write each
// output column sorted by row.
//
// Accumulation is Alg. 5 (HashAdd): an open-addressing table in shared memory
// holding (row, value) pairs, empty = -1, linear probing, insert-or-add.  The
// row key is claimed with atomicCAS and the value added with a shared-memory
// atomicAdd, so the lanes of a warp insert concurrently.  Table size is a power
// of two >= 2 nnz(B(:,j)) (from the symbolic pass).
//
// Thread-block items (CTA-class columns and heavy-column windows) use that
// open-addressing table with the scrambled hash, then sort (the last step of
// Alg. 5): occupied slots are compacted, bucketed by an order-preserving map
// of the row onto [rmin, rmax], placed by a counting sort and ranked inside
// their bucket.  Warp-class columns use a bucketed, order-preserving hash
// instead (spk_warp.cu), which makes the sort step a counting placement.
#include <type_traits>

#include "spk_common.cuh"
#include "spk_launch.h"

namespace spk {

// Padded layouts of the thread-block kernel: table slot p lives at sp(p) (one
// pad slot per 32) and counter word w at cw(w) (one pad word per 4), so a
// thread that walks a contiguous run of slots or words starts on its own bank.
__device__ __forceinline__ int sp(int p) { return p + (p >> 5); }
__host__ __device__ __forceinline__ int cw(int w) { return w + (w >> 2); }
__device__ __forceinline__ uint32_t get16p(const uint32_t* c, uint32_t h) {
  return (c[cw((int)(h >> 1))] >> ((h & 1u) << 4)) & 0xffffu;
}
__device__ __forceinline__ uint32_t add16p(uint32_t* c, uint32_t h) {
  const uint32_t sh = (h & 1u) << 4;
  return (atomicAdd(&c[cw((int)(h >> 1))], 1u << sh) >> sh) & 0xffffu;
}
template <int BLOCK>
__device__ __forceinline__ void block_scan16p(uint32_t* c, int n, int* red) {
  const int nw = n >> 1;
  const int per = (nw + BLOCK - 1) / BLOCK;
  const int w0 = threadIdx.x * per;
  int loc = 0;
  for (int t = 0; t < per; ++t)
    if (w0 + t < nw) {
      const uint32_t x = c[cw(w0 + t)];
      loc += (int)(x & 0xffffu) + (int)(x >> 16);
    }
  int total;
  int run = block_excl_scan<BLOCK>(loc, red, &total);
  for (int t = 0; t < per; ++t)
    if (w0 + t < nw) {
      const uint32_t x = c[cw(w0 + t)];
      const int lo = (int)(x & 0xffffu), hi = (int)(x >> 16);
      c[cw(w0 + t)] = (uint32_t)run | ((uint32_t)(run + lo) << 16);
      run += lo + hi;
    }
}

// Order-preserving bucket of row r on [rmin, rmin + span): floor((r-rmin)*NB/span).
__device__ __forceinline__ uint32_t bucket_of(int32_t r, int32_t rmin, uint64_t bmul) {
  return (uint32_t)(((uint64_t)(uint32_t)(r - rmin) * bmul) >> 32);
}

// Insert-or-add with the padded slot layout (slot h at sp(h)).
__device__ __forceinline__ int table_insert_pad(int32_t* keys, uint32_t h, uint32_t mask, int32_t r, bool& fresh) {
  fresh = false;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int old = atomicCAS(&keys[sp((int)h)], -1, r);
    if (old == -1) {
      fresh = true;
      return (int)h;
    }
    if (old == r) return (int)h;
    h = (h + 1) & mask;
  }
  return -1;
}

// One thread-block work item: a CTA-class column or a heavy column's row
// window (Alg. 8: B(r1:r2, j) <- HashAdd(A_1(r1:r2, j), ..., A_k(r1:r2, j))).
// `sm_raw` holds the table (values sized for V), then the row keys, then the
// padded 16-bit bucket counters.
template <typename V, int BLOCK, int U, int SMAX>
__device__ __forceinline__ void cta_item(const Inputs& in, const Window& W, const Inst* I, const int32_t* offs,
                                         int32_t* __restrict__ out_row, V* __restrict__ out_val,
                                         unsigned char* sm_raw, int tmax, int* red, int* s_rng, Counters* ctr_w) {
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  V* vals = reinterpret_cast<V*>(sm_raw);
  int32_t* keys = reinterpret_cast<int32_t*>(vals + sp(tmax));
  uint32_t* cnt = reinterpret_cast<uint32_t*>(keys + sp(tmax));  // tmax/2 16-bit counters, padded
  const int u = W.u;
  const int k = I->k, off = I->ptr_off, j = W.col - I->colbase;
  const int q = max(7, ceil_log2(2 * u));  // >= 64 counters: enough buckets for any span at M = 1
  const int T = 1 << q;
  if (T > tmax || T / BLOCK > SMAX) {
    if (threadIdx.x == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);
    return;
  }
  const uint32_t mask = (uint32_t)T - 1u;
  for (int p = threadIdx.x; p < T; p += BLOCK) {
    keys[sp(p)] = -1;
    vals[sp(p)] = V(0);
  }
  for (int p = threadIdx.x; p < cw(T / 4); p += BLOCK) cnt[p] = 0u;
  if (threadIdx.x == 0) {
    s_rng[0] = INT32_MAX;
    s_rng[1] = -1;
  }
  __syncthreads();
  int rmin = INT32_MAX, rmax = -1;
  for (int cb = 0; cb < k; cb += 32) {
    const int i = cb + lane;
    int beg = 0, len = 0;
    if (i < k) {
      if (W.search < 0) {
        const int32_t* cp = in.cp[off + i];
        beg = __ldg(cp + j);
        len = __ldg(cp + j + 1) - beg;
      } else {
        const int32_t* o = offs + ((int64_t)W.search * in.kmax + i) * 2;
        beg = o[0];
        len = o[1] - beg;
      }
    }
    SegWalk w;
    w.init(beg, len, lane);
    for (int e0 = wid * 32 * U; e0 < w.total; e0 += NW * 32 * U) {
      int32_t r[U];
      V v[U];
#pragma unroll
      for (int t = 0; t < U; ++t) {
        const int e = e0 + t * 32 + lane;
        const int seg = w.find(e);
        const int idx = w.index_in_input(e, seg);
        r[t] = -1;
        v[t] = V(0);
        if (e < w.total) {
          r[t] = __ldg(in.ri[off + cb + seg] + idx);
          v[t] = __ldg(static_cast<const V*>(in.val[off + cb + seg]) + idx);
        }
      }
#pragma unroll
      for (int t = 0; t < U; ++t) {
        if (r[t] < 0) continue;
        bool fresh;
        const int h = table_insert_pad(keys, hash_scrambled(r[t], q), mask, r[t], fresh);
        if (h < 0) continue;  // table full: the count check below reports it
        atomicAdd(&vals[sp(h)], v[t]);
        rmin = min(rmin, r[t]);
        rmax = max(rmax, r[t]);
      }
    }
  }
  rmin = warp_min(rmin);
  rmax = warp_max(rmax);
  if (lane == 0) {
    atomicMin(&s_rng[0], rmin);
    atomicMax(&s_rng[1], rmax);
  }
  __syncthreads();
  rmin = s_rng[0];
  rmax = s_rng[1];
  // Compaction through registers: thread t owns slots [t*S, t*S + S).
  const int S = T >= BLOCK ? T / BLOCK : 1;
  const int p0 = threadIdx.x * S;
  int32_t kk[SMAX];
  V vv[SMAX];
  int mine = 0;
#pragma unroll
  for (int t = 0; t < SMAX; ++t) {
    kk[t] = -1;
    vv[t] = V(0);
    if (t < S && p0 + t < T) {
      kk[t] = keys[sp(p0 + t)];
      vv[t] = vals[sp(p0 + t)];
      mine += kk[t] >= 0;
    }
  }
  int tot;
  int dst = block_excl_scan<BLOCK>(mine, red, &tot);  // synchronises: all reads are done
  const bool ok = (tot == u);
  if (ok) {
#pragma unroll
    for (int t = 0; t < SMAX; ++t)
      if (kk[t] >= 0) {
        keys[sp(dst)] = kk[t];
        vals[sp(dst)] = vv[t];
        ++dst;
      }
  } else if (threadIdx.x == 0) {
    atomicOr(&ctr_w->err, ERR_INTERNAL);
  }
  __syncthreads();
  if (!ok) return;
  const int NB = T / 2;
  const uint32_t span = (uint32_t)(rmax - rmin) + 1u;
  const uint64_t bmul = ((uint64_t)NB << 32) / span;
  for (int x = threadIdx.x; x < u; x += BLOCK) add16p(cnt, bucket_of(keys[sp(x)], rmin, bmul));
  __syncthreads();
  block_scan16p<BLOCK>(cnt, NB, red);
  __syncthreads();
  for (int x = threadIdx.x; x < u; x += BLOCK) {
    const int32_t key = keys[sp(x)];
    const int pos = (int)add16p(cnt, bucket_of(key, rmin, bmul));
    keys[sp(T / 2 + pos)] = key;
    vals[sp(T / 2 + pos)] = vals[sp(x)];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < u; x += BLOCK) {
    const int32_t key = keys[sp(T / 2 + x)];
    const uint32_t b = bucket_of(key, rmin, bmul);
    const int lo = b ? (int)get16p(cnt, b - 1u) : 0;
    const int hi = (int)get16p(cnt, b);
    int rank = lo;
    for (int y = lo; y < hi; ++y) rank += keys[sp(T / 2 + y)] < key;
    out_row[rank] = key;
    out_val[rank] = vals[sp(T / 2 + x)];
  }
}

// DT: 0 = every problem float, 1 = every problem double, 2 = per-problem dtype.
template <int DT, int BLOCK, int U, int SMAX>
__global__ void __launch_bounds__(BLOCK) k_num_cta(Inputs in, const Window* __restrict__ win, int nwin,
                                                   const int32_t* __restrict__ offs,
                                                   const int64_t* __restrict__ col_ptr, Outs o, int tmax,
                                                   Counters* ctr_w) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int red[BLOCK / 32 + 1];
  __shared__ int s_rng[2];
  for (int wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
    const Window W = win[wi];
    const int q = inst_of(in, W.col);
    const Inst* I = in.inst + q;
    const int64_t out = col_ptr[W.col] - (in.col_inst ? col_ptr[I->colbase] : 0) + W.out_off;
    int32_t* out_row = out_row_of(o, q) + out;
    if (DT == 1 || (DT == 2 && I->dtype == 1))
      cta_item<double, BLOCK, U, SMAX>(in, W, I, offs, out_row, static_cast<double*>(out_val_of(o, q)) + out,
                                       sm_raw, tmax, red, s_rng, ctr_w);
    else
      cta_item<float, BLOCK, U, SMAX>(in, W, I, offs, out_row, static_cast<float*>(out_val_of(o, q)) + out,
                                      sm_raw, tmax, red, s_rng, ctr_w);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
static int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

static int blocks_per_sm(const DeviceInfo& dev, size_t smem_per_block, int threads_per_block) {
  const size_t reserve = 1024;
  int b = (int)(dev.smem_per_sm / (smem_per_block + reserve));
  int bt = 2048 / threads_per_block;
  if (b > bt) b = bt;
  if (b > 32) b = 32;
  return b < 1 ? 1 : b;
}

template <int DT>
static cudaError_t launch_num_cta_t(const Inputs& in, const Window* win, int n_win, const int32_t* offs,
                                    const int64_t* col_ptr, const Outs& out, int window_max, Counters* ctr_w,
                                    const DeviceInfo& dev, cudaStream_t st) {
  using V = typename std::conditional<DT == 0, float, double>::type;  // value bytes per slot
  constexpr int BLOCK = 512;
  constexpr int SMAX = 2 * WINDOW_MAX_LIMIT / BLOCK;  // 16 slots per thread at the largest table
  const int tmax = pow2_at_least(2 * window_max);
  const size_t slots = (size_t)tmax + tmax / 32;
  const size_t smem = slots * (sizeof(V) + 4) + (size_t)cw(tmax / 4) * 4 + 16;
  auto kern = k_num_cta<DT, BLOCK, 4, SMAX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = dev.sms * blocks_per_sm(dev, smem, BLOCK);
  if (grid > n_win) grid = n_win;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, BLOCK, smem, st>>>(in, win, n_win, offs, col_ptr, out, tmax, ctr_w);
  return cudaGetLastError();
}

cudaError_t launch_num_cta(const Inputs& in, int dt, const Window* win, int n_win, const int32_t* offs,
                           const int64_t* col_ptr, const Outs& out, int window_max, Counters* ctr_w,
                           const DeviceInfo& dev, cudaStream_t st) {
  if (n_win <= 0) return cudaSuccess;
  if (dt == 0) return launch_num_cta_t<0>(in, win, n_win, offs, col_ptr, out, window_max, ctr_w, dev, st);
  if (dt == 1) return launch_num_cta_t<1>(in, win, n_win, offs, col_ptr, out, window_max, ctr_w, dev, st);
  return launch_num_cta_t<2>(in, win, n_win, offs, col_ptr, out, window_max, ctr_w, dev, st);
}

}  // namespace spk
