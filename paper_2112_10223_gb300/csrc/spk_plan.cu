// spk_plan.cu -- column binning, input validation, the column-pointer scan
// and the per-input offsets of heavy-column row windows.
#include "spk_common.cuh"
#include "spk_launch.h"

namespace spk {

// Appends `value` to `list` for every lane with pred set; one atomic per warp.
// All 32 lanes must be active.
__device__ __forceinline__ void warp_append(bool pred, int32_t* __restrict__ list, int32_t* counter, int32_t value,
                                            int lane) {
  const unsigned m = __ballot_sync(SPK_FULL, pred);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(SPK_FULL, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// a1 of the hot path: s_j = sum_i nnz(A_i(:,j)) and the column's class
// (Sec. III-A: the symbolic phase balances load on the summed input count),
// for every global column of every problem of the batch.
__global__ void __launch_bounds__(256) k_bin(Inputs in, int warp_max, int cta_max, int32_t* __restrict__ s_out,
                                             int32_t* __restrict__ u_out, int32_t* __restrict__ warp_list,
                                             int32_t* __restrict__ cta_list, int32_t* __restrict__ heavy_list,
                                             int32_t* __restrict__ big_list,
                                             Counters* __restrict__ ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < in.ncols; g0 += stride) {
    const int g = (int)(g0 + threadIdx.x);
    const bool live = g < in.ncols;
    int64_t s = 0;
    if (live) {
      const Inst* I = in.inst + inst_of(in, g);
      const int k = __ldg(&I->k), off = __ldg(&I->ptr_off);
      const int j = g - __ldg(&I->colbase);
      for (int i = 0; i < k; ++i) {
        const int32_t* cp = in.cp[off + i];
        s += (int64_t)__ldg(cp + j + 1) - (int64_t)__ldg(cp + j);
      }
    }
    int cls = CLS_EMPTY;
    if (live) {
      if (s > INT32_MAX) {
        atomicOr(&ctr->err, ERR_OVERFLOW);
        s = INT32_MAX;
      }
      if (s <= 0) cls = CLS_EMPTY;
      else if (s <= warp_max) cls = CLS_WARP;
      else if (s <= cta_max) cls = CLS_CTA;
      else cls = CLS_HEAVY;
      s_out[g] = (int32_t)s;
      if (cls == CLS_EMPTY) u_out[g] = 0;
    }
    warp_append(cls == CLS_WARP, warp_list, &ctr->n_warp, g, lane);
    warp_append(cls == CLS_CTA, cta_list, &ctr->n_cta, g, lane);
    // Heavy columns: the largest go to their own list, handed out first.
    warp_append(cls == CLS_HEAVY && s <= BIG_S, heavy_list, &ctr->n_heavy, g, lane);
    warp_append(cls == CLS_HEAVY && s > BIG_S, big_list, &ctr->n_big, g, lane);
  }
}

__global__ void __launch_bounds__(256) k_col_inst(const Inst* __restrict__ inst, int ninst,
                                                  int32_t* __restrict__ col_inst) {
  for (int q = blockIdx.x; q < ninst; q += gridDim.x) {
    const int cb = inst[q].colbase, n = inst[q].n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) col_inst[cb + j] = q;
  }
}

// Optional input check: col_ptr[0] = 0, non-decreasing, col_ptr[n] = nnz;
// rows in [0, m), and strictly increasing inside each column unless the
// inputs are declared unordered.
__global__ void __launch_bounds__(256) k_validate(Inputs in, const int64_t* __restrict__ nnz, Counters* ctr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int err = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < in.ncols; g += stride) {
    const Inst* I = in.inst + inst_of(in, (int)g);
    const int k = I->k, off = I->ptr_off, m = I->m, n = I->n;
    const int64_t j = g - I->colbase;
    for (int i = 0; i < k; ++i) {
      const int32_t* cp = in.cp[off + i];
      const int64_t b = __ldg(cp + j), e = __ldg(cp + j + 1);
      const int64_t nz = nnz[off + i];
      if (j == 0 && b != 0) err |= ERR_RANGE;
      if (j == n - 1 && e != nz) err |= ERR_RANGE;
      if (b < 0 || e < b || e > nz) {
        err |= ERR_RANGE;
        continue;
      }
      const int32_t* ri = in.ri[off + i];
      int32_t prev = -1;
      for (int64_t p = b; p < e; ++p) {
        const int32_t r = __ldg(ri + p);
        if (r < 0 || r >= m) err |= ERR_RANGE;
        if (in.sorted && r <= prev) err |= ERR_UNSORTED;
        prev = r;
      }
    }
  }
  if (err) atomicOr(&ctr->err, err);
}

// ---------------------------------------------------------------------------
// a3: col_ptr_B = exclusive scan of u (int32 counts -> int64 pointers).
// Three passes: tile sums, scan of the tile sums, per-tile scan.
// ---------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ long long warp_incl_scan64(long long x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(SPK_FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of 64-bit values; tmp holds 33 entries.
__device__ __forceinline__ long long block_excl_scan64(long long x, long long* tmp, long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long inc = warp_incl_scan64(x, lane);
  if (lane == 31) tmp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    long long v = lane < SCAN_BLOCK / 32 ? tmp[lane] : 0;
    long long vi = warp_incl_scan64(v, lane);
    if (lane < SCAN_BLOCK / 32) tmp[lane] = vi - v;
    if (lane == 31) tmp[32] = vi;
  }
  __syncthreads();
  long long r = tmp[wid] + inc - x;
  *total = tmp[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_tiles(const int32_t* __restrict__ u, int n,
                                                          long long* __restrict__ tile_sum) {
  __shared__ long long tmp[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  long long acc = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    const int64_t j = base + (int64_t)t * SCAN_BLOCK + threadIdx.x;
    if (j < n) acc += u[j];
  }
  long long total;
  block_excl_scan64(acc, tmp, &total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(long long* __restrict__ tile_sum, int tiles,
                                                         long long* __restrict__ grand_total) {
  __shared__ long long tmp[33];
  long long carry = 0;
  for (int b = 0; b < tiles; b += SCAN_BLOCK) {
    const int t = b + threadIdx.x;
    long long v = t < tiles ? tile_sum[t] : 0;
    long long total;
    long long ex = block_excl_scan64(v, tmp, &total);
    if (t < tiles) tile_sum[t] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *grand_total = carry;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_apply(const int32_t* __restrict__ u, int n,
                                                          const long long* __restrict__ tile_off,
                                                          const long long* __restrict__ grand_total,
                                                          int64_t* __restrict__ col_ptr) {
  __shared__ long long tmp[33];
  // Each thread owns SCAN_ITEMS consecutive counts of the tile.
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  long long acc = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    const int64_t j = base + t;
    v[t] = j < n ? u[j] : 0;
    acc += v[t];
  }
  long long total;
  long long run = block_excl_scan64(acc, tmp, &total) + tile_off[blockIdx.x];
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    const int64_t j = base + t;
    if (j < n) col_ptr[j] = run;
    run += v[t];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) col_ptr[n] = *grand_total;
}

// Per-input offsets of split row windows (Sec. III-B: "partition rows ...
// using binary searches"): for window w and input i, the first entry of
// A_i(:,col) with row >= r_lo and the first with row >= r_hi.  One thread per
// (window, input) pair (measured faster than a warp-wide 32-way search per
// pair: with thousands of pairs in flight the per-pair setup dominates);
// rows of the offset table are kmax inputs wide.
// Split windows of one column partition its rows, and consecutive search rows
// hold consecutive windows (a slab's windows are listed together, in row
// order), so a window's end in input i is the next window's start there.
// The search kernel finds each window's start (lower bound of r_lo) and, only
// for a window not followed by the next window of its column, its end; the
// second kernel copies the other ends from the next row.
__device__ __forceinline__ bool next_window_follows(const Window* __restrict__ win,
                                                    const int32_t* __restrict__ search_list, int n_search, int s,
                                                    const Window& w) {
  if (s + 1 >= n_search) return false;
  const Window& v = win[search_list[s + 1]];
  return v.col == w.col && v.r_lo == w.r_hi;
}

__global__ void __launch_bounds__(256) k_window_search(Inputs in, const Window* __restrict__ win,
                                                       const int32_t* __restrict__ search_list, int n_search,
                                                       int32_t* __restrict__ offs) {
  const int64_t total = (int64_t)n_search * in.kmax;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int s = (int)(t / in.kmax), i = (int)(t - (int64_t)s * in.kmax);
    const Window w = win[search_list[s]];
    const Inst* I = in.inst + inst_of(in, w.col);
    if (i >= I->k) continue;
    const int j = w.col - I->colbase;
    const int32_t* cp = in.cp[I->ptr_off + i];
    const int b = __ldg(cp + j), e = __ldg(cp + j + 1);
    const int32_t* ri = in.ri[I->ptr_off + i];
    const int lo = lower_bound_i32(ri, b, e, w.r_lo);
    offs[2 * t] = lo;
    if (!next_window_follows(win, search_list, n_search, s, w)) offs[2 * t + 1] = lower_bound_i32(ri, lo, e, w.r_hi);
  }
}

__global__ void __launch_bounds__(256) k_window_ends(Inputs in, const Window* __restrict__ win,
                                                     const int32_t* __restrict__ search_list, int n_search,
                                                     int32_t* __restrict__ offs) {
  const int64_t total = (int64_t)n_search * in.kmax;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int s = (int)(t / in.kmax), i = (int)(t - (int64_t)s * in.kmax);
    const Window w = win[search_list[s]];
    if (i >= in.inst[inst_of(in, w.col)].k) continue;
    if (next_window_follows(win, search_list, n_search, s, w)) offs[2 * t + 1] = offs[2 * (t + in.kmax)];
  }
}

// B's column pointers per problem: out_cp[j] = col_ptr[colbase + j] - col_ptr[colbase].
__global__ void __launch_bounds__(256) k_out_colptr(Inputs in, Outs o, const int64_t* __restrict__ col_ptr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (int64_t)in.ncols + in.ninst; g += stride) {
    if (g < in.ncols) {
      const int q = inst_of(in, (int)g);
      const int cb = in.inst[q].colbase;
      out_cp_of(o, q)[g - cb] = col_ptr[g] - col_ptr[cb];
    } else {  // the closing entry of problem q
      const int q = (int)(g - in.ncols);
      const Inst& I = in.inst[q];
      out_cp_of(o, q)[I.n] = col_ptr[I.colbase + I.n] - col_ptr[I.colbase];
    }
  }
}

__global__ void __launch_bounds__(256) k_inst_nnz(Inputs in, const int64_t* __restrict__ col_ptr,
                                                  int64_t* __restrict__ nnz) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < in.ninst; q += gridDim.x * blockDim.x) {
    const Inst& I = in.inst[q];
    nnz[q] = col_ptr[I.colbase + I.n] - col_ptr[I.colbase];
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_bin(const Inputs& in, int warp_max, int cta_max, int32_t* s, int32_t* u, int32_t* wl, int32_t* cl,
                       int32_t* hl, Counters* ctr, int sms, cudaStream_t st) {
  if (in.ncols == 0) return cudaSuccess;
  int64_t blocks = ((int64_t)in.ncols + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  k_bin<<<(int)blocks, 256, 0, st>>>(in, warp_max, cta_max, s, u, wl, cl, hl, hl + in.ncols, ctr);
  return cudaGetLastError();
}

cudaError_t launch_col_inst(const Inputs& in, int32_t* col_inst, int sms, cudaStream_t st) {
  int blocks = in.ninst < sms * 8 ? in.ninst : sms * 8;
  if (blocks < 1) return cudaSuccess;
  k_col_inst<<<blocks, 256, 0, st>>>(in.inst, in.ninst, col_inst);
  return cudaGetLastError();
}

cudaError_t launch_validate(const Inputs& in, const int64_t* nnz, Counters* ctr, int sms, cudaStream_t st) {
  if (in.ncols == 0) return cudaSuccess;
  int64_t blocks = ((int64_t)in.ncols + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  k_validate<<<(int)blocks, 256, 0, st>>>(in, nnz, ctr);
  return cudaGetLastError();
}

size_t scan_tiles(int64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 1; }

// Loads the scan kernels' code onto the current device now (CUDA loads
// modules lazily, at a kernel's first launch, and loading takes device
// memory); a caller that must not allocate during later calls runs this once
// at set-up.
cudaError_t load_scan_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_scan_tiles);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_scan_sums);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_scan_apply);
  return e;
}

cudaError_t launch_scan(const int32_t* u, int n, long long* tile_buf, int64_t* col_ptr, cudaStream_t st) {
  const int tiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
  long long* grand = tile_buf + tiles;
  if (tiles > 0) k_scan_tiles<<<tiles, SCAN_BLOCK, 0, st>>>(u, n, tile_buf);
  k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(tile_buf, tiles, grand);
  k_scan_apply<<<tiles > 0 ? tiles : 1, SCAN_BLOCK, 0, st>>>(u, n, tile_buf, grand, col_ptr);
  return cudaGetLastError();
}

cudaError_t launch_window_search(const Inputs& in, const Window* win, const int32_t* search_list, int n_search,
                                 int32_t* offs, int sms, cudaStream_t st) {
  if (n_search <= 0) return cudaSuccess;
  const int64_t total = (int64_t)n_search * in.kmax;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)sms * 32) blocks = (int64_t)sms * 32;
  k_window_search<<<(int)blocks, 256, 0, st>>>(in, win, search_list, n_search, offs);
  k_window_ends<<<(int)blocks, 256, 0, st>>>(in, win, search_list, n_search, offs);
  return cudaGetLastError();
}

cudaError_t launch_inst_nnz(const Inputs& in, const int64_t* col_ptr, int64_t* nnz, cudaStream_t st) {
  const int blocks = (in.ninst + 255) / 256;
  k_inst_nnz<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(in, col_ptr, nnz);
  return cudaGetLastError();
}

cudaError_t launch_out_colptr(const Inputs& in, const Outs& o, const int64_t* col_ptr, int sms, cudaStream_t st) {
  int64_t blocks = ((int64_t)in.ncols + in.ninst + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  if (blocks < 1) blocks = 1;
  k_out_colptr<<<(int)blocks, 256, 0, st>>>(in, o, col_ptr);
  return cudaGetLastError();
}

// Column pointers between the int64 form of B and the int32 form of an input
// (a streamed running sum is the next add's input 0; its nnz fits int32).
__global__ void k_colptr_narrow(const int64_t* __restrict__ src, int32_t* __restrict__ dst, int64_t n1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (int32_t)src[i];
}
__global__ void k_colptr_widen(const int32_t* __restrict__ src, int64_t* __restrict__ dst, int64_t n1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (int64_t)src[i];
}

static int colptr_blocks(int64_t n1, int sms) {
  int64_t b = (n1 + 255) / 256;
  if (b > (int64_t)sms * 8) b = (int64_t)sms * 8;
  return b < 1 ? 1 : (int)b;
}

cudaError_t launch_colptr_narrow(const int64_t* src, int32_t* dst, int64_t n1, int sms, cudaStream_t st) {
  k_colptr_narrow<<<colptr_blocks(n1, sms), 256, 0, st>>>(src, dst, n1);
  return cudaGetLastError();
}

cudaError_t launch_colptr_widen(const int32_t* src, int64_t* dst, int64_t n1, int sms, cudaStream_t st) {
  k_colptr_widen<<<colptr_blocks(n1, sms), 256, 0, st>>>(src, dst, n1);
  return cudaGetLastError();
}

}  // namespace spk
