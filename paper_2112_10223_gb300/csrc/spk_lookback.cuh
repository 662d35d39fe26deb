// spk_lookback.cuh -- decoupled look-back over column tiles (Merrill &
// Garland, "Single-pass parallel prefix scan with decoupled look-back", 2016):
// the scan of Sec. II-D's per-column counts done inside the pass that
// produces them, so B's column offsets need no separate symbolic pass.
#pragma once

#include <cstdint>

#include "spk_common.cuh"

namespace spk {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Relaxed gpu-scope accesses of the look-back words: each word is read and
// written whole; no other memory is ordered by them.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Look-back words, one per tile, zero before the launch: the top two bits say
// what the low 62 hold.
constexpr unsigned long long LB_AGG = 1ull << 62;  // the tile's own sum is published
constexpr unsigned long long LB_INC = 2ull << 62;  // the inclusive prefix is published
constexpr unsigned long long LB_BAD = 3ull << 62;  // a wait gave up: no valid prefix
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;

__device__ __forceinline__ long long lb_warp_sum64(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(SPK_FULL, x, o);
  return x;
}

// Decoupled look-back over the tiles: publishes tile t's sum, returns the sum
// of all earlier tiles, publishes the inclusive prefix.  *bad: a predecessor
// (or this wait) gave up.  All 32 lanes call it.  Each round reads 128
// predecessors (4 per lane, nearest first), so the walk covers more tiles per
// memory round trip than the GPU completes in one.
__device__ __forceinline__ long long tile_lookback(unsigned long long* status, int t, long long agg,
                                                   unsigned long long limit, bool stall, bool* bad, int lane) {
  if (t == 0) {
    if (lane == 0) st_relaxed_u64(status, LB_INC | (unsigned long long)agg);
    *bad = false;
    return 0;
  }
  if (lane == 0) st_relaxed_u64(status + t, LB_AGG | (unsigned long long)agg);
  long long excl = 0;
  bool poisoned = false;
  for (int base = t - 1;; base -= 128) {
    unsigned long long w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = base - 4 * lane - q;
      w[q] = idx >= 0 ? ld_relaxed_u64(status + idx) : LB_INC;  // before tile 0: prefix 0
      if (stall && lane == 0 && q == 0) w[q] = 0ull;  // test switch: a predecessor that never publishes
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = base - 4 * lane - q;
      if ((w[q] >> 62) == 0) {
        const unsigned long long t0 = global_ns();
        while ((w[q] >> 62) == 0) {
          if (global_ns() - t0 > limit) {
            w[q] = LB_BAD;
            break;
          }
          __nanosleep(100);
          if (!stall && idx >= 0) w[q] = ld_relaxed_u64(status + idx);
        }
      }
    }
    int first = 4;  // this lane's nearest inclusive word
    bool bad_here = false;
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const unsigned f = (unsigned)(w[q] >> 62);
      if (f == 2u) first = q;
      if (f == 3u) bad_here = true;
    }
    if (__any_sync(SPK_FULL, bad_here)) {
      poisoned = true;
      break;
    }
    const unsigned inc = __ballot_sync(SPK_FULL, first < 4);
    const int L = inc ? __ffs(inc) - 1 : 32;
    long long v = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (lane < L || (lane == L && q <= first)) v += (long long)(w[q] & LB_VAL);
    excl += lb_warp_sum64(v);
    if (inc) break;
  }
  if (lane == 0)
    st_relaxed_u64(status + t, (poisoned ? LB_BAD : LB_INC) | ((unsigned long long)(excl + agg) & LB_VAL));
  *bad = poisoned;
  return excl;
}

}  // namespace spk
