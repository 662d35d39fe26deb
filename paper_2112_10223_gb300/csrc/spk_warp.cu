// spk_warp.cu -- warp-class columns (s_j = sum_i nnz(A_i(:,j)) <= warp_max):
// one warp per column, for both the symbolic count (Alg. 6's role) and the
// numeric sum (Alg. 5's role).
//
// The table is a bucketed hash whose hash is order-preserving,
// b(r) = floor(r * NB / m) with NB = 2^q >= s_j buckets: a bucket holds about
// one entry and every row of bucket b is smaller than every row of a later
// bucket.  Insert-or-add by row key happens inside a bucket; the sort of
// Alg. 5's last step becomes a counting placement plus tiny per-bucket sorts.
//
//   pass 1   read the column's rows (coalesced, k segments), count per bucket
//   scan     exclusive scan of the counts: bucket starts
//   pass 2   read the rows (and values) again -- they are in L1 now -- and
//            file every entry at its bucket's next free slot in shared memory
//   sort     the buckets with two or more entries (listed during the scan)
//            are insertion-sorted, one per lane; the slots are then the column
//            sorted by row.  Symbolic: nnz(B(:,j)) = s_j minus the repeated
//            rows those sorts meet.
//   finish   numeric: a row's first slot is its leader; it sums its run of
//            equal rows and writes at (leaders before it).  When the symbolic
//            pass saw no repeated row (u_j == s_j) the slots are copied out.
// Output is written in slot order, i.e. row order, so stores coalesce.
//
// Entry loads: the k segments of a column are read as one flattened sequence,
// 32 consecutive positions per warp round (coalesced inside each segment).
// When every segment has the same length L (Erdos-Renyi and partial-product
// inputs), position e lies in segment umulhi(e, ceil(2^32/L)); full rounds run
// without bounds checks.
#include <type_traits>

#include "spk_common.cuh"
#include "spk_launch.h"
#include "spk_lookback.cuh"


namespace spk {

// One pad word after every 16 counters: a lane that scans 16 consecutive
// counters then starts on its own bank (17 l mod 32 is a permutation).
__device__ __forceinline__ int pad16(int b) { return b + (b >> 4); }
__host__ __device__ constexpr int padded_words(int n) { return n + (n >> 4) + 1; }

// Per-warp shared memory: values (numeric), row keys, padded bucket counters
// and the list of buckets holding two or more entries.
template <typename V, bool NUMERIC>
__host__ __device__ constexpr size_t warp_col_bytes(int smax) {
  return ((size_t)smax * ((NUMERIC ? sizeof(V) : 0) + sizeof(int32_t)) +
          (size_t)padded_words(smax) * sizeof(uint32_t) + (size_t)(smax / 2 + 1) * sizeof(uint32_t) +
          (NUMERIC ? 0 : (size_t)1024 * sizeof(uint32_t)) + 15) &
         ~(size_t)15;
}

struct WarpColArgs {
  const int32_t* list;     // warp-class global column ids
  const Counters* ctr;     // n_warp
  const int32_t* s_arr;    // s_j
  const int32_t* u_arr;    // numeric: u_j from the symbolic pass
  const int64_t* col_ptr;  // numeric: global column pointers of B
  int32_t* u_out;          // symbolic: u_j
  Outs out;                // numeric: where B goes
  Counters* ctr_w;
  int smax;
  int force_dedup;         // numeric: sort_mode 1
  int unsorted_out;        // numeric: sort_mode 2
  int only_dtype;          // numeric, mixed batch: process only this dtype's columns (-1: all)
};

// Runs f on every entry of the chunk (32 inputs at most), lane by lane in
// flattened order; e is the entry's position in that order.  Per-entry work is
// split in two: f.pre(row, value, valid, e) issues the shared-memory atomic
// and returns its result, f.post(result, row, value, valid, e) consumes it.
// A round calls pre for all its U entries before any post, so the U atomics
// are in flight together instead of each one's result stalling the next
// (warps issue in order).  Equal-length chunks map positions with one
// multiply-high and run their full rounds without bounds checks.
template <bool VALS, int U, typename V, typename F>
__device__ __forceinline__ void for_each_entry(const ChunkMap& cm, const int32_t* srow, const V* svals, int lane,
                                               F& f) {
  if (cm.equal) {
    const uint32_t M = cm.magic32;
    const int L = cm.L;
    const int full = cm.total - cm.total % (32 * U);
    for (int e0 = 0; e0 < full; e0 += 32 * U) {
      int32_t r[U];
      V v[U];
#pragma unroll
      for (int t = 0; t < U; ++t) {
        const int e = e0 + t * 32 + lane;
        const int sg = (int)__umulhi((uint32_t)e, M);
        const int off = e - sg * L;
        r[t] = __ldg(shfl_iptr(srow, sg) + off);
        if constexpr (VALS) v[t] = __ldg(shfl_vptr(svals, sg) + off);
      }
      uint32_t tok[U];
#pragma unroll
      for (int t = 0; t < U; ++t) tok[t] = f.pre(r[t], v[t], true, e0 + t * 32 + lane);
#pragma unroll
      for (int t = 0; t < U; ++t) f.post(tok[t], r[t], v[t], true, e0 + t * 32 + lane);
    }
    for (int e0 = full; e0 < cm.total; e0 += 32) {
      const int e = e0 + lane;
      const bool ok = e < cm.total;
      const int sg = ok ? (int)__umulhi((uint32_t)e, M) : 0;
      const int off = e - sg * L;
      const int32_t* rp = shfl_iptr(srow, sg);
      int32_t r = -1;
      V v = V(0);
      if (ok) r = __ldg(rp + off);
      if constexpr (VALS) {
        const V* vp = shfl_vptr(svals, sg);
        if (ok) v = __ldg(vp + off);
      }
      f.post(f.pre(r, v, ok, e), r, v, ok, e);
    }
    return;
  }
  for (int e0 = 0; e0 < cm.total; e0 += 32 * U) {
    int32_t r[U];
    V v[U];
    bool ok[U];
#pragma unroll
    for (int t = 0; t < U; ++t) {
      const int e = e0 + t * 32 + lane;
      ok[t] = e < cm.total;
      r[t] = -1;
      if constexpr (VALS) v[t] = V(0);
      if (e0 + t * 32 >= cm.total) continue;  // (warp-uniform) slot wholly past the chunk's end
      const int sg = cm.w.find(e);
      const int off = e - __shfl_sync(SPK_FULL, cm.w.P, sg);
      const int32_t* rp = shfl_iptr(srow, sg);
      if (ok[t]) r[t] = __ldg(rp + off);
      if constexpr (VALS) {
        const V* vp = shfl_vptr(svals, sg);
        if (ok[t]) v[t] = __ldg(vp + off);
      }
    }
    uint32_t tok[U];
#pragma unroll
    for (int t = 0; t < U; ++t) tok[t] = f.pre(r[t], v[t], ok[t], e0 + t * 32 + lane);
#pragma unroll
    for (int t = 0; t < U; ++t) f.post(tok[t], r[t], v[t], ok[t], e0 + t * 32 + lane);
  }
}

// Adds the chunk's first flattened position to e.
template <typename V, typename F>
struct ChunkOffset {
  F& f;
  int base;
  __device__ __forceinline__ uint32_t pre(int32_t r, V v, bool ok, int e) { return f.pre(r, v, ok, base + e); }
  __device__ __forceinline__ void post(uint32_t t, int32_t r, V v, bool ok, int e) { f.post(t, r, v, ok, base + e); }
};

// All entries of local column j of the problem whose inputs are pointer-table
// entries [off, off + k): chunk by chunk of 32 inputs.  Resident mode (a batch
// of one with k <= 32): the lane's input pointers and (beg, len) come from
// the caller.
// A lane's segment bounds in the first two chunks of a non-resident column,
// kept from the first pass over the column for the next (which then skips
// the chain of pointer-table and column-pointer loads).
struct ChunkCache {
  int beg[2], len[2];
  bool valid;
};

template <bool VALS, int U, typename V, typename F>
__device__ __forceinline__ void for_each_column_entry(const Inputs& in, int k, int off, int j, bool resident,
                                                      int rbeg, int rlen, const int32_t* my_ri, const V* my_va,
                                                      int lane, F& f, ChunkCache& cc) {
  if (resident) {
    ChunkMap cm;
    cm.init(rbeg, rlen, lane, k);
    for_each_entry<VALS, U, V>(cm, my_ri + rbeg, VALS ? my_va + rbeg : my_va, lane, f);
    return;
  }
  int base = 0;
  for (int cb = 0; cb < k; cb += 32) {
    const int i = cb + lane;
    const int ci = cb >> 5;
    int beg = 0, len = 0;
    const int32_t* ri = nullptr;
    const V* va = nullptr;
    if (i < k) {
      if (ci < 2 && cc.valid) {
        beg = cc.beg[ci];
        len = cc.len[ci];
      } else {
        const int32_t* cp = in.cp[off + i];
        beg = __ldg(cp + j);
        len = __ldg(cp + j + 1) - beg;
      }
      ri = in.ri[off + i] + beg;
      if constexpr (VALS) va = static_cast<const V*>(in.val[off + i]) + beg;
    }
    if (ci == 0) {
      cc.beg[0] = beg;
      cc.len[0] = len;
    } else if (ci == 1) {
      cc.beg[1] = beg;
      cc.len[1] = len;
    }
    ChunkMap cm;
    cm.init(beg, len, lane, min(32, k - cb));
    ChunkOffset<V, F> fo{f, base};
    for_each_entry<VALS, U, V>(cm, ri, va, lane, fo);
    base += cm.total;
  }
  cc.valid = true;
}

// Scalars of one warp-class column, loaded one column ahead of their use.
struct ColState {
  int g;    // global column id, -1 past the end of the list
  int q;    // its problem
  int beg;  // resident mode: this lane's segment begin
  int len;  //                and length
  int s;    // sum of input lengths
  int u;    // numeric: distinct rows
  int64_t out;  // numeric: global col_ptr_B[g]
};

template <bool NUMERIC, bool BATCH>
__device__ __forceinline__ ColState load_col(const Inputs& in, const WarpColArgs& a, int cc, int ncols,
                                             bool resident, const int32_t* my_cp, int lane, int k0) {
  ColState st{-1, 0, 0, 0, 0, 0, 0};
  if (cc >= ncols) return st;
  st.g = a.list[cc];
  if (BATCH) st.q = __ldg(in.col_inst + st.g);
  st.s = a.s_arr[st.g];
  if (NUMERIC) {
    st.u = a.u_arr[st.g];
    st.out = a.col_ptr[st.g];
  }
  if (resident && lane < k0) {
    st.beg = __ldg(my_cp + st.g);
    st.len = __ldg(my_cp + st.g + 1) - st.beg;
  }
  return st;
}

// Per-entry actions of the three passes.
template <typename V>
struct BucketCount {  // pass 1: entries per order-preserving bucket
  uint32_t* cnt;
  uint32_t mul;
  __device__ __forceinline__ uint32_t pre(int32_t r, V, bool ok, int) {
    if (ok) atomicAdd(&cnt[pad16((int)bucket_hi(r, mul))], 1u);
    return 0u;
  }
  __device__ __forceinline__ void post(uint32_t, int32_t, V, bool, int) {}
};

template <typename V>
struct BucketCountChecked {  // pass 1 of the one-pass kernel: rows outside [0, m) are flagged, never counted
  uint32_t* cnt;
  uint32_t mul;
  uint32_t m;
  bool bad;
  __device__ __forceinline__ uint32_t pre(int32_t r, V, bool ok, int) {
    if (ok) {
      if ((uint32_t)r < m) atomicAdd(&cnt[pad16((int)bucket_hi(r, mul))], 1u);
      else bad = true;
    }
    return 0u;
  }
  __device__ __forceinline__ void post(uint32_t, int32_t, V, bool, int) {}
};

template <typename V, bool NUMERIC>
struct BucketFile {  // pass 2: file the row (and value) at the bucket's next slot
  uint32_t* cnt;
  int32_t* skey;
  V* sval;
  uint32_t mul;
  // Numeric filing keeps each atomic next to its stores (measured faster
  // there than issuing a round's atomics first); symbolic filing splits them.
  __device__ __forceinline__ uint32_t pre(int32_t r, V v, bool ok, int) {
    if (!ok) return 0u;
    const uint32_t pos = atomicAdd(&cnt[pad16((int)bucket_hi(r, mul))], 1u);
    if constexpr (NUMERIC) {
      skey[pos] = r;
      sval[pos] = v;
    }
    return pos;
  }
  __device__ __forceinline__ void post(uint32_t pos, int32_t r, V, bool ok, int) {
    if constexpr (!NUMERIC)
      if (ok) skey[pos] = r;
  }
};

// ---------------------------------------------------------------------------
// Symbolic fast path: the number of repeated rows of a column of s <= 512
// entries, without sorting.  Every entry sets one bit of a 2^15-bit filter
// indexed by a multiplicative hash of its row; an entry that finds its bit
// already set is "marked" (a repeated row or a hash collision; about
// s^2 / 2^16 false collisions, i.e. 4 for s = 512).  Rows are staged in
// shared memory with the mark in bit 31.  An entry is a repeat exactly when
// it is marked and another entry of the same row is unmarked or earlier in
// the staging order: in a group of g equal rows the first to set the bit is
// the only unmarked one, unless a collision marked it too, and then the
// earliest entry of the group is not counted; either way g - 1 entries count.
// Only marked entries are compared, against all staged rows (one warp vote
// each).  More marks than the list holds (MARK_MAX, less for small tables)
// hand the column to the bucket path.
// ---------------------------------------------------------------------------
constexpr int FILTER_WORDS = 1024;  // 2^15 bits per warp
constexpr int MARK_MAX = 48;

__device__ __forceinline__ uint32_t filter_hash(int32_t r) { return (static_cast<uint32_t>(r) * 0x9E3779B1u) >> 17; }

struct FilterMark {
  uint32_t* filt;    // FILTER_WORDS words, zero on entry
  int32_t* stage;    // s rows (bit 31: marked)
  __device__ __forceinline__ uint32_t pre(int32_t r, int32_t, bool ok, int) {
    if (!ok) return 0u;
    const uint32_t h = filter_hash(r);
    const uint32_t bit = 1u << (h & 31);
    return atomicOr(&filt[h >> 5], bit) & bit;
  }
  __device__ __forceinline__ void post(uint32_t seen, int32_t r, int32_t, bool ok, int e) {
    if (ok) stage[e] = seen ? (r | INT32_MIN) : r;
  }
};

// Repeated rows of the column, -1 when the marks overflow (then the caller
// runs the bucket path), or -2 when a row lies outside [0, m) (the bucket
// passes index their counters by row and are never run on such a column).
// Leaves the filter zero on all three outcomes.
template <int U>
__device__ __forceinline__ int warp_repeats_filtered(const Inputs& in, int k, int off, int j, bool resident, int rbeg,
                                                     int rlen, const int32_t* my_ri, int s, const int* m_ptr,
                                                     uint32_t* filt, int32_t* stage, uint32_t* marks, int cap,
                                                     int lane) {
  FilterMark fm{filt, stage};
  ChunkCache cc{{0, 0}, {0, 0}, false};
  for_each_column_entry<false, U, int32_t>(in, k, off, j, resident, rbeg, rlen, my_ri, nullptr, lane, fm, cc);
  __syncwarp();
  // Every entry has set its bit: clear the whole filter for the next column
  // (the marks are in the staged rows), so it is left zero on every path.
#pragma unroll
  for (int t = 0; t < FILTER_WORDS / 32; ++t) filt[t * 32 + lane] = 0u;
  constexpr int Q = 16;  // s <= 32 * Q
  // v[q] = staged row of position lane + 32q (INT32_MAX past s: no valid
  // row equals it, since rows are below m < 2^31 - 1).
  // v[q] keeps the row without its mark bit; the marks live in `mine`, so the
  // comparisons below need no masking.
  int32_t v[Q];
  uint32_t mine = 0u;  // bit q: position lane + 32q is marked
  uint32_t top = 0u;   // largest row (a negative row, mark bit cleared, lands at 2^31 - 1 or near)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = lane + 32 * q;
    const int32_t x = e < s ? stage[e] : INT32_MAX;
    v[q] = x & INT32_MAX;
    if (e < s) {
      if (x < 0) mine |= 1u << q;
      top = max(top, (uint32_t)v[q]);
    }
  }
  if (__any_sync(SPK_FULL, top >= (uint32_t)*m_ptr)) return -2;
  // List the marked positions: per-lane counts, one warp scan, then each
  // lane writes its own (few) positions.
  const int cnt = __popc(mine);
  const int inc = warp_incl_scan(cnt, lane);
  const int nmark = __shfl_sync(SPK_FULL, inc, 31);
  if (nmark > cap) return -1;
  int pos = inc - cnt;
  for (uint32_t b = mine; b; b &= b - 1) marks[pos++] = (uint32_t)(lane + 32 * (__ffs(b) - 1));
  __syncwarp();
  int reps = 0;
  for (int i = 0; i < nmark; ++i) {
    const int em = (int)marks[i];
    const int32_t xm = stage[em] & INT32_MAX;
    // Cheap screen first: how many of this lane's rows equal xm, the marked
    // entry itself (in its own lane) not counted?  Most marks are hash
    // collisions, and then no lane goes on to the exact test.
    int eq = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) eq += v[q] == xm;
    if (lane == (em & 31)) --eq;
    bool found = false;
    if (eq > 0) {  // rare: a true repeat of the marked row
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int e = lane + 32 * q;
        if (v[q] == xm && e != em && (!((mine >> q) & 1u) || e < em)) found = true;
      }
    }
    reps += __any_sync(SPK_FULL, found) ? 1 : 0;
  }
  return reps;
}

// Exclusive scan of the NB bucket counts into bucket starts (in place); the
// buckets holding two or more entries -- the only ones that need sorting --
// are listed in mlist as (start | size << 16).  Returns their number.
__device__ __forceinline__ int bucket_scan(uint32_t* cnt, uint32_t* mlist, int NB, int lane) {
  int nmulti = 0;
  const int per = NB >> 5;
  const int b0 = lane * per;
  int loc = 0;
  for (int t = 0; t < per; ++t) loc += (int)cnt[pad16(b0 + t)];
  const int inc = warp_incl_scan(loc, lane);
  int run = inc - loc;
  for (int t = 0; t < per; ++t) {
    const int p = pad16(b0 + t);
    const int x = (int)cnt[p];
    cnt[p] = (uint32_t)run;
    const bool multi = x >= 2;
    const unsigned bal = __ballot_sync(SPK_FULL, multi);
    if (multi) mlist[nmulti + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)run | ((uint32_t)x << 16);
    nmulti += __popc(bal);
    run += x;
  }
  return nmulti;
}

// Insertion sort of the listed multi-entry buckets, one bucket per lane (they
// hold 2-3 entries mostly).  Returns this lane's count of repeated rows met
// (the symbolic count uses it).
template <typename V, bool NUMERIC, bool COUNT = !NUMERIC>
__device__ __forceinline__ int sort_buckets(int32_t* skey, V* sval, const uint32_t* mlist, int nmulti, int lane) {
  int dups = 0;
  for (int i = lane; i < nmulti; i += 32) {
    const uint32_t w = mlist[i];
    const int lo = (int)(w & 0xffffu), hi = lo + (int)(w >> 16);
    for (int x = lo + 1; x < hi; ++x) {
      const int32_t kx = skey[x];
      V vx;
      if constexpr (NUMERIC) vx = sval[x];
      int y = x - 1;
      while (y >= lo && skey[y] > kx) {
        skey[y + 1] = skey[y];
        if constexpr (NUMERIC) sval[y + 1] = sval[y];
        --y;
      }
      skey[y + 1] = kx;
      if constexpr (NUMERIC) sval[y + 1] = vx;
    }
    if constexpr (COUNT)
      for (int x = lo + 1; x < hi; ++x) dups += skey[x] == skey[x - 1];
  }
  return dups;
}

// The s slots hold the column's entries sorted by row: write B(:,j).  Without
// repeated rows (u == s) the slots are copied out; otherwise a row's first
// slot is its leader, which sums its run of equal rows and writes at (leaders
// before it) = ballot prefix.
template <typename V>
__device__ __forceinline__ void write_sorted(const int32_t* skey, const V* sval, int s, int u, bool force_dedup,
                                             int32_t* out_row, V* out_val, Counters* ctr_w, int lane) {
  if (!force_dedup && u == s) {
    // Four slots per lane and round: their loads are issued before any store.
    int q = lane;
    for (; q + 96 < s; q += 128) {
      int32_t r[4];
      V v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        r[t] = skey[q + 32 * t];
        v[t] = sval[q + 32 * t];
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        out_row[q + 32 * t] = r[t];
        out_val[q + 32 * t] = v[t];
      }
    }
    for (; q < s; q += 32) {
      out_row[q] = skey[q];
      out_val[q] = sval[q];
    }
    return;
  }
  int before = 0;
  int32_t carry = -1;  // last row of the previous 32 slots
  for (int q0 = 0; q0 < s; q0 += 32) {
    const int q = q0 + lane;
    const int32_t key = q < s ? skey[q] : -2;
    int32_t prev = __shfl_up_sync(SPK_FULL, key, 1);
    if (lane == 0) prev = carry;
    const bool lead = q < s && key != prev;
    const unsigned bal = __ballot_sync(SPK_FULL, lead);
    if (lead) {
      double sum = (double)sval[q];  // float runs round once, at the end
      for (int y = q + 1; y < s && skey[y] == key; ++y) sum += (double)sval[y];
      const int pos = before + __popc(bal & ((1u << lane) - 1u));
      if (pos < u) {
        out_row[pos] = key;
        out_val[pos] = (V)sum;
      }
    }
    before += __popc(bal);
    carry = __shfl_sync(SPK_FULL, key, 31);
  }
  if (before != u && lane == 0) atomicOr(&ctr_w->err, ERR_INTERNAL);  // symbolic and numeric disagree
}

// Per-warp shared buffers.
struct WarpSmem {
  unsigned char* vals;  // numeric values
  int32_t* skey;
  uint32_t* cnt;
  uint32_t* mlist;      // (start | size << 16) of multi-entry buckets
  uint32_t* filt;       // symbolic: FILTER_WORDS-word filter, kept zero between columns
};

// One column: the three passes, the bucket sorts and (numeric) the write of
// B(:,j).  Symbolic returns the number of repeated rows; numeric returns 0.
template <typename V, bool NUMERIC, int U>
__device__ __forceinline__ int warp_column(const Inputs& in, const WarpColArgs& a, const WarpSmem& sm,
                                           const ColState& cur, int k, int off, int j, uint32_t mul, int NB,
                                           int32_t* out_row, void* out_val_raw, bool resident,
                                           const int32_t* my_ri, const void* my_va_raw, int lane) {
  const int s = cur.s;
  V* sval = reinterpret_cast<V*>(sm.vals);
  int32_t* skey = sm.skey;
  uint32_t* cnt = sm.cnt;
  uint32_t* mlist = sm.mlist;
  const V* my_va = static_cast<const V*>(my_va_raw);
  if (NUMERIC && resident && cur.len > 0) {
    // The lane's value segment is first read in pass 2: start moving it into
    // L2 now, so that pass 2's loads wait on L2, not DRAM.
    // (Prefetching the next column's segments instead ran slower: ER numeric
    // 4.44 -> 5.1 ms.)
    l2_prefetch(my_va + cur.beg, (size_t)cur.len * sizeof(V));
  }
  for (int b = lane; b < padded_words(NB); b += 32) cnt[b] = 0u;
  __syncwarp();
  // Pass 1: entries per bucket.
  BucketCount<V> count{cnt, mul};
  ChunkCache cc{{0, 0}, {0, 0}, false};
  for_each_column_entry<false, U, V>(in, k, off, j, resident, cur.beg, cur.len, my_ri, my_va, lane, count, cc);
  __syncwarp();
  int nmulti = bucket_scan(cnt, mlist, NB, lane);
  __syncwarp();
  // Pass 2: file every entry at its bucket's next slot.
  BucketFile<V, NUMERIC> file{cnt, skey, sval, mul};
  for_each_column_entry<NUMERIC, U, V>(in, k, off, j, resident, cur.beg, cur.len, my_ri, my_va, lane, file, cc);
  __syncwarp();
  // Sort the multi-entry buckets, one bucket per lane (insertion sort; they
  // hold 2-3 entries mostly).  Symbolic: count the repeated rows met.
  // Unsorted output and no repeated row: the bucket order is all that is kept.
  if (NUMERIC && a.unsorted_out && cur.u == s) nmulti = 0;
  const int dups = sort_buckets<V, NUMERIC>(skey, sval, mlist, nmulti, lane);
  __syncwarp();
  if constexpr (!NUMERIC) return warp_sum(dups);
  if constexpr (NUMERIC) {
    write_sorted<V>(skey, sval, s, cur.u, a.force_dedup, out_row, static_cast<V*>(out_val_raw), a.ctr_w, lane);
    return 0;
  }
}

// DT: 0 = float values, 1 = double values (a batch mixing both runs the
// numeric kernel once per dtype, skipping the other dtype's columns).  BATCH:
// columns of several problems (looked up per column); otherwise one problem.
// RES (one problem with k <= 32): lanes hold the inputs' pointers for the
// whole launch (resident mode); the host picks it, so each instantiation
// carries only the code of its mode.
template <int DT, bool NUMERIC, bool BATCH, bool RES, int WARPS, int U>
__global__ void __launch_bounds__(WARPS * 32, 3) k_warp_col(Inputs in, WarpColArgs a) {
  using VB = typename std::conditional<DT == 1, double, float>::type;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int smax = a.smax;
  unsigned char* base = sm_raw + (size_t)wid * warp_col_bytes<VB, NUMERIC>(smax);
  WarpSmem sm;
  sm.vals = base;
  sm.skey = reinterpret_cast<int32_t*>(base + (NUMERIC ? (size_t)smax * sizeof(VB) : 0));
  sm.cnt = reinterpret_cast<uint32_t*>(sm.skey + smax);
  sm.mlist = sm.cnt + padded_words(smax);
  sm.filt = sm.mlist + (smax / 2 + 1);
  if constexpr (!NUMERIC) {
    for (int x = lane; x < FILTER_WORDS; x += 32) sm.filt[x] = 0u;
    __syncwarp();
  }
  __shared__ uint32_t s_mul[16];
  __shared__ int s_m0;
  if (!BATCH && threadIdx.x < 16) s_mul[threadIdx.x] = in.inst[0].bucket_mul[threadIdx.x];
  if (!BATCH && threadIdx.x == 0) s_m0 = in.inst[0].m;
  __syncthreads();
  const int ncols = a.ctr->n_warp;
  const int k0 = in.inst[0].k;
  const bool resident = RES;
  if (RES && (BATCH || k0 > 32)) {  // the host never launches this; never index lanes past k
    if (threadIdx.x == 0) atomicOr(&a.ctr_w->err, ERR_INTERNAL);
    return;
  }
  const int32_t* my_cp = nullptr;
  const int32_t* my_ri = nullptr;
  const void* my_va = nullptr;
  if (resident && lane < k0) {
    my_cp = in.cp[lane];
    my_ri = in.ri[lane];
    if constexpr (NUMERIC) my_va = in.val[lane];
  }
  const int stride = gridDim.x * WARPS;
  int c = blockIdx.x * WARPS + wid;
  // Scalars of the current column and of the next one (loaded a column ahead).
  ColState cur = load_col<NUMERIC, BATCH>(in, a, c, ncols, resident, my_cp, lane, k0);
  ColState nxt = load_col<NUMERIC, BATCH>(in, a, c + stride, ncols, resident, my_cp, lane, k0);
  int n_unique = 0;
  while (cur.g >= 0) {
    // One problem: its scalars were hoisted; a batch looks them up per column.
    const Inst* I = in.inst + cur.q;
    const int k = BATCH ? I->k : k0;
    const int off = BATCH ? I->ptr_off : 0;
    const int j = BATCH ? cur.g - I->colbase : cur.g;
    const int qb = max(5, ceil_log2(cur.s));
    const int NB = 1 << qb;
    if (NUMERIC && BATCH && a.only_dtype >= 0 && I->dtype != a.only_dtype) {
      // another launch handles this column
    } else if (NB > smax) {  // not reachable for a warp-class column
      if (lane == 0) atomicOr(&a.ctr_w->err, ERR_INTERNAL);
    } else {
      const uint32_t mul = BATCH ? __ldg(&I->bucket_mul[qb]) : s_mul[qb];
      if constexpr (!NUMERIC) {
        int dups = -1;
        if (cur.s <= 512)
          dups = warp_repeats_filtered<U>(in, k, off, j, resident, cur.beg, cur.len, my_ri, cur.s,
                                          BATCH ? &I->m : &s_m0, sm.filt, sm.skey, sm.mlist,
                                          min(MARK_MAX, smax / 2 + 1), lane);
        __syncwarp();
        if (dups == -2) {  // a row outside [0, m): reported; B is never computed
          if (lane == 0) atomicOr(&a.ctr_w->err, ERR_RANGE);
          dups = 0;
        }
        if (dups < 0)
          dups = warp_column<int32_t, false, U>(in, a, sm, cur, k, off, j, mul, NB, nullptr, nullptr, resident,
                                                my_ri, my_va, lane);
        if (lane == 0) {
          a.u_out[cur.g] = cur.s - dups;
          n_unique += (dups == 0);
        }
      } else {
        // B(:,j) starts at col_ptr_B[g] - col_ptr_B[colbase] in its problem's buffers.
        const int64_t out = cur.out - (BATCH ? a.col_ptr[I->colbase] : 0);
        int32_t* orow = (BATCH ? out_row_of(a.out, cur.q) : a.out.row0) + out;
        void* oval = BATCH ? out_val_of(a.out, cur.q) : a.out.val0;
        warp_column<VB, true, U>(in, a, sm, cur, k, off, j, mul, NB, orow, static_cast<VB*>(oval) + out, resident,
                                 my_ri, my_va, lane);
      }
    }
    __syncwarp();
    c += stride;
    cur = nxt;
    nxt = load_col<NUMERIC, BATCH>(in, a, c + stride, ncols, resident, my_cp, lane, k0);
  }
  if (!NUMERIC && lane == 0 && n_unique) atomicAdd(&a.ctr_w->n_unique, n_unique);
}

// ---------------------------------------------------------------------------
// One pass over the inputs (spkadd_onepass).  Sec. II-D's symbolic phase exists
// so that B can be allocated before the numeric phase; here B goes into
// buffers sized by nnz(B) <= sum_i nnz(A_i) (Sec. II-A), and each column's
// offset comes from a decoupled look-back over tiles of WARPS consecutive
// columns, so no pass reads the rows only to count them.  A block takes a
// tile from a ticket counter (tiles start in ticket order, which the
// look-back needs); each warp runs the numeric passes above on its column,
// counts the repeated rows its bucket sorts meet (nnz(B(:,j)) = s_j minus
// them: Alg. 6's count), and once warp 0 has the tile's offset writes B(:,j).
// ---------------------------------------------------------------------------
struct OnepassArgs {
  const int32_t* s_arr;        // s_j (plan)
  int64_t* col_ptr;            // B: n + 1 int64
  int32_t* out_row;            // B: `capacity` rows
  void* out_val;               // B: `capacity` values
  long long capacity;
  unsigned int* queue;         // tile ticket counter, zero at launch
  unsigned long long* status;  // look-back words, one per tile, zero at launch
  Counters* ctr_w;
  int n;
  int ntiles;
  int smax;
  int force_dedup;
  int debug_stall;             // test switch: tile 1's look-back also waits on a word nothing writes
  unsigned long long wait_ns;  // bound of every device-side wait
};

template <int WARPS>
struct OnepassTile {
  int ticket;
  int bad;                     // the look-back gave up
  long long off;               // the tile's first entry in B
  int u[2][WARPS];             // nnz(B(:,j)) of the tile's columns, by iteration parity
  int uq[WARPS];               // 1: column without repeated rows
};

template <int DT, bool RES, int WARPS, int U>
__global__ void __launch_bounds__(WARPS * 32, 3) k_warp_onepass(Inputs in, OnepassArgs a) {
  using VB = typename std::conditional<DT == 1, double, float>::type;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ OnepassTile<WARPS> T;
  __shared__ uint32_t s_mul[16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int smax = a.smax;
  unsigned char* base = sm_raw + (size_t)wid * warp_col_bytes<VB, true>(smax);
  VB* sval = reinterpret_cast<VB*>(base);
  int32_t* skey = reinterpret_cast<int32_t*>(base + (size_t)smax * sizeof(VB));
  uint32_t* cnt = reinterpret_cast<uint32_t*>(skey + smax);
  uint32_t* mlist = cnt + padded_words(smax);
  if (threadIdx.x < 16) s_mul[threadIdx.x] = in.inst[0].bucket_mul[threadIdx.x];
  const int k = in.inst[0].k;
  const uint32_t m = (uint32_t)in.inst[0].m;
  if (RES && k > 32) {  // the host never launches this; never index lanes past k
    if (threadIdx.x == 0) atomicOr(&a.ctr_w->err, ERR_INTERNAL);
    return;
  }
  const int32_t* my_cp = nullptr;
  const int32_t* my_ri = nullptr;
  const VB* my_va = nullptr;
  if (RES && lane < k) {
    my_cp = in.cp[lane];
    my_ri = in.ri[lane];
    my_va = static_cast<const VB*>(in.val[lane]);
  }
  for (int it = 0;; ++it) {
    if (threadIdx.x == 0) T.ticket = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int tile = T.ticket;
    if (tile >= a.ntiles) break;
    int* tu = T.u[it & 1];
    const int j = tile * WARPS + wid;
    const bool live = j < a.n;
    int beg = 0, len = 0, s = 0;
    if (live) {
      if (RES) {
        if (lane < k) {
          beg = __ldg(my_cp + j);
          len = __ldg(my_cp + j + 1) - beg;
        }
        s = warp_sum(len);
      } else {
        s = __ldg(a.s_arr + j);
      }
    }
    int dups = 0;
    bool bad = false;
    if (s > 0) {
      const int qb = max(5, ceil_log2(s));
      const int NB = 1 << qb;
      if (NB > smax) {  // not reachable when every column is light
        if (lane == 0) atomicOr(&a.ctr_w->err, ERR_INTERNAL);
        bad = true;
      } else {
        const uint32_t mul = s_mul[qb];
        if (RES && len > 0)  // the value segment, first read in pass 2, toward L2 now
          l2_prefetch(static_cast<const VB*>(my_va) + beg, (size_t)len * sizeof(VB));
        for (int b = lane; b < padded_words(NB); b += 32) cnt[b] = 0u;
        __syncwarp();
        // Pass 1: entries per bucket; rows outside [0, m) are flagged.
        BucketCountChecked<VB> count{cnt, mul, m, false};
        ChunkCache cc{{0, 0}, {0, 0}, false};
        for_each_column_entry<false, U, VB>(in, k, 0, j, RES, beg, len, my_ri, my_va, lane, count, cc);
        bad = __any_sync(SPK_FULL, count.bad);
        if (!bad) {
          __syncwarp();
          const int nmulti = bucket_scan(cnt, mlist, NB, lane);
          __syncwarp();
          // Pass 2: file every entry at its bucket's next slot.
          BucketFile<VB, true> file{cnt, skey, sval, mul};
          for_each_column_entry<true, U, VB>(in, k, 0, j, RES, beg, len, my_ri, my_va, lane, file, cc);
          __syncwarp();
          dups = warp_sum(sort_buckets<VB, true, true>(skey, sval, mlist, nmulti, lane));
          __syncwarp();
        } else if (lane == 0) {
          atomicOr(&a.ctr_w->err, ERR_RANGE);  // B is not computed for such a column
        }
      }
    }
    const int u = (s > 0 && !bad) ? s - dups : 0;
    if (lane == 0) {
      tu[wid] = u;
      T.uq[wid] = (s > 0 && !bad && dups == 0) ? 1 : 0;
    }
    __syncthreads();
    if (wid == 0) {
      long long agg = lane < WARPS ? tu[lane] : 0;
      agg = lb_warp_sum64(agg);
      bool pois = false;
      const long long excl = tile_lookback(a.status, tile, agg, a.wait_ns, a.debug_stall && tile == 1, &pois, lane);
      const int uq = __popc(__ballot_sync(SPK_FULL, lane < WARPS && T.uq[lane < WARPS ? lane : 0]));
      if (lane == 0) {
        if (uq) atomicAdd(&a.ctr_w->n_unique, uq);
        T.off = excl;
        T.bad = pois ? 1 : 0;
        if (pois) atomicOr(&a.ctr_w->err, ERR_TIMEOUT);
      }
    }
    __syncthreads();
    if (live && !T.bad) {
      long long o = T.off;
      for (int c = 0; c < wid; ++c) o += tu[c];
      if (lane == 0) {
        a.col_ptr[j] = o;
        if (j == a.n - 1) a.col_ptr[a.n] = o + u;
      }
      if (u > 0) {
        if (o + u <= a.capacity)
          write_sorted<VB>(skey, sval, s, u, a.force_dedup, a.out_row + o, static_cast<VB*>(a.out_val) + o, a.ctr_w,
                           lane);
        else if (lane == 0)
          atomicOr(&a.ctr_w->err, ERR_INTERNAL);
      }
    }
    __syncwarp();
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

template <int DT, bool NUMERIC>
static cudaError_t launch_warp_col(const Inputs& in, WarpColArgs a, int warp_max, int n_cols_hint,
                                   const DeviceInfo& dev, cudaStream_t st) {
  using VB = typename std::conditional<DT == 1, double, float>::type;
  constexpr int WARPS = 8;
  a.smax = pow2_at_least(warp_max) < 32 ? 32 : pow2_at_least(warp_max);
  const size_t smem = (size_t)WARPS * warp_col_bytes<VB, NUMERIC>(a.smax);
  constexpr int U = NUMERIC ? 8 : 16;
  auto kern = in.col_inst ? k_warp_col<DT, NUMERIC, true, false, WARPS, U>
              : in.kmax <= 32 ? k_warp_col<DT, NUMERIC, false, true, WARPS, U>
                              : k_warp_col<DT, NUMERIC, false, false, WARPS, U>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = dev.sms * blocks_per_sm(dev, smem + 128, WARPS * 32);
  if (n_cols_hint >= 0) {
    const int need = (n_cols_hint + WARPS - 1) / WARPS;
    if (grid > need) grid = need;
    if (grid < 1) return cudaSuccess;
  }
  kern<<<grid, WARPS * 32, smem, st>>>(in, a);
  return cudaGetLastError();
}

cudaError_t launch_sym_warp(const Inputs& in, const int32_t* list, const int32_t* s, const Counters* ctr,
                            int32_t* u, int warp_max, Counters* ctr_w, const DeviceInfo& dev, cudaStream_t st) {
  WarpColArgs a{};
  a.list = list;
  a.ctr = ctr;
  a.s_arr = s;
  a.u_out = u;
  a.ctr_w = ctr_w;
  a.only_dtype = -1;
  return launch_warp_col<0, false>(in, a, warp_max, -1, dev, st);
}

cudaError_t launch_num_warp(const Inputs& in, int dt, const int32_t* list, const Counters* ctr, int n_cols,
                            const int32_t* s, const int32_t* u, const int64_t* col_ptr, const Outs& out,
                            int warp_max, int sort_mode, Counters* ctr_w, const DeviceInfo& dev,
                            cudaStream_t st) {
  if (n_cols <= 0) return cudaSuccess;
  WarpColArgs a{};
  a.list = list;
  a.ctr = ctr;
  a.s_arr = s;
  a.u_arr = u;
  a.col_ptr = col_ptr;
  a.out = out;
  a.ctr_w = ctr_w;
  a.force_dedup = sort_mode == 1;
  a.unsorted_out = sort_mode == 2;
  a.only_dtype = -1;
  if (dt == 0) return launch_warp_col<0, true>(in, a, warp_max, n_cols, dev, st);
  if (dt == 1) return launch_warp_col<1, true>(in, a, warp_max, n_cols, dev, st);
  // Mixed batch: one launch per dtype, each skipping the other dtype's columns.
  a.only_dtype = 0;
  cudaError_t e = launch_warp_col<0, true>(in, a, warp_max, n_cols, dev, st);
  a.only_dtype = 1;
  if (e == cudaSuccess) e = launch_warp_col<1, true>(in, a, warp_max, n_cols, dev, st);
  return e;
}

template <int DT>
static cudaError_t launch_onepass_t(const Inputs& in, OnepassArgs a, int warp_max, const DeviceInfo& dev,
                                    cudaStream_t st, int* grid_out) {
  using VB = typename std::conditional<DT == 1, double, float>::type;
  constexpr int WARPS = 8;  // columns per tile (warps per block)
  constexpr int U = 8;
  a.smax = pow2_at_least(warp_max) < 32 ? 32 : pow2_at_least(warp_max);
  const size_t smem = (size_t)WARPS * warp_col_bytes<VB, true>(a.smax);
  auto kern = in.kmax <= 32 ? k_warp_onepass<DT, true, WARPS, U> : k_warp_onepass<DT, false, WARPS, U>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WARPS * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int grid = dev.sms * occ;
  if (grid > a.ntiles) grid = a.ntiles;
  *grid_out = grid;
  kern<<<grid, WARPS * 32, smem, st>>>(in, a);
  return cudaGetLastError();
}

int onepass_tile_cols() { return 8; }

size_t onepass_scratch_bytes(int64_t ncols) { return 8 + (size_t)((ncols + 7) / 8) * 8 + 8; }

cudaError_t launch_onepass(const Inputs& in, int dt, const int32_t* s, int n, int warp_max, int64_t* col_ptr,
                           int32_t* out_row, void* out_val, long long capacity, void* scratch, int force_dedup,
                           int debug_stall, unsigned long long wait_ns, Counters* ctr, const DeviceInfo& dev,
                           cudaStream_t st, int* grid_out) {
  *grid_out = 0;
  if (warp_max < 1 || warp_max > WARP_MAX_LIMIT || in.col_inst) return cudaErrorInvalidValue;
  OnepassArgs a{};
  a.s_arr = s;
  a.col_ptr = col_ptr;
  a.out_row = out_row;
  a.out_val = out_val;
  a.capacity = capacity;
  a.ctr_w = ctr;
  a.n = n;
  a.ntiles = (n + onepass_tile_cols() - 1) / onepass_tile_cols();
  a.force_dedup = force_dedup;
  a.debug_stall = debug_stall;
  a.wait_ns = wait_ns;
  a.queue = static_cast<unsigned int*>(scratch);
  a.status = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + 8);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 8 + (size_t)a.ntiles * 8, st);
  if (e != cudaSuccess || a.ntiles == 0) return e;
  return dt == 1 ? launch_onepass_t<1>(in, a, warp_max, dev, st, grid_out)
                 : launch_onepass_t<0>(in, a, warp_max, dev, st, grid_out);
}

}  // namespace spk
