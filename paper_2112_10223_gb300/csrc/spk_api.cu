// spk_api.cu -- the C ABI (include/spkadd.h): argument checks, workspace,
// phase ordering and kernel launches.  No compute happens on the host.
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "spkadd.h"
#include "spk_common.cuh"
#include "spk_launch.h"

#define SPK_API extern "C" __attribute__((visibility("default")))

using spk::Counters;
using spk::DeviceInfo;
using spk::Inputs;
using spk::Window;

namespace {

enum State { ST_PLANNED = 1, ST_SYMBOLIC = 2, ST_NUMERIC = 3 };

struct Pinned {  // per-thread pinned readback block
  Counters ctr;
  long long nnz;
};

Pinned* pinned_block() {
  static thread_local Pinned* p = nullptr;
  if (!p) {
    void* q = nullptr;
    if (cudaMallocHost(&q, sizeof(Pinned)) != cudaSuccess) return nullptr;
    p = static_cast<Pinned*>(q);
  }
  return p;
}

std::mutex g_dev_mu;
DeviceInfo g_dev[64];
bool g_dev_ok[64];

cudaError_t device_info(int dev, DeviceInfo* out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_dev_ok[dev]) {
    DeviceInfo d{};
    cudaError_t e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    // Keep freed stream-ordered memory cached in this process's default pool,
    // so a plan/destroy cycle per call does not return memory to the driver.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_dev[dev] = d;
    g_dev_ok[dev] = true;
  }
  *out = g_dev[dev];
  return cudaSuccess;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Carver {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    size_t o = align_up(off, 256);
    off = o + count * sizeof(T);
    return o;
  }
};

spkadd_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SPKADD_OK;
  if (e == cudaErrorMemoryAllocation) return SPKADD_ERR_NOMEM;
  return SPKADD_ERR_CUDA;
}

spkadd_status from_device_err(int32_t err) {
  if (err & spk::ERR_OVERFLOW) return SPKADD_ERR_OVERFLOW;
  if (err & spk::ERR_RANGE) return SPKADD_ERR_INDEX_RANGE;
  if (err & spk::ERR_UNSORTED) return SPKADD_ERR_UNSORTED;
  if (err & spk::ERR_TIMEOUT) return SPKADD_ERR_TIMEOUT;
  if (err & (spk::ERR_WINDOW_CAP | spk::ERR_INTERNAL)) return SPKADD_ERR_INTERNAL;
  return SPKADD_OK;
}

}  // namespace

// Device memory through the caller's allocator (options.alloc / free), else
// stream-ordered cudaMallocAsync / cudaFreeAsync on st.
static void* ws_alloc(const spkadd_options& o, cudaStream_t st, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (o.alloc) return o.alloc(bytes, (void*)st, o.alloc_ctx);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
static void ws_free(const spkadd_options& o, cudaStream_t st, void* p) {
  if (!p) return;
  if (o.alloc) o.free(p, (void*)st, o.alloc_ctx);
  else cudaFreeAsync(p, st);
}

struct spkadd_handle {
  bool batch = false;       // made by spkadd_batch_plan
  int count = 0;            // problems (1 for spkadd_plan)
  int total_k = 0;          // inputs of all problems
  int kmax = 0;
  int64_t mmax = 0;
  int64_t ncols = 0;        // columns of all problems
  int64_t nnz_in = 0;
  int dt_mode = 0;          // 0 = all float, 1 = all double, 2 = mixed
  int f32_kinds = 0;        // float problems held: bit 0 k <= 167, bit 1 167 < k <= FP32_PHASED_MAX_K, bit 2 larger
  spkadd_dtype dt0 = SPKADD_F64;
  cudaStream_t st = nullptr;
  spkadd_options opt{};
  int device = 0;
  DeviceInfo dev{};
  char* ws = nullptr;
  size_t ws_bytes = 0;
  char* offs_buf = nullptr;
  size_t offs_bytes = 0;
  Inputs in{};
  const int64_t* d_nnz = nullptr;      // per (problem, input) nnz
  int32_t* d_col_inst = nullptr;       // batch: global column -> problem
  int64_t* d_inst_nnz = nullptr;       // batch: per-problem nnz(B)
  void** d_out_tab = nullptr;          // batch: B row / value / col_ptr pointer tables
  int32_t *d_s = nullptr, *d_u = nullptr;
  int32_t *d_wl = nullptr, *d_cl = nullptr, *d_hl = nullptr;
  Window* d_win = nullptr;
  int32_t* d_search = nullptr;
  int64_t win_cap = 0;
  Counters* d_ctr = nullptr;
  Window* d_wsort = nullptr;  // thread-block item records grouped by problem kind (batches of several kinds)
  int64_t* d_colptr = nullptr;
  long long* d_scan = nullptr;
  char* d_op = nullptr;                // one-pass: ticket counter and look-back words
  bool onepass = false;                // B last computed by the one-pass kernel
  int32_t* d_offs = nullptr;
  Counters h_ctr{};
  int64_t nnz_out = -1;
  std::vector<int64_t> nnz_each;       // batch: per-problem nnz(B) after symbolic
  int state = 0;
  int64_t launches = 0;  // kernels launched by this handle

  void* dev_alloc(size_t bytes) { return ws_alloc(opt, st, bytes); }
  void dev_free(void* p) { ws_free(opt, st, p); }
};

SPK_API void spkadd_default_options(spkadd_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->validate = 0;
  opt->warp_max = spk::WARP_MAX_LIMIT;
  opt->cta_max = spk::CTA_MAX_LIMIT;
  opt->window_max = spk::WINDOW_MAX_LIMIT;
  opt->sort_mode = 0;
  opt->input_order = 0;
  opt->block_accumulator = 0;
  opt->wait_timeout_ms = 2000;
  opt->test_stall = 0;
}

SPK_API const char* spkadd_status_string(spkadd_status s) {
  switch (s) {
    case SPKADD_OK: return "SPKADD_OK";
    case SPKADD_ERR_INVALID_ARG: return "SPKADD_ERR_INVALID_ARG: invalid argument";
    case SPKADD_ERR_SHAPE_MISMATCH: return "SPKADD_ERR_SHAPE_MISMATCH: inputs disagree on m or n";
    case SPKADD_ERR_UNSORTED: return "SPKADD_ERR_UNSORTED: rows not strictly increasing in a column";
    case SPKADD_ERR_INDEX_RANGE: return "SPKADD_ERR_INDEX_RANGE: row or column pointer out of range";
    case SPKADD_ERR_OVERFLOW: return "SPKADD_ERR_OVERFLOW: size does not fit the index type";
    case SPKADD_ERR_NOMEM: return "SPKADD_ERR_NOMEM: device workspace allocation failed";
    case SPKADD_ERR_CUDA: return "SPKADD_ERR_CUDA: CUDA call or kernel launch failed";
    case SPKADD_ERR_TIMEOUT: return "SPKADD_ERR_TIMEOUT: bounded device wait gave up";
    case SPKADD_ERR_STATE: return "SPKADD_ERR_STATE: call out of order";
    case SPKADD_ERR_UNSUPPORTED: return "SPKADD_ERR_UNSUPPORTED: request not supported by this library";
    case SPKADD_ERR_INTERNAL: return "SPKADD_ERR_INTERNAL: device-side invariant failed";
  }
  return "SPKADD_ERR_?: unknown status";
}

SPK_API int spkadd_version(void) { return 100; }

static spkadd_status check_options(const spkadd_options& o) {
  if (o.warp_max < 1 || o.warp_max > spk::WARP_MAX_LIMIT) return SPKADD_ERR_INVALID_ARG;
  if (o.cta_max < o.warp_max || o.cta_max > spk::CTA_MAX_LIMIT) return SPKADD_ERR_INVALID_ARG;
  if (o.window_max < 1024 || o.window_max > spk::WINDOW_MAX_LIMIT) return SPKADD_ERR_INVALID_ARG;
  if (o.sort_mode < 0 || o.sort_mode > 2) return SPKADD_ERR_INVALID_ARG;
  if (o.input_order != 0 && o.input_order != 1) return SPKADD_ERR_INVALID_ARG;
  if (o.block_accumulator < 0 || o.block_accumulator > 2) return SPKADD_ERR_INVALID_ARG;
  if ((o.alloc == nullptr) != (o.free == nullptr)) return SPKADD_ERR_INVALID_ARG;
  if (o.wait_timeout_ms < 1 || o.wait_timeout_ms > 600000) return SPKADD_ERR_INVALID_ARG;
  if (o.test_stall != 0 && o.test_stall != 1) return SPKADD_ERR_INVALID_ARG;
  return SPKADD_OK;
}

// Host checks of one problem's descriptors; adds its input count to *nnz.
static spkadd_status check_problem(int k, const spkadd_csc* A, spkadd_dtype dtype, int64_t* nnz) {
  if (k < 1 || !A) return SPKADD_ERR_INVALID_ARG;
  if (k > SPKADD_MAX_K) return SPKADD_ERR_UNSUPPORTED;
  if (dtype != SPKADD_F32 && dtype != SPKADD_F64) return SPKADD_ERR_INVALID_ARG;
  const int64_t m = A[0].m, n = A[0].n;
  for (int i = 0; i < k; ++i) {
    const spkadd_csc& a = A[i];
    if (a.m < 0 || a.n < 0 || a.nnz < 0) return SPKADD_ERR_INVALID_ARG;
    if (a.m >= INT32_MAX || a.n >= INT32_MAX || a.nnz > INT32_MAX) return SPKADD_ERR_OVERFLOW;
    if (a.m != m || a.n != n) return SPKADD_ERR_SHAPE_MISMATCH;
    if (!a.col_ptr) return SPKADD_ERR_INVALID_ARG;
    if (a.nnz > 0 && (!a.row_idx || !a.val)) return SPKADD_ERR_INVALID_ARG;
    *nnz += a.nnz;
  }
  return SPKADD_OK;
}

// Numeric work items one problem can produce: heavy windows <= nnz /
// (window_max - 64) + one per heavy column and slab; CTA columns <=
// min(n, nnz / (warp_max + 1)).
static int64_t window_bound(int64_t m, int64_t n, int64_t nnz, const spkadd_options& o) {
  const int64_t slab_rows = (int64_t)1 << spk::SLAB_BITS;
  const int64_t slabs = m > 0 ? (m + slab_rows - 1) / slab_rows : 1;
  int64_t heavy_cols = nnz / (o.cta_max + 1);
  if (heavy_cols > n) heavy_cols = n;
  int64_t cta_cols = nnz / (o.warp_max + 1);
  if (cta_cols > n) cta_cols = n;
  return nnz / (o.window_max - 64) + heavy_cols * (slabs + 1) + cta_cols + 16;
}

// Plans `count` problems (count = 1 and batch = false for spkadd_plan).
static spkadd_status plan_problems(spkadd_handle** hp, bool batch, int count, const int* ks,
                                   const spkadd_csc* const* As, const spkadd_dtype* dts, void* stream,
                                   const spkadd_options* opt) {
  if (!hp) return SPKADD_ERR_INVALID_ARG;
  *hp = nullptr;
  if (count < 1 || !ks || !As || !dts) return SPKADD_ERR_INVALID_ARG;
  spkadd_options o;
  if (opt) o = *opt;
  else spkadd_default_options(&o);
  spkadd_status os = check_options(o);
  if (os != SPKADD_OK) return os;
  int64_t nnz_in = 0, total_k = 0, ncols = 0, mmax = 0, win_cap = 0;
  int kmax = 0, f32_kinds = 0;
  bool any32 = false, any64 = false;
  for (int q = 0; q < count; ++q) {
    int64_t nz = 0;
    const spkadd_status ps = check_problem(ks[q], As[q], dts[q], &nz);
    if (ps != SPKADD_OK) return ps;
    nnz_in += nz;
    total_k += ks[q];
    ncols += As[q][0].n;
    if (As[q][0].m > mmax) mmax = As[q][0].m;
    if (ks[q] > kmax) kmax = ks[q];
    (dts[q] == SPKADD_F64 ? any64 : any32) = true;
    if (dts[q] == SPKADD_F32)
      f32_kinds |= ks[q] <= spk::FP32_ACC_TERMS ? 1 : (ks[q] <= spk::FP32_PHASED_MAX_K ? 2 : 4);
    win_cap += window_bound(As[q][0].m, As[q][0].n, nz, o);
  }
  if (total_k >= INT32_MAX || ncols >= INT32_MAX || win_cap >= INT32_MAX) return SPKADD_ERR_OVERFLOW;

  spkadd_handle* h = new (std::nothrow) spkadd_handle();
  if (!h) return SPKADD_ERR_NOMEM;
  h->batch = batch;
  h->count = count;
  h->total_k = (int)total_k;
  h->kmax = kmax;
  h->mmax = mmax;
  h->ncols = ncols;
  h->nnz_in = nnz_in;
  h->dt_mode = any32 && any64 ? 2 : (any64 ? 1 : 0);
  h->f32_kinds = f32_kinds;
  h->dt0 = dts[0];
  h->st = static_cast<cudaStream_t>(stream);
  h->opt = o;
  h->win_cap = win_cap;
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce == cudaSuccess) ce = device_info(h->device, &h->dev);
  if (ce != cudaSuccess) {
    delete h;
    return from_cuda(ce);
  }
  const bool multi = count > 1;

  Carver cv;
  const size_t o_inst = cv.take<spk::Inst>(count);
  const size_t o_cp = cv.take<const int32_t*>(total_k);
  const size_t o_ri = cv.take<const int32_t*>(total_k);
  const size_t o_va = cv.take<const void*>(total_k);
  const size_t o_nnz = cv.take<int64_t>(total_k);
  const size_t o_ctr = cv.take<Counters>(1);
  const size_t o_out = cv.take<void*>(batch ? 3 * (size_t)count : 0);
  const size_t o_inz = cv.take<int64_t>(batch ? count : 0);
  const size_t o_ci = cv.take<int32_t>(multi ? ncols : 0);
  const size_t o_s = cv.take<int32_t>(ncols);
  const size_t o_u = cv.take<int32_t>(ncols);
  const size_t o_wl = cv.take<int32_t>(ncols);
  const size_t o_cl = cv.take<int32_t>(ncols);
  const size_t o_hl = cv.take<int32_t>(2 * ncols);
  const size_t o_win = cv.take<Window>(win_cap);
  const size_t o_srch = cv.take<int32_t>(win_cap);
  const int cta_kinds = spk::num_cta_kinds(any32 && any64 ? 2 : (any64 ? 1 : 0), f32_kinds);
  const size_t o_ws = cv.take<Window>(__builtin_popcount(cta_kinds) > 1 ? win_cap : 0);
  const size_t o_colp = cv.take<int64_t>(ncols + 1);
  const size_t o_scan = cv.take<long long>(spk::scan_tiles(ncols));
  const size_t o_op = cv.take<char>(batch ? 0 : spk::onepass_scratch_bytes(ncols));
  h->ws_bytes = align_up(cv.off, 256);
  h->ws = static_cast<char*>(h->dev_alloc(h->ws_bytes));
  if (!h->ws) {
    delete h;
    return SPKADD_ERR_NOMEM;
  }
  h->d_nnz = reinterpret_cast<const int64_t*>(h->ws + o_nnz);
  h->d_ctr = reinterpret_cast<Counters*>(h->ws + o_ctr);
  h->d_out_tab = batch ? reinterpret_cast<void**>(h->ws + o_out) : nullptr;
  h->d_inst_nnz = batch ? reinterpret_cast<int64_t*>(h->ws + o_inz) : nullptr;
  h->d_col_inst = multi ? reinterpret_cast<int32_t*>(h->ws + o_ci) : nullptr;
  h->d_s = reinterpret_cast<int32_t*>(h->ws + o_s);
  h->d_u = reinterpret_cast<int32_t*>(h->ws + o_u);
  h->d_wl = reinterpret_cast<int32_t*>(h->ws + o_wl);
  h->d_cl = reinterpret_cast<int32_t*>(h->ws + o_cl);
  h->d_hl = reinterpret_cast<int32_t*>(h->ws + o_hl);
  h->d_win = reinterpret_cast<Window*>(h->ws + o_win);
  h->d_search = reinterpret_cast<int32_t*>(h->ws + o_srch);
  h->d_wsort = __builtin_popcount(cta_kinds) > 1 ? reinterpret_cast<Window*>(h->ws + o_ws) : nullptr;
  h->d_colptr = reinterpret_cast<int64_t*>(h->ws + o_colp);
  h->d_scan = reinterpret_cast<long long*>(h->ws + o_scan);
  h->d_op = batch ? nullptr : h->ws + o_op;

  // Problem and pointer tables plus zeroed counters: one host staging
  // buffer, one copy.
  const size_t desc_bytes = o_ctr + sizeof(Counters);
  std::vector<char> host(desc_bytes, 0);
  spk::Inst* hi = reinterpret_cast<spk::Inst*>(host.data() + o_inst);
  int ptr = 0, colbase = 0;
  for (int q = 0; q < count; ++q) {
    const spkadd_csc* A = As[q];
    spk::Inst& I = hi[q];
    I.k = ks[q];
    I.m = (int32_t)A[0].m;
    I.n = (int32_t)A[0].n;
    I.dtype = dts[q] == SPKADD_F64 ? 1 : 0;
    I.colbase = colbase;
    I.ptr_off = ptr;
    for (int b = 0; b < 16; ++b) {
      const uint64_t nb = 1ull << b;
      I.bucket_mul[b] = (I.m == 0 || nb >= (uint64_t)I.m) ? 0xFFFFFFFFu : (uint32_t)((nb << 32) / (uint64_t)I.m);
    }
    for (int i = 0; i < ks[q]; ++i, ++ptr) {
      reinterpret_cast<const int32_t**>(host.data() + o_cp)[ptr] = A[i].col_ptr;
      reinterpret_cast<const int32_t**>(host.data() + o_ri)[ptr] = A[i].row_idx;
      reinterpret_cast<const void**>(host.data() + o_va)[ptr] = A[i].val;
      reinterpret_cast<int64_t*>(host.data() + o_nnz)[ptr] = A[i].nnz;
    }
    colbase += I.n;
  }
  ce = cudaMemcpyAsync(h->ws, host.data(), desc_bytes, cudaMemcpyHostToDevice, h->st);
  if (ce != cudaSuccess) {
    spkadd_destroy(h);
    return from_cuda(ce);
  }
  h->in.inst = reinterpret_cast<const spk::Inst*>(h->ws + o_inst);
  h->in.col_inst = h->d_col_inst;
  h->in.cp = reinterpret_cast<const int32_t* const*>(h->ws + o_cp);
  h->in.ri = reinterpret_cast<const int32_t* const*>(h->ws + o_ri);
  h->in.val = reinterpret_cast<const void* const*>(h->ws + o_va);
  h->in.ninst = count;
  h->in.ncols = (int32_t)ncols;
  h->in.kmax = kmax;
  h->in.mmax = (int32_t)mmax;
  h->in.sorted = o.input_order == 0 ? 1 : 0;
  if (multi) {
    ce = spk::launch_col_inst(h->in, h->d_col_inst, h->dev.sms, h->st);
    h->launches += 1;
    if (ce != cudaSuccess) {
      spkadd_destroy(h);
      return from_cuda(ce);
    }
  }

  if (o.validate) {
    ce = spk::launch_validate(h->in, h->d_nnz, h->d_ctr, h->dev.sms, h->st);
    h->launches += ncols > 0;
    Pinned* pb = pinned_block();
    if (ce == cudaSuccess && !pb) ce = cudaErrorMemoryAllocation;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&pb->ctr, h->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
    if (ce != cudaSuccess) {
      spkadd_destroy(h);
      return from_cuda(ce);
    }
    spkadd_status vs = from_device_err(pb->ctr.err);
    if (vs != SPKADD_OK) {
      spkadd_destroy(h);
      return vs;
    }
  }
  ce = spk::launch_bin(h->in, o.warp_max, o.cta_max, h->d_s, h->d_u, h->d_wl, h->d_cl, h->d_hl, h->d_ctr,
                       h->dev.sms, h->st);
  h->launches += ncols > 0;
  if (ce != cudaSuccess) {
    spkadd_destroy(h);
    return from_cuda(ce);
  }
  h->state = ST_PLANNED;
  *hp = h;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_plan(spkadd_handle** hp, int k, const spkadd_csc* A, spkadd_dtype dtype, void* stream,
                                  const spkadd_options* opt) {
  if (!hp) return SPKADD_ERR_INVALID_ARG;
  *hp = nullptr;
  if (k < 1 || !A) return SPKADD_ERR_INVALID_ARG;
  const spkadd_csc* As[1] = {A};
  return plan_problems(hp, false, 1, &k, As, &dtype, stream, opt);
}

SPK_API spkadd_status spkadd_batch_plan(spkadd_handle** hp, int count, const int* k, const spkadd_csc* const* A,
                                        const spkadd_dtype* dtype, void* stream, const spkadd_options* opt) {
  return plan_problems(hp, true, count, k, A, dtype, stream, opt);
}

// The symbolic phase of every problem of the handle; one stream
// synchronisation.  Fills h->nnz_out (all problems) and, for a batch,
// h->nnz_each.
static spkadd_status run_symbolic(spkadd_handle* h) {
  cudaError_t ce = cudaSuccess;
  if (h->ncols > 0) {
    ce = spk::launch_sym_heavy(h->in, h->d_hl, h->d_s, h->d_ctr, h->d_u, h->d_win, h->d_search, h->win_cap, h->d_ctr,
                               h->opt.window_max, h->opt.block_accumulator, h->dev, h->st);
    if (ce == cudaSuccess)
      ce = spk::launch_sym_cta(h->in, h->d_cl, h->d_s, h->d_ctr, h->d_u, h->d_win, h->win_cap, h->d_ctr,
                               h->opt.cta_max, h->dev, h->st);
    if (ce == cudaSuccess)
      ce = spk::launch_sym_warp(h->in, h->d_wl, h->d_s, h->d_ctr, h->d_u, h->opt.warp_max, h->d_ctr, h->dev,
                                h->st);
    h->launches += 3;
    // Several problem kinds: the thread-block items grouped by kind for the numeric launches.
    if (ce == cudaSuccess && h->d_wsort) {
      ce = spk::launch_kind_sort(h->in, h->d_win, (int)h->win_cap, h->d_wsort, h->d_ctr, h->dev, h->st);
      h->launches += 2;
    }
  }
  if (ce == cudaSuccess) ce = spk::launch_scan(h->d_u, (int)h->ncols, h->d_scan, h->d_colptr, h->st);
  h->launches += h->ncols > 0 ? 3 : 2;
  if (ce == cudaSuccess && h->batch) {
    ce = spk::launch_inst_nnz(h->in, h->d_colptr, h->d_inst_nnz, h->st);
    h->launches += 1;
  }
  Pinned* pb = pinned_block();
  if (ce == cudaSuccess && !pb) ce = cudaErrorMemoryAllocation;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&pb->ctr, h->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(&pb->nnz, h->d_colptr + h->ncols, sizeof(long long), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess && h->batch) {
    h->nnz_each.assign(h->count, 0);
    ce = cudaMemcpyAsync(h->nnz_each.data(), h->d_inst_nnz, sizeof(int64_t) * h->count, cudaMemcpyDeviceToHost,
                         h->st);
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  h->h_ctr = pb->ctr;
  const spkadd_status ds = from_device_err(h->h_ctr.err);
  if (ds != SPKADD_OK) return ds;
  h->nnz_out = pb->nnz;

  // Per-input offsets of split windows (sized now that their count is known).
  const int64_t ns = h->h_ctr.n_search;
  if (ns > 0) {
    const size_t need = (size_t)ns * h->kmax * 2 * sizeof(int32_t);
    if (need > h->offs_bytes) {
      h->dev_free(h->offs_buf);
      h->offs_buf = static_cast<char*>(h->dev_alloc(need));
      h->offs_bytes = h->offs_buf ? need : 0;
      if (!h->offs_buf) return SPKADD_ERR_NOMEM;
    }
    h->d_offs = reinterpret_cast<int32_t*>(h->offs_buf);
    ce = spk::launch_window_search(h->in, h->d_win, h->d_search, (int)ns, h->d_offs, h->dev.sms, h->st);
    if (ce != cudaSuccess) return from_cuda(ce);
    h->launches += 2;
  }
  h->state = ST_SYMBOLIC;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_symbolic(spkadd_handle* h, int64_t* nnz_B) {
  if (!h || !nnz_B || h->batch) return SPKADD_ERR_INVALID_ARG;
  if (h->state < ST_PLANNED) return SPKADD_ERR_STATE;
  if (h->state < ST_SYMBOLIC) {
    const spkadd_status s = run_symbolic(h);
    if (s != SPKADD_OK) return s;
  }
  *nnz_B = h->nnz_out;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_batch_symbolic(spkadd_handle* h, int64_t* nnz_B) {
  if (!h || !nnz_B) return SPKADD_ERR_INVALID_ARG;
  if (h->state < ST_PLANNED) return SPKADD_ERR_STATE;
  if (h->state < ST_SYMBOLIC) {
    const spkadd_status s = run_symbolic(h);
    if (s != SPKADD_OK) return s;
  }
  if (h->batch) std::memcpy(nnz_B, h->nnz_each.data(), sizeof(int64_t) * h->count);
  else nnz_B[0] = h->nnz_out;
  return SPKADD_OK;
}

// The numeric kernels of every problem, writing through `out`.
static spkadd_status run_numeric(spkadd_handle* h, const spk::Outs& out) {
  cudaError_t ce = cudaSuccess;
  const int cta_items = h->h_ctr.n_windows;
  int item_launches = 0;
  if (cta_items > 0)
    ce = spk::launch_num_cta(h->in, h->dt_mode, h->f32_kinds, h->d_win, cta_items, h->d_wsort, h->h_ctr.kind_n,
                             h->d_offs, h->d_colptr, out,
                             h->opt.window_max > h->opt.cta_max ? h->opt.window_max : h->opt.cta_max,
                             h->opt.block_accumulator, h->d_ctr, h->dev, h->st, &item_launches);
  h->launches += item_launches;
  if (ce == cudaSuccess && h->h_ctr.n_warp > 0)
    ce = spk::launch_num_warp(h->in, h->dt_mode, h->d_wl, h->d_ctr, h->h_ctr.n_warp, h->d_s, h->d_u, h->d_colptr,
                              out, h->opt.warp_max, h->opt.sort_mode, h->d_ctr, h->dev, h->st);
  h->launches += (h->h_ctr.n_warp > 0) * (h->dt_mode == 2 ? 2 : 1);
  return from_cuda(ce);
}

SPK_API spkadd_status spkadd_numeric(spkadd_handle* h, int64_t* B_col_ptr, int32_t* B_row_idx, void* B_val) {
  if (!h || !B_col_ptr || h->batch) return SPKADD_ERR_INVALID_ARG;
  if (h->state < ST_SYMBOLIC) return SPKADD_ERR_STATE;
  if (h->nnz_out > 0 && (!B_row_idx || !B_val)) return SPKADD_ERR_INVALID_ARG;
  cudaError_t ce = cudaMemcpyAsync(B_col_ptr, h->d_colptr, (size_t)(h->ncols + 1) * sizeof(int64_t),
                                   cudaMemcpyDeviceToDevice, h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  h->onepass = false;
  spk::Outs out{};
  out.row0 = B_row_idx;
  out.val0 = B_val;
  out.cp0 = B_col_ptr;
  const spkadd_status s = run_numeric(h, out);
  if (s != SPKADD_OK) return s;
  h->state = ST_NUMERIC;
  return SPKADD_OK;
}

// One pass over the inputs (symbolic count, scan by decoupled look-back and
// numeric sum fused) into buffers sized by sum_i nnz(A_i); the phases of
// spkadd_symbolic / spkadd_numeric when the problem does not qualify.
SPK_API spkadd_status spkadd_onepass(spkadd_handle* h, int64_t* B_col_ptr, int32_t* B_row_idx, void* B_val,
                                     int64_t capacity, int64_t* nnz_B) {
  if (!h || !B_col_ptr || !nnz_B || h->batch) return SPKADD_ERR_INVALID_ARG;
  if (h->state < ST_PLANNED) return SPKADD_ERR_STATE;
  if (capacity < h->nnz_in) return SPKADD_ERR_INVALID_ARG;
  if (h->nnz_in > 0 && (!B_row_idx || !B_val)) return SPKADD_ERR_INVALID_ARG;
  Pinned* pb = pinned_block();
  if (!pb) return SPKADD_ERR_NOMEM;
  cudaError_t ce = cudaMemcpyAsync(&pb->ctr, h->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  spkadd_status ds = from_device_err(pb->ctr.err);
  if (ds != SPKADD_OK) return ds;
  const Counters c = pb->ctr;
  const bool fits = h->ncols > 0 && c.n_cta == 0 && c.n_heavy == 0 && c.n_big == 0 && h->dt_mode != 2;
  if (!fits) {
    h->onepass = false;
    spkadd_status s = SPKADD_OK;
    if (h->state < ST_SYMBOLIC) s = run_symbolic(h);
    if (s != SPKADD_OK) return s;
    s = spkadd_numeric(h, B_col_ptr, B_row_idx, B_val);
    if (s != SPKADD_OK) return s;
    *nnz_B = h->nnz_out;
    return SPKADD_OK;
  }
  h->h_ctr = c;
  int grid = 0;
  ce = cudaMemsetAsync(&h->d_ctr->n_unique, 0, sizeof(int32_t), h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  ce = spk::launch_onepass(h->in, h->dt_mode, h->d_s, (int)h->ncols, h->opt.warp_max, B_col_ptr,
                           B_row_idx, B_val, capacity, h->d_op, h->opt.sort_mode == 1, h->opt.test_stall,
                           (unsigned long long)h->opt.wait_timeout_ms * 1000000ull, h->d_ctr, h->dev, h->st, &grid);
  if (ce != cudaSuccess) return from_cuda(ce);
  h->launches += grid > 0 ? 1 : 0;
  ce = cudaMemcpyAsync(&pb->ctr, h->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(&pb->nnz, B_col_ptr + h->ncols, sizeof(long long), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  h->h_ctr = pb->ctr;
  ds = from_device_err(pb->ctr.err);
  if (ds != SPKADD_OK) return ds;
  h->nnz_out = pb->nnz;
  h->onepass = true;
  h->state = ST_NUMERIC;
  *nnz_B = h->nnz_out;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_batch_numeric(spkadd_handle* h, int64_t* const* B_col_ptr, int32_t* const* B_row_idx,
                                           void* const* B_val) {
  if (!h || !B_col_ptr || !B_row_idx || !B_val) return SPKADD_ERR_INVALID_ARG;
  if (h->state < ST_SYMBOLIC) return SPKADD_ERR_STATE;
  if (!h->batch) return spkadd_numeric(h, B_col_ptr[0], B_row_idx[0], B_val[0]);
  const int n = h->count;
  std::vector<void*> tab(3 * (size_t)n);
  for (int q = 0; q < n; ++q) {
    if (!B_col_ptr[q]) return SPKADD_ERR_INVALID_ARG;
    if (h->nnz_each[q] > 0 && (!B_row_idx[q] || !B_val[q])) return SPKADD_ERR_INVALID_ARG;
    tab[q] = B_row_idx[q];
    tab[n + q] = B_val[q];
    tab[2 * (size_t)n + q] = B_col_ptr[q];
  }
  // Pageable source: the call returns once the table is staged, so `tab`
  // may go out of scope right after.
  cudaError_t ce =
      cudaMemcpyAsync(h->d_out_tab, tab.data(), sizeof(void*) * tab.size(), cudaMemcpyHostToDevice, h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  spk::Outs out{};
  out.row0 = B_row_idx[0];
  out.val0 = B_val[0];
  out.cp0 = B_col_ptr[0];
  out.rows = reinterpret_cast<int32_t* const*>(h->d_out_tab);
  out.vals = reinterpret_cast<void* const*>(h->d_out_tab + n);
  out.cps = reinterpret_cast<int64_t* const*>(h->d_out_tab + 2 * (size_t)n);
  ce = spk::launch_out_colptr(h->in, out, h->d_colptr, h->dev.sms, h->st);
  h->launches += 1;
  if (ce != cudaSuccess) return from_cuda(ce);
  const spkadd_status s = run_numeric(h, out);
  if (s != SPKADD_OK) return s;
  h->state = ST_NUMERIC;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_get_info(spkadd_handle* h, spkadd_info* info) {
  if (!h || !info) return SPKADD_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->k = h->total_k;
  info->m = h->mmax;
  info->n = h->ncols;
  info->problems = h->count;
  info->nnz_in = h->nnz_in;
  info->nnz_out = h->state >= ST_SYMBOLIC ? h->nnz_out : -1;
  Pinned* pb = pinned_block();
  if (!pb) return SPKADD_ERR_NOMEM;
  cudaError_t ce = cudaMemcpyAsync(&pb->ctr, h->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  const Counters c = pb->ctr;
  info->cols_warp = c.n_warp;
  info->cols_cta = c.n_cta;
  info->cols_heavy = (int64_t)c.n_heavy + c.n_big;
  info->windows = c.n_windows;
  info->windows_split = c.n_search;
  info->cols_unique = c.n_unique;
  info->workspace_bytes = (int64_t)(h->ws_bytes + h->offs_bytes);
  info->kernel_launches = h->launches;
  info->onepass = h->onepass ? 1 : 0;
  return from_device_err(c.err);
}

SPK_API spkadd_status spkadd_destroy(spkadd_handle* h) {
  if (!h) return SPKADD_OK;
  h->dev_free(h->offs_buf);
  h->dev_free(h->ws);
  delete h;
  return SPKADD_OK;
}

// ---------------------------------------------------------------------------
// Streaming accumulation (Sec. IV, distributed SpGEMM: the stage results of
// sparse SUMMA are added; Sec. V: inputs that arrive in batches, or do not fit
// in memory together, are arranged in batches and each batch is added with
// SpKAdd).  The stream keeps the running sum B on the device; each add of k
// inputs is one (k+1)-way SpKAdd with B as input 0, so only one batch of
// inputs need be resident at a time.
// ---------------------------------------------------------------------------
struct spkadd_stream {
  int64_t m = 0, n = 0;
  spkadd_dtype dtype = SPKADD_F64;
  cudaStream_t st = nullptr;
  spkadd_options opt{};
  int sms = 1;
  int32_t* cp = nullptr;  // running sum B: int32 col_ptr[n + 1], rows, values
  int32_t* ri = nullptr;
  void* va = nullptr;
  int64_t nnz = 0;
  int64_t adds = 0;
  int64_t launches = 0;   // kernels launched by the stream's adds and reads
};

SPK_API spkadd_status spkadd_stream_create(spkadd_stream** sp, int64_t m, int64_t n, spkadd_dtype dtype, void* stream,
                                           const spkadd_options* opt) {
  if (!sp) return SPKADD_ERR_INVALID_ARG;
  *sp = nullptr;
  if (m < 0 || n < 0) return SPKADD_ERR_INVALID_ARG;
  if (m >= INT32_MAX || n >= INT32_MAX) return SPKADD_ERR_OVERFLOW;
  if (dtype != SPKADD_F32 && dtype != SPKADD_F64) return SPKADD_ERR_INVALID_ARG;
  spkadd_options o;
  spkadd_default_options(&o);
  if (opt) o = *opt;
  const spkadd_status cs = check_options(o);
  if (cs != SPKADD_OK) return cs;
  int device = 0, sms = 0;
  cudaError_t ce = cudaGetDevice(&device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (ce != cudaSuccess) return from_cuda(ce);
  spkadd_stream* s = new (std::nothrow) spkadd_stream;
  if (!s) return SPKADD_ERR_NOMEM;
  s->m = m;
  s->n = n;
  s->dtype = dtype;
  s->st = static_cast<cudaStream_t>(stream);
  s->opt = o;
  s->sms = sms > 0 ? sms : 1;
  s->cp = static_cast<int32_t*>(ws_alloc(o, s->st, (size_t)(n + 1) * sizeof(int32_t)));
  if (!s->cp) {
    delete s;
    return SPKADD_ERR_NOMEM;
  }
  ce = cudaMemsetAsync(s->cp, 0, (size_t)(n + 1) * sizeof(int32_t), s->st);  // B = 0: every column empty
  if (ce != cudaSuccess) {
    ws_free(o, s->st, s->cp);
    delete s;
    return from_cuda(ce);
  }
  *sp = s;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_stream_add(spkadd_stream* s, int k, const spkadd_csc* A) {
  if (!s || k < 1 || !A) return SPKADD_ERR_INVALID_ARG;
  if (k >= SPKADD_MAX_K) return SPKADD_ERR_UNSUPPORTED;  // k + 1 inputs with the running sum
  for (int i = 0; i < k; ++i)
    if (A[i].m != s->m || A[i].n != s->n) return SPKADD_ERR_SHAPE_MISMATCH;
  std::vector<spkadd_csc> all;
  try {
    all.resize((size_t)k + 1);
  } catch (...) {
    return SPKADD_ERR_NOMEM;
  }
  all[0] = spkadd_csc{s->m, s->n, s->nnz, s->cp, s->nnz ? s->ri : nullptr, s->nnz ? s->va : nullptr};
  for (int i = 0; i < k; ++i) all[(size_t)i + 1] = A[i];
  spkadd_handle* h = nullptr;
  spkadd_status r = spkadd_plan(&h, k + 1, all.data(), s->dtype, (void*)s->st, &s->opt);
  if (r != SPKADD_OK) return r;
  int64_t nnz = 0;
  r = spkadd_symbolic(h, &nnz);
  if (r == SPKADD_OK && nnz > INT32_MAX) r = SPKADD_ERR_OVERFLOW;  // the sum must stay usable as an input
  int32_t* cp = nullptr;
  int32_t* ri = nullptr;
  void* va = nullptr;
  if (r == SPKADD_OK) {
    const size_t vs = s->dtype == SPKADD_F64 ? 8 : 4;
    cp = static_cast<int32_t*>(ws_alloc(s->opt, s->st, (size_t)(s->n + 1) * sizeof(int32_t)));
    ri = static_cast<int32_t*>(ws_alloc(s->opt, s->st, (size_t)nnz * sizeof(int32_t)));
    va = ws_alloc(s->opt, s->st, (size_t)nnz * vs);
    if (!cp || !ri || !va) r = SPKADD_ERR_NOMEM;
  }
  if (r == SPKADD_OK) {
    const cudaError_t ce = spk::launch_colptr_narrow(h->d_colptr, cp, s->n + 1, s->sms, s->st);
    if (ce != cudaSuccess) r = from_cuda(ce);
  }
  if (r == SPKADD_OK) {
    spk::Outs out{};
    out.row0 = ri;
    out.val0 = va;
    r = run_numeric(h, out);
  }
  if (r == SPKADD_OK) s->launches += h->launches + 1;
  spkadd_destroy(h);  // stream-ordered: its workspace is released after the kernels above
  if (r != SPKADD_OK) {
    ws_free(s->opt, s->st, cp);
    ws_free(s->opt, s->st, ri);
    ws_free(s->opt, s->st, va);
    return r;
  }
  ws_free(s->opt, s->st, s->cp);
  ws_free(s->opt, s->st, s->ri);
  ws_free(s->opt, s->st, s->va);
  s->cp = cp;
  s->ri = ri;
  s->va = va;
  s->nnz = nnz;
  s->adds += 1;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_stream_query(spkadd_stream* s, int64_t* nnz_B, int64_t* adds, int64_t* kernel_launches) {
  if (!s || !nnz_B) return SPKADD_ERR_INVALID_ARG;
  *nnz_B = s->nnz;
  if (adds) *adds = s->adds;
  if (kernel_launches) *kernel_launches = s->launches;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_stream_view(spkadd_stream* s, spkadd_csc* B) {
  if (!s || !B) return SPKADD_ERR_INVALID_ARG;
  *B = spkadd_csc{s->m, s->n, s->nnz, s->cp, s->nnz ? s->ri : nullptr, s->nnz ? s->va : nullptr};
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_stream_result(spkadd_stream* s, int64_t* B_col_ptr, int32_t* B_row_idx, void* B_val) {
  if (!s || !B_col_ptr) return SPKADD_ERR_INVALID_ARG;
  if (s->nnz > 0 && (!B_row_idx || !B_val)) return SPKADD_ERR_INVALID_ARG;
  cudaError_t ce = spk::launch_colptr_widen(s->cp, B_col_ptr, s->n + 1, s->sms, s->st);
  if (ce == cudaSuccess && s->nnz > 0)
    ce = cudaMemcpyAsync(B_row_idx, s->ri, (size_t)s->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s->st);
  if (ce == cudaSuccess && s->nnz > 0)
    ce = cudaMemcpyAsync(B_val, s->va, (size_t)s->nnz * (s->dtype == SPKADD_F64 ? 8 : 4), cudaMemcpyDeviceToDevice,
                         s->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  s->launches += 1;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_stream_destroy(spkadd_stream* s) {
  if (!s) return SPKADD_OK;
  ws_free(s->opt, s->st, s->cp);
  ws_free(s->opt, s->st, s->ri);
  ws_free(s->opt, s->st, s->va);
  delete s;
  return SPKADD_OK;
}
