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
  if (err & (spk::ERR_WINDOW_CAP | spk::ERR_INTERNAL)) return SPKADD_ERR_INTERNAL;
  return SPKADD_OK;
}

}  // namespace

struct spkadd_handle {
  int k = 0;
  int64_t m = 0, n = 0, nnz_in = 0;
  spkadd_dtype dt = SPKADD_F64;
  cudaStream_t st = nullptr;
  spkadd_options opt{};
  int device = 0;
  DeviceInfo dev{};
  char* ws = nullptr;
  size_t ws_bytes = 0;
  char* offs_buf = nullptr;
  size_t offs_bytes = 0;
  Inputs in{};
  const int64_t* d_nnz = nullptr;
  int32_t *d_s = nullptr, *d_u = nullptr;
  int32_t *d_wl = nullptr, *d_cl = nullptr, *d_hl = nullptr;
  Window* d_win = nullptr;
  int32_t* d_search = nullptr;
  int64_t win_cap = 0;
  Counters* d_ctr = nullptr;
  int64_t* d_colptr = nullptr;
  long long* d_scan = nullptr;
  int32_t* d_offs = nullptr;
  Counters h_ctr{};
  int64_t nnz_out = -1;
  int state = 0;
  int64_t launches = 0;  // kernels launched by this handle

  void* dev_alloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (opt.alloc) return opt.alloc(bytes, (void*)st, opt.alloc_ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void dev_free(void* p) {
    if (!p) return;
    if (opt.alloc) opt.free(p, (void*)st, opt.alloc_ctx);
    else cudaFreeAsync(p, st);
  }
};

SPK_API void spkadd_default_options(spkadd_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->validate = 0;
  opt->warp_max = spk::WARP_MAX_LIMIT;
  opt->cta_max = spk::CTA_MAX_LIMIT;
  opt->window_max = spk::WINDOW_MAX_LIMIT;
  opt->sort_mode = 0;
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
    case SPKADD_ERR_UNSUPPORTED: return "SPKADD_ERR_UNSUPPORTED: request not supported by this build";
    case SPKADD_ERR_INTERNAL: return "SPKADD_ERR_INTERNAL: device-side invariant failed";
  }
  return "SPKADD_ERR_?: unknown status";
}

SPK_API int spkadd_version(void) { return 100; }

static spkadd_status check_options(const spkadd_options& o) {
  if (o.warp_max < 1 || o.warp_max > spk::WARP_MAX_LIMIT) return SPKADD_ERR_INVALID_ARG;
  if (o.cta_max < o.warp_max || o.cta_max > spk::CTA_MAX_LIMIT) return SPKADD_ERR_INVALID_ARG;
  if (o.window_max < 1024 || o.window_max > spk::WINDOW_MAX_LIMIT) return SPKADD_ERR_INVALID_ARG;
  if (o.sort_mode != 0 && o.sort_mode != 1) return SPKADD_ERR_INVALID_ARG;
  if ((o.alloc == nullptr) != (o.free == nullptr)) return SPKADD_ERR_INVALID_ARG;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_plan(spkadd_handle** hp, int k, const spkadd_csc* A, spkadd_dtype dtype, void* stream,
                                  const spkadd_options* opt) {
  if (!hp) return SPKADD_ERR_INVALID_ARG;
  *hp = nullptr;
  if (k < 1 || !A) return SPKADD_ERR_INVALID_ARG;
  if (k > SPKADD_MAX_K) return SPKADD_ERR_UNSUPPORTED;
  if (dtype != SPKADD_F32 && dtype != SPKADD_F64) return SPKADD_ERR_INVALID_ARG;
  spkadd_options o;
  if (opt) o = *opt;
  else spkadd_default_options(&o);
  spkadd_status os = check_options(o);
  if (os != SPKADD_OK) return os;
  const int64_t m = A[0].m, n = A[0].n;
  int64_t nnz_in = 0;
  for (int i = 0; i < k; ++i) {
    const spkadd_csc& a = A[i];
    if (a.m < 0 || a.n < 0 || a.nnz < 0) return SPKADD_ERR_INVALID_ARG;
    if (a.m >= INT32_MAX || a.n >= INT32_MAX || a.nnz > INT32_MAX) return SPKADD_ERR_OVERFLOW;
    if (a.m != m || a.n != n) return SPKADD_ERR_SHAPE_MISMATCH;
    if (!a.col_ptr) return SPKADD_ERR_INVALID_ARG;
    if (a.nnz > 0 && (!a.row_idx || !a.val)) return SPKADD_ERR_INVALID_ARG;
    nnz_in += a.nnz;
  }

  spkadd_handle* h = new (std::nothrow) spkadd_handle();
  if (!h) return SPKADD_ERR_NOMEM;
  h->k = k;
  h->m = m;
  h->n = n;
  h->nnz_in = nnz_in;
  h->dt = dtype;
  h->st = static_cast<cudaStream_t>(stream);
  h->opt = o;
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce == cudaSuccess) ce = device_info(h->device, &h->dev);
  if (ce != cudaSuccess) {
    delete h;
    return from_cuda(ce);
  }

  // Window capacity: heavy windows <= nnz_in / (window_max - 32) + one per
  // heavy column and slab; CTA columns <= min(n, nnz_in / (warp_max + 1)).
  const int64_t slab_rows = (int64_t)1 << spk::SLAB_BITS;
  const int64_t slabs = m > 0 ? (m + slab_rows - 1) / slab_rows : 1;
  int64_t heavy_cols = nnz_in / (o.cta_max + 1);
  if (heavy_cols > n) heavy_cols = n;
  int64_t cta_cols = nnz_in / (o.warp_max + 1);
  if (cta_cols > n) cta_cols = n;
  h->win_cap = nnz_in / (o.window_max - 32) + heavy_cols * (slabs + 1) + cta_cols + 16;

  Carver cv;
  const size_t o_cp = cv.take<const int32_t*>(k);
  const size_t o_ri = cv.take<const int32_t*>(k);
  const size_t o_va = cv.take<const void*>(k);
  const size_t o_nnz = cv.take<int64_t>(k);
  const size_t o_ctr = cv.take<Counters>(1);
  const size_t o_s = cv.take<int32_t>(n);
  const size_t o_u = cv.take<int32_t>(n);
  const size_t o_wl = cv.take<int32_t>(n);
  const size_t o_cl = cv.take<int32_t>(n);
  const size_t o_hl = cv.take<int32_t>(n);
  const size_t o_win = cv.take<Window>(h->win_cap);
  const size_t o_srch = cv.take<int32_t>(h->win_cap);
  const size_t o_colp = cv.take<int64_t>(n + 1);
  const size_t o_scan = cv.take<long long>(spk::scan_tiles(n));
  h->ws_bytes = align_up(cv.off, 256);
  h->ws = static_cast<char*>(h->dev_alloc(h->ws_bytes));
  if (!h->ws) {
    delete h;
    return SPKADD_ERR_NOMEM;
  }
  h->d_nnz = reinterpret_cast<const int64_t*>(h->ws + o_nnz);
  h->d_ctr = reinterpret_cast<Counters*>(h->ws + o_ctr);
  h->d_s = reinterpret_cast<int32_t*>(h->ws + o_s);
  h->d_u = reinterpret_cast<int32_t*>(h->ws + o_u);
  h->d_wl = reinterpret_cast<int32_t*>(h->ws + o_wl);
  h->d_cl = reinterpret_cast<int32_t*>(h->ws + o_cl);
  h->d_hl = reinterpret_cast<int32_t*>(h->ws + o_hl);
  h->d_win = reinterpret_cast<Window*>(h->ws + o_win);
  h->d_search = reinterpret_cast<int32_t*>(h->ws + o_srch);
  h->d_colptr = reinterpret_cast<int64_t*>(h->ws + o_colp);
  h->d_scan = reinterpret_cast<long long*>(h->ws + o_scan);

  // Descriptor tables (one host staging buffer, one copy).
  const size_t desc_bytes = o_ctr;  // tables occupy [0, o_ctr)
  std::vector<char> host(desc_bytes + sizeof(Counters), 0);
  for (int i = 0; i < k; ++i) {
    reinterpret_cast<const int32_t**>(host.data() + o_cp)[i] = A[i].col_ptr;
    reinterpret_cast<const int32_t**>(host.data() + o_ri)[i] = A[i].row_idx;
    reinterpret_cast<const void**>(host.data() + o_va)[i] = A[i].val;
    reinterpret_cast<int64_t*>(host.data() + o_nnz)[i] = A[i].nnz;
  }
  ce = cudaMemcpyAsync(h->ws, host.data(), desc_bytes + sizeof(Counters), cudaMemcpyHostToDevice, h->st);
  if (ce != cudaSuccess) {
    spkadd_destroy(h);
    return from_cuda(ce);
  }
  h->in.cp = reinterpret_cast<const int32_t* const*>(h->ws + o_cp);
  h->in.ri = reinterpret_cast<const int32_t* const*>(h->ws + o_ri);
  h->in.val = reinterpret_cast<const void* const*>(h->ws + o_va);
  h->in.k = k;
  h->in.m = (int32_t)m;
  h->in.n = (int32_t)n;
  h->in.home_mul = m > 0 ? (((uint64_t)1 << 48) / (uint64_t)m) : 0;

  if (o.validate) {
    ce = spk::launch_validate(h->in, h->d_nnz, h->d_ctr, h->dev.sms, h->st);
    h->launches += n > 0;
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
  h->launches += n > 0;
  if (ce != cudaSuccess) {
    spkadd_destroy(h);
    return from_cuda(ce);
  }
  h->state = ST_PLANNED;
  *hp = h;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_symbolic(spkadd_handle* h, int64_t* nnz_B) {
  if (!h || !nnz_B) return SPKADD_ERR_INVALID_ARG;
  if (h->state < ST_PLANNED) return SPKADD_ERR_STATE;
  if (h->state >= ST_SYMBOLIC) {  // already counted: the workspace holds the result
    *nnz_B = h->nnz_out;
    return SPKADD_OK;
  }
  cudaError_t ce = cudaSuccess;
  if (h->n > 0) {
    ce = spk::launch_sym_heavy(h->in, h->d_hl, h->d_ctr, h->d_u, h->d_win, h->d_search, h->win_cap, h->d_ctr,
                               h->opt.window_max, h->dev, h->st);
    if (ce == cudaSuccess)
      ce = spk::launch_sym_cta(h->in, h->d_cl, h->d_s, h->d_ctr, h->d_u, h->d_win, h->win_cap, h->d_ctr,
                               h->opt.cta_max, h->dev, h->st);
    if (ce == cudaSuccess)
      ce = spk::launch_sym_warp(h->in, h->d_wl, h->d_s, h->d_ctr, h->d_u, h->opt.warp_max, h->d_ctr, h->dev,
                                h->st);
    h->launches += 3;
  }
  if (ce == cudaSuccess) ce = spk::launch_scan(h->d_u, (int)h->n, h->d_scan, h->d_colptr, h->st);
  h->launches += h->n > 0 ? 3 : 2;
  Pinned* pb = pinned_block();
  if (ce == cudaSuccess && !pb) ce = cudaErrorMemoryAllocation;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&pb->ctr, h->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(&pb->nnz, h->d_colptr + h->n, sizeof(long long), cudaMemcpyDeviceToHost, h->st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
  if (ce != cudaSuccess) return from_cuda(ce);
  h->h_ctr = pb->ctr;
  const spkadd_status ds = from_device_err(h->h_ctr.err);
  if (ds != SPKADD_OK) return ds;
  h->nnz_out = pb->nnz;

  // Per-input offsets of split windows (sized now that their count is known).
  const int64_t ns = h->h_ctr.n_search;
  if (ns > 0) {
    const size_t need = (size_t)ns * h->k * 2 * sizeof(int32_t);
    if (need > h->offs_bytes) {
      h->dev_free(h->offs_buf);
      h->offs_buf = static_cast<char*>(h->dev_alloc(need));
      h->offs_bytes = h->offs_buf ? need : 0;
      if (!h->offs_buf) return SPKADD_ERR_NOMEM;
    }
    h->d_offs = reinterpret_cast<int32_t*>(h->offs_buf);
    ce = spk::launch_window_search(h->in, h->d_win, h->d_search, (int)ns, h->d_offs, h->dev.sms, h->st);
    if (ce != cudaSuccess) return from_cuda(ce);
    h->launches += 1;
  }
  h->state = ST_SYMBOLIC;
  *nnz_B = h->nnz_out;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_numeric(spkadd_handle* h, int64_t* B_col_ptr, int32_t* B_row_idx, void* B_val) {
  if (!h || !B_col_ptr) return SPKADD_ERR_INVALID_ARG;
  if (h->state < ST_SYMBOLIC) return SPKADD_ERR_STATE;
  if (h->nnz_out > 0 && (!B_row_idx || !B_val)) return SPKADD_ERR_INVALID_ARG;
  cudaError_t ce = cudaMemcpyAsync(B_col_ptr, h->d_colptr, (size_t)(h->n + 1) * sizeof(int64_t),
                                   cudaMemcpyDeviceToDevice, h->st);
  const bool f64 = h->dt == SPKADD_F64;
  const int cta_items = h->h_ctr.n_windows;
  if (ce == cudaSuccess && cta_items > 0)
    ce = spk::launch_num_cta(h->in, f64, h->d_win, cta_items, h->d_offs, h->d_colptr, B_row_idx, B_val,
                             h->opt.window_max > h->opt.cta_max ? h->opt.window_max : h->opt.cta_max, h->d_ctr,
                             h->dev, h->st);
  h->launches += cta_items > 0;
  if (ce == cudaSuccess && h->h_ctr.n_warp > 0)
    ce = spk::launch_num_warp(h->in, f64, h->d_wl, h->d_ctr, h->h_ctr.n_warp, h->d_s, h->d_u, h->d_colptr, B_row_idx,
                              B_val, h->opt.warp_max, h->opt.sort_mode, h->d_ctr, h->dev, h->st);
  h->launches += h->h_ctr.n_warp > 0;
  if (ce != cudaSuccess) return from_cuda(ce);
  h->state = ST_NUMERIC;
  return SPKADD_OK;
}

SPK_API spkadd_status spkadd_get_info(spkadd_handle* h, spkadd_info* info) {
  if (!h || !info) return SPKADD_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->k = h->k;
  info->m = h->m;
  info->n = h->n;
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
  info->cols_heavy = c.n_heavy;
  info->windows = c.n_windows;
  info->windows_split = c.n_search;
  info->cols_unique = c.n_unique;
  info->workspace_bytes = (int64_t)(h->ws_bytes + h->offs_bytes);
  info->kernel_launches = h->launches;
  return from_device_err(c.err);
}

SPK_API spkadd_status spkadd_destroy(spkadd_handle* h) {
  if (!h) return SPKADD_OK;
  h->dev_free(h->offs_buf);
  h->dev_free(h->ws);
  delete h;
  return SPKADD_OK;
}
