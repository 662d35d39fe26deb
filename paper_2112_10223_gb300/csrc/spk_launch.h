// spk_launch.h -- host-side launchers of the SpKAdd kernels (internal).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace spk {

struct Inputs;
struct Outs;
struct Counters;
struct Window;

// Per-launch limits shared by host and device code.
constexpr int WARP_MAX_LIMIT = 512;     // warp class: s_j <= 512 -> table <= 1024 slots
constexpr int CTA_MAX_LIMIT = 4096;     // CTA class: s_j <= 4096 -> table <= 8192 slots
constexpr int WINDOW_MAX_LIMIT = 4096;  // numeric window: u <= 4096 -> table <= 8192 slots
constexpr int SLAB_BITS = 20;           // heavy symbolic bitmap covers 2^20 rows per pass

struct DeviceInfo {
  int sms;
  int smem_optin;  // max dynamic shared memory per block (opt-in)
  int smem_per_sm;
};

// Resident blocks per SM of kernel `fn` at `block` threads and `smem` bytes of
// dynamic shared memory (sets the kernel's shared-memory limit to smem; cached).
// 0 on error.
int resident_blocks(const void* fn, int block, size_t smem);

// heavy_list holds 2 * ncols entries: heavy columns with s_j <= BIG_S from the
// start, the larger ones from entry ncols (Counters::n_heavy, ::n_big).
cudaError_t launch_bin(const Inputs& in, int warp_max, int cta_max, int32_t* s, int32_t* u, int32_t* warp_list,
                       int32_t* cta_list, int32_t* heavy_list, Counters* ctr, int sms, cudaStream_t st);
// Batch: col_inst[colbase + j] = q for every column j of every problem q.
cudaError_t launch_col_inst(const Inputs& in, int32_t* col_inst, int sms, cudaStream_t st);
cudaError_t launch_validate(const Inputs& in, const int64_t* nnz, Counters* ctr, int sms, cudaStream_t st);
size_t scan_tiles(int64_t n);
cudaError_t launch_scan(const int32_t* u, int n, long long* tile_buf, int64_t* col_ptr, cudaStream_t st);
// Loads the scan kernels onto the current device (module loading is lazy).
cudaError_t load_scan_kernels();
cudaError_t launch_window_search(const Inputs& in, const Window* win, const int32_t* search_list, int n_search,
                                 int32_t* offs, int sms, cudaStream_t st);

cudaError_t launch_sym_warp(const Inputs& in, const int32_t* list, const int32_t* s, const Counters* ctr,
                            int32_t* u, int warp_max, Counters* ctr_w, const DeviceInfo& dev, cudaStream_t st);
cudaError_t launch_sym_cta(const Inputs& in, const int32_t* list, const int32_t* s, const Counters* ctr, int32_t* u,
                           Window* win, int64_t win_cap, Counters* ctr_w, int cta_max, const DeviceInfo& dev,
                           cudaStream_t st);
cudaError_t launch_sym_heavy(const Inputs& in, const int32_t* list, const int32_t* s, const Counters* ctr, int32_t* u,
                             Window* win,
                             int32_t* search_list, int64_t win_cap, Counters* ctr_w, int window_max,
                             int accumulator, const DeviceInfo& dev, cudaStream_t st);

// dt: 0 = every problem float, 1 = every problem double, 2 = mixed batch.
cudaError_t launch_num_warp(const Inputs& in, int dt, const int32_t* list, const Counters* ctr, int n_cols,
                            const int32_t* s, const int32_t* u, const int64_t* col_ptr, const Outs& out,
                            int warp_max, int sort_mode, Counters* ctr_w, const DeviceInfo& dev, cudaStream_t st);
// Problem kinds of the thread-block numeric launches present in a batch
// (bit 0 float k <= FP32_ACC_TERMS, bit 1 float up to FP32_PHASED_MAX_K, bit 2
// larger float, bit 3 double); f32_kinds holds bits 0-2 of the float problems.
int num_cta_kinds(int dt, int f32_kinds);
// Several kinds: copies the symbolic phase's window records (at most `cap`)
// into wsort grouped by kind; ctr->kind_n gets the count of each.
cudaError_t launch_kind_sort(const Inputs& in, const Window* win, int cap, Window* wsort, Counters* ctr_w,
                             const DeviceInfo& dev, cudaStream_t st);
// One launch per kind present: over win[0, n_win) when the batch has one
// kind, else over the kind's group of wsort (host copy of kind_n).
cudaError_t launch_num_cta(const Inputs& in, int dt, int f32_kinds, const Window* win, int n_win,
                           const Window* wsort, const int32_t* kind_n, const int32_t* offs, const int64_t* col_ptr,
                           const Outs& out, int window_max, int accumulator, Counters* ctr_w, const DeviceInfo& dev,
                           cudaStream_t st, int* launches);
// Per-problem column pointers of B (a batch): out_cp[q][j] = col_ptr[colbase + j] - col_ptr[colbase].
cudaError_t launch_out_colptr(const Inputs& in, const Outs& o, const int64_t* col_ptr, int sms, cudaStream_t st);
// Per-problem nnz(B): nnz[q] = col_ptr[colbase + n] - col_ptr[colbase].
// B's int64 column pointers to int32 (a streamed running sum; nnz < 2^31) and back.
cudaError_t launch_colptr_narrow(const int64_t* src, int32_t* dst, int64_t n1, int sms, cudaStream_t st);
cudaError_t launch_colptr_widen(const int32_t* src, int64_t* dst, int64_t n1, int sms, cudaStream_t st);
cudaError_t launch_inst_nnz(const Inputs& in, const int64_t* col_ptr, int64_t* nnz, cudaStream_t st);

// One-pass path (one problem, every column s_j <= warp_max): B written into
// buffers of `capacity` entries; `scratch` holds onepass_scratch_bytes(n)
// bytes (ticket counter and look-back words).
int onepass_tile_cols();
size_t onepass_scratch_bytes(int64_t ncols);
cudaError_t launch_onepass(const Inputs& in, int dt, const int32_t* s, int n, int warp_max, int64_t* col_ptr,
                           int32_t* out_row, void* out_val, long long capacity, void* scratch, int force_dedup,
                           int debug_stall, unsigned long long wait_ns, Counters* ctr, const DeviceInfo& dev,
                           cudaStream_t st, int* grid_out);

}  // namespace spk
