// Host runtime of the SpGEMM library (internal): the plan object and the pass drivers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "spgemm.h"
#include "kernels.h"

namespace spg {

// Device workspace of one plan: every block comes from the caller's allocator, or from
// cudaMallocAsync on the plan's stream, and is released in stream order.
struct Workspace {
  spgemm_allocator alloc{};
  bool has_alloc = false;
  void* stream = nullptr;
  std::vector<void*> blocks;
  int64_t total = 0;
  void* get(size_t bytes);
  void release_all();
};

spgemm_status set_error_msg(spgemm_status st, const char* fmt, ...);
void clear_error_msg();
spgemm_status cuda_status(cudaError_t e, const char* what);
int device_sm_count();
cudaMemPool_t library_pool();   // the library's stream-ordered pool on the current device (null if none)
spgemm_status check_csr_in(const spgemm_csr_in* M, const char* name, spgemm_prec prec);

}  // namespace spg

struct spgemm_plan_s {
  spg::DevCsr A{}, B{};
  spgemm_prec prec = SPGEMM_F64;
  spgemm_opts opts{};
  spg::ClassParams cp{};
  spg::Workspace ws;
  int num_sms = 1;
  int64_t ntiles = 0;
  int64_t* P = nullptr;
  int32_t* nnz_row = nullptr;
  int32_t* perm_s = nullptr;
  int32_t* perm_n = nullptr;
  int64_t* c_off = nullptr;
  int32_t* tile_hist = nullptr;
  int64_t* tile_sum = nullptr;
  int64_t* tile_max = nullptr;
  int64_t* tile_sum_off = nullptr;
  spg::Summary* summary = nullptr;   // device
  int32_t* counters = nullptr;       // device, 16 ints
  int32_t* win_slot = nullptr;
  uint16_t* blockcnt = nullptr;
  int64_t nblocks = 0;
  int32_t* cursor = nullptr;
  int32_t* split = nullptr;          // column-block split table of B (windowed numeric rows)
  uint32_t* wbits = nullptr;         // column bitmaps of windowed rows, stored by the symbolic pass
  int64_t wcap = 0;                  // words wbits holds
  unsigned long long* wcur = nullptr;   // device cursor into wbits
  int64_t* woff = nullptr;           // per windowed row slot: its first word in wbits, or -1
  double* rerun_dense = nullptr;     // FP64 rows of a rerun group (FP32-compensated plans)
  int64_t rerun_group = 0;           // rows per rerun group
  // Column space of the rows: [abase[i], abase[i] + awidth[i]) for row i of A (and B's rows start
  // at bbase[k]); width is the widest row. A single product has no bases and width = n. A batch
  // run as one block-diagonal product gives every row the columns of its own job.
  const int32_t* abase = nullptr;
  const int32_t* awidth = nullptr;
  const int32_t* bbase = nullptr;
  int64_t width = 0;
  bool split_tried = false;
  bool lists_tried = false;        // windowed rows: lists of long rows' window segments
  int64_t* list_bs = nullptr;
  int32_t* list_len = nullptr;
  double* list_av = nullptr;
  int64_t list_cap = 0;           // entries per block of the windowed kernel
  // FP32-compensated path
  int32_t* rerun_flag = nullptr;     // per row: 1 = recompute in FP64
  uint16_t* bexp = nullptr;          // largest biased exponent per row of B (exact FP64 accumulation)
  bool fx_rerun_pending = false;     // the last numeric pass listed FP64 reruns in counters[6]
  bool small = false;                // the small-product path (k_small.cu) holds this plan
  int small_cap = 0;                 // small path: longest row of C (from the symbolic pass)
  spg::SmallGrid small_grid{};       // small path: the symbolic kernel's runs of rows
  int32_t* small_loc = nullptr;      // small path: row offsets within their run
  int64_t* small_blk = nullptr;      // small path: offsets of the runs (and nnz(C) last)
  spgemm_csr_in a_in{}, b_in{};      // small path: the inputs as the caller gave them
  void* small_host = nullptr;        // small path: mapped staging block the symbolic kernel writes its summary to
  int32_t* rerun_list = nullptr;
  int64_t sym_off[spg::kMaxClasses + 1] = {};
  int64_t num_off[spg::kMaxClasses + 1] = {};
  int64_t total_products = 0;
  int64_t max_row_products = 0;
  int64_t nnz_c = -1;
  int64_t f32c_rerun_rows = 0;
  int64_t launches = 0;
  unsigned long long cls_sums[spg::kMaxClasses][3] = {};
  // stage timing (record_timings)
  cudaEvent_t ev[16][2] = {};
  bool ev_made = false;
  int ev_dev = 0;                // device of the plan's timing events
  bool ev_rec[16] = {};
  int ev_launches[16] = {};
  int state = 0;
};

namespace spg {

spgemm_status plan_run(spgemm_plan_s* p, const spgemm_csr_in* A, const spgemm_csr_in* B,
                       cudaStream_t s);
template <typename T>
T* ws_alloc(spgemm_plan_s* p, int64_t count, spgemm_status* st);
spgemm_status symbolic_run(spgemm_plan_s* p, cudaStream_t s);
spgemm_status numeric_run(spgemm_plan_s* p, spgemm_csr_out* C, cudaStream_t s);
spgemm_status read_device_error(spgemm_plan_s* p, cudaStream_t s);
// Synchronous read of a few bytes of device state (a multiple of 4, at most 4 KB) on stream s,
// by a kernel storing into mapped page-locked memory (copies to the host queue behind every bulk
// copy in flight); `launches` (may be null) counts the kernel.
spgemm_status read_small(void* dst, const void* src, size_t bytes, cudaStream_t s, int64_t* launches,
                         const char* what);
// Gives a small plan's summary staging block back (after waiting for the plan's stream while its
// symbolic kernel may still write to it).
void release_small_host(spgemm_plan_s* p);
// Below this many micro rows (at most 8 A entries and 32 partial products) the rows take the
// warp-per-row tiny kernels instead of the thread-per-row merge, whose dependent loads make it
// pay only when many rows run at once.
constexpr int64_t kMicroMinRows = 32768;
// Bytes of FP64 scratch the FP32 rerun of windowed rows works in (rows of the plan's width).
constexpr int64_t kRerunScratchBytes = int64_t(256) << 20;
// Device bytes the numeric pass of a plan past its symbolic pass will still allocate (FP32 rerun
// lists and scratch, the split table of B), rounded as the workspace rounds them.
int64_t numeric_extra_bytes(const spgemm_plan_s* p);
// Bounds on the workspace bytes spgemm_plan and spgemm_symbolic allocate for an m-row A with
// a_nnz entries and output rows `width` columns wide: *lo is always allocated, *hi is never
// exceeded.
void plan_bytes_bounds(int64_t m, int64_t a_nnz, int64_t width, int a_rowptr32, int b_rowptr32, int64_t b_rows,
                       int64_t b_nnz, int validate, int32_t wbits_mb, int64_t* lo, int64_t* hi);
// Bytes the workspace takes for a request of `bytes`.
inline int64_t ws_rounded(int64_t bytes) { return ((bytes <= 0 ? 16 : bytes) + 255) & ~int64_t(255); }
void stage_begin(spgemm_plan_s* p, int stage, cudaStream_t s);
void stage_end(spgemm_plan_s* p, int stage, int launches, cudaStream_t s);
void destroy_events(spgemm_plan_s* p);

}  // namespace spg
