// C ABI and host runtime of the SpGEMM library: argument checks, workspace management,
// the launch sequence of the plan / symbolic / numeric passes, and the host-buffer entry.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "spgemm.h"
#include "kernels.h"
#include "runtime.h"

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace spg {

spgemm_status set_error_msg(spgemm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

void clear_error_msg() { g_last_error.clear(); }

spgemm_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SPGEMM_OK;
  cudaGetLastError();  // clear the sticky-free error state of the runtime for this thread
  return set_error_msg(SPGEMM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int device_sm_count() {
  static std::mutex mu;
  static std::vector<int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> g(mu);
  if (static_cast<int>(cache.size()) <= dev) cache.resize(dev + 1, 0);
  if (cache[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 1;
  }
  return cache[dev];
}

// The library's own stream-ordered memory pool on the current device, created on first use.
// It keeps freed memory reserved (release threshold = max) so repeated products reuse it
// instead of mapping fresh pages every call; the default pool of the process is untouched.
cudaMemPool_t library_pool() {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (static_cast<int>(pools.size()) <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t threshold = ~uint64_t(0);
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    pools[dev] = pool;
  }
  return pools[dev];
}

void* Workspace::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (has_alloc) {
    p = alloc.alloc(bytes, stream, alloc.ctx);
  } else {
    cudaMemPool_t pool = library_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, static_cast<cudaStream_t>(stream))
                         : cudaMallocAsync(&p, bytes, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (p) {
    blocks.push_back(p);
    total += static_cast<int64_t>(bytes);
  }
  return p;
}

void Workspace::release_all() {
  for (void* p : blocks) {
    if (has_alloc) alloc.free(p, stream, alloc.ctx);
    else cudaFreeAsync(p, static_cast<cudaStream_t>(stream));
  }
  blocks.clear();
  total = 0;
}

spgemm_status check_csr_in(const spgemm_csr_in* M, const char* name, spgemm_prec prec) {
  if (!M) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "%s is NULL", name);
  if (M->rows < 0 || M->cols < 0 || M->nnz < 0)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "%s has a negative size", name);
  if (M->rows >= (int64_t(1) << 31) - 1 || M->cols >= (int64_t(1) << 31) - 1)
    return set_error_msg(SPGEMM_ERR_UNSUPPORTED, "%s: rows and cols must be < 2^31-1 (int32 indices)", name);
  if (!M->row_ptr) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "%s.row_ptr is NULL", name);
  if (M->nnz > 0 && (!M->col || !M->val))
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "%s.col or %s.val is NULL", name, name);
  if (!M->idx64_rowptr && M->nnz > 0x7fffffffLL)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "%s: nnz does not fit an int32 row_ptr", name);
  (void)prec;
  return SPGEMM_OK;
}

}  // namespace spg

using namespace spg;

extern "C" {

void spgemm_opts_default(spgemm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->validate = 1;
  o->tiny_max = 32;
  o->warp_max = 1024;
  o->block_max = 2048;
  o->window_hash_fill = 4096;
  o->force_window = 0;
  o->rowptr32_limit = 0x7fffffffLL;
  o->f32c_rerun_all = 0;
  o->f32c_rerun_none = 0;
  o->num_streams = 4;
  o->record_timings = 0;
  o->window_split_max_mb = 4096;
  o->window_cols_max_mb = 49152;
}

const char* spgemm_last_error(void) { return g_last_error.c_str(); }

const char* spgemm_version(void) { return "gb300-spgemm 0.1 (sm_103a)"; }

spgemm_status spgemm_plan(const spgemm_csr_in* A, const spgemm_csr_in* B, spgemm_prec prec,
                          const spgemm_opts* opts, const spgemm_allocator* alloc, void* stream,
                          spgemm_plan_t** out_plan) {
  clear_error_msg();
  if (!out_plan) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "out_plan is NULL");
  *out_plan = nullptr;
  spgemm_status st;
  if ((st = check_csr_in(A, "A", prec)) != SPGEMM_OK) return st;
  if ((st = check_csr_in(B, "B", prec)) != SPGEMM_OK) return st;
  if (A->cols != B->rows)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "A.cols (%lld) != B.rows (%lld)", (long long)A->cols,
                         (long long)B->rows);
  if (prec != SPGEMM_F64 && prec != SPGEMM_F32_COMPENSATED)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "unknown precision %d", int(prec));
  if (alloc && (!alloc->alloc || !alloc->free))
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "allocator callbacks are NULL");
  spgemm_plan_t* p = new (std::nothrow) spgemm_plan_t();
  if (!p) return set_error_msg(SPGEMM_ERR_OOM, "host allocation of the plan failed");
  spgemm_opts_default(&p->opts);
  if (opts) p->opts = *opts;
  p->prec = prec;
  p->ws.stream = stream;
  if (alloc) { p->ws.alloc = *alloc; p->ws.has_alloc = true; }
  st = plan_run(p, A, B, static_cast<cudaStream_t>(stream));
  if (st != SPGEMM_OK) {
    const std::string msg = g_last_error;
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    release_small_host(p);
    destroy_events(p);
    p->ws.release_all();
    delete p;
    g_last_error = msg;
    return st;
  }
  *out_plan = p;
  return SPGEMM_OK;
}

spgemm_status spgemm_symbolic(spgemm_plan_t* plan, void* stream, int64_t* nnz_c,
                              int32_t* needs_rowptr64) {
  clear_error_msg();
  if (!plan) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "plan is NULL");
  if (plan->state != 0) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "symbolic already ran on this plan");
  spgemm_status st = symbolic_run(plan, static_cast<cudaStream_t>(stream));
  if (st != SPGEMM_OK) return st;
  if (nnz_c) *nnz_c = plan->nnz_c;
  if (needs_rowptr64) *needs_rowptr64 = plan->nnz_c > plan->opts.rowptr32_limit ? 1 : 0;
  return SPGEMM_OK;
}

spgemm_status spgemm_numeric(spgemm_plan_t* plan, spgemm_csr_out* C, void* stream) {
  clear_error_msg();
  if (!plan) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "plan is NULL");
  if (plan->state < 1) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "spgemm_symbolic has not run on this plan");
  if (!C) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C is NULL");
  if (C->rows != plan->A.rows || C->cols != plan->B.cols || C->nnz != plan->nnz_c)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C shape (%lld x %lld, nnz %lld) != expected (%lld x %lld, nnz %lld)",
                         (long long)C->rows, (long long)C->cols, (long long)C->nnz, (long long)plan->A.rows,
                         (long long)plan->B.cols, (long long)plan->nnz_c);
  if (!C->row_ptr || (C->nnz > 0 && (!C->col || !C->val)))
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C arrays are NULL");
  if (!C->idx64_rowptr && plan->nnz_c > plan->opts.rowptr32_limit)
    return set_error_msg(SPGEMM_ERR_INDEX_OVERFLOW, "nnz(C) = %lld needs an int64 row_ptr", (long long)plan->nnz_c);
  return numeric_run(plan, C, static_cast<cudaStream_t>(stream));
}

spgemm_status spgemm_plan_get_info(const spgemm_plan_t* plan, spgemm_plan_info* info) {
  clear_error_msg();
  if (!plan || !info) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->rows = plan->A.rows;
  info->inner = plan->A.cols;
  info->cols = plan->B.cols;
  info->products = plan->total_products;
  info->nnz_c = plan->state >= 1 ? plan->nnz_c : -1;
  info->max_row_products = plan->max_row_products;
  for (int c = 0; c < kSymNumClasses; ++c) info->sym_class_rows[c] = plan->sym_off[c + 1] - plan->sym_off[c];
  if (plan->state >= 1) {
    for (int c = 0; c < kNumNumClasses; ++c) {
      info->num_class_rows[c] = plan->num_off[c + 1] - plan->num_off[c];
      info->num_class_products[c] = static_cast<int64_t>(plan->cls_sums[c][0]);
      info->num_class_annz[c] = static_cast<int64_t>(plan->cls_sums[c][1]);
      info->num_class_cnnz[c] = static_cast<int64_t>(plan->cls_sums[c][2]);
    }
  }
  info->workspace_bytes = plan->ws.total;
  info->f32c_rerun_rows = plan->f32c_rerun_rows;
  info->kernel_launches = plan->launches;
  info->needs_rowptr64 = plan->state >= 1 && plan->nnz_c > plan->opts.rowptr32_limit;
  info->state = plan->state;
  return SPGEMM_OK;
}

spgemm_status spgemm_plan_check(spgemm_plan_t* plan, void* stream) {
  clear_error_msg();
  if (!plan) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "plan is NULL");
  const spgemm_status st = read_device_error(plan, static_cast<cudaStream_t>(stream));
  if (st == SPGEMM_OK && plan->fx_rerun_pending) {
    int32_t n = 0;
    const spgemm_status rs = read_small(&n, plan->counters + 6, sizeof(n), static_cast<cudaStream_t>(stream),
                                        &plan->launches, "reading the FP64 rerun count");
    if (rs != SPGEMM_OK) return rs;
    plan->f32c_rerun_rows = n;
  }
  return st;
}

spgemm_status spgemm_plan_get_timings(spgemm_plan_t* plan, spgemm_timings* t) {
  clear_error_msg();
  if (!plan || !t) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  std::memset(t, 0, sizeof(*t));
  if (!plan->ev_made) return SPGEMM_OK;
  for (int i = 0; i < SPGEMM_NUM_STAGES; ++i) {
    if (!plan->ev_rec[i]) continue;
    cudaError_t e = cudaEventSynchronize(plan->ev[i][1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, plan->ev[i][0], plan->ev[i][1]);
    if (e != cudaSuccess) return cuda_status(e, "reading stage timings");
    t->ms[i] = ms;
    t->launches[i] = plan->ev_launches[i];
  }
  return SPGEMM_OK;
}

spgemm_status spgemm_plan_destroy(spgemm_plan_t* plan) {
  if (!plan) return SPGEMM_OK;
  release_small_host(plan);
  destroy_events(plan);
  plan->ws.release_all();
  delete plan;
  return SPGEMM_OK;
}

}  // extern "C"
