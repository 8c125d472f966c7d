// Pass drivers: the launch sequence of plan (validate, count, class scan, scatter),
// symbolic (per-class symbolic kernels, row-offset scan, numeric classes) and numeric
// (per-class numeric kernels). Two host synchronisations per product: after the plan
// (class sizes, sum of P_i) and after the symbolic pass (nnz(C), so the caller can
// allocate C); one, after the symbolic pass, on the small-product path.
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "runtime.h"

namespace spg {

template <typename T>
T* ws_alloc(spgemm_plan_s* p, int64_t count, spgemm_status* st) {
  if (*st != SPGEMM_OK) return nullptr;
  void* ptr = p->ws.get(static_cast<size_t>(count < 1 ? 1 : count) * sizeof(T));
  if (!ptr) *st = set_error_msg(SPGEMM_ERR_OOM, "device workspace allocation of %lld bytes failed",
                                (long long)(count * (int64_t)sizeof(T)));
  return static_cast<T*>(ptr);
}
template int32_t* ws_alloc<int32_t>(spgemm_plan_s*, int64_t, spgemm_status*);
template int64_t* ws_alloc<int64_t>(spgemm_plan_s*, int64_t, spgemm_status*);

namespace {

template <typename T>
T* ws_get(spgemm_plan_s* p, int64_t count, spgemm_status* st) { return ws_alloc<T>(p, count, st); }


spgemm_status read_summary(spgemm_plan_s* p, Summary* h, cudaStream_t s) {
  return read_small(h, p->summary, sizeof(Summary), s, &p->launches, "reading the pass summary");
}

spgemm_status error_bits_status(uint32_t err) {
  if (err & kErrInvalidCsr)
    return set_error_msg(SPGEMM_ERR_INVALID_CSR, "an input is not canonical CSR (row pointers or column indices)");
  if (err) return set_error_msg(SPGEMM_ERR_INTERNAL, "device consistency check failed (error bits 0x%x)", err);
  return SPGEMM_OK;
}

int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

}  // namespace

namespace {

// Page-locked, mapped staging blocks shared by all reads: a read takes one from the free list
// (allocating it on first need) and gives it back.
constexpr size_t kStageBytes = 4096;
std::mutex g_stage_mu;
std::vector<void*> g_stage_free;

void* stage_take() {
  {
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (!g_stage_free.empty()) {
      void* h = g_stage_free.back();
      g_stage_free.pop_back();
      return h;
    }
  }
  void* h = nullptr;
  if (cudaHostAlloc(&h, kStageBytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return h;
}

void stage_give(void* h) {
  std::lock_guard<std::mutex> lk(g_stage_mu);
  g_stage_free.push_back(h);
}

}  // namespace

spgemm_status read_small(void* dst, const void* src, size_t bytes, cudaStream_t s, int64_t* launches,
                         const char* what) {
  void* hp = bytes <= kStageBytes && bytes % 4 == 0 ? stage_take() : nullptr;
  void* dp = nullptr;
  cudaError_t e;
  if (hp && cudaHostGetDevicePointer(&dp, hp, 0) == cudaSuccess) {
    const int n = launch_fetch(src, dp, static_cast<int64_t>(bytes), s);
    if (launches) *launches += n;
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) std::memcpy(dst, hp, bytes);
  } else {
    cudaGetLastError();
    e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (hp) stage_give(hp);
  if (e != cudaSuccess) return cuda_status(e, what);
  return SPGEMM_OK;
}

void release_small_host(spgemm_plan_s* p) {
  if (!p->small_host) return;
  cudaStreamSynchronize(static_cast<cudaStream_t>(p->ws.stream));
  stage_give(p->small_host);
  p->small_host = nullptr;
}

spgemm_status read_device_error(spgemm_plan_s* p, cudaStream_t s) {
  Summary h;
  spgemm_status st = read_summary(p, &h, s);
  if (st != SPGEMM_OK) return st;
  return error_bits_status(h.err);
}

namespace {

// Timing events come from a process-wide free list (per device) and go back to it when the plan
// is destroyed: an instrumented plan pays two event records per stage it runs, not the creation
// of events.
std::mutex g_ev_mu;
std::vector<std::pair<int, cudaEvent_t>> g_ev_free;

cudaEvent_t event_take(int dev) {
  {
    std::lock_guard<std::mutex> lk(g_ev_mu);
    for (size_t i = g_ev_free.size(); i-- > 0;)
      if (g_ev_free[i].first == dev) {
        const cudaEvent_t e = g_ev_free[i].second;
        g_ev_free[i] = g_ev_free.back();
        g_ev_free.pop_back();
        return e;
      }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

}  // namespace

void stage_begin(spgemm_plan_s* p, int stage, cudaStream_t s) {
  if (!p->opts.record_timings) return;
  if (!p->ev_made) {
    if (cudaGetDevice(&p->ev_dev) != cudaSuccess) return;
    p->ev_made = true;
  }
  for (int j = 0; j < 2; ++j)
    if (!p->ev[stage][j]) p->ev[stage][j] = event_take(p->ev_dev);
  if (p->ev[stage][0]) cudaEventRecord(p->ev[stage][0], s);
}

void stage_end(spgemm_plan_s* p, int stage, int launches, cudaStream_t s) {
  p->launches += launches;
  if (!p->opts.record_timings || !p->ev[stage][0] || !p->ev[stage][1]) return;
  cudaEventRecord(p->ev[stage][1], s);
  p->ev_rec[stage] = true;
  p->ev_launches[stage] = launches;
}

void destroy_events(spgemm_plan_s* p) {
  if (!p->ev_made) return;
  std::lock_guard<std::mutex> lk(g_ev_mu);
  for (int i = 0; i < SPGEMM_NUM_STAGES; ++i)
    for (int j = 0; j < 2; ++j)
      if (p->ev[i][j]) {
        g_ev_free.emplace_back(p->ev_dev, p->ev[i][j]);
        p->ev[i][j] = nullptr;
      }
  p->ev_made = false;
}

namespace {

SmallCsr small_csr(const spgemm_csr_in& M, const int32_t* cbase = nullptr) {
  return SmallCsr{M.rows, M.cols, M.nnz, M.row_ptr, M.idx64_rowptr, static_cast<const int32_t*>(M.col), M.val,
                  cbase};
}

// Width of a small plan's column space: n, or a stacked batch's widest job.
int64_t small_width(const spgemm_plan_s* p) { return p->abase ? p->width : p->B.cols; }

// The small-product path's plan: one workspace block for the summary, the row counts, their
// offsets within the symbolic kernel's runs of rows and the runs' offsets; nothing is launched
// but the summary's clearing (the symbolic kernel checks A and B itself) and nothing is read
// back.
spgemm_status plan_small(spgemm_plan_s* p, const spgemm_csr_in* A, const spgemm_csr_in* B, cudaStream_t s) {
  spgemm_status st = SPGEMM_OK;
  const int64_t m = A->rows;
  auto r256 = [](int64_t b) { return static_cast<size_t>((b + 255) & ~int64_t(255)); };
  p->small_grid = small_sym_grid(small_csr(*A), p->abase ? p->width : B->cols, p->num_sms);
  const size_t sum_bytes = r256(sizeof(Summary));
  const size_t blk_bytes = r256(8 * (p->small_grid.blocks + 1));
  const size_t row_bytes = r256(4 * m);
  unsigned char* w = ws_get<unsigned char>(p, static_cast<int64_t>(sum_bytes + blk_bytes + 2 * row_bytes), &st);
  if (st) return st;
  p->summary = reinterpret_cast<Summary*>(w);
  p->small_blk = reinterpret_cast<int64_t*>(w + sum_bytes);
  p->nnz_row = reinterpret_cast<int32_t*>(w + sum_bytes + blk_bytes);
  p->small_loc = reinterpret_cast<int32_t*>(w + sum_bytes + blk_bytes + row_bytes);
  p->a_in = *A;
  p->b_in = *B;
  p->A = DevCsr{m, A->cols, A->nnz, nullptr, static_cast<const int32_t*>(A->col), A->val};
  p->B = DevCsr{B->rows, B->cols, B->nnz, nullptr, static_cast<const int32_t*>(B->col), B->val};
  cudaMemsetAsync(p->summary, 0, sizeof(Summary), s);
  stage_end(p, SPGEMM_STAGE_VALIDATE, 0, s);
  if ((st = cuda_status(cudaGetLastError(), "clearing the plan summary")) != SPGEMM_OK) return st;
  // the summary's host copy: the symbolic kernel's last block stores it into a mapped staging
  // block, so spgemm_symbolic reads it after one wait, with no copy; small_flags starts at a value
  // the kernel never writes, so a summary the kernel did not store is caught
  Summary* hsum = nullptr;
  if (!p->small_host) p->small_host = stage_take();
  if (p->small_host) {
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&hsum), p->small_host, 0) == cudaSuccess) {
      static_cast<Summary*>(p->small_host)->small_flags = kSmallUnwritten;
    } else {
      cudaGetLastError();
      stage_give(p->small_host);
      p->small_host = nullptr;
      hsum = nullptr;
    }
  }
  // the symbolic kernel starts now, on the plan's stream: spgemm_symbolic only reads its summary
  stage_begin(p, SPGEMM_STAGE_SYM_WARP, s);
  const int nl = launch_small_symbolic(small_csr(p->a_in, p->abase), small_csr(p->b_in), small_width(p),
                                       p->small_grid, p->opts.validate, p->nnz_row, p->small_loc, p->small_blk,
                                       p->summary, hsum, s);
  stage_end(p, SPGEMM_STAGE_SYM_WARP, nl, s);
  if ((st = cuda_status(cudaGetLastError(), "launching the small-product symbolic pass")) != SPGEMM_OK) return st;
  p->state = 0;
  return SPGEMM_OK;
}


}  // namespace

spgemm_status plan_run(spgemm_plan_s* p, const spgemm_csr_in* A, const spgemm_csr_in* B,
                       cudaStream_t s) {
  spgemm_status st = SPGEMM_OK;
  const int64_t m = A->rows, n = B->cols;
  p->num_sms = device_sm_count();
  if (p->opts.max_sms > 0 && p->opts.max_sms < p->num_sms) p->num_sms = p->opts.max_sms;
  // internal int64 row pointers
  const int64_t* arp = static_cast<const int64_t*>(A->row_ptr);
  const int64_t* brp = static_cast<const int64_t*>(B->row_ptr);
  int conv = 0;
  stage_begin(p, SPGEMM_STAGE_VALIDATE, s);
  const spgemm_opts& o = p->opts;
  // small narrow F64 products with the default class options: a warp per row over a bitmap of all
  // columns (k_small.cu), one host read in all
  // (also a stacked batch whose widest job has at most kSmallMaxCols columns)
  p->small = p->prec == SPGEMM_F64 && !o.general_path && !o.force_window && o.fp64_accumulate == 0 &&
             o.tiny_max == 32 && o.warp_max == 1024 && o.block_max == 2048 && o.window_hash_fill == 4096 &&
             m > 0 &&
             (p->abase ? m <= kSmallMaxBatchRows && p->width > 0 && p->width <= kSmallMaxCols
                       : small_path_fits(m, n));
  if (p->small) return plan_small(p, A, B, s);
  if (!A->idx64_rowptr) {
    int64_t* t = ws_get<int64_t>(p, m + 1, &st);
    if (st) return st;
    conv += launch_rowptr_to64(static_cast<const int32_t*>(A->row_ptr), t, m + 1, s);
    arp = t;
  }
  if (!B->idx64_rowptr) {
    int64_t* t = ws_get<int64_t>(p, B->rows + 1, &st);
    if (st) return st;
    conv += launch_rowptr_to64(static_cast<const int32_t*>(B->row_ptr), t, B->rows + 1, s);
    brp = t;
  }
  p->A = DevCsr{m, A->cols, A->nnz, arp, A->col, A->val};
  p->B = DevCsr{B->rows, n, B->nnz, brp, B->col, B->val};
  if (p->width <= 0) p->width = n;
  p->cp.n = p->width;
  p->cp.rwidth = p->awidth;
  p->cp.tiny_max = clampi(o.tiny_max, 0, 32);
  p->cp.warp_max = clampi(o.warp_max, 0, 1024);
  p->cp.block_max = clampi(o.block_max, p->cp.warp_max > 32 ? p->cp.warp_max : 32, 4096);
  // deterministic FP64 (fp64_accumulate 2): every non-empty row takes the exact windowed path
  p->cp.force_window = (o.force_window || (p->prec == SPGEMM_F64 && o.fp64_accumulate == 2)) ? 1 : 0;
  p->cp.window_all = p->prec == SPGEMM_F32_COMPENSATED ? 1 : 0;
  if (o.window_hash_fill < 1 || o.window_hash_fill > 4096) p->opts.window_hash_fill = 4096;

  p->ntiles = (m + kTileRows - 1) / kTileRows;
  p->summary = ws_get<Summary>(p, 1, &st);
  p->counters = ws_get<int32_t>(p, 16, &st);
  p->P = ws_get<int64_t>(p, m, &st);
  p->nnz_row = ws_get<int32_t>(p, m, &st);
  p->perm_s = ws_get<int32_t>(p, m, &st);
  p->perm_n = ws_get<int32_t>(p, m, &st);
  p->c_off = ws_get<int64_t>(p, m + 1, &st);
  p->tile_hist = ws_get<int32_t>(p, p->ntiles * kMaxClasses, &st);
  p->tile_sum = ws_get<int64_t>(p, p->ntiles, &st);
  p->tile_max = ws_get<int64_t>(p, p->ntiles, &st);
  p->tile_sum_off = ws_get<int64_t>(p, p->ntiles, &st);
  if (st) return st;
  cudaMemsetAsync(p->summary, 0, sizeof(Summary), s);
  cudaMemsetAsync(p->c_off, 0, sizeof(int64_t), s);
  if (p->prec == SPGEMM_F32_COMPENSATED && m > 0) {
    // FP32 compensated: the short rows take the block and warp hash kernels when no value of A or
    // B is negative (their bound then needs only the row length); otherwise every non-tiny row
    // takes the windowed kernel, which keeps the full bound
    launch_negative_check(p->A.val, A->nnz, p->B.val, B->nnz, p->counters + 8, p->num_sms, s);
    int32_t neg = 1;
    st = read_small(&neg, p->counters + 8, sizeof(neg), s, &p->launches, "reading the sign check of the FP32 values");
    if (st) return st;
    p->cp.window_all = neg ? 1 : 0;
  }

  Summary h;
  if (o.validate) {
    uint32_t* starts = ws_get<uint32_t>(p, validate_words(A->nnz > B->nnz ? A->nnz : B->nnz), &st);
    if (st) return st;
    // no wait here: the count kernels clamp every access, and the error word is read with the
    // plan's summary below (an invalid input is reported before any other pass runs)
    conv += launch_validate(p->A, starts, &p->summary->err, s);
    conv += launch_validate(p->B, starts, &p->summary->err, s);
    stage_end(p, SPGEMM_STAGE_VALIDATE, conv, s);
    if ((st = cuda_status(cudaGetLastError(), "launching validation")) != SPGEMM_OK) return st;
  } else {
    stage_end(p, SPGEMM_STAGE_VALIDATE, conv, s);
  }
  if (m > 0) {
    stage_begin(p, SPGEMM_STAGE_COUNT, s);
    int nl = launch_count(p->A, p->B, p->cp, p->P, p->nnz_row, p->tile_hist, p->tile_sum, p->tile_max, s);
    nl += launch_class_scan(p->ntiles, kSymNumClasses, p->tile_hist, p->tile_sum, p->tile_max, nullptr,
                            p->summary, s);
    nl += launch_scatter_sym(p->A, p->cp, p->P, p->tile_hist, p->perm_s, s);
    stage_end(p, SPGEMM_STAGE_COUNT, nl, s);
    if ((st = cuda_status(cudaGetLastError(), "launching the plan kernels")) != SPGEMM_OK) return st;
    if ((st = read_summary(p, &h, s)) != SPGEMM_OK) return st;
    if (h.err) return error_bits_status(h.err);
    std::memcpy(p->sym_off, h.class_off, sizeof(p->sym_off));
    p->total_products = h.total;
    p->max_row_products = h.max_row;
  } else if (o.validate) {
    if ((st = read_summary(p, &h, s)) != SPGEMM_OK) return st;
    if (h.err) return error_bits_status(h.err);
  }
  const int64_t nwin = p->sym_off[kSymWin3 + 1] - p->sym_off[kSymWin0];
  if (nwin > 0) {
    p->nblocks = (p->width + kBlockCols - 1) / kBlockCols;
    const int64_t cnt_bytes = nwin * p->nblocks * 2;
    if (cnt_bytes > (int64_t(8) << 30))
      return set_error_msg(SPGEMM_ERR_UNSUPPORTED, "windowed rows need %lld bytes of block counts", (long long)cnt_bytes);
    p->blockcnt = ws_get<uint16_t>(p, nwin * p->nblocks, &st);
    p->win_slot = ws_get<int32_t>(p, m, &st);
    p->cursor = ws_get<int32_t>(p, A->nnz, &st);
    if (st) return st;
    // room for the windowed rows' column bitmaps (one 128-word block per 4096 columns of the row),
    // within the budget; rows that find it full keep the marking pass in the numeric kernel
    const int64_t budget = (int64_t(p->opts.window_cols_max_mb > 0 ? p->opts.window_cols_max_mb : 0) << 20) / 4;
    const int64_t need = nwin * p->nblocks * kBlockWords;
    p->wcap = need < budget ? need : budget;
    if (p->wcap > 0) {
      p->wbits = ws_get<uint32_t>(p, p->wcap, &st);
      p->wcur = ws_get<unsigned long long>(p, 1, &st);
      p->woff = ws_get<int64_t>(p, nwin, &st);
      if (st) return st;
    }
  }
  p->state = 0;
  return SPGEMM_OK;
}

spgemm_status symbolic_run(spgemm_plan_s* p, cudaStream_t s) {
  spgemm_status st;
  const int64_t m = p->A.rows;
  if (p->small) {
    // the plan launched the symbolic kernel on its own stream; read its summary there (the host
    // wait orders every later stream after it)
    Summary h;
    if (p->small_host) {
      const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(p->ws.stream));
      if (e != cudaSuccess) return cuda_status(e, "waiting for the small-product symbolic pass");
      std::memcpy(&h, p->small_host, sizeof(Summary));
      release_small_host(p);
      if (h.small_flags == kSmallUnwritten)
        return set_error_msg(SPGEMM_ERR_INTERNAL, "the small-product symbolic pass left no summary");
    } else if ((st = read_summary(p, &h, static_cast<cudaStream_t>(p->ws.stream))) != SPGEMM_OK) {
      return st;
    }
    if (h.err) return error_bits_status(h.err);
    if (h.small_flags) {
      // a row of C is too long for the small path: plan and count again through the row classes
      const spgemm_csr_in a = p->a_in, b = p->b_in;
      p->opts.general_path = 1;
      p->small = false;
      if ((st = plan_run(p, &a, &b, s)) != SPGEMM_OK) return st;
      return symbolic_run(p, s);
    }
    p->total_products = static_cast<int64_t>(h.small_products);
    p->nnz_c = h.total;
    p->small_cap = static_cast<int>(h.max_row);
    if (p->abase) {
      // a stacked batch reads its jobs' offsets from the row offsets of C
      p->c_off = ws_get<int64_t>(p, m + 1, &st);
      if (st) return st;
      launch_small_offsets(p->small_loc, p->small_blk, p->small_grid, m, p->c_off, s);
    }
    // every row counts as one warp-table row in the plan's class counters
    for (int c = 0; c <= kMaxClasses; ++c) {
      p->sym_off[c] = c <= kSymWarp3 ? 0 : m;
      p->num_off[c] = c <= kNumWarp3 ? 0 : m;
    }
    std::memset(p->cls_sums, 0, sizeof(p->cls_sums));
    p->cls_sums[kNumWarp3][0] = static_cast<unsigned long long>(h.small_products);
    p->cls_sums[kNumWarp3][1] = static_cast<unsigned long long>(p->A.nnz);
    p->cls_sums[kNumWarp3][2] = static_cast<unsigned long long>(h.total);
    p->state = 1;
    return SPGEMM_OK;
  }
  auto seg = [&](int c) { return p->perm_s + p->sym_off[c]; };
  auto cnt = [&](int c) { return p->sym_off[c + 1] - p->sym_off[c]; };
  uint32_t* err = &p->summary->err;
  if (m > 0) {
    int nl;
    stage_begin(p, SPGEMM_STAGE_SYM_WINDOW, s);
    if (p->wcur) cudaMemsetAsync(p->wcur, 0, sizeof(unsigned long long), s);
    nl = launch_sym_window(p->A, p->B, seg(kSymWin0), p->sym_off[kSymWin3 + 1] - p->sym_off[kSymWin0],
                           p->counters + 0, p->nnz_row, p->win_slot, p->blockcnt, p->nblocks, p->cursor,
                           p->abase, p->awidth, p->width, p->wbits, p->wcap, p->wcur, p->woff, p->num_sms, err,
                           s);
    stage_end(p, SPGEMM_STAGE_SYM_WINDOW, nl, s);
    stage_begin(p, SPGEMM_STAGE_SYM_BLOCK, s);
    nl = launch_sym_block(13, p->A, p->B, seg(kSymBlock), cnt(kSymBlock), p->nnz_row, err, p->num_sms, s);
    stage_end(p, SPGEMM_STAGE_SYM_BLOCK, nl, s);
    stage_begin(p, SPGEMM_STAGE_SYM_WARP, s);
    nl = launch_sym_warp(11, p->A, p->B, seg(kSymWarp3), cnt(kSymWarp3), p->nnz_row, err, p->num_sms, s);
    nl += launch_sym_warp(9, p->A, p->B, seg(kSymWarp2), cnt(kSymWarp2), p->nnz_row, err, p->num_sms, s);
    nl += launch_sym_warp(7, p->A, p->B, seg(kSymWarp1), cnt(kSymWarp1), p->nnz_row, err, p->num_sms, s);
    stage_end(p, SPGEMM_STAGE_SYM_WARP, nl, s);
    stage_begin(p, SPGEMM_STAGE_SYM_TINY, s);
    if (cnt(kSymMicro) < kMicroMinRows) {
      // few micro rows: a thread-per-row merge is one long chain of dependent loads, so they join
      // the tiny rows (a warp per row; every micro row qualifies), which come just before them
      nl = launch_sym_tiny(p->A, p->B, seg(kSymTiny), cnt(kSymTiny) + cnt(kSymMicro), p->nnz_row, p->num_sms, s);
    } else {
      nl = launch_sym_tiny(p->A, p->B, seg(kSymTiny), cnt(kSymTiny), p->nnz_row, p->num_sms, s);
      nl += launch_sym_micro(p->A, p->B, seg(kSymMicro), cnt(kSymMicro), p->nnz_row, p->num_sms, s);
    }
    stage_end(p, SPGEMM_STAGE_SYM_TINY, nl, s);
    stage_begin(p, SPGEMM_STAGE_SYM_SCAN, s);
    nl = launch_num_tiles(p->A, p->cp, p->P, p->nnz_row, p->tile_hist, p->tile_sum, &p->summary->cls_sums[0][0], s);
    nl += launch_class_scan(p->ntiles, kNumNumClasses, p->tile_hist, p->tile_sum, nullptr, p->tile_sum_off,
                            p->summary, s);
    nl += launch_scatter_num(p->A, p->cp, p->P, p->nnz_row, p->tile_hist, p->tile_sum_off, p->perm_n,
                             p->c_off, s);
    stage_end(p, SPGEMM_STAGE_SYM_SCAN, nl, s);
    if ((st = cuda_status(cudaGetLastError(), "launching the symbolic kernels")) != SPGEMM_OK) return st;
    Summary h;
    if ((st = read_summary(p, &h, s)) != SPGEMM_OK) return st;
    if (h.err) return error_bits_status(h.err);
    std::memcpy(p->num_off, h.class_off, sizeof(p->num_off));
    std::memcpy(p->cls_sums, h.cls_sums, sizeof(p->cls_sums));
    p->nnz_c = h.total;
  } else {
    if ((st = cuda_status(cudaStreamSynchronize(s), "symbolic pass")) != SPGEMM_OK) return st;
    p->nnz_c = 0;
  }
  p->state = 1;
  return SPGEMM_OK;
}

void plan_bytes_bounds(int64_t m, int64_t a_nnz, int64_t width, int a_rowptr32, int b_rowptr32, int64_t b_rows,
                       int64_t b_nnz, int validate, int32_t wbits_mb, int64_t* lo, int64_t* hi) {
  const int64_t ntiles = (m + kTileRows - 1) / kTileRows;
  int64_t fixed = ws_rounded(sizeof(Summary)) + ws_rounded(16 * 4) + ws_rounded(8 * m) + 3 * ws_rounded(4 * m) +
                  ws_rounded(8 * (m + 1));
  if (a_rowptr32) fixed += ws_rounded(8 * (m + 1));
  if (b_rowptr32) fixed += ws_rounded(8 * (b_rows + 1));
  if (validate) fixed += ws_rounded(4 * validate_words(a_nnz > b_nnz ? a_nnz : b_nnz));
  const int64_t tiles = ws_rounded(4 * ntiles * kMaxClasses) + 3 * ws_rounded(8 * ntiles);
  const int64_t nblocks = (width + kBlockCols - 1) / kBlockCols;
  const int64_t stored_words = wbits_mb > 0 ? (int64_t(wbits_mb) << 20) / 4 : 0;
  const int64_t row_words = m * nblocks * kBlockWords;
  const int64_t stored = stored_words > 0 ? ws_rounded(4 * (row_words < stored_words ? row_words : stored_words)) +
                                                ws_rounded(8) + ws_rounded(8 * m)
                                          : 0;
  const int64_t window = ws_rounded(2 * m * nblocks) + ws_rounded(4 * m) + ws_rounded(4 * a_nnz) + stored;
  *lo = fixed;
  *hi = fixed + tiles + window;
}

namespace {

// Entries of each windowed-kernel block's window lists (rows with more than 512 A entries list
// their segments per window; a batch of windows whose lists exceed this keeps chunks of A entries):
// 16 per A entry of the windowed rows, spread over the blocks, at most 2^20 (20 MB a block). None
// for the exact fixed-point mode or without a split table.
constexpr int64_t kListCapMax = int64_t(1) << 20;
constexpr int64_t kListBytesPerEntry = 8 + 4 + 8;

int64_t window_list_cap(const spgemm_plan_s* p, int64_t nwin) {
  if (nwin <= 0 || (p->prec == SPGEMM_F64 && p->opts.fp64_accumulate != 0)) return 0;
  unsigned long long annz = 0;
  for (int c = kNumWin0; c <= kNumWin3; ++c) annz += p->cls_sums[c][1];
  if (annz <= 512) return 0;
  const int64_t cap = static_cast<int64_t>(annz) * 16 / num_window_blocks(nwin, p->num_sms);
  return cap < kListCapMax ? cap : kListCapMax;
}

}  // namespace

int64_t numeric_extra_bytes(const spgemm_plan_s* p) {
  const int64_t m = p->A.rows;
  if (m <= 0) return 0;
  int64_t extra = 0;
  const int64_t nwin = p->num_off[kNumWin3 + 1] - p->num_off[kNumWin0];
  if (p->prec == SPGEMM_F32_COMPENSATED && !p->rerun_flag) {
    extra += 2 * ws_rounded(4 * m);
    const int64_t nwh = p->num_off[kNumWarp1 + 1] - p->num_off[kNumWin0];
    if (nwh > 0) extra += ws_rounded(8 * rerun_group_rows(p->width, kRerunScratchBytes) * p->width);
  }
  if (p->prec == SPGEMM_F64 && p->opts.fp64_accumulate != 0 && nwin > 0) {
    if (!p->rerun_flag) extra += 2 * ws_rounded(4 * m);   // flags and list of FP64 reruns
    if (!p->bexp) extra += ws_rounded(2 * p->B.rows);     // exponent bound per row of B
  }
  if (nwin > 0 && !p->split_tried) {
    const int64_t bytes = split_table_bytes(p->B.rows, p->nblocks);
    if (bytes <= (int64_t(p->opts.window_split_max_mb) << 20)) {
      extra += ws_rounded(bytes);
      if (!p->lists_tried) {
        const int64_t n = num_window_blocks(nwin, p->num_sms) * window_list_cap(p, nwin);
        if (n > 0) extra += ws_rounded(8 * n) + ws_rounded(4 * n) + ws_rounded(8 * n);
      }
    }
  }
  return extra;
}

spgemm_status numeric_run(spgemm_plan_s* p, spgemm_csr_out* C, cudaStream_t s) {
  spgemm_status st = SPGEMM_OK;
  const int64_t m = p->A.rows;
  const bool f32c = p->prec == SPGEMM_F32_COMPENSATED;
  const int mode = f32c ? kModeF32C : kModeF64;
  // FP64 windowed rows: exact fixed-point accumulation when the caller asks for it
  const bool fx = !f32c && p->opts.fp64_accumulate != 0;
  p->f32c_rerun_rows = 0;
  int nl;
  if (p->small) {
    // the numeric kernel writes C's row pointers as well
    stage_begin(p, SPGEMM_STAGE_NUM_WARP, s);
    nl = launch_small_numeric(small_csr(p->a_in, p->abase), small_csr(p->b_in), small_width(p), p->small_grid,
                              p->small_cap, p->nnz_row,
                              p->small_loc, p->small_blk, C->row_ptr, C->idx64_rowptr, C->col,
                              static_cast<double*>(C->val), &p->summary->err, p->num_sms, s);
    stage_end(p, SPGEMM_STAGE_NUM_WARP, nl, s);
    if ((st = cuda_status(cudaGetLastError(), "launching the small-product numeric pass")) != SPGEMM_OK) return st;
    p->state = 2;
    return SPGEMM_OK;
  }
  stage_begin(p, SPGEMM_STAGE_NUM_ROWPTR, s);
  nl = launch_write_rowptr(p->c_off, m + 1, C->row_ptr, C->idx64_rowptr, s);
  stage_end(p, SPGEMM_STAGE_NUM_ROWPTR, nl, s);
  if (m > 0) {
    auto seg = [&](int c) { return p->perm_n + p->num_off[c]; };
    auto cnt = [&](int c) { return p->num_off[c + 1] - p->num_off[c]; };
    uint32_t* err = &p->summary->err;
    const int64_t nwin = p->num_off[kNumWin3 + 1] - p->num_off[kNumWin0];
    const int64_t nslots = p->sym_off[kSymWin3 + 1] - p->sym_off[kSymWin0];
    // windowed, block and warp rows (consecutive classes): the FP32 rows the dense FP64 rerun takes
    const int64_t nwh = p->num_off[kNumWarp1 + 1] - p->num_off[kNumWin0];
    if (f32c) {
      if (!p->rerun_flag) {
        p->rerun_flag = ws_get<int32_t>(p, m, &st);
        p->rerun_list = ws_get<int32_t>(p, m, &st);
        if (nwh > 0) {
          p->rerun_group = rerun_group_rows(p->width, kRerunScratchBytes);
          p->rerun_dense = ws_get<double>(p, p->rerun_group * p->width, &st);
        }
        if (st) return st;
      }
      cudaMemsetAsync(p->rerun_flag, 0, sizeof(int32_t) * m, s);
    }
    if (fx && nwin > 0) {
      if (!p->rerun_flag) {
        p->rerun_flag = ws_get<int32_t>(p, m, &st);
        p->rerun_list = ws_get<int32_t>(p, m, &st);
      }
      if (!p->bexp) p->bexp = ws_get<uint16_t>(p, p->B.rows, &st);
      if (st) return st;
      cudaMemsetAsync(p->rerun_flag, 0, sizeof(int32_t) * m, s);
      cudaMemsetAsync(p->counters + 6, 0, sizeof(int32_t), s);
    }
    stage_begin(p, SPGEMM_STAGE_NUM_WINDOW, s);
    nl = 0;
    if (fx && nwin > 0) nl += launch_brow_exponent(p->B, p->bexp, p->num_sms, s);
    // FP32 compensated: whether every value of A and B is non-negative (then the windowed rows'
    // error bound needs no sum of |p|), read by the window kernel on the device
    if (f32c && nwh > 0) nl += launch_negative_check(p->A.val, p->A.nnz, p->B.val, p->B.nnz, p->counters + 8,
                                                     p->num_sms, s);
    if (nwin > 0 && !p->split_tried) {
      // split table of B, once per plan, when it fits the budget (else the kernel searches)
      p->split_tried = true;
      const int64_t bytes = split_table_bytes(p->B.rows, p->nblocks);
      if (bytes <= (int64_t(p->opts.window_split_max_mb) << 20)) {
        p->split = static_cast<int32_t*>(p->ws.get(static_cast<size_t>(bytes)));
        if (p->split) nl += launch_bsplit(p->B, p->nblocks, p->bbase, p->split, s);
      }
    }
    if (nwin > 0 && !p->lists_tried && !fx) {
      p->lists_tried = true;
      const int64_t cap = p->split ? window_list_cap(p, nwin) : 0;
      const int64_t n = num_window_blocks(nwin, p->num_sms) * cap;
      if (n > 0) {
        p->list_bs = static_cast<int64_t*>(p->ws.get(static_cast<size_t>(8 * n)));
        p->list_len = static_cast<int32_t*>(p->ws.get(static_cast<size_t>(4 * n)));
        p->list_av = static_cast<double*>(p->ws.get(static_cast<size_t>(8 * n)));
        if (p->list_bs && p->list_len && p->list_av) p->list_cap = cap;
      }
    }
    nl += launch_num_window(fx ? kModeF64X : mode, p->A, p->B, seg(kNumWin0), nwin, p->counters + 1, p->c_off,
                            p->win_slot, p->blockcnt, p->nblocks, nslots, p->split, p->opts.window_hash_fill, C->col,
                            C->val, p->rerun_flag, p->abase, p->awidth, p->width, p->wbits, p->woff, p->bexp,
                            nullptr, f32c ? p->counters + 8 : nullptr, fx ? nullptr : p->list_bs,
                            fx ? nullptr : p->list_len, fx ? nullptr : p->list_av, fx ? 0 : p->list_cap, p->num_sms,
                            err, s);
    if (fx && nwin > 0) {
      // rows outside the fixed-point range (a very wide spread of product magnitudes, subnormal or
      // non-finite values) are redone with FP64 shared atomics; the list stays on the device
      nl += launch_collect_flagged(seg(kNumWin0), nwin, p->rerun_flag, 0, p->rerun_list, p->counters + 6, s);
      nl += launch_num_window(kModeF64, p->A, p->B, p->rerun_list, nwin, p->counters + 7, p->c_off, p->win_slot,
                              p->blockcnt, p->nblocks, nslots, p->split, p->opts.window_hash_fill, C->col, C->val,
                              nullptr, p->abase, p->awidth, p->width, p->wbits, p->woff, nullptr, p->counters + 6,
                              nullptr, nullptr, nullptr, nullptr, 0, p->num_sms, err, s);
      p->fx_rerun_pending = true;
    }
    stage_end(p, SPGEMM_STAGE_NUM_WINDOW, nl, s);
    stage_begin(p, SPGEMM_STAGE_NUM_EXPAND, s);
    nl = launch_expand_cols(seg(kNumWin0), nwin, p->win_slot, p->woff, p->wbits, p->blockcnt, p->nblocks, p->c_off,
                            p->awidth, p->width, C->col, p->num_sms, err, s);
    stage_end(p, SPGEMM_STAGE_NUM_EXPAND, nl, s);
    {
      int32_t* flag = f32c ? p->rerun_flag : nullptr;
      const int32_t* neg = f32c ? p->counters + 8 : nullptr;
      stage_begin(p, SPGEMM_STAGE_NUM_BLOCK, s);
      nl = launch_num_block(13, mode, p->A, p->B, seg(kNumBlock2), cnt(kNumBlock2), p->c_off, C->col, C->val,
                            p->abase, flag, neg, err, p->num_sms, s);
      nl += launch_num_block(11, mode, p->A, p->B, seg(kNumBlock1), cnt(kNumBlock1), p->c_off, C->col, C->val,
                             p->abase, flag, neg, err, p->num_sms, s);
      stage_end(p, SPGEMM_STAGE_NUM_BLOCK, nl, s);
      stage_begin(p, SPGEMM_STAGE_NUM_WARP, s);
      nl = launch_num_warp(10, mode, p->A, p->B, seg(kNumWarp3), cnt(kNumWarp3), p->c_off, C->col, C->val, p->abase,
                           flag, neg, err, p->num_sms, s);
      nl += launch_num_warp(8, mode, p->A, p->B, seg(kNumWarp2), cnt(kNumWarp2), p->c_off, C->col, C->val, p->abase,
                            flag, neg, err, p->num_sms, s);
      nl += launch_num_warp(6, mode, p->A, p->B, seg(kNumWarp1), cnt(kNumWarp1), p->c_off, C->col, C->val, p->abase,
                            flag, neg, err, p->num_sms, s);
      stage_end(p, SPGEMM_STAGE_NUM_WARP, nl, s);
    }
    stage_begin(p, SPGEMM_STAGE_NUM_TINY, s);
    const bool micro_as_tiny = f32c || cnt(kNumMicro) < kMicroMinRows;   // (F32 plans have no micro rows)
    nl = launch_num_tiny(mode, p->A, p->B, seg(kNumTiny), cnt(kNumTiny) + (micro_as_tiny ? cnt(kNumMicro) : 0),
                         p->c_off, C->col, C->val, p->rerun_flag, p->abase, err, p->num_sms, s);
    if (!micro_as_tiny)
      nl += launch_num_micro(p->A, p->B, seg(kNumMicro), cnt(kNumMicro), p->c_off, C->col,
                             static_cast<double*>(C->val), p->abase, err, p->num_sms, s);
    stage_end(p, SPGEMM_STAGE_NUM_TINY, nl, s);
    if (f32c && !p->opts.f32c_rerun_none) {
      // rows with an entry over the compensated bound are recomputed in FP64 and rounded once
      stage_begin(p, SPGEMM_STAGE_NUM_RERUN, s);
      int32_t* list_w = p->rerun_list;
      int32_t* list_t = p->rerun_list + nwh;
      cudaMemsetAsync(p->counters + 4, 0, 2 * sizeof(int32_t), s);
      const int all = p->opts.f32c_rerun_all ? 1 : 0;
      nl = launch_collect_flagged(seg(kNumWin0), nwh, p->rerun_flag, all, list_w, p->counters + 4, s);
      nl += launch_collect_flagged(seg(kNumTiny), cnt(kNumTiny), p->rerun_flag, all, list_t, p->counters + 5, s);
      int32_t hc[2] = {0, 0};
      spgemm_status rs = read_small(hc, p->counters + 4, sizeof(hc), s, &p->launches, "reading the FP64 rerun counts");
      if (rs) return rs;
      if (hc[0] > 0)
        nl += launch_rerun_dense(p->A, p->B, list_w, hc[0], p->c_off, C->col, static_cast<float*>(C->val), p->abase,
                                 p->width, p->rerun_dense, p->rerun_group, p->num_sms, err, s);
      nl += launch_num_tiny(kModeF32R, p->A, p->B, list_t, hc[1], p->c_off, C->col, C->val, nullptr, p->abase, err, p->num_sms,
                            s);
      stage_end(p, SPGEMM_STAGE_NUM_RERUN, nl, s);
      p->f32c_rerun_rows = int64_t(hc[0]) + hc[1];
    }
  }
  if ((st = cuda_status(cudaGetLastError(), "launching the numeric kernels")) != SPGEMM_OK) return st;
  p->state = 2;
  return SPGEMM_OK;
}

}  // namespace spg
