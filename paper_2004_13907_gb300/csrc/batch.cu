// Batched products C_j = A_j * B_j for many independent jobs, run as ONE product.
//
// The jobs are stacked into a block-diagonal product: A = diag(A_1, ..., A_n) and
// B = diag(B_1, ..., B_n) give C = diag(A_1 B_1, ..., A_n B_n). One plan, one symbolic pass and
// one numeric pass then cover every job, so thousands of small products cost the launches of one
// (about twenty kernels in all) instead of twenty each. Every row of the stacked product keeps the
// column space of its own job (its column base and the widest job's width), so the windowed
// kernels count blocks from the job's first column and the output columns come out job-local.
//
// The result is one concatenated CSR owned by the batch: job j's rows are rows
// [row0_j, row0_j + m_j) of it, and spgemm_batch_result hands out a standalone CSR view per job
// (its own int64 row_ptr starting at 0, col and val pointers into the shared arrays).
// spgemm_batch_replay re-copies the jobs' current values and re-runs the numeric pass through a
// CUDA graph captured on first use (the sparsity patterns must be unchanged).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "batch.h"

namespace spg {

namespace {

constexpr int64_t kTile = 1 << 15;

// One stacked matrix (A or B side) of one job.
struct Part {
  const void* rp;
  const int32_t* col;
  const void* val;
  int64_t rows, nnz;
  int64_t row0, nnz0;     // where the job's rows / entries start in the stacked matrix
  int64_t col_shift;      // added to the job's column indices
  int64_t col_limit;      // the job's own column count (indices must be below it)
  int32_t base;           // column base of the job's rows in the stacked product
  int32_t idx64;
  int32_t width;          // A side: the job's column count of C (the width of its rows)
  int32_t pad_;
};

struct Tile {
  int32_t part;
  int32_t kind;           // 0: row pointers (+ base), 1: columns and values, 2: values only
  int64_t start;
};

__global__ void __launch_bounds__(256) k_stack(const Part* __restrict__ parts, const Tile* __restrict__ tiles,
                                               int64_t* __restrict__ rp_out, int32_t* __restrict__ col_out,
                                               unsigned char* __restrict__ val_out, int32_t* __restrict__ base_out,
                                               int32_t* __restrict__ width_out, int val_bytes, uint32_t* err) {
  const Tile t = tiles[blockIdx.x];
  const Part pt = parts[t.part];
  if (t.kind == 0) {
    const int64_t end = t.start + kTile < pt.rows ? t.start + kTile : pt.rows;
    for (int64_t r = t.start + threadIdx.x; r < end; r += blockDim.x) {
      const int64_t v = pt.idx64 ? static_cast<const int64_t*>(pt.rp)[r] : static_cast<const int32_t*>(pt.rp)[r];
      rp_out[pt.row0 + r] = v + pt.nnz0;
      base_out[pt.row0 + r] = pt.base;
      if (width_out) width_out[pt.row0 + r] = pt.width;
    }
  } else {
    const int64_t end = t.start + kTile < pt.nnz ? t.start + kTile : pt.nnz;
    for (int64_t e = t.start + threadIdx.x; e < end; e += blockDim.x) {
      if (t.kind == 1) {
        const int32_t c = pt.col[e];
        if (c < 0 || c >= pt.col_limit) set_error(err, kErrInvalidCsr);
        col_out[pt.nnz0 + e] = static_cast<int32_t>(c + pt.col_shift);
      }
      if (val_bytes == 8)
        reinterpret_cast<double*>(val_out)[pt.nnz0 + e] = static_cast<const double*>(pt.val)[e];
      else
        reinterpret_cast<float*>(val_out)[pt.nnz0 + e] = static_cast<const float*>(pt.val)[e];
    }
  }
}

// Per-job row pointers starting at 0: out[row0_j + j + r] = c_off[row0_j + r] - c_off[row0_j].
__global__ void __launch_bounds__(256) k_job_rowptr(const Part* __restrict__ parts, const Tile* __restrict__ tiles,
                                                    const int64_t* __restrict__ c_off, int64_t* __restrict__ out) {
  const Tile t = tiles[blockIdx.x];
  const Part pt = parts[t.part];
  const int64_t job = t.part;   // tiles of this kernel index the A side, one part per job
  const int64_t end = t.start + kTile < pt.rows + 1 ? t.start + kTile : pt.rows + 1;
  const int64_t first = c_off[pt.row0];
  for (int64_t r = t.start + threadIdx.x; r < end; r += blockDim.x)
    out[pt.row0 + job + r] = c_off[pt.row0 + r] - first;
}

void add_tiles(std::vector<Tile>& tiles, int part, int kind, int64_t count) {
  for (int64_t s = 0; s < count; s += kTile) tiles.push_back(Tile{part, kind, s});
}

}  // namespace

}  // namespace spg

using namespace spg;

struct spgemm_batch_s {
  int64_t n_jobs = 0;
  spgemm_prec prec = SPGEMM_F64;
  Workspace ws;                       // stacked inputs, outputs, tables
  spgemm_plan_t* plan = nullptr;
  std::vector<Part> parts;            // A parts [0, n), B parts [n, 2n)
  Part* d_parts = nullptr;
  // tile lists, A side first then B side: [0, a_tiles) stack A, [a_tiles, end) stack B
  std::vector<Tile> stack_tiles, value_tiles, rowptr_tiles;
  int64_t stack_a = 0, value_a = 0;
  Tile* d_stack_tiles = nullptr;
  Tile* d_value_tiles = nullptr;
  Tile* d_rowptr_tiles = nullptr;
  int64_t* a_rp = nullptr;
  int32_t* a_col = nullptr;
  void* a_val = nullptr;
  int32_t* abase = nullptr;
  int32_t* awidth = nullptr;
  int64_t* b_rp = nullptr;
  int32_t* b_col = nullptr;
  void* b_val = nullptr;
  int32_t* bbase = nullptr;
  uint32_t* err = nullptr;
  int64_t rows = 0, inner = 0, cols = 0, a_nnz = 0, b_nnz = 0;
  std::vector<int64_t> job_nnz0;      // entry offset of each job in the output (n_jobs + 1)
  int32_t* c_col = nullptr;
  void* c_val = nullptr;
  int64_t* job_rp = nullptr;          // per-job row pointers, rows_j + 1 each
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;   // private stream the graph is captured on
  int64_t launches = 0;               // stacking and row-pointer kernels (the plan counts its own)
};

namespace spg {

spgemm_status batch_prepare(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B, spgemm_prec prec,
                            const spgemm_opts* opts, const spgemm_allocator* alloc, void* stream,
                            spgemm_batch_t** out) {
  if (!out) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_jobs < 1 || !A || !B) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "need n_jobs >= 1 and job arrays");
  if (prec != SPGEMM_F64 && prec != SPGEMM_F32_COMPENSATED)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "unknown precision %d", int(prec));
  spgemm_status st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spgemm_batch_t* b = new (std::nothrow) spgemm_batch_t();
  if (!b) return set_error_msg(SPGEMM_ERR_OOM, "host allocation of the batch failed");
  b->n_jobs = n_jobs;
  b->prec = prec;
  b->ws.stream = stream;
  if (alloc) { b->ws.alloc = *alloc; b->ws.has_alloc = true; }
  auto fail = [&](spgemm_status code) {
    const std::string msg = spgemm_last_error();
    cudaStreamSynchronize(s);
    if (b->plan) spgemm_plan_destroy(b->plan);
    b->ws.release_all();
    delete b;
    set_error_msg(code, "%s", msg.c_str());
    return code;
  };
  // job tables: stacked row, entry and column offsets
  int64_t width = 0;
  b->parts.resize(static_cast<size_t>(2 * n_jobs));
  for (int64_t j = 0; j < n_jobs; ++j) {
    char name[32];
    std::snprintf(name, sizeof(name), "A[%lld]", (long long)j);
    if ((st = check_csr_in(&A[j], name, prec)) != SPGEMM_OK) return fail(st);
    std::snprintf(name, sizeof(name), "B[%lld]", (long long)j);
    if ((st = check_csr_in(&B[j], name, prec)) != SPGEMM_OK) return fail(st);
    if (A[j].cols != B[j].rows) {
      set_error_msg(SPGEMM_ERR_INVALID_ARG, "job %lld: A.cols != B.rows", (long long)j);
      return fail(SPGEMM_ERR_INVALID_ARG);
    }
    Part& pa = b->parts[j];
    pa = Part{A[j].row_ptr, A[j].col, A[j].val, A[j].rows, A[j].nnz, b->rows, b->a_nnz, b->inner, A[j].cols,
              static_cast<int32_t>(b->cols), A[j].idx64_rowptr, static_cast<int32_t>(B[j].cols), 0};
    Part& pb = b->parts[n_jobs + j];
    pb = Part{B[j].row_ptr, B[j].col, B[j].val, B[j].rows, B[j].nnz, b->inner, b->b_nnz, b->cols, B[j].cols,
              static_cast<int32_t>(b->cols), B[j].idx64_rowptr, static_cast<int32_t>(B[j].cols), 0};
    b->rows += A[j].rows;
    b->inner += B[j].rows;
    b->cols += B[j].cols;
    b->a_nnz += A[j].nnz;
    b->b_nnz += B[j].nnz;
    width = B[j].cols > width ? B[j].cols : width;
  }
  if (b->rows >= 0x7fffffffLL || b->inner >= 0x7fffffffLL || b->cols >= 0x7fffffffLL) {
    set_error_msg(SPGEMM_ERR_UNSUPPORTED, "the stacked batch exceeds int32 row/column indices");
    return fail(SPGEMM_ERR_UNSUPPORTED);
  }
  for (int64_t j = 0; j < n_jobs; ++j) {
    add_tiles(b->stack_tiles, static_cast<int>(j), 0, b->parts[j].rows);
    add_tiles(b->stack_tiles, static_cast<int>(j), 1, b->parts[j].nnz);
    add_tiles(b->value_tiles, static_cast<int>(j), 2, b->parts[j].nnz);
    add_tiles(b->rowptr_tiles, static_cast<int>(j), 0, b->parts[j].rows + 1);
  }
  b->stack_a = static_cast<int64_t>(b->stack_tiles.size());
  b->value_a = static_cast<int64_t>(b->value_tiles.size());
  for (int64_t j = 0; j < n_jobs; ++j) {
    add_tiles(b->stack_tiles, static_cast<int>(n_jobs + j), 0, b->parts[n_jobs + j].rows);
    add_tiles(b->stack_tiles, static_cast<int>(n_jobs + j), 1, b->parts[n_jobs + j].nnz);
    add_tiles(b->value_tiles, static_cast<int>(n_jobs + j), 2, b->parts[n_jobs + j].nnz);
  }
  const int vb = prec == SPGEMM_F64 ? 8 : 4;
  auto get = [&](size_t bytes) { return b->ws.get(bytes); };
  b->d_parts = static_cast<Part*>(get(sizeof(Part) * b->parts.size()));
  b->d_stack_tiles = static_cast<Tile*>(get(sizeof(Tile) * (b->stack_tiles.size() + 1)));
  b->d_value_tiles = static_cast<Tile*>(get(sizeof(Tile) * (b->value_tiles.size() + 1)));
  b->d_rowptr_tiles = static_cast<Tile*>(get(sizeof(Tile) * (b->rowptr_tiles.size() + 1)));
  b->a_rp = static_cast<int64_t*>(get(sizeof(int64_t) * (b->rows + 1)));
  b->a_col = static_cast<int32_t*>(get(sizeof(int32_t) * b->a_nnz));
  b->a_val = get(static_cast<size_t>(vb) * b->a_nnz);
  b->abase = static_cast<int32_t*>(get(sizeof(int32_t) * b->rows));
  b->awidth = static_cast<int32_t*>(get(sizeof(int32_t) * b->rows));
  b->b_rp = static_cast<int64_t*>(get(sizeof(int64_t) * (b->inner + 1)));
  b->b_col = static_cast<int32_t*>(get(sizeof(int32_t) * b->b_nnz));
  b->b_val = get(static_cast<size_t>(vb) * b->b_nnz);
  b->bbase = static_cast<int32_t*>(get(sizeof(int32_t) * b->inner));
  b->err = static_cast<uint32_t*>(get(sizeof(uint32_t)));
  if (!b->d_parts || !b->d_stack_tiles || !b->d_value_tiles || !b->d_rowptr_tiles || !b->a_rp || !b->a_col ||
      !b->a_val || !b->abase || !b->awidth || !b->b_rp || !b->b_col || !b->b_val || !b->bbase || !b->err) {
    set_error_msg(SPGEMM_ERR_OOM, "device allocation of the stacked batch failed");
    return fail(SPGEMM_ERR_OOM);
  }
  cudaError_t e = cudaMemcpyAsync(b->d_parts, b->parts.data(), sizeof(Part) * b->parts.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !b->stack_tiles.empty())
    e = cudaMemcpyAsync(b->d_stack_tiles, b->stack_tiles.data(), sizeof(Tile) * b->stack_tiles.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !b->value_tiles.empty())
    e = cudaMemcpyAsync(b->d_value_tiles, b->value_tiles.data(), sizeof(Tile) * b->value_tiles.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !b->rowptr_tiles.empty())
    e = cudaMemcpyAsync(b->d_rowptr_tiles, b->rowptr_tiles.data(), sizeof(Tile) * b->rowptr_tiles.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->a_rp + b->rows, &b->a_nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->b_rp + b->inner, &b->b_nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { cuda_status(e, "staging the batch tables"); return fail(SPGEMM_ERR_CUDA); }
  // stack A (columns shifted to the job's B rows) and B (columns shifted to the job's columns)
  {
    const int64_t na = b->stack_a, nb = static_cast<int64_t>(b->stack_tiles.size()) - b->stack_a;
    if (na > 0)
      k_stack<<<static_cast<unsigned>(na), 256, 0, s>>>(b->d_parts, b->d_stack_tiles, b->a_rp, b->a_col,
                                                        static_cast<unsigned char*>(b->a_val), b->abase, b->awidth, vb,
                                                        b->err);
    if (nb > 0)
      k_stack<<<static_cast<unsigned>(nb), 256, 0, s>>>(b->d_parts, b->d_stack_tiles + na, b->b_rp, b->b_col,
                                                        static_cast<unsigned char*>(b->b_val), b->bbase, nullptr, vb,
                                                        b->err);
    b->launches += (na > 0) + (nb > 0);
  }
  uint32_t herr = 0;
  if ((st = read_small(&herr, b->err, sizeof(herr), s, &b->launches, "stacking the batch")) != SPGEMM_OK)
    return fail(st);
  if (herr) {
    set_error_msg(SPGEMM_ERR_INVALID_CSR, "a job has a column index outside its matrix");
    return fail(SPGEMM_ERR_INVALID_CSR);
  }
  // one plan over the stacked product, each row in its job's column space
  spgemm_csr_in SA{b->rows, b->inner, b->a_nnz, 1, 0, b->a_rp, b->a_col, b->a_val};
  spgemm_csr_in SB{b->inner, b->cols, b->b_nnz, 1, 0, b->b_rp, b->b_col, b->b_val};
  spgemm_plan_t* p = new (std::nothrow) spgemm_plan_t();
  if (!p) { set_error_msg(SPGEMM_ERR_OOM, "host allocation of the plan failed"); return fail(SPGEMM_ERR_OOM); }
  spgemm_opts_default(&p->opts);
  if (opts) p->opts = *opts;
  p->prec = prec;
  p->ws.stream = stream;
  if (alloc) { p->ws.alloc = *alloc; p->ws.has_alloc = true; }
  p->abase = b->abase;
  p->awidth = b->awidth;
  p->bbase = b->bbase;
  p->width = width > 0 ? width : 1;
  b->plan = p;
  if ((st = plan_run(p, &SA, &SB, s)) != SPGEMM_OK) return fail(st);
  if ((st = symbolic_run(p, s)) != SPGEMM_OK) return fail(st);
  // per-job entry offsets from the row offsets of C
  std::vector<int64_t> row0(static_cast<size_t>(n_jobs) + 1);
  for (int64_t j = 0; j < n_jobs; ++j) row0[j] = b->parts[j].row0;
  row0[n_jobs] = b->rows;
  b->job_nnz0.resize(static_cast<size_t>(n_jobs) + 1);
  std::vector<int64_t> h_off(static_cast<size_t>(b->rows) + 1);
  e = cudaMemcpyAsync(h_off.data(), p->c_off, sizeof(int64_t) * (b->rows + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cuda_status(e, "reading the batch row offsets"); return fail(SPGEMM_ERR_CUDA); }
  for (int64_t j = 0; j <= n_jobs; ++j) b->job_nnz0[j] = h_off[row0[j]];
  *out = b;
  return SPGEMM_OK;
}

void batch_prepare_bounds(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B, spgemm_prec prec,
                          const spgemm_opts* opts, int64_t* lo, int64_t* hi) {
  const int vb = prec == SPGEMM_F64 ? 8 : 4;
  int64_t rows = 0, inner = 0, a_nnz = 0, b_nnz = 0, width = 1, stack_tiles = 0, value_tiles = 0, rp_tiles = 0;
  for (int64_t j = 0; j < n_jobs; ++j) {
    rows += A[j].rows;
    inner += B[j].rows;
    a_nnz += A[j].nnz;
    b_nnz += B[j].nnz;
    width = B[j].cols > width ? B[j].cols : width;
    auto t = [](int64_t c) { return (c + kTile - 1) / kTile; };
    stack_tiles += t(A[j].rows) + t(A[j].nnz) + t(B[j].rows) + t(B[j].nnz);
    value_tiles += t(A[j].nnz) + t(B[j].nnz);
    rp_tiles += t(A[j].rows + 1);
  }
  const int64_t stacked = ws_rounded(int64_t(sizeof(Part)) * 2 * n_jobs) +
                          ws_rounded(int64_t(sizeof(Tile)) * (stack_tiles + 1)) +
                          ws_rounded(int64_t(sizeof(Tile)) * (value_tiles + 1)) +
                          ws_rounded(int64_t(sizeof(Tile)) * (rp_tiles + 1)) + ws_rounded(8 * (rows + 1)) +
                          ws_rounded(4 * a_nnz) + ws_rounded(vb * a_nnz) + 2 * ws_rounded(4 * rows) +
                          ws_rounded(8 * (inner + 1)) + ws_rounded(4 * b_nnz) + ws_rounded(vb * b_nnz) +
                          ws_rounded(4 * inner) + ws_rounded(4);
  int64_t plo = 0, phi = 0;
  plan_bytes_bounds(rows, a_nnz, width, 0, 0, inner, b_nnz, opts->validate, opts->window_cols_max_mb, &plo, &phi);
  *lo = stacked + plo;
  *hi = stacked + phi;
}

int64_t batch_output_bytes(const spgemm_batch_t* b) {
  const int vb = b->prec == SPGEMM_F64 ? 8 : 4;
  const int64_t nnz = b->plan->nnz_c > 0 ? b->plan->nnz_c : 1;
  return ws_rounded(4 * nnz) + ws_rounded(vb * nnz) + ws_rounded(8 * (b->rows + b->n_jobs));
}

int64_t batch_device_bytes(const spgemm_batch_t* b) {
  return b->ws.total + (b->plan ? b->plan->ws.total : 0);
}

int64_t batch_needed_bytes(const spgemm_batch_t* b) {
  return batch_device_bytes(b) + numeric_extra_bytes(b->plan) + batch_output_bytes(b);
}

int64_t batch_nnz(const spgemm_batch_t* b) { return b->plan ? b->plan->nnz_c : 0; }

void batch_set_release_stream(spgemm_batch_t* b, void* stream) {
  b->ws.stream = stream;
  if (b->plan) b->plan->ws.stream = stream;
}

int64_t batch_products(const spgemm_batch_t* b) { return b->plan ? b->plan->total_products : 0; }

spgemm_status batch_row_offsets(const spgemm_batch_t* b, int64_t* host_off, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(host_off, b->plan->c_off, sizeof(int64_t) * (b->rows + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SPGEMM_OK : cuda_status(e, "reading the batch row offsets");
}

int64_t batch_rows(const spgemm_batch_t* b) { return b->rows; }

int64_t batch_jobs(const spgemm_batch_t* b) { return b->n_jobs; }

spgemm_status batch_execute(spgemm_batch_t* b, void* stream) {
  spgemm_status st;
  cudaError_t e;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spgemm_plan_t* p = b->plan;
  const int vb = b->prec == SPGEMM_F64 ? 8 : 4;
  auto get = [&](size_t bytes) { return b->ws.get(bytes); };
  const int64_t n_jobs = b->n_jobs;
  // outputs, owned by the batch
  const int64_t nnz = p->nnz_c;
  b->c_col = static_cast<int32_t*>(get(sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
  b->c_val = get(static_cast<size_t>(vb) * (nnz > 0 ? nnz : 1));
  b->job_rp = static_cast<int64_t*>(get(sizeof(int64_t) * (b->rows + n_jobs)));
  if (!b->c_col || !b->c_val || !b->job_rp) return set_error_msg(SPGEMM_ERR_OOM, "device allocation of the batch output failed");
  spgemm_csr_out C{b->rows, b->cols, nnz, 1, 0, p->c_off, b->c_col, b->c_val};
  if ((st = numeric_run(p, &C, s)) != SPGEMM_OK) return st;
  if (!b->rowptr_tiles.empty()) {
    k_job_rowptr<<<static_cast<unsigned>(b->rowptr_tiles.size()), 256, 0, s>>>(b->d_parts, b->d_rowptr_tiles,
                                                                                  p->c_off, b->job_rp);
    ++b->launches;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "launching the batch");
  return SPGEMM_OK;
}

}  // namespace spg

extern "C" spgemm_status spgemm_batch(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B,
                                      spgemm_prec prec, const spgemm_opts* opts, const spgemm_allocator* alloc,
                                      void* stream, spgemm_batch_t** out) {
  clear_error_msg();
  spgemm_batch_t* b = nullptr;
  spgemm_status st = batch_prepare(n_jobs, A, B, prec, opts, alloc, stream, &b);
  if (st != SPGEMM_OK) return st;
  if ((st = batch_execute(b, stream)) != SPGEMM_OK) {
    const std::string msg = spgemm_last_error();
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    spgemm_batch_destroy(b);
    set_error_msg(st, "%s", msg.c_str());
    return st;
  }
  *out = b;
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_batch_result(const spgemm_batch_t* b, int64_t job, spgemm_csr_out* C) {
  clear_error_msg();
  if (!b || !C) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  if (job < 0 || job >= b->n_jobs) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "job %lld out of range", (long long)job);
  const Part& pa = b->parts[job];
  const int vb = b->prec == SPGEMM_F64 ? 8 : 4;
  C->rows = pa.rows;
  C->cols = b->parts[b->n_jobs + job].col_limit;
  C->nnz = b->job_nnz0[job + 1] - b->job_nnz0[job];
  C->idx64_rowptr = 1;
  C->row_ptr = b->job_rp + pa.row0 + job;
  C->col = b->c_col + b->job_nnz0[job];
  C->val = static_cast<unsigned char*>(b->c_val) + static_cast<size_t>(vb) * b->job_nnz0[job];
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_batch_get_info(const spgemm_batch_t* b, spgemm_plan_info* info) {
  clear_error_msg();
  if (!b || !info) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  const spgemm_status st = spgemm_plan_get_info(b->plan, info);
  info->kernel_launches += b->launches;
  return st;
}

extern "C" spgemm_status spgemm_batch_check(spgemm_batch_t* b, void* stream) {
  clear_error_msg();
  if (!b) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  return read_device_error(b->plan, static_cast<cudaStream_t>(stream));
}

extern "C" spgemm_status spgemm_batch_replay(spgemm_batch_t* b, void* stream) {
  clear_error_msg();
  if (!b) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "batch is NULL");
  if (b->prec != SPGEMM_F64)
    return set_error_msg(SPGEMM_ERR_UNSUPPORTED, "graph replay takes FP64 batches (the FP32 rerun reads a count)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spgemm_plan_t* p = b->plan;
  cudaError_t e;
  if (!b->graph_exec) {
    // capture on a private stream (the legacy default stream cannot be captured); the graph is
    // launched on the caller's stream
    if (!b->capture_stream) {
      e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_status(e, "creating the capture stream");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "waiting for the batch stream");
    const cudaStream_t cs = b->capture_stream;
    const int saved = p->opts.record_timings;
    p->opts.record_timings = 0;   // no event records inside the graph
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { p->opts.record_timings = saved; return cuda_status(e, "beginning the graph capture"); }
    // refresh the stacked values from the jobs' arrays, then the numeric pass
    const int vb = 8;
    const int64_t na = b->value_a, nb = static_cast<int64_t>(b->value_tiles.size()) - b->value_a;
    if (na > 0)
      k_stack<<<static_cast<unsigned>(na), 256, 0, cs>>>(b->d_parts, b->d_value_tiles, b->a_rp, b->a_col,
                                                         static_cast<unsigned char*>(b->a_val), b->abase, nullptr, vb,
                                                         b->err);
    if (nb > 0)
      k_stack<<<static_cast<unsigned>(nb), 256, 0, cs>>>(b->d_parts, b->d_value_tiles + na, b->b_rp, b->b_col,
                                                         static_cast<unsigned char*>(b->b_val), b->bbase, nullptr, vb,
                                                         b->err);
    spgemm_csr_out C{b->rows, b->cols, p->nnz_c, 1, 0, p->c_off, b->c_col, b->c_val};
    spgemm_status st = numeric_run(p, &C, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    p->opts.record_timings = saved;
    if (st != SPGEMM_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_status(e, "ending the graph capture");
    e = cudaGraphInstantiate(&b->graph_exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_status(e, "instantiating the graph"); }
    b->graph = g;
  }
  e = cudaGraphLaunch(b->graph_exec, s);
  if (e != cudaSuccess) return cuda_status(e, "launching the graph");
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_batch_destroy(spgemm_batch_t* b) {
  if (!b) return SPGEMM_OK;
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->plan) spgemm_plan_destroy(b->plan);
  b->ws.release_all();
  delete b;
  return SPGEMM_OK;
}
