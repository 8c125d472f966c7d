// spgemm_multiply_host: one product through host buffers (the end-to-end entry point).
// Copies A and B to the device, runs plan / symbolic / numeric, and copies C back.
#include <cstring>

#include "runtime.h"

using namespace spg;

namespace {

size_t rp_bytes(int64_t rows, int idx64) { return static_cast<size_t>(rows + 1) * (idx64 ? 8 : 4); }
size_t val_bytes(spgemm_prec p) { return p == SPGEMM_F64 ? 8 : 4; }

struct HostStage {
  Workspace ws;
  ~HostStage() { ws.release_all(); }
};

spgemm_status stage_in(HostStage& hs, const spgemm_csr_in* H, spgemm_prec prec, cudaStream_t s,
                       spgemm_csr_in* D) {
  *D = *H;
  const size_t rb = rp_bytes(H->rows, H->idx64_rowptr);
  void* rp = hs.ws.get(rb);
  void* col = hs.ws.get(static_cast<size_t>(H->nnz) * 4);
  void* val = hs.ws.get(static_cast<size_t>(H->nnz) * val_bytes(prec));
  if (!rp || !col || !val) return set_error_msg(SPGEMM_ERR_OOM, "device staging allocation failed");
  cudaError_t e = cudaMemcpyAsync(rp, H->row_ptr, rb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && H->nnz > 0)
    e = cudaMemcpyAsync(col, H->col, static_cast<size_t>(H->nnz) * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && H->nnz > 0)
    e = cudaMemcpyAsync(val, H->val, static_cast<size_t>(H->nnz) * val_bytes(prec), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e, "copying an input to the device");
  D->row_ptr = rp;
  D->col = static_cast<const int32_t*>(col);
  D->val = val;
  return SPGEMM_OK;
}

}  // namespace

extern "C" spgemm_status spgemm_multiply_host(const spgemm_csr_in* A_host, const spgemm_csr_in* B_host,
                                              spgemm_prec prec, const spgemm_opts* opts,
                                              const spgemm_allocator* alloc, void* stream,
                                              spgemm_csr_out* C_host, int64_t nnz_capacity,
                                              int64_t* nnz_c) {
  clear_error_msg();
  if (!C_host || !nnz_c) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C_host or nnz_c is NULL");
  spgemm_status st;
  if ((st = check_csr_in(A_host, "A", prec)) != SPGEMM_OK) return st;
  if ((st = check_csr_in(B_host, "B", prec)) != SPGEMM_OK) return st;
  if (A_host->cols != B_host->rows) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "A.cols != B.rows");
  if (!C_host->row_ptr) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C_host->row_ptr is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostStage hs;
  hs.ws.stream = stream;
  if (alloc) { hs.ws.alloc = *alloc; hs.ws.has_alloc = true; }
  spgemm_csr_in dA, dB;
  if ((st = stage_in(hs, A_host, prec, s, &dA)) != SPGEMM_OK) return st;
  if ((st = stage_in(hs, B_host, prec, s, &dB)) != SPGEMM_OK) return st;
  spgemm_plan_t* plan = nullptr;
  if ((st = spgemm_plan(&dA, &dB, prec, opts, alloc, stream, &plan)) != SPGEMM_OK) return st;
  int64_t nnz = 0;
  if ((st = spgemm_symbolic(plan, stream, &nnz, nullptr)) != SPGEMM_OK) { spgemm_plan_destroy(plan); return st; }
  *nnz_c = nnz;
  if (nnz > nnz_capacity) {
    spgemm_plan_destroy(plan);
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "nnz(C) = %lld exceeds the host capacity %lld",
                         (long long)nnz, (long long)nnz_capacity);
  }
  if (nnz > 0 && (!C_host->col || !C_host->val)) {
    spgemm_plan_destroy(plan);
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C_host arrays are NULL");
  }
  spgemm_csr_out dC{};
  dC.rows = A_host->rows;
  dC.cols = B_host->cols;
  dC.nnz = nnz;
  dC.idx64_rowptr = C_host->idx64_rowptr;
  const size_t crb = rp_bytes(dC.rows, dC.idx64_rowptr);
  dC.row_ptr = hs.ws.get(crb);
  dC.col = static_cast<int32_t*>(hs.ws.get(static_cast<size_t>(nnz) * 4));
  dC.val = hs.ws.get(static_cast<size_t>(nnz) * val_bytes(prec));
  if (!dC.row_ptr || !dC.col || !dC.val) {
    spgemm_plan_destroy(plan);
    return set_error_msg(SPGEMM_ERR_OOM, "device allocation of C failed");
  }
  if ((st = spgemm_numeric(plan, &dC, stream)) != SPGEMM_OK) { spgemm_plan_destroy(plan); return st; }
  cudaError_t e = cudaMemcpyAsync(C_host->row_ptr, dC.row_ptr, crb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(C_host->col, dC.col, static_cast<size_t>(nnz) * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(C_host->val, dC.val, static_cast<size_t>(nnz) * val_bytes(prec), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { spgemm_plan_destroy(plan); return cuda_status(e, "copying C to the host"); }
  st = read_device_error(plan, s);
  spgemm_plan_destroy(plan);
  C_host->rows = dC.rows;
  C_host->cols = dC.cols;
  C_host->nnz = nnz;
  return st;
}
