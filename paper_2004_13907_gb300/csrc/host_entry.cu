// spgemm_multiply_host: one product through host buffers (the end-to-end entry point).
// Copies A and B to the device, runs plan / symbolic / numeric, and copies C back.
#include <cstdint>
#include <cstring>
#include <vector>

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

// Row panels of A for the pipelined host path, with equal shares of the partial products:
// host_panels N > 0 of them, or by default kDefaultPanels when the estimated partial products (A's
// entries times B's mean row length) reach kPanelMinProducts (else one). Copying C to the host
// takes longer than computing it (C2C at about 190 GB/s against HBM), so after the first panel
// the copy stream never waits: the call lasts the first panel's product plus the copy of C. More panels shorten the
// first but pay a plan, a symbolic pass and buffer growth each, and the first panel cannot end
// before the longest row of A does (R-MAT's heaviest rows all fall into it).
constexpr int kDefaultPanels = 4;
constexpr double kPanelMinProducts = 1e8;
constexpr int kMaxPanels = 64;

int64_t host_rp(const spgemm_csr_in* M, int64_t r) {
  return M->idx64_rowptr ? static_cast<const int64_t*>(M->row_ptr)[r] : static_cast<const int32_t*>(M->row_ptr)[r];
}

// Interior panel boundaries as fractions of the work, increasing in (0, 1); empty for one panel.
std::vector<double> panel_bounds(const spgemm_csr_in* A, const spgemm_csr_in* B, int requested) {
  int np = 1;
  if (requested > 0) {
    np = requested < kMaxPanels ? requested : kMaxPanels;
  } else {
    const double est = B->rows > 0 ? static_cast<double>(A->nnz) * static_cast<double>(B->nnz) / B->rows : 0.0;
    if (est >= kPanelMinProducts) np = kDefaultPanels;
  }
  std::vector<double> bounds;
  if (A->rows < 2 * static_cast<int64_t>(np)) return bounds;
  for (int q = 1; q < np; ++q) bounds.push_back(static_cast<double>(q) / np);
  return bounds;
}

// Panel q holds rows [cut[q], cut[q + 1]): boundary b falls on the first row r at which
// prefix(r), the work of the rows before r (non-decreasing, prefix(m) = the total), reaches
// b times the total. Empty panels are dropped.
template <typename Prefix>
std::vector<int64_t> cut_rows(const std::vector<double>& bounds, int64_t m, Prefix prefix) {
  std::vector<int64_t> cut{0};
  const double total = static_cast<double>(prefix(m));
  for (double b : bounds) {
    const int64_t target = static_cast<int64_t>(b * total);
    int64_t lo = cut.back(), hi = m;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (prefix(mid) < target) lo = mid + 1;
      else hi = mid;
    }
    if (lo > cut.back() && lo < m) cut.push_back(lo);
  }
  cut.push_back(m);
  return cut;
}

void* pool_alloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  cudaMemPool_t pool = library_pool();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, pool, s)
                             : cudaMallocAsync(&p, bytes ? bytes : 16, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

// The pipelined host path: A's row panels are multiplied one after another on `s` while the
// previous panels' rows of C travel to the host on a copy stream. Two device buffers of C take
// turns (panel q writes buffer q % 2 once the copy of panel q - 2 out of it has finished), so the
// product waits for a copy only when it runs ahead by two panels; nothing allocated on one stream
// is freed on the other. The row pointers come back panel-relative and are shifted on the host.
struct PanelBuf {
  void* rp = nullptr;
  int32_t* col = nullptr;
  void* val = nullptr;
  int64_t rows = 0, cap = 0;
};

spgemm_status multiply_panels(const std::vector<int64_t>& cut, const spgemm_csr_in* A_host, const spgemm_csr_in& dA,
                              const spgemm_csr_in& dB, spgemm_prec prec, const spgemm_opts* opts,
                              const spgemm_allocator* alloc, cudaStream_t s, HostStage& hs, spgemm_csr_out* C_host,
                              int64_t nnz_capacity, int64_t* nnz_c) {
  const size_t vb = val_bytes(prec);
  const int idx64 = C_host->idx64_rowptr;
  const size_t eb = idx64 ? 8 : 4;
  const int np = static_cast<int>(cut.size()) - 1;
  int64_t* prp = static_cast<int64_t*>(hs.ws.get(sizeof(int64_t) * static_cast<size_t>(A_host->rows + 1)));
  if (!prp) return set_error_msg(SPGEMM_ERR_OOM, "device staging allocation failed");
  cudaStream_t cs = nullptr;
  cudaEvent_t computed = nullptr, copied[2] = {nullptr, nullptr};
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&computed, cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
  PanelBuf buf[2];
  auto release = [&]() {
    cudaStreamSynchronize(cs);
    for (PanelBuf& pb : buf)
      for (void* ptr : {pb.rp, static_cast<void*>(pb.col), pb.val})
        if (ptr) cudaFreeAsync(ptr, s);
    cudaStreamSynchronize(s);
    for (cudaEvent_t ev : {computed, copied[0], copied[1]})
      if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_status(e, "creating the copy stream");
  }
  std::vector<int64_t> nnz0(static_cast<size_t>(np) + 1, 0);
  spgemm_status st = SPGEMM_OK;
  bool fits = true;
  for (int q = 0; q < np && st == SPGEMM_OK; ++q) {
    const int64_t r0 = cut[q], r1 = cut[q + 1], rows = r1 - r0;
    const int64_t base = host_rp(A_host, r0);
    // panel q of A: rebased row pointers, columns and values from its first entry
    launch_rowptr_rebase(dA.row_ptr, dA.idx64_rowptr, r0, rows + 1, base, prp + r0, s);
    spgemm_csr_in ap{rows, dA.cols, host_rp(A_host, r1) - base, 1, 0, prp + r0,
                     static_cast<const int32_t*>(dA.col) + base,
                     static_cast<const unsigned char*>(dA.val) + static_cast<size_t>(base) * vb};
    spgemm_plan_t* plan = nullptr;
    if ((st = spgemm_plan(&ap, &dB, prec, opts, alloc, s, &plan)) != SPGEMM_OK) break;
    int64_t nnz = 0;
    st = spgemm_symbolic(plan, s, &nnz, nullptr);
    nnz0[q + 1] = nnz0[q] + nnz;
    if (st == SPGEMM_OK && (nnz0[q + 1] > nnz_capacity || (!idx64 && nnz0[q + 1] > INT32_MAX))) fits = false;
    if (st == SPGEMM_OK && fits) {
      PanelBuf& pb = buf[q & 1];
      // the copy of panel q - 2 out of this buffer must be done before the buffer is written
      if (q >= 2) cudaStreamWaitEvent(s, copied[q & 1], 0);
      if (pb.rows < rows + 1 || pb.cap < nnz) {
        for (void* ptr : {pb.rp, static_cast<void*>(pb.col), pb.val})
          if (ptr) cudaFreeAsync(ptr, s);
        pb.rows = rows + 1 > pb.rows ? rows + 1 : pb.rows;
        pb.cap = nnz > pb.cap ? nnz + nnz / 8 : pb.cap;
        pb.rp = pool_alloc(eb * static_cast<size_t>(pb.rows), s);
        pb.col = static_cast<int32_t*>(pool_alloc(4 * static_cast<size_t>(pb.cap), s));
        pb.val = pool_alloc(vb * static_cast<size_t>(pb.cap), s);
        if (!pb.rp || !pb.col || !pb.val) st = set_error_msg(SPGEMM_ERR_OOM, "device allocation of a panel of C failed");
      }
      if (st == SPGEMM_OK) {
        spgemm_csr_out pc{};
        pc.rows = rows;
        pc.cols = dB.cols;
        pc.nnz = nnz;
        pc.idx64_rowptr = idx64;
        pc.row_ptr = pb.rp;
        pc.col = pb.col;
        pc.val = pb.val;
        if ((st = spgemm_numeric(plan, &pc, s)) == SPGEMM_OK) st = spgemm_plan_check(plan, s);
      }
      if (st == SPGEMM_OK) {
        e = cudaEventRecord(computed, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, computed, 0);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(static_cast<unsigned char*>(C_host->row_ptr) + eb * static_cast<size_t>(r0), pb.rp,
                              eb * static_cast<size_t>(rows), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && nnz > 0)
          e = cudaMemcpyAsync(C_host->col + nnz0[q], pb.col, 4 * static_cast<size_t>(nnz), cudaMemcpyDeviceToHost,
                              cs);
        if (e == cudaSuccess && nnz > 0)
          e = cudaMemcpyAsync(static_cast<unsigned char*>(C_host->val) + vb * static_cast<size_t>(nnz0[q]), pb.val,
                              vb * static_cast<size_t>(nnz), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaEventRecord(copied[q & 1], cs);
        if (e != cudaSuccess) st = cuda_status(e, "copying a panel of C to the host");
      }
    }
    spgemm_plan_destroy(plan);
  }
  e = cudaStreamSynchronize(cs);
  release();
  if (st != SPGEMM_OK) return st;
  if (e != cudaSuccess) return cuda_status(e, "copying C to the host");
  *nnz_c = nnz0[np];
  if (!fits) {
    if (!idx64 && nnz0[np] > INT32_MAX)
      return set_error_msg(SPGEMM_ERR_INDEX_OVERFLOW, "nnz(C) = %lld needs an int64 row_ptr", (long long)nnz0[np]);
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "nnz(C) = %lld exceeds the host capacity %lld",
                         (long long)nnz0[np], (long long)nnz_capacity);
  }
  // panel-relative row pointers to C's
  for (int q = 1; q < np; ++q) {
    const int64_t add = nnz0[q];
    if (idx64) {
      int64_t* rp = static_cast<int64_t*>(C_host->row_ptr);
      for (int64_t r = cut[q]; r < cut[q + 1]; ++r) rp[r] += add;
    } else {
      int32_t* rp = static_cast<int32_t*>(C_host->row_ptr);
      for (int64_t r = cut[q]; r < cut[q + 1]; ++r) rp[r] += static_cast<int32_t>(add);
    }
  }
  if (idx64) static_cast<int64_t*>(C_host->row_ptr)[A_host->rows] = nnz0[np];
  else static_cast<int32_t*>(C_host->row_ptr)[A_host->rows] = static_cast<int32_t>(nnz0[np]);
  C_host->rows = A_host->rows;
  C_host->cols = dB.cols;
  C_host->nnz = nnz0[np];
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
  const std::vector<double> bounds = panel_bounds(A_host, B_host, opts ? opts->host_panels : 0);
  std::vector<int64_t> cut = cut_rows(bounds, A_host->rows, [&](int64_t r) { return host_rp(A_host, r); });
  if (cut.size() > 2) {
    // shares of the partial products (the plan of the whole product counts P_i per row on the
    // device), which the time to compute and to copy a panel follows, rather than of A's entries
    spgemm_plan_t* whole = nullptr;
    if ((st = spgemm_plan(&dA, &dB, prec, opts, alloc, stream, &whole)) != SPGEMM_OK) return st;
    if (!whole->small && whole->P) {
      const int64_t m = A_host->rows;
      std::vector<int64_t> pre(static_cast<size_t>(m) + 1, 0);
      cudaError_t e = cudaMemcpyAsync(pre.data() + 1, whole->P, sizeof(int64_t) * static_cast<size_t>(m),
                                      cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        spgemm_plan_destroy(whole);
        return cuda_status(e, "reading the partial products per row");
      }
      for (int64_t r = 0; r < m; ++r) pre[r + 1] += pre[r];
      cut = cut_rows(bounds, m, [&](int64_t r) { return pre[static_cast<size_t>(r)]; });
    }
    spgemm_plan_destroy(whole);
  }
  if (cut.size() > 2) {
    if (nnz_capacity > 0 && (!C_host->col || !C_host->val))
      return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C_host arrays are NULL");
    return multiply_panels(cut, A_host, dA, dB, prec, opts, alloc, s, hs, C_host, nnz_capacity, nnz_c);
  }
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
