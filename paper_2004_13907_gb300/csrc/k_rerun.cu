// FP64 recomputation of the FP32 rows (windowed, block or warp hash rows) whose compensated sums
// may exceed their bound.
//
// These rows are few and long (R-MAT 2^20: 21 rows, the heaviest of the matrix), so instead of
// one block per row the whole GPU works on a group of them at once: every partial product
// a_ik*b_kj (exact in FP64 for FP32 inputs) is added with a global FP64 atomic into a dense FP64
// row of the group's scratch, indexed by the column within the row's job; then each entry of the
// row, whose column the first pass already wrote, takes its sum rounded once to FP32.
#include "kernels.h"

namespace spg {

namespace {

constexpr int kRerunThreads = 256;
constexpr int kRerunGroupMax = 1024;   // rows per group (the per-row A-entry prefix lives in shared memory)

// Warp per A entry of the group's rows (flattened over rows: the entry's row is found in the
// group's prefix of nnz(A_i)); lanes stride the entry's B row.
__global__ void __launch_bounds__(kRerunThreads) k_rerun_accumulate(DevCsr A, DevCsr B, const int32_t* __restrict__ rows,
                                                                     int nrows, const int32_t* __restrict__ abase,
                                                                     int64_t width, double* __restrict__ dense) {
  __shared__ int64_t s_pre[kRerunGroupMax + 1];
  __shared__ int64_t s_a0[kRerunGroupMax];
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int q = 0; q < nrows; ++q) {
      const int32_t i = rows[q];
      s_pre[q] = run;
      s_a0[q] = A.rp[i];
      run += A.rp[i + 1] - A.rp[i];
    }
    s_pre[nrows] = run;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t total = s_pre[nrows];
  const int64_t nwarps = (int64_t(gridDim.x) * kRerunThreads) >> 5;
  const float* av = static_cast<const float*>(A.val);
  const float* bv = static_cast<const float*>(B.val);
  for (int64_t e = (blockIdx.x * int64_t(kRerunThreads) + threadIdx.x) >> 5; e < total; e += nwarps) {
    int lo = 0, hi = nrows - 1;   // the row q with s_pre[q] <= e < s_pre[q + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pre[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const int64_t a = s_a0[lo] + (e - s_pre[lo]);
    const int32_t k = A.col[a];
    const double aik = static_cast<double>(av[a]);
    const int64_t cb = abase ? abase[rows[lo]] : 0;
    double* drow = dense + int64_t(lo) * width;
    for (int64_t j = B.rp[k] + lane; j < B.rp[k + 1]; j += 32)
      atomicAdd(&drow[B.col[j] - cb], aik * static_cast<double>(bv[j]));
  }
}

// Block per row of the group: every entry of the row takes its FP64 sum, rounded once to FP32.
__global__ void __launch_bounds__(kRerunThreads) k_rerun_gather(const int32_t* __restrict__ rows, int nrows,
                                                                 const int64_t* __restrict__ c_off,
                                                                 const int32_t* __restrict__ ccol, int64_t width,
                                                                 const double* __restrict__ dense,
                                                                 float* __restrict__ cval, uint32_t* err) {
  for (int q = blockIdx.x; q < nrows; q += gridDim.x) {
    const int32_t i = rows[q];
    const double* drow = dense + int64_t(q) * width;
    for (int64_t e = c_off[i] + threadIdx.x; e < c_off[i + 1]; e += kRerunThreads) {
      const int32_t c = ccol[e];
      if (c < 0 || c >= width) {
        set_error(err, kErrWindowPlan);
        continue;
      }
      cval[e] = static_cast<float>(drow[c]);
    }
  }
}

}  // namespace

int64_t rerun_group_rows(int64_t width, int64_t budget_bytes) {
  const int64_t row_bytes = (width > 0 ? width : 1) * 8;
  int64_t g = budget_bytes / row_bytes;
  if (g < 1) g = 1;
  if (g > kRerunGroupMax) g = kRerunGroupMax;
  return g;
}

int launch_rerun_dense(const DevCsr& A, const DevCsr& B, const int32_t* rows, int64_t nrows, const int64_t* c_off,
                       int32_t* ccol, float* cval, const int32_t* abase, int64_t width, double* dense,
                       int64_t group_rows, int num_sms, uint32_t* err, cudaStream_t s) {
  int nl = 0;
  for (int64_t g0 = 0; g0 < nrows; g0 += group_rows) {
    const int n = static_cast<int>(nrows - g0 < group_rows ? nrows - g0 : group_rows);
    cudaMemsetAsync(dense, 0, sizeof(double) * width * n, s);
    k_rerun_accumulate<<<num_sms * 8, kRerunThreads, 0, s>>>(A, B, rows + g0, n, abase, width, dense);
    k_rerun_gather<<<n, kRerunThreads, 0, s>>>(rows + g0, n, c_off, ccol, width, dense, cval, err);
    nl += 2;
  }
  return nl;
}

}  // namespace spg
