// spgemm_multiply_noalloc: C = A*B for small products without any device allocation.
//
// Some callers cannot allocate device memory while they call into this library: services
// that reserve the whole device up front and hand out fixed buffers (an allocation would
// fail or steal memory another tenant was promised), and real-time loops that must never
// block in an allocator or risk its failure. This entry point serves them. The caller passes A, B and C's arrays (with a capacity); the scratch the
// kernels need (row counts of C, row offsets, an error word and the total) lives in one
// file-scope device array of fixed size, kScratchBytes, which every GPU that loads the library
// keeps until the process exits.
//
// Limits: A has at most kMaxRows rows, and every row of C has at most kMaxRowEntries entries
// (a larger row is reported as SPGEMM_ERR_UNSUPPORTED); FP64 only.
//
// The kernels are variants of the block-wide hash-table symbolic and numeric kernels of this
// library that process rows in index order and keep their per-row state in that array.
#include <cstring>
#include <mutex>
#include <vector>

#include "enumerate.cuh"
#include "runtime.h"

namespace spg {

namespace {

constexpr int64_t kMaxRows = 1 << 16;
constexpr int kMaxRowEntries = 4096;
constexpr int kLog2Slots = 13;                 // hash table of 8192 slots per block
constexpr int kSlots = 1 << kLog2Slots;
constexpr int kThreads = 512;

// scratch layout: [err uint32 | pad | total int64] [nnz_row int32 x kMaxRows] [c_off int64 x kMaxRows+1]
constexpr size_t kHeaderBytes = 256;
constexpr size_t kNnzOff = kHeaderBytes;
constexpr size_t kOffOff = kNnzOff + sizeof(int32_t) * kMaxRows;
constexpr size_t kScratchBytes = kOffOff + sizeof(int64_t) * (kMaxRows + 1);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Scratch {
  uint32_t* err;
  int64_t* total;
  int32_t* nnz_row;
  int64_t* c_off;
};

struct RowPtr {
  const void* p;
  int idx64;
  __device__ __forceinline__ int64_t operator[](int64_t i) const {
    return idx64 ? static_cast<const int64_t*>(p)[i] : static_cast<const int32_t*>(p)[i];
  }
};

struct InCsr {
  int64_t rows, cols;
  RowPtr rp;
  const int32_t* col;
  const double* val;
};

enum : uint32_t { kNaInvalid = 1u, kNaTooLarge = 2u, kNaHashFull = 4u, kNaCount = 8u };

// Products of row i: f(j, e) for every stored (e-th) entry (k, a) of row i of A and every
// stored entry j of row k of B. Block-flattened, as in the library's block kernels.
template <typename F>
__device__ __forceinline__ void na_for_each_product(const InCsr& A, const InCsr& B, int64_t a0, int64_t na,
                                                    int32_t* s_excl, int64_t* s_bs, int32_t* s_scan,
                                                    uint32_t* err, F&& f) {
  for (int64_t base = 0; base < na; base += kThreads) {
    const int64_t e = base + threadIdx.x;
    int32_t len = 0;
    int64_t bs = 0;
    if (e < na) {
      const int32_t k = A.col[a0 + e];
      if (k < 0 || k >= B.rows) {
        atomicOr(err, kNaInvalid);
      } else {
        bs = B.rp[k];
        const int64_t l = B.rp[k + 1] - bs;
        if (l > kMaxRowEntries) atomicOr(err, kNaTooLarge);   // its row of C would be too long
        else len = static_cast<int32_t>(l);
      }
    }
    int32_t total;
    const int32_t ex = block_excl_scan<int32_t>(len, s_scan, &total);
    s_excl[threadIdx.x] = ex;
    s_bs[threadIdx.x] = bs;
    const int nvalid = static_cast<int>(na - base < kThreads ? na - base : kThreads);
    __syncthreads();
    int owner = 0;
    for (int32_t p = threadIdx.x; p < total; p += kThreads) {
      owner = find_owner(s_excl, nvalid, p, owner);
      const int64_t j = s_bs[owner] + (p - s_excl[owner]);
      const int32_t c = B.col[j];
      if (c < 0 || c >= B.cols) atomicOr(err, kNaInvalid);   // B is not canonical: no product for it
      else f(j, base + owner);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int na_insert(int32_t* keys, int32_t key, uint32_t* err) {
  uint32_t h = hash_slot(key, kLog2Slots);
  for (int probe = 0; probe < kSlots; ++probe) {
    const int32_t cur = *reinterpret_cast<volatile int32_t*>(&keys[h]);
    if (cur == key) return -1 - static_cast<int>(h);
    if (cur == kEmpty) {
      const int32_t old = atomicCAS(&keys[h], kEmpty, key);
      if (old == kEmpty) return static_cast<int>(h);
      if (old == key) return -1 - static_cast<int>(h);
    }
    h = (h + 1) & (kSlots - 1);
  }
  atomicOr(err, kNaHashFull);
  return -1 - kSlots;
}

// nnz(C_i) for every row, one block per row (grid-stride).
__global__ void __launch_bounds__(kThreads) k_na_symbolic(InCsr A, InCsr B, Scratch sc) {
  extern __shared__ int32_t na_keys[];
  __shared__ int32_t s_excl[kThreads];
  __shared__ int64_t s_bs[kThreads];
  __shared__ int32_t s_scan[33];
  __shared__ int32_t s_cnt;
  for (int64_t i = blockIdx.x; i < A.rows; i += gridDim.x) {
    for (int s = threadIdx.x; s < kSlots; s += kThreads) na_keys[s] = kEmpty;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    int cnt = 0;
    na_for_each_product(A, B, a0, na, s_excl, s_bs, s_scan, sc.err, [&](int64_t j, int64_t) {
      if (na_insert(na_keys, B.col[j], sc.err) >= 0) ++cnt;
    });
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
      sc.nnz_row[i] = s_cnt;
      if (s_cnt > kMaxRowEntries) atomicOr(sc.err, kNaTooLarge);
    }
    __syncthreads();
  }
}

// Row offsets of C (one block): c_off[i] = sum of nnz_row[0..i), total = c_off[m].
__global__ void __launch_bounds__(1024) k_na_scan(int64_t m, Scratch sc) {
  __shared__ int64_t s_scan[33];
  int64_t carry = 0;
  for (int64_t b = 0; b < m; b += 1024) {
    const int64_t i = b + threadIdx.x;
    const int64_t v = i < m ? sc.nnz_row[i] : 0;
    int64_t tot;
    const int64_t ex = block_excl_scan<int64_t>(v, s_scan, &tot);
    if (i < m) sc.c_off[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    sc.c_off[m] = carry;
    *sc.total = carry;
  }
}

__global__ void k_na_rowptr(int64_t m1, Scratch sc, void* out, int idx64) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m1; i += int64_t(gridDim.x) * blockDim.x) {
    if (idx64) static_cast<int64_t*>(out)[i] = sc.c_off[i];
    else static_cast<int32_t*>(out)[i] = static_cast<int32_t>(sc.c_off[i]);
  }
}

// Values and sorted columns of every row, one block per row (grid-stride): hash
// accumulation, compaction of the occupied slots, bitonic sort by column, write-out.
__global__ void __launch_bounds__(kThreads) k_na_numeric(InCsr A, InCsr B, Scratch sc, int32_t* ccol,
                                                         double* cval) {
  extern __shared__ double na_smem[];
  double* vals = na_smem;
  int32_t* keys = reinterpret_cast<int32_t*>(na_smem + kSlots);
  __shared__ int32_t s_excl[kThreads];
  __shared__ int64_t s_bs[kThreads];
  __shared__ int32_t s_scan[33];
  for (int64_t i = blockIdx.x; i < A.rows; i += gridDim.x) {
    for (int s = threadIdx.x; s < kSlots; s += kThreads) { keys[s] = kEmpty; vals[s] = 0.0; }
    __syncthreads();
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    na_for_each_product(A, B, a0, na, s_excl, s_bs, s_scan, sc.err, [&](int64_t j, int64_t e) {
      int h = na_insert(keys, B.col[j], sc.err);
      if (h < 0) h = -1 - h;
      if (h < kSlots) atomicAdd(&vals[h], A.val[a0 + e] * B.val[j]);
    });
    int cnt = 0;
    for (int base = 0; base < kSlots; base += kThreads) {
      const int32_t k = keys[base + threadIdx.x];
      const double v = vals[base + threadIdx.x];
      const int occ = k != kEmpty;
      int32_t tot;
      const int32_t pos = cnt + block_excl_scan<int32_t>(occ, s_scan, &tot);
      if (occ) { keys[pos] = k; vals[pos] = v; }
      cnt += tot;
      __syncthreads();
    }
    const int64_t off = sc.c_off[i];
    const int64_t len = sc.c_off[i + 1] - off;
    if (threadIdx.x == 0 && len != cnt) atomicOr(sc.err, kNaCount);
    int N = 1;
    while (N < cnt) N <<= 1;
    for (int t = cnt + threadIdx.x; t < N; t += kThreads) keys[t] = kNoCol;
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < (N >> 1); t += kThreads) {
          const int a = ((t / j) * 2 * j) + (t % j);
          const int b = a + j;
          const bool up = (a & k) == 0;
          const int32_t ka = keys[a], kb = keys[b];
          if ((ka > kb) == up) {
            keys[a] = kb; keys[b] = ka;
            const double va = vals[a]; vals[a] = vals[b]; vals[b] = va;
          }
        }
        __syncthreads();
      }
    }
    const int nout = cnt < len ? cnt : static_cast<int>(len);
    for (int t = threadIdx.x; t < nout; t += kThreads) {
      ccol[off + t] = keys[t];
      cval[off + t] = vals[t];
    }
    __syncthreads();
  }
}

// Device address of the scratch array, looked up once per device (with that device current).
spgemm_status scratch_for_current_device(Scratch* out) {
  static std::mutex mu;
  static std::vector<void*> addr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  std::lock_guard<std::mutex> g(mu);
  if (static_cast<int>(addr.size()) <= dev) addr.resize(dev + 1, nullptr);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress of the scratch array");
    addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(addr[dev]);
  out->err = reinterpret_cast<uint32_t*>(base);
  out->total = reinterpret_cast<int64_t*>(base + 8);
  out->nnz_row = reinterpret_cast<int32_t*>(base + kNnzOff);
  out->c_off = reinterpret_cast<int64_t*>(base + kOffOff);
  return SPGEMM_OK;
}

}  // namespace

}  // namespace spg

using namespace spg;

extern "C" spgemm_status spgemm_multiply_noalloc(const spgemm_csr_in* A, const spgemm_csr_in* B,
                                                 spgemm_csr_out* C, int64_t nnz_capacity, int64_t* nnz_c,
                                                 void* stream) {
  clear_error_msg();
  spgemm_status st;
  if ((st = check_csr_in(A, "A", SPGEMM_F64)) != SPGEMM_OK) return st;
  if ((st = check_csr_in(B, "B", SPGEMM_F64)) != SPGEMM_OK) return st;
  if (A->cols != B->rows) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "A.cols != B.rows");
  if (!C || !nnz_c || !C->row_ptr) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C, C->row_ptr or nnz_c is NULL");
  if (A->rows > kMaxRows)
    return set_error_msg(SPGEMM_ERR_UNSUPPORTED, "A has %lld rows; this entry point takes at most %lld",
                         (long long)A->rows, (long long)kMaxRows);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc;
  if ((st = scratch_for_current_device(&sc)) != SPGEMM_OK) return st;
  const InCsr a{A->rows, A->cols, RowPtr{A->row_ptr, A->idx64_rowptr}, A->col, static_cast<const double*>(A->val)};
  const InCsr b{B->rows, B->cols, RowPtr{B->row_ptr, B->idx64_rowptr}, B->col, static_cast<const double*>(B->val)};
  cudaError_t e = cudaMemsetAsync(sc.err, 0, 16, s);
  if (e != cudaSuccess) return cuda_status(e, "clearing the scratch header");
  const unsigned grid = static_cast<unsigned>(A->rows < 4 * 152 ? (A->rows > 0 ? A->rows : 1) : 4 * 152);
  if (A->rows > 0) {
    k_na_symbolic<<<grid, kThreads, kSlots * 4, s>>>(a, b, sc);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "launching the no-allocation symbolic pass");
  }
  k_na_scan<<<1, 1024, 0, s>>>(A->rows, sc);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "launching the no-allocation row scan");
  uint32_t herr = 0;
  int64_t htotal = 0;
  e = cudaMemcpyAsync(&herr, sc.err, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&htotal, sc.total, sizeof(htotal), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "symbolic pass of the no-allocation product");
  if (herr & kNaInvalid)
    return set_error_msg(SPGEMM_ERR_INVALID_CSR, "a column index of A is outside B's rows, or of B outside B's columns");
  if (herr & (kNaTooLarge | kNaHashFull))
    return set_error_msg(SPGEMM_ERR_UNSUPPORTED, "a row of C has more than %d entries", kMaxRowEntries);
  *nnz_c = htotal;
  if (htotal > nnz_capacity)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "nnz(C) = %lld exceeds the capacity %lld", (long long)htotal,
                         (long long)nnz_capacity);
  if (!C->idx64_rowptr && htotal > 0x7fffffffLL)
    return set_error_msg(SPGEMM_ERR_INDEX_OVERFLOW, "nnz(C) needs an int64 row_ptr");
  if (htotal > 0 && (!C->col || !C->val)) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "C arrays are NULL");
  k_na_rowptr<<<static_cast<unsigned>((A->rows + 256) / 256), 256, 0, s>>>(A->rows + 1, sc, C->row_ptr,
                                                                            C->idx64_rowptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "launching the no-allocation row pointers");
  if (A->rows > 0 && htotal > 0) {
    e = cudaFuncSetAttribute(k_na_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize, kSlots * 12);
    if (e != cudaSuccess) return cuda_status(e, "raising the numeric kernel's shared memory limit");
    k_na_numeric<<<grid, kThreads, kSlots * 12, s>>>(a, b, sc, C->col, static_cast<double*>(C->val));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "launching the no-allocation numeric pass");
  }
  e = cudaMemcpyAsync(&herr, sc.err, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "numeric pass of the no-allocation product");
  if (herr) return set_error_msg(SPGEMM_ERR_INTERNAL, "device consistency check failed (0x%x)", herr);
  C->rows = A->rows;
  C->cols = B->cols;
  C->nnz = htotal;
  return SPGEMM_OK;
}
