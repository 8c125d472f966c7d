// Shared device-side definitions of the SpGEMM library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spg {

constexpr int kWarp = 32;
constexpr int32_t kEmpty = -1;           // empty hash slot (columns are >= 0)
constexpr int32_t kNoCol = 0x7fffffff;   // "no next column" sentinel

// Device error word bits (OR-ed; read back by the host after each pass).
enum : uint32_t {
  kErrInvalidCsr = 1u,
  kErrHashFull = 2u,       // a hash table ran out of slots (cannot happen with exact sizing)
  kErrWindowPlan = 4u,     // a window held more entries than its table
  kErrCount = 16u,         // a row wrote a different number of entries than counted
};

constexpr int kMicroNa = 8;   // micro rows: at most this many A entries (B rows merged per thread)

// Row classes. A row's class fixes the kernel that handles it. The class order is the
// order of the rows in the permutation, so the windowed classes come first, largest
// work first, which lets persistent blocks take the heaviest rows earliest.
enum SymClass : int {
  kSymWin0 = 0,   // windowed, P_i >= 2^22
  kSymWin1,       // windowed, P_i >= 2^20
  kSymWin2,       // windowed, P_i >= 2^17
  kSymWin3,       // windowed, the rest
  kSymBlock,      // block-wide hash table (min(P_i, n) <= block_max)
  kSymWarp3,      // warp table of 2048 keys (min(P_i,n) <= 1024)
  kSymWarp2,      // warp table of 512 keys  (<= 256)
  kSymWarp1,      // warp table of 128 keys  (<= 64)
  kSymTiny,       // P_i <= tiny_max and nnz(A_i) <= 32: registers only, one warp per row
  kSymMicro,      // tiny with nnz(A_i) <= kMicroNa: one thread per row merges the B rows
  kSymZero,       // P_i == 0
  kSymNumClasses
};

enum NumClass : int {
  kNumWin0 = 0,
  kNumWin1,
  kNumWin2,
  kNumWin3,
  kNumBlock2,     // block hash of 8192 slots (nnz <= 4096)
  kNumBlock1,     // block hash of 2048 slots (nnz <= 1024)
  kNumWarp3,      // warp hash of 1024 slots (nnz <= 512)
  kNumWarp2,      // warp hash of 256 slots  (nnz <= 128)
  kNumWarp1,      // warp hash of 64 slots   (nnz <= 32)
  kNumTiny,
  kNumMicro,      // tiny with nnz(A_i) <= kMicroNa, FP64: one thread per row merges the B rows
  kNumZero,
  kNumNumClasses
};

// Thresholds the class functions use (copied from spgemm_opts by the host).
struct ClassParams {
  int64_t n;              // columns of B (and C)
  int32_t tiny_max;
  int32_t warp_max;       // symbolic warp tables take min(P,n) <= warp_max
  int32_t block_max;      // block tables take <= block_max; larger rows are windowed
  int32_t force_window;
  int32_t window_all;     // every row that is not tiny takes the windowed path (FP32-compensated)
  const int32_t* rwidth;  // per-row column count of C (device, NULL: every row has n columns)
};

// The column count of row `row` of C: its own width in a stacked batch, else n.
__device__ inline ClassParams row_params(const ClassParams& cp, int64_t row) {
  ClassParams c = cp;
  if (cp.rwidth) c.n = cp.rwidth[row];
  return c;
}

__host__ __device__ inline int win_subclass(int64_t P) {
  return P >= (int64_t(1) << 22) ? 0 : P >= (int64_t(1) << 20) ? 1 : P >= (int64_t(1) << 17) ? 2 : 3;
}

__host__ __device__ inline int sym_class(int64_t P, int32_t na, const ClassParams& cp) {
  if (P == 0) return kSymZero;
  const int64_t U = P < cp.n ? P : cp.n;
  if (cp.force_window) return kSymWin0 + win_subclass(P);
  if (P <= cp.tiny_max && na <= kWarp) return na <= kMicroNa ? kSymMicro : kSymTiny;
  if (cp.window_all) return kSymWin0 + win_subclass(P);
  if (U <= 64 && cp.warp_max >= 64) return kSymWarp1;
  if (U <= 256 && cp.warp_max >= 256) return kSymWarp2;
  if (U <= cp.warp_max) return kSymWarp3;
  if (U <= cp.block_max) return kSymBlock;
  return kSymWin0 + win_subclass(P);
}

__host__ __device__ inline int num_class(int64_t P, int32_t na, int32_t nnz,
                                         const ClassParams& cp) {
  if (nnz == 0) return kNumZero;
  if (cp.force_window) return kNumWin0 + win_subclass(P);
  if (P <= cp.tiny_max && na <= kWarp) return (na <= kMicroNa && !cp.window_all) ? kNumMicro : kNumTiny;
  if (cp.window_all) return kNumWin0 + win_subclass(P);
  if (nnz <= 32 && cp.warp_max >= 64) return kNumWarp1;
  if (nnz <= 128 && cp.warp_max >= 256) return kNumWarp2;
  if (nnz <= 512 && cp.warp_max >= 1024) return kNumWarp3;
  if (nnz <= 1024 && cp.block_max >= 1024) return kNumBlock1;
  if (nnz <= cp.block_max) return kNumBlock2;
  return kNumWin0 + win_subclass(P);
}

// Windowed path geometry. The symbolic pass records, for every windowed row, how many
// entries of C fall in each block of kBlockCols columns; the numeric pass groups blocks
// into windows from those counts.
constexpr int kBlockShift = 12;
constexpr int kBlockCols = 1 << kBlockShift;   // columns per block, 4096
constexpr int kBlockWords = kBlockCols / 32;   // bitmap words per block
constexpr int kSymWinBits = 1 << 20;           // symbolic bitmap window (128 KB)
constexpr int kSymWinThreads = 1024;           // threads of the windowed symbolic kernel

__device__ __forceinline__ void set_error(uint32_t* err, uint32_t code) { atomicOr(err, code); }

// Error bound of the compensated FP32 accumulation. A result res = s + c of t partial products
// accumulated with an error-free product and a compensated sum (Ogita, Rump and Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 2005, algorithm Dot2) satisfies
//   |res - exact| <= u |exact| + gamma_t^2 * sum|p|,  u = 2^-24,  gamma_t = t u / (1 - t u).
// The entry counts as within the FP32 bound when gamma_t^2 * sum|p| <= u |res| (its error is then
// about 2u|exact|); `mag` is the FP32 running sum of |p|, inflated here for its own rounding.
__device__ __forceinline__ bool f32c_within_bound(float res, float mag, int t) {
  const float u = 5.9604644775390625e-8f;   // 2^-24
  const float tu = static_cast<float>(t) * u;
  if (tu >= 0.5f) return false;
  const float g = tu / (1.0f - tu);
  const float mag_ub = mag * (1.0f + 2.0f * g + 8.0f * u);
  return g * g * mag_ub <= u * fabsf(res) * (1.0f - 8.0f * u);
}

// Modes of the accumulating kernels: FP64 values; FP32 values with compensated FP32
// accumulation; FP32 values recomputed in FP64 and rounded once to FP32.
enum : int { kModeF64 = 0, kModeF32C = 1, kModeF32R = 2 };

// Knuth's multiplicative hash: the top log2S bits of key * floor(2^32 / phi).
__device__ __forceinline__ uint32_t hash_slot(int32_t key, int log2S) {
  return (static_cast<uint32_t>(key) * 2654435769u) >> (32 - log2S);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, d);
    if (static_cast<int>(lane_id()) >= d) v += t;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    T o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o < v ? o : v;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread. `scratch` holds >= 33 T.
// Returns the exclusive prefix; *total receives the block sum. Contains __syncthreads.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* scratch, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T incl = warp_incl_scan(v);
  if (lane == 31) scratch[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? scratch[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < nw) scratch[lane] = wi - w;
    if (lane == nw - 1) scratch[32] = wi;
  }
  __syncthreads();
  T r = scratch[wid] + incl - v;
  *total = scratch[32];
  __syncthreads();
  return r;
}

}  // namespace spg
