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

// The same bound when every partial product is non-negative (A's and B's values are): then
// sum|p| equals the exact sum S, and |res - S| <= (u + gamma_t^2) S gives S <= |res| / (1 - u -
// gamma_t^2), so the test gamma_t^2 S <= u |res| holds whenever gamma_t^2 <= u (1 - 8u) (1 - u -
// gamma_t^2): a condition on the term count alone (t up to about 4,000).
__device__ __forceinline__ bool f32c_within_count(int t) {
  const float u = 5.9604644775390625e-8f;   // 2^-24
  const float tu = static_cast<float>(t) * u;
  if (tu >= 0.5f) return false;
  const float g = tu / (1.0f - tu);
  const float g2 = g * g * (1.0f + 8.0f * u);
  return g2 <= u * (1.0f - 8.0f * u) * (1.0f - u - g2);
}

// Modes of the accumulating kernels: FP64 values summed with FP64 shared atomics; FP32 values
// with compensated FP32 accumulation; FP32 values recomputed in FP64 and rounded once to FP32;
// FP64 values summed exactly in integer fixed point (below).
enum : int { kModeF64 = 0, kModeF32C = 1, kModeF32R = 2, kModeF64X = 3 };

// Exact fixed-point accumulation of FP64 partial products (kModeF64X).
//
// GB300 runs FP64 arithmetic at 2 lanes per clock per SM and a shared-memory FP64 atomic add at
// about one per clock per SM, while a 32-bit shared integer atomic add runs at about 12-15 per
// clock per SM. So an entry of C is accumulated as an integer: every partial product p = a*b
// (rounded once, as any FP64 product) is written as q * 2^lsb with q an integer, and q is split
// into four 32-bit limbs (three unsigned 22-bit chunks and a signed top part) that are added
// with integer atomics. Integer addition is exact and associative, so the sum of an entry does
// not depend on the order of its terms; it is rounded once to FP64 at the end.
//
// lsb is chosen per row from bounds of the operands: |p| < 2^(eA + eB - 2044) for biased
// exponents eA, eB of a and b, and the row's bound E is the largest eA + eB' over its A entries
// (eB' the largest exponent in the named B row). With H = ceil(log2(nnz(A_i) + 1)) (an entry has
// at most nnz(A_i) terms) and Q = kFxTopBits - H, lsb = E - 2044 - Q keeps |q| < 2^(Q+1), and the
// signed top limb below 2^31 for any number of terms up to 2^H. Products whose q would keep fewer
// than 45 significant bits, subnormal products and non-finite ones make the row fall back to the
// FP64 path; every other product is exact (q >= 2^44 * 2^lsb when it is truncated at all), so an
// entry's error is at most 2^-44 * sum|p| plus the final rounding, 2^-53 |c|.
// The lower limbs take at most 2^9 products between normalisations (512 A entries per chunk),
// so they never wrap: 513 * (2^22 - 1) < 2^32.
constexpr int kFxLimbBits = 22;
constexpr uint32_t kFxLimbMask = (1u << kFxLimbBits) - 1u;
constexpr int kFxTopBits = 95;
constexpr int kFxMinShift = -8;   // q keeps 53 + shift significant bits

// Biased exponent field of x.
__device__ __forceinline__ int fx_exponent(double x) {
  return static_cast<int>((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ffu);
}

// Limbs of p / 2^lsb, with sh0 = 1075 + lsb. Returns false when p cannot be taken exactly
// enough (non-finite, subnormal, or fewer than 45 significant bits left); ±0 gives zero limbs.
__device__ __forceinline__ bool fx_split(double p, int sh0, uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                         int32_t& ct) {
  const unsigned long long pb = static_cast<unsigned long long>(__double_as_longlong(p));
  const int e = static_cast<int>((pb >> 52) & 0x7ffu);
  const unsigned long long f = pb & ((1ull << 52) - 1ull);
  c0 = c1 = c2 = 0u;
  ct = 0;
  if (e == 0) return f == 0ull;
  if (e == 0x7ff) return false;
  const int sh = e - sh0;   // q = (f + 2^52) * 2^sh, sh <= kFxTopBits - 52 < 64 by the choice of lsb
  if (sh < kFxMinShift) return false;
  const unsigned long long m = f | (1ull << 52);
  unsigned long long lo, hi;
  if (sh >= 0) {
    lo = m << sh;
    hi = sh > 0 ? (m >> (64 - sh)) : 0ull;
  } else {
    lo = m >> (-sh);
    hi = 0ull;
  }
  if (pb >> 63) {   // two's complement of the 128-bit hi:lo
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    lo = 0ull - lo;
  }
  c0 = static_cast<uint32_t>(lo) & kFxLimbMask;
  c1 = static_cast<uint32_t>(lo >> kFxLimbBits) & kFxLimbMask;
  c2 = static_cast<uint32_t>((lo >> (2 * kFxLimbBits)) | (hi << (64 - 2 * kFxLimbBits))) & kFxLimbMask;
  ct = static_cast<int32_t>(static_cast<long long>(hi) >> (3 * kFxLimbBits - 64));
  return true;
}

// Carries the low limbs of one accumulator into the next, leaving each below 2^22.
__device__ __forceinline__ void fx_normalise(uint32_t& l0, uint32_t& l1, uint32_t& l2, int32_t& lt) {
  l1 += l0 >> kFxLimbBits;
  l0 &= kFxLimbMask;
  l2 += l1 >> kFxLimbBits;
  l1 &= kFxLimbMask;
  lt += static_cast<int32_t>(l2 >> kFxLimbBits);
  l2 &= kFxLimbMask;
}

// The accumulated value (lt * 2^66 + l2 * 2^44 + l1 * 2^22 + l0) * 2^lsb rounded to the nearest
// FP64 (ties to even). Sets *bad when the result overflows or is subnormal (the row then takes
// the FP64 path). An exact zero gives +0. The low limbs may hold up to 32 bits each.
__device__ __forceinline__ double fx_to_double(uint32_t l0, uint32_t l1, uint32_t l2, int32_t lt, int lsb,
                                               bool* bad) {
  // the value as a signed 128-bit hi:lo (hi two's complement)
  const unsigned long long lo1 = static_cast<unsigned long long>(l0) + (static_cast<unsigned long long>(l1) << 22);
  const unsigned long long t2 = static_cast<unsigned long long>(l2) << 44;   // low 64 bits of l2 * 2^44
  unsigned long long lo = lo1 + t2;
  long long hi = static_cast<long long>(lt) * 4 + static_cast<long long>(l2 >> 20) + (lo < lo1 ? 1 : 0);
  if (hi == 0 && lo == 0ull) return 0.0;
  const bool neg = hi < 0;
  unsigned long long uh = static_cast<unsigned long long>(hi);
  if (neg) {
    uh = ~uh + (lo == 0ull ? 1ull : 0ull);
    lo = 0ull - lo;
  }
  // normalise so that the leading one is bit 127 of uh:lo
  const int lz = uh ? __clzll(static_cast<long long>(uh)) : 64 + __clzll(static_cast<long long>(lo));
  if (lz >= 64) {
    uh = lo << (lz - 64);
    lo = 0ull;
  } else if (lz > 0) {
    uh = (uh << lz) | (lo >> (64 - lz));
    lo <<= lz;
  }
  int b = 127 - lz;   // position of the leading one in the unnormalised value
  unsigned long long mant = uh >> 11;
  const bool rbit = (uh >> 10) & 1ull;
  const bool sticky = (uh & 0x3ffull) != 0ull || lo != 0ull;
  if (rbit && (sticky || (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++b;
    }
  }
  const int biased = b + lsb + 1023;
  if (biased <= 0 || biased >= 2047) {
    *bad = true;
    return 0.0;
  }
  const unsigned long long bits = (static_cast<unsigned long long>(neg) << 63) |
                                  (static_cast<unsigned long long>(biased) << 52) | (mant & ((1ull << 52) - 1ull));
  return __longlong_as_double(static_cast<long long>(bits));
}

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
