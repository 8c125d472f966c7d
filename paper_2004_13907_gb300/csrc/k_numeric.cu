// Numeric pass, FP64: forms every partial product a_ik*b_kj of row i (the match
// and multiply unit of Sec. III-A), merges the products of equal column (the merge unit)
// and writes row i of C sorted by column (the sort unit; Algorithm 1 sorts PP and emits
// one entry per column of COLB, including sums that cancel to zero).
//
// Row classes (chosen from nnz(C_i) after the symbolic pass):
//  * tiny  : P_i <= 32: one warp, one product per lane; equal columns are grouped with a
//            warp match and summed by the lowest lane of the group in product order; the
//            output position is the number of smaller columns in the row.
//  * warp  : one warp per row, a shared hash table (column -> FP64 sum) of 64/256/1024
//            slots, then the occupied slots are compacted and bitonic-sorted by column.
//  * block : one block per row, a hash table of 2048 or 8192 slots, compaction, bitonic sort.
//  * window: rows with more entries than a block table (k_window.cu).
// Sums are accumulated with shared-memory FP64 atomics, so their order (and the last bits of
// a value) can change from run to run; the pattern is always exact.
#include "enumerate.cuh"

namespace spg {

namespace {

template <int Mode>
__global__ void __launch_bounds__(256) k_num_tiny(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                  int64_t count, const int64_t* __restrict__ c_off,
                                                  int32_t* __restrict__ ccol, void* __restrict__ cval_,
                                                  int32_t* __restrict__ row_flag, const int32_t* __restrict__ abase,
                                                  uint32_t* err) {
  __shared__ int32_t s_col[8][32];
  __shared__ double s_val[8][32];   // FP64 product (kModeF64, kModeF32R) or the FP32 high part
  __shared__ float s_lo[8][32];     // kModeF32C: the FP32 low part of the product
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = gw; r < count; r += nw) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int32_t na = static_cast<int32_t>(A.rp[i + 1] - a0);
    int32_t len = 0;
    int64_t bs = 0;
    double av = 0.0;
    if (lane < na) {
      const int32_t k = A.col[a0 + lane];
      av = Mode == kModeF64 ? static_cast<const double*>(A.val)[a0 + lane]
                            : static_cast<double>(static_cast<const float*>(A.val)[a0 + lane]);
      bs = B.rp[k];
      len = static_cast<int32_t>(B.rp[k + 1] - bs);
    }
    const int32_t incl = warp_incl_scan(len);
    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
    int o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int32_t v = __shfl_sync(0xffffffffu, incl, o + step - 1);
      if (v <= lane) o += step;
    }
    const int32_t incl_o = __shfl_sync(0xffffffffu, incl, o & 31);
    const int32_t len_o = __shfl_sync(0xffffffffu, len, o & 31);
    const int64_t bs_o = __shfl_sync(0xffffffffu, bs, o & 31);
    const double av_o = __shfl_sync(0xffffffffu, av, o & 31);
    int32_t col = -2 - lane;
    double val = 0.0;
    float lo = 0.f;
    if (lane < total) {
      const int64_t j = bs_o + (lane - (incl_o - len_o));
      col = B.col[j];
      if constexpr (Mode == kModeF64) {
        val = av_o * static_cast<const double*>(B.val)[j];
      } else if constexpr (Mode == kModeF32R) {
        val = av_o * static_cast<double>(static_cast<const float*>(B.val)[j]);   // exact in FP64
      } else {
        const float a = static_cast<float>(av_o);
        const float b = static_cast<const float*>(B.val)[j];
        const float ph = a * b;
        val = ph;
        lo = fmaf(a, b, -ph);   // a*b = ph + lo exactly
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, col);
    s_col[wid][lane] = col;
    s_val[wid][lane] = val;
    s_lo[wid][lane] = lo;
    __syncwarp();
    const bool lead = lane < total && (__ffs(peers) - 1) == lane;
    const unsigned leaders = __ballot_sync(0xffffffffu, lead);
    bool missed = false;
    if (lead) {
      int rank = 0;
      for (unsigned m = leaders; m; m &= m - 1) rank += s_col[wid][__ffs(m) - 1] < col;
      if (rank < c_off[i + 1] - c_off[i]) {   // a miscount raises kErrCount, never writes out of the row
        const int64_t out = c_off[i] + rank;
        ccol[out] = col - (abase ? abase[i] : 0);
        if constexpr (Mode == kModeF32C) {
          // compensated sum of the group's products in product order (Dot2)
          float sum = 0.f, comp = 0.f, mag = 0.f;
          int t = 0;
          for (unsigned m = peers; m; m &= m - 1) {
            const int q = __ffs(m) - 1;
            const float ph = static_cast<float>(s_val[wid][q]);
            const float nsum = sum + ph;
            const float bp = nsum - sum;
            comp += (sum - (nsum - bp)) + (ph - bp) + s_lo[wid][q];
            sum = nsum;
            mag += fabsf(ph);
            ++t;
          }
          const float res = sum + comp;
          static_cast<float*>(cval_)[out] = res;
          missed = !f32c_within_bound(res, mag, t);
        } else {
          double sum = 0.0;
          for (unsigned m = peers; m; m &= m - 1) sum += s_val[wid][__ffs(m) - 1];
          if constexpr (Mode == kModeF64) static_cast<double*>(cval_)[out] = sum;
          else static_cast<float*>(cval_)[out] = static_cast<float>(sum);
        }
      }
    }
    if constexpr (Mode == kModeF32C) {
      if (__any_sync(0xffffffffu, missed) && lane == 0) row_flag[i] = 1;
    }
    if (lane == 0 && c_off[i + 1] - c_off[i] != __popc(leaders)) set_error(err, kErrCount);
    __syncwarp();
  }
}

// Micro rows (nnz(A_i) <= kMicroNa, P_i <= tiny_max), FP64: one thread per row merges the row's
// sorted B rows head by head. The smallest head column is the next column of C; the products of
// every head holding it are summed in A-entry order and those heads advance. The output comes out
// sorted, with no shared memory and no atomics.
__global__ void __launch_bounds__(256) k_num_micro(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                   int64_t count, const int64_t* __restrict__ c_off,
                                                   int32_t* __restrict__ ccol, double* __restrict__ cval,
                                                   const int32_t* __restrict__ abase, uint32_t* err) {
  constexpr int NA = kMicroNa;
  constexpr int32_t kEnd = 0x7fffffff;
  const double* av64 = static_cast<const double*>(A.val);
  const double* bv64 = static_cast<const double*>(B.val);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < count; r += stride) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int na = static_cast<int>(A.rp[i + 1] - a0);
    int64_t out = c_off[i];
    const int64_t out_end = c_off[i + 1];
    const int32_t cb = abase ? abase[i] : 0;
    int64_t pos[NA];
    int32_t left[NA], hc[NA];
    double av[NA];
#pragma unroll
    for (int h = 0; h < NA; ++h) {
      pos[h] = 0; left[h] = 0; hc[h] = kEnd; av[h] = 0.0;
      if (h < na) {
        const int32_t k = A.col[a0 + h];
        av[h] = av64[a0 + h];
        pos[h] = B.rp[k];
        left[h] = static_cast<int32_t>(B.rp[k + 1] - pos[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < NA; ++h) if (left[h] > 0) hc[h] = B.col[pos[h]];
    for (;;) {
      int32_t m = hc[0];
#pragma unroll
      for (int h = 1; h < NA; ++h) m = hc[h] < m ? hc[h] : m;
      if (m == kEnd) break;
      double sum = 0.0;
#pragma unroll
      for (int h = 0; h < NA; ++h) {
        if (hc[h] == m) {
          sum += av[h] * bv64[pos[h]];
          ++pos[h];
          --left[h];
          hc[h] = left[h] > 0 ? B.col[pos[h]] : kEnd;
        }
      }
      if (out < out_end) {   // a miscount raises kErrCount, never writes out of the row
        ccol[out] = m - cb;
        cval[out] = sum;
      }
      ++out;
    }
    if (out != out_end) set_error(err, kErrCount);
  }
}

// Value q of an FP64 (kModeF64) or FP32 (kModeF32C) array, as a double (exact).
template <int Mode>
__device__ __forceinline__ double value_at(const void* v, int64_t q) {
  if constexpr (Mode == kModeF32C) return static_cast<double>(static_cast<const float*>(v)[q]);
  else return static_cast<const double*>(v)[q];
}

// The slot of `key` (linear probing; keys are columns, kEmpty = free), claimed if new; -1 when
// the table is full.
template <int LOG2S>
__device__ __forceinline__ int hash_claim(int32_t* keys, int32_t key) {
  constexpr int S = 1 << LOG2S;
  uint32_t h = hash_slot(key, LOG2S);
  for (int probe = 0; probe < S; ++probe) {
    const int32_t cur = *reinterpret_cast<volatile int32_t*>(&keys[h]);
    if (cur == key) return static_cast<int>(h);
    if (cur == kEmpty) {
      const int32_t old = atomicCAS(&keys[h], kEmpty, key);
      if (old == kEmpty || old == key) return static_cast<int>(h);
    }
    h = (h + 1) & (S - 1);
  }
  return -1;
}

// Adds the partial product a*b into the slot of `key`. kModeF64: one FP64 atomic. kModeF32C: the
// slot's 8 bytes hold an FP32 sum and its compensation; the error-free product a*b = ph + pl and
// the sum's own rounding error (TwoSum, rebuilt from the value the atomic returns) go to the
// compensation, as in the windowed kernel (Dot2 accumulated concurrently).
template <int LOG2S, int Mode>
__device__ __forceinline__ void hash_accumulate(int32_t* keys, double* vals, int32_t key, double a, double b,
                                                uint32_t* err) {
  const int h = hash_claim<LOG2S>(keys, key);
  if (h < 0) {
    set_error(err, kErrHashFull);
    return;
  }
  if constexpr (Mode == kModeF32C) {
    float* sc = reinterpret_cast<float*>(&vals[h]);
    const float fa = static_cast<float>(a), fb = static_cast<float>(b);
    const float ph = fa * fb;
    const float pl = fmaf(fa, fb, -ph);
    const float old = atomicAdd(&sc[0], ph);
    const float nw = old + ph;
    const float bp = nw - old;
    const float q = (old - (nw - bp)) + (ph - bp);
    atomicAdd(&sc[1], q + pl);
  } else {
    atomicAdd(&vals[h], a * b);
  }
}

// Value of an entry of C from its slot's 8 bytes (an FP64 sum, or an FP32 sum and compensation).
template <int Mode>
__device__ __forceinline__ void store_value(void* cval, int64_t at, double slot) {
  if constexpr (Mode == kModeF32C) {
    const float2 sc = *reinterpret_cast<const float2*>(&slot);
    static_cast<float*>(cval)[at] = sc.x + sc.y;
  } else {
    static_cast<double*>(cval)[at] = slot;
  }
}

// kModeF32C rows of the hash kernels: every partial product must be non-negative (no negative value
// in A or B, *negflag == 0) and the row's A length must pass the term-count bound, so that no
// entry can exceed Dot2's bound; otherwise the row is listed for the FP64 recomputation.
__device__ __forceinline__ bool f32c_hash_row_ok(const int32_t* negflag, int64_t na) {
  return negflag != nullptr && *negflag == 0 &&
         f32c_within_count(na < (int64_t(1) << 30) ? static_cast<int>(na) : (1 << 30));
}

// In-warp bitonic sort of keys/vals[0, N), N a power of two.
__device__ __forceinline__ void warp_bitonic(int32_t* keys, double* vals, int N) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < (N >> 1); t += 32) {
        const int a = ((t / j) * 2 * j) + (t % j);
        const int b = a + j;
        const bool up = (a & k) == 0;
        const int32_t ka = keys[a], kb = keys[b];
        if ((ka > kb) == up) {
          keys[a] = kb; keys[b] = ka;
          const double va = vals[a]; vals[a] = vals[b]; vals[b] = va;
        }
      }
      __syncwarp();
    }
  }
}

template <int NT>
__device__ __forceinline__ void block_bitonic(int32_t* keys, double* vals, int N) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (N >> 1); t += NT) {
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
}

__device__ __forceinline__ int pow2_ceil(int x) {
  return x <= 1 ? 1 : 1 << (32 - __clz(x - 1));
}

template <int LOG2S, int Mode>
__global__ void __launch_bounds__(256) k_num_warp(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                  int64_t count, const int64_t* __restrict__ c_off,
                                                  int32_t* __restrict__ ccol, void* __restrict__ cval,
                                                  const int32_t* __restrict__ abase, int32_t* __restrict__ row_flag,
                                                  const int32_t* __restrict__ negflag, uint32_t* err) {
  constexpr int S = 1 << LOG2S;
  extern __shared__ double smem_f64[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* vals = smem_f64 + wid * S;
  int32_t* keys = reinterpret_cast<int32_t*>(smem_f64 + 8 * S) + wid * S;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = gw; r < count; r += nw) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    if (Mode == kModeF32C && lane == 0 && !f32c_hash_row_ok(negflag, na)) row_flag[i] = 1;
    for (int s = lane; s < S; s += 32) { keys[s] = kEmpty; vals[s] = 0.0; }
    __syncwarp();
    warp_for_each_product(A, B, a0, na, [&](int64_t j, int64_t e) {
      hash_accumulate<LOG2S, Mode>(keys, vals, B.col[j], value_at<Mode>(A.val, a0 + e), value_at<Mode>(B.val, j),
                                   err);
    });
    __syncwarp();
    // compact in place (a write position never passes the slot being read)
    int cnt = 0;
    for (int base = 0; base < S; base += 32) {
      const int32_t k = keys[base + lane];
      const double v = vals[base + lane];
      const bool occ = k != kEmpty;
      const unsigned b = __ballot_sync(0xffffffffu, occ);
      const int pos = cnt + __popc(b & ((1u << lane) - 1u));
      __syncwarp();
      if (occ) { keys[pos] = k; vals[pos] = v; }
      cnt += __popc(b);
      __syncwarp();
    }
    const int64_t off = c_off[i];
    const int64_t len = c_off[i + 1] - off;
    if (lane == 0 && len != cnt) set_error(err, kErrCount);
    const int N = pow2_ceil(cnt);
    for (int t = cnt + lane; t < N; t += 32) keys[t] = kNoCol;
    __syncwarp();
    warp_bitonic(keys, vals, N);
    const int nw_out = cnt < len ? cnt : static_cast<int>(len);
    const int32_t cb = abase ? abase[i] : 0;
    for (int t = lane; t < nw_out; t += 32) {
      ccol[off + t] = keys[t] - cb;
      store_value<Mode>(cval, off + t, vals[t]);
    }
    __syncwarp();
  }
}

template <int LOG2S, int NT, int Mode>
__global__ void __launch_bounds__(NT) k_num_block(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                  int64_t count, const int64_t* __restrict__ c_off,
                                                  int32_t* __restrict__ ccol, void* __restrict__ cval,
                                                  const int32_t* __restrict__ abase, int32_t* __restrict__ row_flag,
                                                  const int32_t* __restrict__ negflag, uint32_t* err) {
  constexpr int S = 1 << LOG2S;
  extern __shared__ double smem_f64[];
  double* vals = smem_f64;
  int32_t* keys = reinterpret_cast<int32_t*>(smem_f64 + S);
  __shared__ int32_t s_excl[NT];
  __shared__ int64_t s_bs[NT];
  __shared__ int32_t s_scan[33];
  for (int64_t r = blockIdx.x; r < count; r += gridDim.x) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    if (Mode == kModeF32C && threadIdx.x == 0 && !f32c_hash_row_ok(negflag, na)) row_flag[i] = 1;
    for (int s = threadIdx.x; s < S; s += NT) { keys[s] = kEmpty; vals[s] = 0.0; }
    __syncthreads();
    block_for_each_product<NT>(A, B, a0, na, s_excl, s_bs, s_scan, [&](int64_t j, int64_t e) {
      hash_accumulate<LOG2S, Mode>(keys, vals, B.col[j], value_at<Mode>(A.val, a0 + e), value_at<Mode>(B.val, j),
                                   err);
    });
    // compact in place, one block-wide chunk at a time
    int cnt = 0;
    for (int base = 0; base < S; base += NT) {
      const int32_t k = keys[base + threadIdx.x];
      const double v = vals[base + threadIdx.x];
      const int occ = k != kEmpty;
      int32_t tot;
      const int32_t pos = cnt + block_excl_scan<int32_t>(occ, s_scan, &tot);
      if (occ) { keys[pos] = k; vals[pos] = v; }
      cnt += tot;
      __syncthreads();
    }
    const int64_t off = c_off[i];
    const int64_t len = c_off[i + 1] - off;
    if (threadIdx.x == 0 && len != cnt) set_error(err, kErrCount);
    const int N = pow2_ceil(cnt);
    for (int t = cnt + threadIdx.x; t < N; t += NT) keys[t] = kNoCol;
    __syncthreads();
    block_bitonic<NT>(keys, vals, N);
    const int nb_out = cnt < len ? cnt : static_cast<int>(len);
    const int32_t cb = abase ? abase[i] : 0;
    for (int t = threadIdx.x; t < nb_out; t += NT) {
      ccol[off + t] = keys[t] - cb;
      store_value<Mode>(cval, off + t, vals[t]);
    }
    __syncthreads();
  }
}

inline unsigned grid_rows(int64_t count, int rows_per_block, int max_blocks) {
  int64_t g = (count + rows_per_block - 1) / rows_per_block;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return static_cast<unsigned>(g);
}

}  // namespace

int launch_num_tiny(int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                    const int64_t* c_off, int32_t* ccol, void* cval, int32_t* row_flag, const int32_t* abase,
                    uint32_t* err, int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  const unsigned g = grid_rows(count, 8, num_sms * 64);
  if (mode == kModeF32C) k_num_tiny<kModeF32C><<<g, 256, 0, s>>>(A, B, perm, count, c_off, ccol, cval, row_flag, abase, err);
  else if (mode == kModeF32R) k_num_tiny<kModeF32R><<<g, 256, 0, s>>>(A, B, perm, count, c_off, ccol, cval, row_flag, abase, err);
  else k_num_tiny<kModeF64><<<g, 256, 0, s>>>(A, B, perm, count, c_off, ccol, cval, row_flag, abase, err);
  return 1;
}

int launch_num_micro(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     const int64_t* c_off, int32_t* ccol, double* cval, const int32_t* abase, uint32_t* err,
                     int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  k_num_micro<<<grid_rows(count, 256, num_sms * 16), 256, 0, s>>>(A, B, perm, count, c_off, ccol, cval, abase, err);
  return 1;
}

int launch_num_warp(int log2S, int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                    const int64_t* c_off, int32_t* ccol, void* cval, const int32_t* abase, int32_t* row_flag,
                    const int32_t* negflag, uint32_t* err, int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  const unsigned g = grid_rows(count, 8, num_sms * 32);
  const size_t sm = size_t(8) * (size_t(1) << log2S) * 12;
  auto go = [&](auto kernel) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    kernel<<<g, 256, sm, s>>>(A, B, perm, count, c_off, ccol, cval, abase, row_flag, negflag, err);
  };
  const bool f32c = mode == kModeF32C;
  switch (log2S) {
    case 6: f32c ? go(k_num_warp<6, kModeF32C>) : go(k_num_warp<6, kModeF64>); break;
    case 8: f32c ? go(k_num_warp<8, kModeF32C>) : go(k_num_warp<8, kModeF64>); break;
    case 10: f32c ? go(k_num_warp<10, kModeF32C>) : go(k_num_warp<10, kModeF64>); break;
    default: break;
  }
  return 1;
}

int launch_num_block(int log2S, int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     const int64_t* c_off, int32_t* ccol, void* cval, const int32_t* abase, int32_t* row_flag,
                     const int32_t* negflag, uint32_t* err, int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  const size_t sm = (size_t(1) << log2S) * 12;
  const bool f32c = mode == kModeF32C;
  auto go = [&](auto kernel, int nt, int per_sm) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    kernel<<<grid_rows(count, 1, num_sms * per_sm), nt, sm, s>>>(A, B, perm, count, c_off, ccol, cval, abase, row_flag,
                                                                 negflag, err);
  };
  if (log2S == 11) {
    f32c ? go(k_num_block<11, 256, kModeF32C>, 256, 8) : go(k_num_block<11, 256, kModeF64>, 256, 8);
  } else if (log2S == 13) {
    f32c ? go(k_num_block<13, 512, kModeF32C>, 512, 4) : go(k_num_block<13, 512, kModeF64>, 512, 4);
  }
  return 1;
}

}  // namespace spg
