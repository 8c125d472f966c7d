// Plan-phase and scan kernels: CSR validation, the per-row product count, the
// class histogram scan, the class scatter that groups rows by work, and the row-offset
// scan of C after the symbolic pass.
//
// The count is the number of partial products Algorithm 1 forms for row i (Sec. III-A):
// P_i = sum over the stored columns k of row i of A of nnz(row k of B), i.e. only the B
// rows named by row i are "streamed" (Sec. III-A, selective streaming of B rows).
// Grouping rows by P_i on the device plays the role of the CPU-side scheduling of RIR
// bundles (Sec. II, "RIR includes scheduling"; Sec. III-A, long rows split into bundles):
// every row class gets a kernel shaped for its size.
#include "kernels.h"

namespace spg {

namespace {

// Row pointers of rows [r0, r0 + n1 - 1) of a CSR matrix, rebased to start at 0 (int64).
__global__ void k_rowptr_rebase(const void* __restrict__ in, int idx64, int64_t r0, int64_t n1, int64_t base,
                                int64_t* __restrict__ out) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n1; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t v = idx64 ? static_cast<const int64_t*>(in)[r0 + t] : static_cast<const int32_t*>(in)[r0 + t];
    out[t] = v - base;
  }
}

// Small reads of device state: a grid of SMs stores the words into mapped page-locked host
// memory, so the read never queues on the copy engine behind bulk copies to the host.
__global__ void k_fetch(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int64_t words) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < words; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_rowptr_to64(const int32_t* __restrict__ in, int64_t* __restrict__ out, int64_t n1) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n1;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] = in[i];
}

// One warp per row: row pointers in range and non-decreasing, columns strictly increasing
// in [0, cols). Any violation sets kErrInvalidCsr.
// Canonical-CSR check in two bandwidth-shaped passes. Rows: a thread per row checks its row
// pointers and marks the row's first entry in a bitmap over the entries. Entries: a thread per
// entry checks its column range and, unless the entry starts a row, that it is larger than the
// entry before it.
__global__ void __launch_bounds__(256) k_validate_rows(DevCsr M, uint32_t* __restrict__ starts, uint32_t* err) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t t0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t0 == 0 && (M.rp[0] != 0 || M.rp[M.rows] != M.nnz)) set_error(err, kErrInvalidCsr);
  bool bad = false;
  for (int64_t i = t0; i < M.rows; i += stride) {
    const int64_t s = M.rp[i], e = M.rp[i + 1];
    if (s < 0 || e < s || e > M.nnz) bad = true;
    else if (s < e) atomicOr(&starts[s >> 5], 1u << (s & 31));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_error(err, kErrInvalidCsr);
}

__global__ void __launch_bounds__(256) k_validate_cols(DevCsr M, const uint32_t* __restrict__ starts,
                                                       uint32_t* err) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  bool bad = false;
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < M.nnz; j += stride) {
    const int32_t c = M.col[j];
    bad |= c < 0 || c >= M.cols;
    if (j > 0 && !((starts[j >> 5] >> (j & 31)) & 1u)) bad |= M.col[j - 1] >= c;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_error(err, kErrInvalidCsr);
}

// Warp-aggregated increment of a shared counter per class; returns this lane's slot.
__device__ __forceinline__ int32_t aggregated_slot(int32_t* counters, int cls, bool valid) {
  const unsigned lane = lane_id();
  const unsigned peers = __match_any_sync(0xffffffffu, valid ? cls : 1000 + static_cast<int>(lane));
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  int32_t base = 0;
  if (valid && static_cast<int>(lane) == leader) base = atomicAdd(&counters[cls], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + rank;
}

// P_i for 256 rows (a quarter of a tile of kTileRows rows; one row per thread, so that even a
// small matrix spreads over many blocks). Short rows are summed by their own thread, rows with
// more than 64 entries by the whole warp, and rows with more than kCountBlockNa entries by the
// whole block after the others. The block adds its class counts, sum and maximum of P_i into its
// tile's (zeroed) histogram with global atomics.
// Rows with more entries than this are counted by the whole block of k_count.
constexpr int64_t kCountBlockNa = 2048;

// Row `row` of A as [a0, a0 + na) clamped to the stored entries, so that an input the
// validation kernels have not yet rejected cannot send a read outside A's arrays.
__device__ __forceinline__ void clamped_row(const DevCsr& A, int64_t row, int64_t& a0, int64_t& na) {
  int64_t s = A.rp[row], e = A.rp[row + 1];
  s = s < 0 ? 0 : (s > A.nnz ? A.nnz : s);
  e = e < s ? s : (e > A.nnz ? A.nnz : e);
  a0 = s;
  na = e - s;
}

__global__ void __launch_bounds__(256) k_count(DevCsr A, DevCsr B, ClassParams cp, int64_t* P,
                                               int32_t* nnz_row, int32_t* tile_hist,
                                               int64_t* tile_sum, int64_t* tile_max) {
  __shared__ int32_t hist[kMaxClasses];
  __shared__ unsigned long long s_sum, s_max;
  __shared__ int32_t s_ndef;                 // rows left to the whole block (longest rows)
  __shared__ int64_t s_def[256];
  __shared__ long long s_red[8];
  if (threadIdx.x < kMaxClasses) hist[threadIdx.x] = 0;
  if (threadIdx.x == 0) { s_sum = 0; s_max = 0; s_ndef = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t t = blockIdx.x / (kTileRows / 256);   // the tile this block belongs to
  unsigned long long my_sum = 0, my_max = 0;
  {
    const int64_t row = blockIdx.x * int64_t(256) + threadIdx.x;
    const bool valid = row < A.rows;
    int64_t a0 = 0, na = 0;
    if (valid) {
      // the validation kernels run ahead in the same stream and the host reads their verdict
      // only after this pass, so a row range or column of an invalid input is clamped here
      // (its counts are then meaningless, but every access stays inside the arrays)
      clamped_row(A, row, a0, na);
    }
    int64_t p = 0;
    const bool blockrow = valid && na > kCountBlockNa;   // summed by the whole block below
    const bool longrow = valid && na > 64 && !blockrow;
    if (blockrow) s_def[atomicAdd(&s_ndef, 1)] = row;
    if (valid && !longrow && !blockrow) {
#pragma unroll 4
      for (int64_t j = 0; j < na; ++j) {
        const int32_t k = A.col[a0 + j];
        if (k >= 0 && k < B.rows) p += B.rp[k + 1] - B.rp[k];
      }
    }
    unsigned lm = __ballot_sync(0xffffffffu, longrow);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int64_t sa0 = __shfl_sync(0xffffffffu, a0, src);
      const int64_t sna = __shfl_sync(0xffffffffu, na, src);
      int64_t acc = 0;
      for (int64_t j = lane; j < sna; j += 32) {
        const int32_t k = A.col[sa0 + j];
        if (k >= 0 && k < B.rows) acc += B.rp[k + 1] - B.rp[k];
      }
      acc = warp_sum(acc);
      if (lane == src) p = acc;
    }
    int cls = kSymZero;
    if (valid && !blockrow) {
      const int32_t na32 = na > 0x7fffffff ? 0x7fffffff : static_cast<int32_t>(na);
      cls = sym_class(p, na32, row_params(cp, row));
      P[row] = p;
      if (cls == kSymZero) nnz_row[row] = 0;
      my_sum += static_cast<unsigned long long>(p);
      my_max = my_max > static_cast<unsigned long long>(p) ? my_max : static_cast<unsigned long long>(p);
    }
    aggregated_slot(hist, cls, valid && !blockrow);
  }
  __syncthreads();
  // the longest rows of the tile, one at a time, their entries spread over all 256 threads
  const int ndef = s_ndef;
  for (int d = 0; d < ndef; ++d) {
    const int64_t row = s_def[d];
    int64_t a0, na;
    clamped_row(A, row, a0, na);
    long long acc = 0;
    for (int64_t j = threadIdx.x; j < na; j += 256) {
      const int32_t k = A.col[a0 + j];
      if (k >= 0 && k < B.rows) acc += B.rp[k + 1] - B.rp[k];
    }
    acc = warp_sum(acc);
    if (lane == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long p = 0;
      for (int w = 0; w < 8; ++w) p += s_red[w];
      const int32_t na32 = na > 0x7fffffff ? 0x7fffffff : static_cast<int32_t>(na);
      const int cls = sym_class(p, na32, row_params(cp, row));
      P[row] = p;
      if (cls == kSymZero) nnz_row[row] = 0;
      atomicAdd(&hist[cls], 1);
      my_sum += static_cast<unsigned long long>(p);
      my_max = my_max > static_cast<unsigned long long>(p) ? my_max : static_cast<unsigned long long>(p);
    }
    __syncthreads();
  }
  my_sum = warp_sum(my_sum);
  my_max = warp_min(~my_max);
  my_max = ~my_max;
  if (lane == 0) {
    atomicAdd(&s_sum, my_sum);
    atomicMax(&s_max, my_max);
  }
  __syncthreads();
  if (threadIdx.x < kMaxClasses && hist[threadIdx.x]) atomicAdd(&tile_hist[t * kMaxClasses + threadIdx.x], hist[threadIdx.x]);
  if (threadIdx.x == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&tile_sum[t]), s_sum);
    if (tile_max) atomicMax(reinterpret_cast<unsigned long long*>(&tile_max[t]), s_max);
  }
}

// One block: turns the per-tile class counts into per-tile base offsets (in place),
// writes the class offsets, and scans the per-tile sums. Warp c handles class c.
__global__ void __launch_bounds__(544) k_class_scan(int64_t ntiles, int nclasses, int32_t* tile_hist,
                                                    const int64_t* tile_sum, const int64_t* tile_max,
                                                    int64_t* tile_sum_off, Summary* summary) {
  __shared__ int64_t tot[kMaxClasses];
  __shared__ int64_t off[kMaxClasses + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < nclasses) {
    int64_t s = 0;
    for (int64_t t = lane; t < ntiles; t += 32) s += tile_hist[t * kMaxClasses + w];
    s = warp_sum(s);
    if (lane == 0) tot[w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t o = 0;
    for (int c = 0; c < nclasses; ++c) { off[c] = o; summary->class_off[c] = o; o += tot[c]; }
    for (int c = nclasses; c <= kMaxClasses; ++c) { off[c] = o; summary->class_off[c] = o; }
  }
  __syncthreads();
  if (w < nclasses) {
    int64_t run = off[w];
    for (int64_t t0 = 0; t0 < ntiles; t0 += 32) {
      const int64_t t = t0 + lane;
      const int64_t v = t < ntiles ? tile_hist[t * kMaxClasses + w] : 0;
      const int64_t incl = warp_incl_scan(v);
      if (t < ntiles) tile_hist[t * kMaxClasses + w] = static_cast<int32_t>(run + incl - v);
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  } else if (w == kMaxClasses) {
    int64_t run = 0, mx = 0;
    for (int64_t t0 = 0; t0 < ntiles; t0 += 32) {
      const int64_t t = t0 + lane;
      const int64_t v = t < ntiles ? tile_sum[t] : 0;
      if (tile_max && t < ntiles) mx = mx > tile_max[t] ? mx : tile_max[t];
      const int64_t incl = warp_incl_scan(v);
      if (tile_sum_off && t < ntiles) tile_sum_off[t] = run + incl - v;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    mx = ~warp_min(~mx);
    if (lane == 0) {
      summary->total = run;
      summary->max_row = mx;
    }
  }
}

__global__ void __launch_bounds__(256) k_scatter_sym(DevCsr A, ClassParams cp, const int64_t* P,
                                                     const int32_t* tile_hist, int32_t* perm) {
  __shared__ int32_t base[kMaxClasses];
  const int64_t t = blockIdx.x;
  if (threadIdx.x < kMaxClasses) base[threadIdx.x] = tile_hist[t * kMaxClasses + threadIdx.x];
  __syncthreads();
  for (int r = 0; r < kTileRows / 256; ++r) {
    const int64_t row = t * kTileRows + r * 256 + threadIdx.x;
    const bool valid = row < A.rows;
    int cls = 0;
    if (valid) {
      int64_t a0, na;
      clamped_row(A, row, a0, na);   // the same row length k_count classified (before validation's verdict)
      cls = sym_class(P[row], na > 0x7fffffff ? 0x7fffffff : static_cast<int32_t>(na), row_params(cp, row));
    }
    const int32_t pos = aggregated_slot(base, cls, valid);
    if (valid) perm[pos] = static_cast<int32_t>(row);
  }
}

__global__ void __launch_bounds__(256) k_num_tiles(DevCsr A, ClassParams cp, const int64_t* P,
                                                   const int32_t* nnz_row, int32_t* tile_hist,
                                                   int64_t* tile_sum, unsigned long long* cls_sums) {
  __shared__ int32_t hist[kMaxClasses];
  __shared__ unsigned long long s_sum;
  __shared__ unsigned long long s_cls[kMaxClasses][3];
  if (threadIdx.x < kMaxClasses) hist[threadIdx.x] = 0;
  if (threadIdx.x < kMaxClasses * 3) (&s_cls[0][0])[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_sum = 0;
  __syncthreads();
  const int64_t t = blockIdx.x;
  unsigned long long my = 0;
  for (int r = 0; r < kTileRows / 256; ++r) {
    const int64_t row = t * kTileRows + r * 256 + threadIdx.x;
    const bool valid = row < A.rows;
    int cls = 0;
    unsigned long long vp = 0, vn = 0, vz = 0;
    if (valid) {
      const int64_t na = A.rp[row + 1] - A.rp[row];
      const int32_t z = nnz_row[row];
      cls = num_class(P[row], na > 0x7fffffff ? 0x7fffffff : static_cast<int32_t>(na), z, cp);
      my += static_cast<unsigned long long>(z);
      vp = static_cast<unsigned long long>(P[row]);
      vn = static_cast<unsigned long long>(na);
      vz = static_cast<unsigned long long>(z);
    }
    // per-class sums: one warp reduction per distinct class of the warp (a stencil has one), so
    // the shared counters see one atomic per class and warp instead of one per row
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
      const int lc = __shfl_sync(0xffffffffu, cls, __ffs(todo) - 1);
      const bool mine = valid && cls == lc;
      const unsigned long long sp = warp_sum(mine ? vp : 0ull);
      const unsigned long long sn = warp_sum(mine ? vn : 0ull);
      const unsigned long long sz = warp_sum(mine ? vz : 0ull);
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_cls[lc][0], sp);
        atomicAdd(&s_cls[lc][1], sn);
        atomicAdd(&s_cls[lc][2], sz);
      }
      todo &= ~__ballot_sync(0xffffffffu, mine);
    }
    aggregated_slot(hist, cls, valid);
  }
  my = warp_sum(my);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_sum, my);
  __syncthreads();
  if (threadIdx.x < kMaxClasses) tile_hist[t * kMaxClasses + threadIdx.x] = hist[threadIdx.x];
  if (threadIdx.x == 0) tile_sum[t] = static_cast<int64_t>(s_sum);
  if (threadIdx.x < kMaxClasses * 3) {
    const unsigned long long v = (&s_cls[0][0])[threadIdx.x];
    if (v) atomicAdd(&cls_sums[threadIdx.x], v);
  }
}

// Row offsets of C (exclusive scan of nnz(C_i), int64) and the numeric class scatter.
__global__ void __launch_bounds__(256) k_scatter_num(DevCsr A, ClassParams cp, const int64_t* P,
                                                     const int32_t* nnz_row, const int32_t* tile_hist,
                                                     const int64_t* tile_sum_off, int32_t* perm,
                                                     int64_t* c_off) {
  __shared__ int32_t base[kMaxClasses];
  __shared__ int64_t scratch[33];
  const int64_t t = blockIdx.x;
  if (threadIdx.x < kMaxClasses) base[threadIdx.x] = tile_hist[t * kMaxClasses + threadIdx.x];
  __syncthreads();
  int64_t carry = tile_sum_off[t];
  for (int r = 0; r < kTileRows / 256; ++r) {
    const int64_t row = t * kTileRows + r * 256 + threadIdx.x;
    const bool valid = row < A.rows;
    int cls = 0;
    int64_t z = 0;
    if (valid) {
      const int64_t na = A.rp[row + 1] - A.rp[row];
      z = nnz_row[row];
      cls = num_class(P[row], na > 0x7fffffff ? 0x7fffffff : static_cast<int32_t>(na),
                      static_cast<int32_t>(z), cp);
    }
    int64_t tot;
    const int64_t ex = block_excl_scan<int64_t>(z, scratch, &tot);
    if (valid) {
      c_off[row] = carry + ex;
      if (row == A.rows - 1) c_off[A.rows] = carry + ex + z;
    }
    carry += tot;
    const int32_t pos = aggregated_slot(base, cls, valid);
    if (valid) perm[pos] = static_cast<int32_t>(row);
  }
}

__global__ void __launch_bounds__(256) k_collect_flagged(const int32_t* __restrict__ perm, int64_t count,
                                                         const int32_t* __restrict__ row_flag, int all,
                                                         int32_t* __restrict__ list, int32_t* list_count) {
  for (int64_t r0 = blockIdx.x * int64_t(blockDim.x); r0 < count; r0 += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = r0 + threadIdx.x;
    int32_t row = 0;
    bool take = false;
    if (r < count) {
      row = perm[r];
      take = all || row_flag[row] != 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, take);
    int32_t base = 0;
    if (lane_id() == 0 && m) base = atomicAdd(list_count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) list[base + __popc(m & ((1u << lane_id()) - 1u))] = row;
  }
}

__global__ void k_write_rowptr(const int64_t* __restrict__ c_off, int64_t m1, void* out, int idx64) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m1;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (idx64) static_cast<int64_t*>(out)[i] = c_off[i];
    else static_cast<int32_t*>(out)[i] = static_cast<int32_t>(c_off[i]);
  }
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 65535LL * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<unsigned>(g);
}

}  // namespace

int launch_rowptr_rebase(const void* in, int idx64, int64_t r0, int64_t n1, int64_t base, int64_t* out,
                         cudaStream_t s) {
  if (n1 <= 0) return 0;
  k_rowptr_rebase<<<grid_for(n1, 256), 256, 0, s>>>(in, idx64, r0, n1, base, out);
  return 1;
}

int launch_fetch(const void* src, void* dst, int64_t bytes, cudaStream_t s) {
  const int64_t words = bytes / 4;
  if (words <= 0) return 0;
  k_fetch<<<grid_for(words, 256), 256, 0, s>>>(static_cast<const uint32_t*>(src), static_cast<uint32_t*>(dst), words);
  return 1;
}

int launch_rowptr_to64(const int32_t* in, int64_t* out, int64_t n1, cudaStream_t s) {
  k_rowptr_to64<<<grid_for(n1, 256), 256, 0, s>>>(in, out, n1);
  return 1;
}

int64_t validate_words(int64_t nnz) { return (nnz + 31) / 32 + 1; }

int launch_validate(const DevCsr& M, uint32_t* starts, uint32_t* err, cudaStream_t s) {
  cudaMemsetAsync(starts, 0, sizeof(uint32_t) * validate_words(M.nnz), s);
  k_validate_rows<<<grid_for(M.rows > 0 ? M.rows : 1, 256, 152 * 16), 256, 0, s>>>(M, starts, err);
  if (M.nnz > 0) k_validate_cols<<<grid_for(M.nnz, 256, 152 * 16), 256, 0, s>>>(M, starts, err);
  return M.nnz > 0 ? 2 : 1;
}

int launch_count(const DevCsr& A, const DevCsr& B, ClassParams cp, int64_t* P, int32_t* nnz_row,
                  int32_t* tile_hist, int64_t* tile_sum, int64_t* tile_max, cudaStream_t s) {
  const int64_t ntiles = (A.rows + kTileRows - 1) / kTileRows;
  if (ntiles == 0) return 0;
  cudaMemsetAsync(tile_hist, 0, sizeof(int32_t) * ntiles * kMaxClasses, s);
  cudaMemsetAsync(tile_sum, 0, sizeof(int64_t) * ntiles, s);
  if (tile_max) cudaMemsetAsync(tile_max, 0, sizeof(int64_t) * ntiles, s);
  const int64_t blocks = (A.rows + 255) / 256;
  k_count<<<static_cast<unsigned>(blocks), 256, 0, s>>>(A, B, cp, P, nnz_row, tile_hist, tile_sum, tile_max);
  return 1;
}

int launch_class_scan(int64_t ntiles, int nclasses, int32_t* tile_hist, const int64_t* tile_sum,
                       const int64_t* tile_max, int64_t* tile_sum_off, Summary* summary,
                       cudaStream_t s) {
  k_class_scan<<<1, 544, 0, s>>>(ntiles, nclasses, tile_hist, tile_sum, tile_max, tile_sum_off,
                                 summary);
  return 1;
}

int launch_scatter_sym(const DevCsr& A, ClassParams cp, const int64_t* P, const int32_t* tile_hist,
                        int32_t* perm, cudaStream_t s) {
  const int64_t ntiles = (A.rows + kTileRows - 1) / kTileRows;
  if (ntiles == 0) return 0;
  k_scatter_sym<<<static_cast<unsigned>(ntiles), 256, 0, s>>>(A, cp, P, tile_hist, perm);
  return 1;
}

int launch_num_tiles(const DevCsr& A, ClassParams cp, const int64_t* P, const int32_t* nnz_row,
                      int32_t* tile_hist, int64_t* tile_sum, unsigned long long* cls_sums,
                      cudaStream_t s) {
  const int64_t ntiles = (A.rows + kTileRows - 1) / kTileRows;
  if (ntiles == 0) return 0;
  k_num_tiles<<<static_cast<unsigned>(ntiles), 256, 0, s>>>(A, cp, P, nnz_row, tile_hist, tile_sum, cls_sums);
  return 1;
}

int launch_scatter_num(const DevCsr& A, ClassParams cp, const int64_t* P, const int32_t* nnz_row,
                        const int32_t* tile_hist, const int64_t* tile_sum_off, int32_t* perm,
                        int64_t* c_off, cudaStream_t s) {
  const int64_t ntiles = (A.rows + kTileRows - 1) / kTileRows;
  if (ntiles == 0) return 0;
  k_scatter_num<<<static_cast<unsigned>(ntiles), 256, 0, s>>>(A, cp, P, nnz_row, tile_hist,
                                                              tile_sum_off, perm, c_off);
  return 1;
}

int launch_collect_flagged(const int32_t* perm, int64_t count, const int32_t* row_flag, int all,
                           int32_t* list, int32_t* list_count, cudaStream_t s) {
  if (count <= 0) return 0;
  k_collect_flagged<<<grid_for(count, 256, 152 * 16), 256, 0, s>>>(perm, count, row_flag, all, list, list_count);
  return 1;
}

int launch_write_rowptr(const int64_t* c_off, int64_t m1, void* out, int idx64, cudaStream_t s) {
  k_write_rowptr<<<grid_for(m1, 256), 256, 0, s>>>(c_off, m1, out, idx64);
  return 1;
}

}  // namespace spg
