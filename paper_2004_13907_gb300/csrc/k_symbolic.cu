// Symbolic pass: nnz(C_i) = |union over the stored k of row i of A of cols(B_k)|,
// the size of the COLB set Algorithm 1 builds for row i (Sec. III-A).
//
// Row classes (chosen by the plan from P_i and min(P_i, n)):
//  * tiny  : P_i <= 32, one warp, each lane holds one column; duplicates are found with a
//            warp match, so no shared table is needed;
//  * warp  : one warp per row, a shared-memory hash table of 128 / 512 / 2048 keys;
//  * block : one block per row, a shared-memory hash table of 8192 keys;
//  * window: one persistent block per row, a shared-memory bitmap of up to 2^20 columns.
//            Besides nnz(C_i) it records how many columns of C_i fall in each block of
//            kBlockCols columns, which the numeric pass uses to plan its windows. When B has
//            more than 2^20 columns the bitmap slides over the columns in windows and a
//            per-entry cursor in global memory remembers where each B row stopped.
// Hash tables are sized to at least twice the row's upper bound min(P_i, n), so probing
// always ends; a probe count over the table size still reports kErrHashFull.
#include "enumerate.cuh"

namespace spg {

namespace {

__global__ void __launch_bounds__(256) k_sym_tiny(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                  int64_t count, int32_t* __restrict__ nnz_row) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = gw; r < count; r += nw) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int32_t na = static_cast<int32_t>(A.rp[i + 1] - a0);
    int32_t col = -2 - lane;
    int32_t total = 0;
    int32_t len = 0;
    int64_t bs = 0;
    if (lane < na) {
      const int32_t k = A.col[a0 + lane];
      bs = B.rp[k];
      len = static_cast<int32_t>(B.rp[k + 1] - bs);
    }
    const int32_t incl = warp_incl_scan(len);
    total = __shfl_sync(0xffffffffu, incl, 31);
    int o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int32_t v = __shfl_sync(0xffffffffu, incl, o + step - 1);
      if (v <= lane) o += step;
    }
    const int32_t incl_o = __shfl_sync(0xffffffffu, incl, o & 31);
    const int32_t len_o = __shfl_sync(0xffffffffu, len, o & 31);
    const int64_t bs_o = __shfl_sync(0xffffffffu, bs, o & 31);
    if (lane < total) col = B.col[bs_o + (lane - (incl_o - len_o))];
    const unsigned peers = __match_any_sync(0xffffffffu, col);
    const bool lead = lane < total && (__ffs(peers) - 1) == lane;
    const int n = __popc(__ballot_sync(0xffffffffu, lead));
    if (lane == 0) nnz_row[i] = n;
  }
}

// Micro rows (nnz(A_i) <= kMicroNa, P_i <= tiny_max): one thread per row merges the row's sorted
// B rows head by head (the smallest head column is the next column of C; every head holding it
// advances) and counts the distinct columns.
__global__ void __launch_bounds__(256) k_sym_micro(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                   int64_t count, int32_t* __restrict__ nnz_row) {
  constexpr int NA = kMicroNa;
  constexpr int32_t kEnd = 0x7fffffff;   // column of an exhausted head (every column is smaller)
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < count; r += stride) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int na = static_cast<int>(A.rp[i + 1] - a0);
    int64_t pos[NA];
    int32_t left[NA], hc[NA];
#pragma unroll
    for (int h = 0; h < NA; ++h) {
      pos[h] = 0; left[h] = 0; hc[h] = kEnd;
      if (h < na) {
        const int32_t k = A.col[a0 + h];
        pos[h] = B.rp[k];
        left[h] = static_cast<int32_t>(B.rp[k + 1] - pos[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < NA; ++h) if (left[h] > 0) hc[h] = B.col[pos[h]];
    int32_t n = 0;
    for (;;) {
      int32_t m = hc[0];
#pragma unroll
      for (int h = 1; h < NA; ++h) m = hc[h] < m ? hc[h] : m;
      if (m == kEnd) break;
      ++n;
#pragma unroll
      for (int h = 0; h < NA; ++h) {
        if (hc[h] == m) {
          ++pos[h];
          --left[h];
          hc[h] = left[h] > 0 ? B.col[pos[h]] : kEnd;
        }
      }
    }
    nnz_row[i] = n;
  }
}

// Insert `key` into an open-addressing table (linear probing). Returns 1 if it was new.
template <int LOG2S>
__device__ __forceinline__ int insert_key(int32_t* table, int32_t key, uint32_t* err) {
  constexpr int S = 1 << LOG2S;
  uint32_t h = hash_slot(key, LOG2S);
  for (int probe = 0; probe < S; ++probe) {
    const int32_t cur = *reinterpret_cast<volatile int32_t*>(&table[h]);
    if (cur == key) return 0;
    if (cur == kEmpty) {
      const int32_t old = atomicCAS(&table[h], kEmpty, key);
      if (old == kEmpty) return 1;
      if (old == key) return 0;
    }
    h = (h + 1) & (S - 1);
  }
  set_error(err, kErrHashFull);
  return 0;
}

template <int LOG2S>
__global__ void __launch_bounds__(256) k_sym_warp(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                  int64_t count, int32_t* __restrict__ nnz_row,
                                                  uint32_t* err) {
  constexpr int S = 1 << LOG2S;
  extern __shared__ int32_t smem_i32[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* table = smem_i32 + wid * S;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = gw; r < count; r += nw) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    for (int s = lane; s < S; s += 32) table[s] = kEmpty;
    __syncwarp();
    int cnt = 0;
    warp_for_each_product(A, B, a0, na, [&](int64_t j, int64_t) {
      cnt += insert_key<LOG2S>(table, B.col[j], err);
    });
    cnt = warp_sum(cnt);
    if (lane == 0) nnz_row[i] = cnt;
    __syncwarp();
  }
}

template <int LOG2S, int NT>
__global__ void __launch_bounds__(NT) k_sym_block(DevCsr A, DevCsr B, const int32_t* __restrict__ perm,
                                                  int64_t count, int32_t* __restrict__ nnz_row,
                                                  uint32_t* err) {
  constexpr int S = 1 << LOG2S;
  extern __shared__ int32_t smem_i32[];
  int32_t* table = smem_i32;
  __shared__ int32_t s_excl[NT];
  __shared__ int64_t s_bs[NT];
  __shared__ int32_t s_scan[33];
  __shared__ int32_t s_cnt;
  for (int64_t r = blockIdx.x; r < count; r += gridDim.x) {
    const int32_t i = perm[r];
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    for (int s = threadIdx.x; s < S; s += NT) table[s] = kEmpty;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int cnt = 0;
    block_for_each_product<NT>(A, B, a0, na, s_excl, s_bs, s_scan, [&](int64_t j, int64_t) {
      cnt += insert_key<LOG2S>(table, B.col[j], err);
    });
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) nnz_row[i] = s_cnt;
    __syncthreads();
  }
}

// Windowed symbolic pass, one row per block at a time (rows handed out by an atomic
// counter, heaviest class first).
__global__ void __launch_bounds__(kSymWinThreads, 1) k_sym_window(DevCsr A, DevCsr B,
                                                               const int32_t* __restrict__ perm,
                                                               int64_t count, int32_t* counter,
                                                               int32_t* __restrict__ nnz_row,
                                                               int32_t* __restrict__ win_slot,
                                                               uint16_t* __restrict__ blockcnt,
                                                               int64_t nblocks, int32_t* cursor,
                                                               const int32_t* __restrict__ abase,
                                                               const int32_t* __restrict__ awidth,
                                                               int64_t width_all, uint32_t* __restrict__ wbits,
                                                               int64_t wcap, unsigned long long* wcur,
                                                               int64_t* __restrict__ woff, uint32_t* err) {
  extern __shared__ uint32_t bm[];  // kSymWinBits / 32 words
  __shared__ int32_t s_excl[kSymWinThreads + 1];
  __shared__ int64_t s_bs[kSymWinThreads];
  __shared__ long long s_scan64[33];
  __shared__ int32_t s_ctl[2];
  __shared__ int32_t s_idx;
  __shared__ unsigned long long s_total;
  __shared__ long long s_woff;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int kWarps = kSymWinThreads / 32;
  // the bitmap is cleared once here; every window's counting pass leaves it clear again
  for (int t = threadIdx.x; t < kSymWinBits / 32; t += kSymWinThreads) bm[t] = 0u;
  if (threadIdx.x == 0) {
    s_idx = atomicAdd(counter, 1);
    s_total = 0;
  }
  for (;;) {
    __syncthreads();
    const int64_t idx = s_idx;
    if (idx >= count) break;
    const int32_t i = perm[idx];
    if (threadIdx.x == 0) win_slot[i] = static_cast<int32_t>(idx);
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    const int64_t cb = abase ? abase[i] : 0;   // the row's columns are [cb, cb + width)
    const int64_t width = awidth ? awidth[i] : width_all;
    uint16_t* cnts = blockcnt + idx * nblocks;
    // a row inside one window stores its bitmap (its blocks, 128 words each) for the numeric
    // pass when wbits has room
    const bool store = wbits != nullptr && width <= kSymWinBits;
    // thread 0 claims the next row and this row's stored-bitmap space now; both results are used
    // only after the marking, so the atomics' latency hides behind it
    int64_t next_idx = 0;
    const int64_t words = store ? (width + kBlockCols - 1) / kBlockCols * kBlockWords : 0;
    unsigned long long woff_at = 0;
    if (threadIdx.x == 0) {
      next_idx = atomicAdd(counter, 1);
      if (store) woff_at = atomicAdd(wcur, static_cast<unsigned long long>(words));
    }
    for (int64_t r0 = 0; r0 < width; r0 += kSymWinBits) {
      const int64_t w0 = cb + r0;
      const int64_t wend = cb + ((r0 + kSymWinBits < width) ? r0 + kSymWinBits : width);
      if (width <= kSymWinBits) {
        // one window covers every column: no cursors; each warp marks a contiguous range of the
        // row's products (eight groups of 32 loaded before they are marked)
        // columns and the window start are below 2^31, so the offset fits 32 bits; a negative one
        // wraps above span
        const uint32_t span = static_cast<uint32_t>(wend - w0);
        const int32_t w0i = static_cast<int32_t>(w0);
        bool outside = false;
        block_range_for_each_product<kSymWinThreads, 8>(
            A, B, a0, na, s_excl, s_bs, s_scan64, s_ctl, [&](const int64_t (&j)[8]) {
              int32_t c[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) c[u] = j[u] >= 0 ? B.col[j[u]] : w0i;
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                if (j[u] < 0) continue;
                const uint32_t rel = static_cast<uint32_t>(c[u] - w0i);
                if (rel < span) atomicOr(&bm[rel >> 5], 1u << (rel & 31));
                else outside = true;
              }
            });
        if (outside) set_error(err, kErrWindowPlan);
      } else {
        for (int64_t e = wid; e < na; e += kWarps) {
          const int32_t k = A.col[a0 + e];
          const int64_t bstart = B.rp[k], bend = B.rp[k + 1];
          int64_t cur = (r0 == 0) ? bstart : bstart + cursor[a0 + e];
          while (cur < bend) {
            const int64_t j = cur + lane;
            const int32_t c = j < bend ? B.col[j] : kNoCol;
            const bool ok = c < wend;
            if (ok && c >= w0) atomicOr(&bm[(c - w0) >> 5], 1u << ((c - w0) & 31));
            const int got = __popc(__ballot_sync(0xffffffffu, ok));
            cur += got;
            if (got < 32) break;
          }
          if (lane == 0) cursor[a0 + e] = static_cast<int32_t>(cur - bstart);
        }
        __syncthreads();
      }
      if (r0 == 0) {
        // the stored copy's place (a stored row has this one window), published for the pass below
        if (threadIdx.x == 0) {
          long long o = -1;
          if (store && woff_at + words <= static_cast<unsigned long long>(wcap)) o = static_cast<long long>(woff_at);
          s_woff = o;
          if (woff) woff[idx] = o;
        }
        __syncthreads();
      }
      const long long wo = s_woff;
      // per-block counts of this window, the stored copy and the clearing of the bitmap in one
      // pass: a warp per block of kBlockWords words (lane: 4), blocks counted from the row's first
      // column cb. A window ends on a block boundary (kSymWinBits is a multiple of kBlockCols), so
      // every block's words lie inside the bitmap; words past the row's width were never marked.
      const int64_t b0 = r0 / kBlockCols;
      const int64_t b1 = (wend - cb + kBlockCols - 1) / kBlockCols;
      for (int64_t b = b0 + wid; b < b1; b += kWarps) {
        uint4* p = reinterpret_cast<uint4*>(bm + (b * kBlockWords - (r0 >> 5))) + lane;
        const uint4 v = *p;
        int c = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        c = warp_sum(c);
        if (lane == 0) {
          cnts[b] = static_cast<uint16_t>(c);
          if (c) atomicAdd(&s_total, static_cast<unsigned long long>(c));
        }
        // a stored row has one window, starting at block 0
        if (wo >= 0) reinterpret_cast<uint4*>(wbits + wo)[b * (kBlockWords / 4) + lane] = v;
        if (v.x | v.y | v.z | v.w) *p = make_uint4(0u, 0u, 0u, 0u);
      }
      __syncthreads();
    }
    // s_total is final (the counting pass ended with a barrier); thread 0 resets it and hands out
    // the next row, which every thread reads after the barrier at the top
    if (threadIdx.x == 0) {
      nnz_row[i] = static_cast<int32_t>(s_total);
      s_total = 0;
      s_idx = next_idx;
    }
  }
}

inline unsigned grid_rows(int64_t count, int rows_per_block, int max_blocks) {
  int64_t g = (count + rows_per_block - 1) / rows_per_block;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return static_cast<unsigned>(g);
}

}  // namespace

int launch_sym_tiny(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     int32_t* nnz_row, int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  k_sym_tiny<<<grid_rows(count, 8, num_sms * 64), 256, 0, s>>>(A, B, perm, count, nnz_row);
  return 1;
}

int launch_sym_micro(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     int32_t* nnz_row, int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  k_sym_micro<<<grid_rows(count, 256, num_sms * 16), 256, 0, s>>>(A, B, perm, count, nnz_row);
  return 1;
}

int launch_sym_warp(int log2S, const DevCsr& A, const DevCsr& B, const int32_t* perm,
                     int64_t count, int32_t* nnz_row, uint32_t* err, int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  const unsigned g = grid_rows(count, 8, num_sms * 32);
  const size_t sm = size_t(8) << log2S << 2;
  switch (log2S) {
    case 7: k_sym_warp<7><<<g, 256, sm, s>>>(A, B, perm, count, nnz_row, err); break;
    case 9: k_sym_warp<9><<<g, 256, sm, s>>>(A, B, perm, count, nnz_row, err); break;
    case 11:
      cudaFuncSetAttribute(k_sym_warp<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
      k_sym_warp<11><<<g, 256, sm, s>>>(A, B, perm, count, nnz_row, err);
      break;
    default: break;
  }
  return 1;
}

int launch_sym_block(int log2S, const DevCsr& A, const DevCsr& B, const int32_t* perm,
                      int64_t count, int32_t* nnz_row, uint32_t* err, int num_sms, cudaStream_t s) {
  if (count <= 0) return 0;
  const size_t sm = size_t(4) << log2S;
  if (log2S == 13) {
    k_sym_block<13, 512><<<grid_rows(count, 1, num_sms * 8), 512, sm, s>>>(A, B, perm, count, nnz_row, err);
  }
  return 1;
}

int launch_sym_window(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                       int32_t* counter, int32_t* nnz_row, int32_t* win_slot, uint16_t* blockcnt,
                       int64_t nblocks, int32_t* cursor, const int32_t* abase, const int32_t* awidth,
                       int64_t width, uint32_t* wbits, int64_t wcap, unsigned long long* wcur, int64_t* woff,
                       int num_sms, uint32_t* err, cudaStream_t s) {
  if (count <= 0) return 0;
  const size_t sm = size_t(kSymWinBits / 32) * 4;
  cudaFuncSetAttribute(k_sym_window, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  const int64_t g = count < num_sms ? count : num_sms;
  k_sym_window<<<static_cast<unsigned>(g), kSymWinThreads, sm, s>>>(A, B, perm, count, counter, nnz_row,
                                                                 win_slot, blockcnt, nblocks, cursor,
                                                                 abase, awidth, width, wbits, wcap, wcur, woff, err);
  return 1;
}

}  // namespace spg
