// Windowed numeric pass for rows with more entries of C than a block-wide hash table holds,
// and the column-block split table of B it reads.
//
// The columns of C are cut into blocks of kBlockCols. The symbolic pass counted, for each
// windowed row, the entries of C_i in every block. The numeric pass takes the blocks of a
// row in column order and groups consecutive blocks into windows of at most kRankCap entries
// of C spanning at most kSpanBlocks blocks. Each window is done in two passes over its partial
// products:
//  1. mark: set one bit per column that receives a partial product (a bitmap of the window's
//     columns); a prefix count over the bitmap then gives every column its rank, i.e. its
//     position among the window's columns in ascending order;
//  2. accumulate: add a_ik * b_kj into an FP64 array indexed by the rank of column j.
// The window is written out by rank: values straight from the rank-indexed array (coalesced),
// columns from the bitmap. The output is therefore sorted by column without any sort
// (Algorithm 1 sorts the partial products of a row and emits one entry per column of COLB,
// Sec. III-A; here the order comes from the bitmap).
//
// Inside a window, every A entry (k, a_ik) contributes the part of B row k whose columns fall
// in the window. The split table holds, for every row k of B and every block boundary b, the
// offset of the first entry of row k with column >= b * kBlockCols, so each A entry's part is
// known with two loads. The parts of a chunk of A entries are numbered consecutively
// ("flattened") and the block's threads take consecutive partial products, so long and short B
// rows keep all lanes busy. Building the split table once per product is the device-side
// counterpart of REAP's CPU-side regularisation of B into bundles (Sec. II): it turns "find
// the B entries of this row in this column range" into a table lookup.
//
// Sums are accumulated with shared-memory FP64 atomics, so their order may differ from run to
// run; the pattern is always exact.
#include "enumerate.cuh"

namespace spg {

namespace {

constexpr int kRankCap = 8192;                     // entries of C per window (>= kBlockCols)
constexpr int kSpanBlocks = 64;                    // blocks a window may span (512K columns)
constexpr int kSpanWords = kSpanBlocks * kBlockWords;    // bitmap words, 16384
constexpr int kGroupWords = 64;                    // words per prefix group
constexpr int kNumThreads = 1024;                  // threads of the windowed numeric kernel
constexpr int kWordsPerThread = kSpanWords / kNumThreads;
constexpr int kCntCache = 1024;                    // block counts kept in shared memory
constexpr int kSmemVals = kRankCap * 8;
constexpr int kSmemBits = kSpanWords * 4;
constexpr int kSmemPre = kSpanWords * 2;
constexpr int kSmemGrp = (kSpanWords / kGroupWords) * 4;
constexpr int kSmemEnt = kNumThreads * (8 + 8 + 8 + 4 + 4);
constexpr int kWinSmemBytes = kSmemVals + kSmemBits + kSmemPre + kSmemGrp + kSmemEnt + kCntCache * 2;
static_assert(kRankCap >= kBlockCols, "a window must hold any single block");
static_assert(kWordsPerThread * kNumThreads == kSpanWords, "words per thread");
static_assert(kGroupWords % kWordsPerThread == 0, "a thread's words lie in one group");
static_assert(kWinSmemBytes + 1024 <= 227 * 1024, "shared memory budget");


// Split table: one warp per row k of B writes split[k * (nblocks + 1) + b] for b in
// [0, nblocks]: the offset within row k of its first entry with column >= b * kBlockCols.
__global__ void __launch_bounds__(256) k_bsplit(DevCsr B, int64_t nblocks, int32_t* __restrict__ split) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  constexpr int kShift = kBlockShift;
  for (int64_t k = gw; k < B.rows; k += nw) {
    const int64_t s = B.rp[k];
    const int32_t len = static_cast<int32_t>(B.rp[k + 1] - s);
    int32_t* out = split + k * (nblocks + 1);
    if (len == 0) {
      for (int64_t b = lane; b <= nblocks; b += 32) out[b] = 0;
      continue;
    }
    for (int32_t t0 = 0; t0 < len; t0 += 32) {
      const int32_t t = t0 + lane;
      if (t < len) {
        const int64_t bc = B.col[s + t] >> kShift;
        const int64_t bp = t == 0 ? -1 : (B.col[s + t - 1] >> kShift);
        for (int64_t b = bp + 1; b <= bc; ++b) out[b] = t;
        if (t == len - 1)
          for (int64_t b = bc + 1; b <= nblocks; ++b) out[b] = len;
      }
    }
  }
}

// First index in col[0, len) with col >= x (col ascending).
__device__ __forceinline__ int32_t lower_bound_col(const int32_t* col, int32_t len, int64_t x) {
  int32_t lo = 0, hi = len;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (col[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Per-entry segment of the current window for the A entry in chunk slot t (e < na).
struct Seg { int64_t bs; int32_t len; };

__device__ __forceinline__ Seg entry_segment(const DevCsr& A, const DevCsr& B, const int32_t* split,
                                             int64_t nblocks, int64_t a0, int64_t e, bool resident,
                                             const int32_t* e_k, const int64_t* e_rs, double* e_av,
                                             int64_t b0, int64_t b1, int64_t w0, int64_t w1) {
  int32_t k;
  int64_t rs;
  if (resident) {
    k = e_k[threadIdx.x];
    rs = e_rs[threadIdx.x];
  } else {
    k = A.col[a0 + e];
    rs = B.rp[k];
    e_av[threadIdx.x] = static_cast<const double*>(A.val)[a0 + e];
  }
  int32_t s0, s1;
  if (split) {
    const int32_t* sp = split + int64_t(k) * (nblocks + 1);
    s0 = sp[b0];
    s1 = sp[b1];
  } else {
    const int32_t rl = static_cast<int32_t>(B.rp[k + 1] - rs);
    s0 = lower_bound_col(B.col + rs, rl, w0);
    s1 = lower_bound_col(B.col + rs, rl, w1);
  }
  return Seg{rs + s0, s1 - s0};
}

// Shared layout (dynamic): rank-indexed FP64 values [kRankCap]; window bitmap [kSpanWords];
// in-group word prefix (uint16) [kSpanWords]; group prefix (int32) [kSpanWords / 64]; per-entry
// state of the current chunk of A entries (B row start, a_ik, segment start, B row number,
// segment prefix); the row's block counts. The values and the bitmap are all zero between
// windows. A row whose A entries fit one chunk keeps their B row numbers, B row starts and
// values across all its windows.
__global__ void __launch_bounds__(kNumThreads, 1) k_num_window(
    DevCsr A, DevCsr B, const int32_t* __restrict__ perm, int64_t count, int32_t* counter,
    const int64_t* __restrict__ c_off, const int32_t* __restrict__ win_slot,
    const uint16_t* __restrict__ blockcnt, int64_t nblocks, int64_t nslots,
    const int32_t* __restrict__ split, int32_t merge_cap, int32_t* __restrict__ ccol,
    double* __restrict__ cval, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char win_smem[];
  double* vals = reinterpret_cast<double*>(win_smem);
  uint32_t* bm = reinterpret_cast<uint32_t*>(win_smem + kSmemVals);
  uint16_t* pre = reinterpret_cast<uint16_t*>(win_smem + kSmemVals + kSmemBits);
  int32_t* grp = reinterpret_cast<int32_t*>(win_smem + kSmemVals + kSmemBits + kSmemPre);
  unsigned char* ent = win_smem + kSmemVals + kSmemBits + kSmemPre + kSmemGrp;
  int64_t* e_rs = reinterpret_cast<int64_t*>(ent);                 // B row start
  double* e_av = reinterpret_cast<double*>(e_rs + kNumThreads);    // a_ik
  int64_t* e_bs = reinterpret_cast<int64_t*>(e_av + kNumThreads);  // window segment start
  int32_t* e_k = reinterpret_cast<int32_t*>(e_bs + kNumThreads);   // B row number
  int32_t* e_excl = e_k + kNumThreads;                              // segment prefix
  uint16_t* s_cnt = reinterpret_cast<uint16_t*>(e_excl + kNumThreads);
  __shared__ int32_t s_scan32[33];
  __shared__ int32_t s_ctl[6];
  const int64_t n = B.cols;
  const double* av_ = static_cast<const double*>(A.val);
  const double* bv_ = static_cast<const double*>(B.val);
  const bool cnt_cached = nblocks <= kCntCache;

  for (int t = threadIdx.x; t < (kSmemVals + kSmemBits) / 16; t += kNumThreads)
    reinterpret_cast<uint4*>(win_smem)[t] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) s_ctl[0] = atomicAdd(counter, 1);
    __syncthreads();
    const int64_t idx = s_ctl[0];
    if (idx >= count) break;
    const int32_t i = perm[idx];
    const int64_t slot = win_slot[i];
    if (slot < 0 || slot >= nslots) {      // the row was not counted by the windowed symbolic pass
      if (threadIdx.x == 0) set_error(err, kErrWindowPlan);
      __syncthreads();
      continue;
    }
    const uint16_t* gcnt = blockcnt + slot * nblocks;
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    const bool resident = na <= kNumThreads;
    if (cnt_cached)
      for (int64_t b = threadIdx.x; b < nblocks; b += kNumThreads) s_cnt[b] = gcnt[b];
    if (resident && threadIdx.x < na) {
      const int32_t k = A.col[a0 + threadIdx.x];
      e_k[threadIdx.x] = k;
      e_rs[threadIdx.x] = B.rp[k];
      e_av[threadIdx.x] = av_[a0 + threadIdx.x];
    }
    const uint16_t* cnts = cnt_cached ? s_cnt : gcnt;
    int64_t out = c_off[i];
    const int64_t out_end = c_off[i + 1];
    int64_t next_b = 0;   // meaningful in thread 0 only
    __syncthreads();
    for (;;) {
      if (threadIdx.x == 0) {
        int64_t b = next_b;
        while (b < nblocks && cnts[b] == 0) ++b;
        if (b >= nblocks) {
          s_ctl[1] = 0;
        } else {
          int64_t e = b;
          int32_t sum = 0;
          do { sum += cnts[e]; ++e; }
          while (e < nblocks && e - b < kSpanBlocks && sum + cnts[e] <= merge_cap);
          s_ctl[1] = 1; s_ctl[2] = static_cast<int32_t>(b); s_ctl[3] = static_cast<int32_t>(e);
          s_ctl[4] = sum;
          next_b = e;
        }
      }
      __syncthreads();
      if (s_ctl[1] == 0) break;
      const int64_t b0 = s_ctl[2], b1 = s_ctl[3];
      const int64_t w0 = b0 * kBlockCols;
      const int64_t w1 = b1 * kBlockCols < n ? b1 * kBlockCols : n;
      const int32_t expect = s_ctl[4];
      const int nwords = static_cast<int>((w1 - w0 + 31) >> 5);

      // pass 1: mark the window's columns
      int32_t p1_total = 0;   // products of the (single) chunk, reused by pass 2 when na fits one chunk
      for (int64_t base = 0; base < na; base += kNumThreads) {
        const int64_t e = base + threadIdx.x;
        Seg sg{0, 0};
        if (e < na) sg = entry_segment(A, B, split, nblocks, a0, e, resident, e_k, e_rs, e_av, b0, b1, w0, w1);
        int32_t total;
        const int32_t ex = block_excl_scan<int32_t>(sg.len, s_scan32, &total);
        e_excl[threadIdx.x] = ex;
        e_bs[threadIdx.x] = sg.bs;
        p1_total = total;
        const int nvalid = static_cast<int>(na - base < kNumThreads ? na - base : kNumThreads);
        __syncthreads();
        int owner = 0;
        for (int32_t p = threadIdx.x; p < total; p += kNumThreads) {
          owner = find_owner(e_excl, nvalid, p, owner);
          const int32_t c = B.col[e_bs[owner] + (p - e_excl[owner])];
          const int64_t rel = c - w0;
          if (rel >= 0 && rel < w1 - w0) atomicOr(&bm[rel >> 5], 1u << (rel & 31));
          else set_error(err, kErrWindowPlan);
        }
        if (na > kNumThreads) __syncthreads();
      }
      __syncthreads();
      // rank prefix: each thread owns kWordsPerThread consecutive words of one group
      {
        const int wlo = threadIdx.x * kWordsPerThread;
        int c = 0;
#pragma unroll
        for (int t = 0; t < kWordsPerThread; ++t) c += __popc(bm[wlo + t]);
        int32_t tot;
        const int32_t tpre = block_excl_scan<int32_t>(c, s_scan32, &tot);
        constexpr int kThreadsPerGroup = kGroupWords / kWordsPerThread;
        const int lead = (threadIdx.x & 31) & ~(kThreadsPerGroup - 1);
        const int32_t gbase = __shfl_sync(0xffffffffu, tpre, lead);
        if ((threadIdx.x & (kThreadsPerGroup - 1)) == 0) grp[wlo / kGroupWords] = gbase;
        int run = tpre - gbase;
#pragma unroll
        for (int t = 0; t < kWordsPerThread; ++t) {
          pre[wlo + t] = static_cast<uint16_t>(run);
          run += __popc(bm[wlo + t]);
        }
        if (threadIdx.x == 0) s_ctl[5] = tot;
      }
      __syncthreads();
      const int32_t cnt = s_ctl[5];
      if (threadIdx.x == 0 && cnt != expect) set_error(err, kErrCount);
      // pass 2: accumulate by rank
      for (int64_t base = 0; base < na; base += kNumThreads) {
        int32_t total;
        if (na > kNumThreads) {
          const int64_t e = base + threadIdx.x;
          Seg sg{0, 0};
          if (e < na) sg = entry_segment(A, B, split, nblocks, a0, e, resident, e_k, e_rs, e_av, b0, b1, w0, w1);
          const int32_t ex = block_excl_scan<int32_t>(sg.len, s_scan32, &total);
          e_excl[threadIdx.x] = ex;
          e_bs[threadIdx.x] = sg.bs;
          __syncthreads();
        } else {
          total = p1_total;   // the single chunk's state from pass 1 is still in shared memory
        }
        const int nvalid = static_cast<int>(na - base < kNumThreads ? na - base : kNumThreads);
        int owner = 0;
        for (int32_t p = threadIdx.x; p < total; p += 2 * kNumThreads) {
          const int o1 = find_owner(e_excl, nvalid, p, owner);
          const int64_t j1 = e_bs[o1] + (p - e_excl[o1]);
          const int32_t p2 = p + kNumThreads;
          const bool two = p2 < total;
          const int o2 = two ? find_owner(e_excl, nvalid, p2, o1) : o1;
          const int64_t j2 = e_bs[o2] + (p2 - e_excl[o2]);
          const int32_t c1 = B.col[j1];
          const double v1 = e_av[o1] * bv_[j1];
          int32_t c2 = 0;
          double v2 = 0.0;
          if (two) { c2 = B.col[j2]; v2 = e_av[o2] * bv_[j2]; }
          {
            const int32_t rel = static_cast<int32_t>(c1 - w0);
            if (rel >= 0 && rel < (int32_t)(w1 - w0)) {
              const int wd = rel >> 5;
              const int r = grp[wd / kGroupWords] + pre[wd] + __popc(bm[wd] & ((1u << (rel & 31)) - 1u));
              if (r < kRankCap) atomicAdd(&vals[r], v1);
            }
          }
          if (two) {
            const int32_t rel = static_cast<int32_t>(c2 - w0);
            if (rel >= 0 && rel < (int32_t)(w1 - w0)) {
              const int wd = rel >> 5;
              const int r = grp[wd / kGroupWords] + pre[wd] + __popc(bm[wd] & ((1u << (rel & 31)) - 1u));
              if (r < kRankCap) atomicAdd(&vals[r], v2);
            }
          }
          owner = o2;
        }
        if (na > kNumThreads) __syncthreads();
      }
      __syncthreads();
      // emit: values by rank (coalesced), columns from the bitmap
      for (int r = threadIdx.x; r < cnt && r < kRankCap; r += kNumThreads) {
        if (out + r < out_end) cval[out + r] = vals[r];
        vals[r] = 0.0;
      }
      {
        const int wlo = threadIdx.x * kWordsPerThread;
        if (wlo < nwords) {
          int r = grp[wlo / kGroupWords] + pre[wlo];
#pragma unroll
          for (int t = 0; t < kWordsPerThread; ++t) {
            uint32_t m = bm[wlo + t];
            if (!m) continue;
            bm[wlo + t] = 0u;
            for (; m; m &= m - 1) {
              if (out + r < out_end) ccol[out + r] = static_cast<int32_t>(w0 + (wlo + t) * 32 + (__ffs(m) - 1));
              ++r;
            }
          }
        }
      }
      out += cnt;
      __syncthreads();
    }
    if (threadIdx.x == 0 && out != out_end) set_error(err, kErrCount);
  }
}

}  // namespace

int64_t split_table_bytes(int64_t brows, int64_t nblocks) { return brows * (nblocks + 1) * 4; }

int launch_bsplit(const DevCsr& B, int64_t nblocks, int32_t* split, cudaStream_t s) {
  if (B.rows <= 0) return 0;
  int64_t g = (B.rows * 32 + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  k_bsplit<<<static_cast<unsigned>(g), 256, 0, s>>>(B, nblocks, split);
  return 1;
}

int launch_num_window(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                      int32_t* counter, const int64_t* c_off, const int32_t* win_slot,
                      const uint16_t* blockcnt, int64_t nblocks, int64_t nslots, const int32_t* split,
                      int32_t hash_fill, int32_t* ccol, double* cval, int num_sms, uint32_t* err,
                      cudaStream_t s) {
  if (count <= 0) return 0;
  cudaFuncSetAttribute(k_num_window, cudaFuncAttributeMaxDynamicSharedMemorySize, kWinSmemBytes);
  cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  const int64_t g = count < num_sms ? count : num_sms;
  k_num_window<<<static_cast<unsigned>(g), kNumThreads, kWinSmemBytes, s>>>(
      A, B, perm, count, counter, c_off, win_slot, blockcnt, nblocks, nslots, split, hash_fill, ccol, cval,
      err);
  return 1;
}

}  // namespace spg
