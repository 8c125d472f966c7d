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
// FP64 sums are accumulated with FP64 shared-memory atomics (kModeF64, the order of the additions
// may vary from run to run) or, on request, exactly in integer fixed point (kModeF64X, see
// common.cuh): a value then does not depend on the order of its terms and repeats bit for bit; a
// row whose products span too wide a range takes kModeF64 afterwards. The pattern is always exact.
#include "enumerate.cuh"

namespace spg {

namespace {

constexpr int kRankCap = 4096;                     // entries of C per window (>= kBlockCols)
constexpr int kNumThreads = 512;                   // threads of the windowed numeric kernel
constexpr int kCntCache = 1024;                    // block counts kept in shared memory
constexpr int kMaxWin = 256;                       // windows planned per batch
constexpr int kUnroll = 4;                         // partial products in flight per thread
// per entry: B row start, a_ik, B row number; per non-empty segment: start, prefix, entry
constexpr int kSmemEnt = kNumThreads * (8 + 8 + 4) + kNumThreads * (8 + 4 + 4) + 16;
// Per rank the windowed kernel keeps an FP64 sum (kModeF64, kModeF32R), in kModeF32C an FP32
// sum, its compensation, sum|p| and the term count, and in kModeF64X four 32-bit fixed-point
// limbs. A window spans at most kSpanBlocks blocks: 64 (256K columns) with 8 bytes per rank, 32
// with 16, so that two blocks fit on an SM in every mode.
template <int Mode>
struct WinGeom {
  static constexpr bool kWide = Mode == kModeF32C || Mode == kModeF64X;
  static constexpr int kSpanBlocks = kWide ? 32 : 64;
  static constexpr int kSpanWords = kSpanBlocks * kBlockWords;   // bitmap words
  static constexpr int kWordsPerThread = kSpanWords / kNumThreads;
  static constexpr int kSmemBits = kSpanWords * 4;
  static constexpr int kSmemPre = kSpanWords * 2;
  static constexpr int kValBytes = kWide ? 16 : 8;
  static constexpr int kSmemVals = kRankCap * kValBytes;
  static constexpr int kSmemBytes = kSmemVals + kSmemBits + kSmemPre + kSmemEnt + kCntCache * 2 + kMaxWin * 12 +
                                    (kMaxWin + 1) * 4;
  static_assert(kSmemPre >= 2 * kMaxWin * 4, "the list counters fit the rank bases' space");
  static constexpr int kBlocksPerSm = 2;
  static_assert(kWordsPerThread * kNumThreads == kSpanWords, "words per thread");
  static_assert(kWordsPerThread % 4 == 0, "a thread's words are copied as 16-byte vectors");
  static_assert(kSmemVals % 16 == 0, "vector clearing of the values");
  static_assert(2 * (kSmemBytes + 1024 + 512) <= 228 * 1024, "two blocks per SM");
};
static_assert(kRankCap >= kBlockCols, "a window must hold any single block");


// Split table: one warp per row k of B writes split[k * (nblocks + 1) + b] for b in
// [0, nblocks]: the offset within row k of its first entry with column >= b * kBlockCols.
__global__ void __launch_bounds__(256) k_bsplit(DevCsr B, int64_t nblocks, const int32_t* __restrict__ bbase,
                                                int32_t* __restrict__ split) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  constexpr int kShift = kBlockShift;
  for (int64_t k = gw; k < B.rows; k += nw) {
    const int64_t s = B.rp[k];
    const int32_t len = static_cast<int32_t>(B.rp[k + 1] - s);
    const int64_t bb = bbase ? bbase[k] : 0;   // blocks are counted from the row's first column
    int32_t* out = split + k * (nblocks + 1);
    if (len == 0) {
      for (int64_t b = lane; b <= nblocks; b += 32) out[b] = 0;
      continue;
    }
    for (int32_t t0 = 0; t0 < len; t0 += 32) {
      const int32_t t = t0 + lane;
      if (t < len) {
        const int64_t bc = (B.col[s + t] - bb) >> kShift;
        const int64_t bp = t == 0 ? -1 : ((B.col[s + t - 1] - bb) >> kShift);
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

// Shared layout (dynamic): rank-indexed FP64 values [kRankCap] (also the staging buffer of
// the window's columns during the write-out); window bitmap [kSpanWords]; in-group word prefix
// (uint16) [kSpanWords]; group prefix (int32) [kSpanWords / 64]; per-entry state of the current
// chunk of A entries (B row start, a_ik, B row number); the chunk's non-empty segments in the
// window (start in B, product prefix, entry); the row's block counts; the planned windows (first
// block, end block, entries). The values and the bitmap are all zero between windows. A row whose
// A entries fit one chunk keeps its entry state across all its windows.
//
// Each chunk's partial products are split into one contiguous range per warp; a warp walks its
// range 32 products at a time (lane l takes product p0 + l), finding the lanes' segments with
// group_owner, so loads of B are coalesced along each segment.
template <int Mode>
__global__ void __launch_bounds__(kNumThreads, WinGeom<Mode>::kBlocksPerSm) k_num_window(
    DevCsr A, DevCsr B, const int32_t* __restrict__ perm, int64_t count, int32_t* counter,
    const int64_t* __restrict__ c_off, const int32_t* __restrict__ win_slot,
    const uint16_t* __restrict__ blockcnt, int64_t nblocks, int64_t nslots,
    const int32_t* __restrict__ split, int32_t merge_cap, int32_t* __restrict__ ccol,
    void* __restrict__ cval_, int32_t* __restrict__ row_flag, const int32_t* __restrict__ abase,
    const int32_t* __restrict__ awidth, int64_t width_all, const uint32_t* __restrict__ wbits,
    const int64_t* __restrict__ woff, const uint16_t* __restrict__ bexp, const int32_t* __restrict__ dev_count,
    const int32_t* __restrict__ negflag, int64_t* __restrict__ list_bs, int32_t* __restrict__ list_len,
    double* __restrict__ list_av, int64_t list_cap, uint32_t* err) {
  using G = WinGeom<Mode>;
  constexpr int kSmemBits = G::kSmemBits;
  constexpr int kSmemPre = G::kSmemPre;
  constexpr int kSpanBlocks = G::kSpanBlocks;
  constexpr int kWordsPerThread = G::kWordsPerThread;
  constexpr int kSmemVals = WinGeom<Mode>::kSmemVals;
  extern __shared__ __align__(16) unsigned char win_smem[];
  double* vals = reinterpret_cast<double*>(win_smem);        // kModeF64, kModeF32R
  float* f_s = reinterpret_cast<float*>(win_smem);            // kModeF32C: sum,
  float* f_c = f_s + kRankCap;                                //   compensation,
  float* f_m = f_c + kRankCap;                                //   sum |p|,
  int32_t* f_t = reinterpret_cast<int32_t*>(f_m + kRankCap);  //   term count
  uint32_t* x_l0 = reinterpret_cast<uint32_t*>(win_smem);     // kModeF64X: low limbs,
  uint32_t* x_l1 = x_l0 + kRankCap;
  uint32_t* x_l2 = x_l1 + kRankCap;
  int32_t* x_lt = reinterpret_cast<int32_t*>(x_l2 + kRankCap); //   signed top limb
  int32_t* colbuf = reinterpret_cast<int32_t*>(win_smem);
  uint32_t* bm = reinterpret_cast<uint32_t*>(win_smem + kSmemVals);
  uint16_t* pre = reinterpret_cast<uint16_t*>(win_smem + kSmemVals + kSmemBits);   // rank base of each word
  unsigned char* ent = win_smem + kSmemVals + kSmemBits + kSmemPre;
  int64_t* e_rs = reinterpret_cast<int64_t*>(ent);                 // B row start
  double* e_av = reinterpret_cast<double*>(e_rs + kNumThreads);    // a_ik
  int64_t* c_bs = reinterpret_cast<int64_t*>(e_av + kNumThreads);  // segment start in B
  int32_t* e_k = reinterpret_cast<int32_t*>(c_bs + kNumThreads);   // B row number
  int32_t* c_ent = e_k + kNumThreads;                               // segment's entry (chunk slot)
  int32_t* c_excl = c_ent + kNumThreads;                            // segment product prefix [+1]
  uint16_t* s_cnt = reinterpret_cast<uint16_t*>(c_excl + kNumThreads + 4);
  int32_t* w_b0 = reinterpret_cast<int32_t*>(s_cnt + kCntCache);
  int32_t* w_b1 = w_b0 + kMaxWin;
  int32_t* w_cnt = w_b1 + kMaxWin;
  int32_t* w_loff = w_cnt + kMaxWin;    // a long row's window list offsets (kMaxWin + 1)
  __shared__ long long s_scan64[33];
  __shared__ int32_t s_scan32[33];
  __shared__ int32_t s_ctl[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int kWarps = kNumThreads / 32;
  const double* av64 = static_cast<const double*>(A.val);
  const double* bv64 = static_cast<const double*>(B.val);
  const float* av32 = static_cast<const float*>(A.val);
  const float* bv32 = static_cast<const float*>(B.val);
  auto a_at = [&](int64_t q) -> double {
    return (Mode == kModeF64 || Mode == kModeF64X) ? av64[q] : static_cast<double>(av32[q]);
  };
  const bool cnt_cached = nblocks <= kCntCache;
  // kModeF32C: every partial product is non-negative (no value of A or B is negative), so the
  // bound needs no sum of |p| (f32c_within_count)
  const bool nonneg = Mode == kModeF32C && negflag != nullptr && *negflag == 0;
  if (dev_count) {   // the rows to redo are listed on the device
    const int64_t dc = *dev_count;
    count = dc < count ? dc : count;
  }

  for (int t = threadIdx.x; t < (kSmemVals + kSmemBits) / 16; t += kNumThreads)
    reinterpret_cast<uint4*>(win_smem)[t] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  // Compacts the non-empty window segments of chunk [base, base + kNumThreads) of the row's A
  // entries into c_bs / c_excl / c_ent; returns (segments, products) through s_ctl[6..7].
  // ps0/ps1 (when >= 0): the entry's split offsets for the window, already in registers.
  auto build_chunk = [&](int64_t a0, int64_t na, int64_t base, bool resident, int64_t b0, int64_t b1,
                         int64_t w0, int64_t w1, int32_t ps0 = -1, int32_t ps1 = -1) {
    const int64_t e = base + threadIdx.x;
    int64_t bs = 0;
    int32_t len = 0;
    if (e < na) {
      int32_t k;
      int64_t rs;
      if (resident) {
        k = e_k[threadIdx.x];
        rs = e_rs[threadIdx.x];
      } else {
        k = A.col[a0 + e];
        rs = B.rp[k];
        e_av[threadIdx.x] = a_at(a0 + e);
      }
      int32_t s0, s1;
      if (ps0 >= 0) {
        s0 = ps0;
        s1 = ps1;
      } else if (split) {
        const int32_t* sp = split + int64_t(k) * (nblocks + 1);
        s0 = sp[b0];
        s1 = sp[b1];
      } else {
        const int32_t rl = static_cast<int32_t>(B.rp[k + 1] - rs);
        s0 = lower_bound_col(B.col + rs, rl, w0);
        s1 = lower_bound_col(B.col + rs, rl, w1);
      }
      bs = rs + s0;
      len = s1 - s0;
    }
    const long long packed = (static_cast<long long>(len > 0) << 32) | static_cast<long long>(len);
    long long tot;
    const long long ex = block_excl_scan<long long>(packed, s_scan64, &tot);
    if (len > 0) {
      const int pos = static_cast<int>(ex >> 32);
      c_bs[pos] = bs;
      c_excl[pos] = static_cast<int32_t>(ex & 0xffffffffLL);
      c_ent[pos] = threadIdx.x;
    }
    if (threadIdx.x == 0) {
      const int nent = static_cast<int>(tot >> 32);
      c_excl[nent] = static_cast<int32_t>(tot & 0xffffffffLL);
      s_ctl[6] = nent;
      s_ctl[7] = static_cast<int32_t>(tot & 0xffffffffLL);
    }
    __syncthreads();
  };
  // This block's lists of a long row's window segments (list_cap entries each; none when null).
  int64_t* const l_bs = list_cap > 0 ? list_bs + int64_t(blockIdx.x) * list_cap : nullptr;
  int32_t* const l_len = list_cap > 0 ? list_len + int64_t(blockIdx.x) * list_cap : nullptr;
  double* const l_av = list_cap > 0 ? list_av + int64_t(blockIdx.x) * list_cap : nullptr;
  // Pass-2 chunk [base, base + kNumThreads) of a window's list (ending at end), compacted as
  // build_chunk does; every listed segment is non-empty.
  auto build_list_chunk = [&](int64_t base, int64_t end) {
    const int64_t q = base + threadIdx.x;
    int64_t bs = 0;
    int32_t len = 0;
    if (q < end) {
      bs = l_bs[q];
      len = l_len[q];
      e_av[threadIdx.x] = l_av[q];
    }
    const long long packed = (static_cast<long long>(len > 0) << 32) | static_cast<long long>(len);
    long long tot;
    const long long ex = block_excl_scan<long long>(packed, s_scan64, &tot);
    if (len > 0) {
      const int pos = static_cast<int>(ex >> 32);
      c_bs[pos] = bs;
      c_excl[pos] = static_cast<int32_t>(ex & 0xffffffffLL);
      c_ent[pos] = threadIdx.x;
    }
    if (threadIdx.x == 0) {
      const int nent = static_cast<int>(tot >> 32);
      c_excl[nent] = static_cast<int32_t>(tot & 0xffffffffLL);
      s_ctl[6] = nent;
      s_ctl[7] = static_cast<int32_t>(tot & 0xffffffffLL);
    }
    __syncthreads();
  };

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
    const int64_t cb = abase ? abase[i] : 0;   // the row's columns are [cb, cb + width)
    const int64_t width = awidth ? awidth[i] : width_all;
    const int64_t row_blocks = (width + kBlockCols - 1) / kBlockCols;   // counted by the symbolic pass
    const bool resident = na <= kNumThreads;
    // kModeF32C with non-negative products: an entry has at most na terms, so when na itself
    // passes the term-count bound no entry needs counting
    const bool count_terms = !nonneg || !f32c_within_count(na < (int64_t(1) << 30) ? static_cast<int>(na) : (1 << 30));
    if (cnt_cached)
      for (int64_t b = threadIdx.x; b < row_blocks; b += kNumThreads) s_cnt[b] = gcnt[b];
    if (resident && threadIdx.x < na) {
      const int32_t k = A.col[a0 + threadIdx.x];
      e_k[threadIdx.x] = k;
      e_rs[threadIdx.x] = B.rp[k];
      e_av[threadIdx.x] = a_at(a0 + threadIdx.x);
    }
    const uint16_t* cnts = cnt_cached ? s_cnt : gcnt;
    // kModeF64X: the row's fixed-point scale from its largest possible product exponent
    int fx_sh0 = 0, fx_lsb = 0;
    bool row_bad = false;   // kModeF64X: the row needs the FP64 path
    if constexpr (Mode == kModeF64X) {
      int emax = 0;
      for (int64_t q = threadIdx.x; q < na; q += kNumThreads)
        emax = max(emax, fx_exponent(av64[a0 + q]) + static_cast<int>(bexp[A.col[a0 + q]]));
      emax = __reduce_max_sync(0xffffffffu, emax);
      if (lane == 0) s_scan32[wid] = emax;
      __syncthreads();
      emax = s_scan32[0];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) emax = max(emax, s_scan32[w]);
      const int hbits = 32 - __clz(static_cast<int>(na < (int64_t(1) << 30) ? na : (int64_t(1) << 30)));
      fx_lsb = emax - 2044 - (kFxTopBits - hbits);
      fx_sh0 = 1075 + fx_lsb;
    }
    int64_t out = c_off[i];
    const int64_t out_end = c_off[i + 1];
    // the symbolic pass stored this row's column bitmap: windows copy it instead of marking
    const int64_t toff = woff ? woff[slot] : -1;
    const bool stored = toff >= 0;
    int64_t next_b = 0;   // meaningful in warp 0 only
    // Split offsets of a resident row's entry (thread t < na holds entry t): a window [b0, b1)
    // needs the entry's offsets at b0 and b1. The blocks between two windows of the row hold none
    // of its entries, so no B row it names has entries there either: the offset at the next
    // window's b0 equals this window's at b1 (sp_prev1). The offset at the next window's b1 is
    // loaded one window ahead (sp_pref), so its latency hides behind the current window.
    const int32_t* sp_row = nullptr;
    int32_t sp_prev1 = -1, sp_pref = -1;
    if (resident && split && threadIdx.x < na) sp_row = split + int64_t(e_k[threadIdx.x]) * (nblocks + 1);
    __syncthreads();
    for (;;) {
      // plan a batch of windows: runs of consecutive blocks holding <= merge_cap entries of C
      if (wid == 0) {
        int nw = 0;
        int64_t b = next_b;
        while (nw < kMaxWin) {
          bool found = false;
          while (b < row_blocks) {
            const int64_t q = b + lane;
            const unsigned m = __ballot_sync(0xffffffffu, q < row_blocks && cnts[q] != 0);
            if (m) { b += __ffs(m) - 1; found = true; break; }
            b += 32;
          }
          if (!found) { b = row_blocks; break; }
          int32_t sum = cnts[b];
          int64_t e = b + 1;
          for (;;) {
            const int64_t q = e + lane;
            const bool in = q < row_blocks && q - b < kSpanBlocks;
            int32_t incl = in ? cnts[q] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
              const int32_t v = __shfl_up_sync(0xffffffffu, incl, d);
              if (lane >= d) incl += v;
            }
            const unsigned okm = __ballot_sync(0xffffffffu, in && sum + incl <= merge_cap);
            const int run = __popc(okm);
            if (run > 0) sum += __shfl_sync(0xffffffffu, incl, run - 1);
            e += run;
            if (run < 32) break;
          }
          if (lane == 0) {
            w_b0[nw] = static_cast<int32_t>(b);
            w_b1[nw] = static_cast<int32_t>(e);
            w_cnt[nw] = sum;
          }
          ++nw;
          b = e;
        }
        next_b = b;
        if (lane == 0) s_ctl[1] = nw;
      }
      __syncthreads();
      const int nwin = s_ctl[1];
      if (nwin == 0) break;
      // A row that is not resident lists its segments per planned window once for the batch: a
      // warp takes one entry at a time and its lanes the windows, reading the entry's split
      // offsets at the windows' bounds from the entry's row of the split table (coalesced). An
      // entry with nothing in a window stays out of that window's list, so pass 2 builds chunks
      // only from what each window holds. The counters live in the rank bases' space, which
      // every window rewrites; a batch whose lists exceed list_cap keeps the chunks of A entries.
      bool listed = false;
      if (Mode != kModeF64X && !resident && split != nullptr && list_cap > 0) {
        int32_t* s_wcnt = reinterpret_cast<int32_t*>(pre);
        int32_t* s_wfill = s_wcnt + kMaxWin;
        for (int w = threadIdx.x; w < nwin; w += kNumThreads) {
          s_wcnt[w] = 0;
          s_wfill[w] = 0;
        }
        __syncthreads();
        for (int64_t e = wid; e < na; e += kWarps) {
          const int32_t* sp = split + int64_t(A.col[a0 + e]) * (nblocks + 1);
          for (int w = lane; w < nwin; w += 32)
            if (sp[w_b1[w]] > sp[w_b0[w]]) atomicAdd(&s_wcnt[w], 1);
        }
        __syncthreads();
        if (wid == 0) {
          int32_t run = 0;
          for (int wb = 0; wb < nwin; wb += 32) {
            const int w = wb + lane;
            const int32_t c = w < nwin ? s_wcnt[w] : 0;
            int32_t incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
              const int32_t v = __shfl_up_sync(0xffffffffu, incl, d);
              if (lane >= d) incl += v;
            }
            if (w < nwin) w_loff[w] = run + incl - c;
            run += __shfl_sync(0xffffffffu, incl, 31);
          }
          if (lane == 0) w_loff[nwin] = run;
        }
        __syncthreads();
        listed = w_loff[nwin] <= list_cap;
        if (listed) {
          for (int64_t e = wid; e < na; e += kWarps) {
            const int32_t k = A.col[a0 + e];
            const int32_t* sp = split + int64_t(k) * (nblocks + 1);
            const int64_t rs = B.rp[k];
            const double av = a_at(a0 + e);
            for (int w = lane; w < nwin; w += 32) {
              const int32_t s0 = sp[w_b0[w]], s1 = sp[w_b1[w]];
              if (s1 > s0) {
                const int32_t pos = w_loff[w] + atomicAdd(&s_wfill[w], 1);
                l_bs[pos] = rs + s0;
                l_len[pos] = s1 - s0;
                l_av[pos] = av;
              }
            }
          }
        }
        __syncthreads();
      }
      for (int wi = 0; wi < nwin; ++wi) {
        const int64_t b0 = w_b0[wi], b1 = w_b1[wi];
        const int64_t w0 = cb + b0 * kBlockCols;
        const int64_t w1 = cb + (b1 * kBlockCols < width ? b1 * kBlockCols : width);
        const int32_t span = static_cast<int32_t>(w1 - w0);
        const int32_t expect = w_cnt[wi];
        const int nwords = (span + 31) >> 5;
        int32_t ps0 = -1, ps1 = -1;
        if (sp_row) {
          ps0 = sp_prev1 >= 0 ? sp_prev1 : sp_row[b0];
          ps1 = sp_pref >= 0 ? sp_pref : sp_row[b1];
          sp_prev1 = ps1;
          sp_pref = wi + 1 < nwin ? sp_row[w_b1[wi + 1]] : -1;
        }

        // pass 1: mark the window's columns (a row with a stored bitmap copies it in the rank
        // prefix below instead)
        for (int64_t base = 0; base < (stored ? 0 : na); base += kNumThreads) {
          build_chunk(a0, na, base, resident, b0, b1, w0, w1, ps0, ps1);
          const int nent = s_ctl[6];
          const int32_t total = s_ctl[7];
          int32_t per = (total + kWarps - 1) / kWarps;
          per = (per + 31) & ~31;
          const int32_t lo = wid * per;
          const int32_t hi = total < lo + per ? total : lo + per;
          if (lo < hi) {
            auto walk = make_walker<int>(c_excl, c_bs, nent, search_owner(c_excl, nent, lo), [](int) { return 0; });
            for (int32_t p0 = lo; p0 < hi; p0 += 32 * kUnroll) {
              int64_t j[kUnroll];
              if (walk.whole(p0, 32 * kUnroll, hi)) {
                const int64_t j0 = walk.first(p0);
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) j[u] = j0 + 32 * u;
              } else {
                int unused[kUnroll];
                walk.template step_many<kUnroll>(p0, hi, j, unused);
              }
              int32_t c[kUnroll];
#pragma unroll
              for (int u = 0; u < kUnroll; ++u) c[u] = j[u] >= 0 ? B.col[j[u]] : -1;
#pragma unroll
              for (int u = 0; u < kUnroll; ++u) {
                if (j[u] < 0) continue;
                const int32_t rel = static_cast<int32_t>(c[u] - w0);
                if (rel >= 0 && rel < span) atomicOr(&bm[rel >> 5], 1u << (rel & 31));
                else set_error(err, kErrWindowPlan);
              }
            }
          }
          __syncthreads();
        }
        // a resident row with a stored bitmap builds its pass-2 chunk inside the rank prefix's scan
        const bool fused = stored && resident && split != nullptr;
        // rank prefix over the window's words: each thread owns kWordsPerThread consecutive
        // words of one group. A stored bitmap is read here straight into the thread's registers
        // and copied to shared memory; its window's whole blocks are stored (zero past the row's
        // width), so every word up to (b1 - b0) * kBlockWords can be read.
        {
          const int wlo = threadIdx.x * kWordsPerThread;
          const int wmine = stored ? static_cast<int>((b1 - b0) * kBlockWords) : nwords;
          const bool mine = wlo < wmine;
          uint32_t wv[kWordsPerThread];
          if (mine && stored) {
            const uint4* src = reinterpret_cast<const uint4*>(wbits + toff + b0 * kBlockWords + wlo);
#pragma unroll
            for (int q = 0; q < kWordsPerThread / 4; ++q) {
              const uint4 v = src[q];
              reinterpret_cast<uint4*>(bm + wlo)[q] = v;
              wv[4 * q] = v.x;
              wv[4 * q + 1] = v.y;
              wv[4 * q + 2] = v.z;
              wv[4 * q + 3] = v.w;
            }
          } else {
#pragma unroll
            for (int t = 0; t < kWordsPerThread; ++t) wv[t] = mine ? bm[wlo + t] : 0u;
          }
          int c = 0;
#pragma unroll
          for (int t = 0; t < kWordsPerThread; ++t) c += __popc(wv[t]);
          int32_t tot, tpre;
          if (fused) {
            // the same scan also numbers the chunk's B segments for pass 2 (whose offsets this
            // thread already holds): one 64-bit word per thread carries its segment length (bits
            // 0-31; a chunk's products fit 32 bits), whether it is non-empty (bits 32-41) and its
            // words' set bits (bits 42-60)
            int64_t bs = 0;
            int32_t len = 0;
            if (threadIdx.x < na) {
              bs = e_rs[threadIdx.x] + ps0;
              len = ps1 - ps0;
            }
            const long long packed = static_cast<long long>(static_cast<uint32_t>(len)) |
                                     (static_cast<long long>(len > 0) << 32) | (static_cast<long long>(c) << 42);
            long long ptot;
            const long long ex = block_excl_scan<long long>(packed, s_scan64, &ptot);
            tpre = static_cast<int32_t>(ex >> 42);
            tot = static_cast<int32_t>(ptot >> 42);
            if (len > 0) {
              const int pos = static_cast<int>((ex >> 32) & 0x3ff);
              c_bs[pos] = bs;
              c_excl[pos] = static_cast<int32_t>(ex & 0xffffffffLL);
              c_ent[pos] = threadIdx.x;
            }
            if (threadIdx.x == 0) {
              const int nent = static_cast<int>((ptot >> 32) & 0x3ff);
              c_excl[nent] = static_cast<int32_t>(ptot & 0xffffffffLL);
              s_ctl[6] = nent;
              s_ctl[7] = static_cast<int32_t>(ptot & 0xffffffffLL);
            }
          } else {
            tpre = block_excl_scan<int32_t>(c, s_scan32, &tot);
          }
          // each word's rank base, absolute in the window (a rank past 65,535 saturates there: any
          // rank at or beyond kRankCap is skipped alike), so a product's rank takes two shared
          // loads, its bitmap word and its base
          if (mine) {
            int run = tpre;
#pragma unroll
            for (int t = 0; t < kWordsPerThread; ++t) {
              pre[wlo + t] = static_cast<uint16_t>(run < 65535 ? run : 65535);
              run += __popc(wv[t]);
            }
          }
          if (threadIdx.x == 0) s_ctl[5] = tot;
        }
        __syncthreads();
        const int32_t cnt = s_ctl[5];
        if (threadIdx.x == 0 && cnt != expect) set_error(err, kErrCount);
        constexpr int kLineThreads = kWordsPerThread >= 32 ? 1 : 32 / kWordsPerThread;   // threads per 128 B
        if (stored && wi + 1 < nwin && (threadIdx.x & (kLineThreads - 1)) == 0) {
          // the next window's stored words (one request per 128-byte line) into L2
          const int64_t nb0 = w_b0[wi + 1], nb1 = w_b1[wi + 1];
          const int wlo = threadIdx.x * kWordsPerThread;
          if (wlo < (nb1 - nb0) * kBlockWords)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(wbits + toff + nb0 * kBlockWords + wlo));
        }
        // pass 2: accumulate a_ik * b_kj by rank
        const int64_t p2_lo = listed ? w_loff[wi] : 0, p2_hi = listed ? w_loff[wi + 1] : na;
        for (int64_t base = p2_lo; base < p2_hi; base += kNumThreads) {
          if (listed) build_list_chunk(base, p2_hi);
          else if (na > kNumThreads || (stored && !fused)) build_chunk(a0, na, base, resident, b0, b1, w0, w1, ps0, ps1);
          const int nent = s_ctl[6];    // a resident row's single chunk: from pass 1 or the prefix scan
          const int32_t total = s_ctl[7];
          int32_t per = (total + kWarps - 1) / kWarps;
          per = (per + 31) & ~31;
          const int32_t lo = wid * per;
          const int32_t hi = total < lo + per ? total : lo + per;
          if (lo < hi) {
            // each segment carries its a_ik, so a group inside one segment reads no shared memory
            auto walk = make_walker<double>(c_excl, c_bs, nent, search_owner(c_excl, nent, lo),
                                            [&](int sgm) { return e_av[c_ent[sgm]]; });
            for (int32_t p0 = lo; p0 < hi; p0 += 32 * kUnroll) {
              int64_t j[kUnroll];
              double av[kUnroll];
              if (walk.whole(p0, 32 * kUnroll, hi)) {
                const int64_t j0 = walk.first(p0);
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                  j[u] = j0 + 32 * u;
                  av[u] = walk.oval;
                }
              } else {
                walk.template step_many<kUnroll>(p0, hi, j, av);
              }
              int32_t c[kUnroll];
              double bv[kUnroll];
#pragma unroll
              for (int u = 0; u < kUnroll; ++u) {
                c[u] = j[u] >= 0 ? B.col[j[u]] : -1;
                bv[u] = j[u] >= 0 ? ((Mode == kModeF64 || Mode == kModeF64X) ? bv64[j[u]]
                                                                             : static_cast<double>(bv32[j[u]]))
                                  : 0.0;
              }
#pragma unroll
              for (int u = 0; u < kUnroll; ++u) {
                if (j[u] < 0) continue;
                const int32_t rel = static_cast<int32_t>(c[u] - w0);
                if (rel < 0 || rel >= span) continue;
                const int wd = rel >> 5;
                const uint32_t word = bm[wd];
                if (stored && !((word >> (rel & 31)) & 1u)) {   // a product outside the stored columns
                  set_error(err, kErrWindowPlan);
                  continue;
                }
                const int r = pre[wd] + __popc(word & ((1u << (rel & 31)) - 1u));
                if (r >= kRankCap) continue;
                if constexpr (Mode == kModeF32C) {
                  // error-free product a*b = ph + pl (TwoProduct with fmaf); the sum's own rounding
                  // error is rebuilt from the value atomicAdd returns (TwoSum) and, with pl, goes
                  // to the compensation term (Ogita, Rump and Oishi's Dot2, accumulated concurrently)
                  const float a = static_cast<float>(av[u]);
                  const float b = static_cast<float>(bv[u]);
                  const float ph = a * b;
                  const float pl = fmaf(a, b, -ph);
                  const float old = atomicAdd(&f_s[r], ph);
                  const float nw = old + ph;
                  const float bp = nw - old;
                  const float q = (old - (nw - bp)) + (ph - bp);
                  atomicAdd(&f_c[r], q + pl);
                  if (!nonneg) atomicAdd(&f_m[r], fabsf(ph));
                  if (count_terms) atomicAdd(&f_t[r], 1);
                } else if constexpr (Mode == kModeF64X) {
                  uint32_t c0, c1, c2;
                  int32_t ct;
                  if (!fx_split(av[u] * bv[u], fx_sh0, c0, c1, c2, ct)) row_bad = true;
                  atomicAdd(&x_l0[r], c0);
                  atomicAdd(&x_l1[r], c1);
                  atomicAdd(&x_l2[r], c2);
                  atomicAdd(&x_lt[r], ct);
                } else {
                  atomicAdd(&vals[r], av[u] * bv[u]);
                }
              }
            }
          }
          __syncthreads();
          if constexpr (Mode == kModeF64X) {
            // a row with more than one chunk of A entries: carry the low limbs before the next chunk
            if (na > kNumThreads && base + kNumThreads < na) {
              const int nr = cnt < kRankCap ? cnt : kRankCap;
              for (int r = threadIdx.x; r < nr; r += kNumThreads) {
                uint32_t l0 = x_l0[r], l1 = x_l1[r], l2 = x_l2[r];
                int32_t lt = x_lt[r];
                fx_normalise(l0, l1, l2, lt);
                x_l0[r] = l0;
                x_l1[r] = l1;
                x_l2[r] = l2;
                x_lt[r] = lt;
              }
              __syncthreads();
            }
          }
        }
        // write-out: values by rank (coalesced); then the columns, staged by rank in the value
        // array's memory (words interleaved across threads for balance), copied out coalesced
        const int ncnt = cnt < kRankCap ? cnt : kRankCap;
        if constexpr (Mode == kModeF32C) {
          bool missed = false;
          for (int r = threadIdx.x; r < ncnt; r += kNumThreads) {
            const float res = f_s[r] + f_c[r];
            if (out + r < out_end) static_cast<float*>(cval_)[out + r] = res;
            missed |= nonneg ? count_terms && !f32c_within_count(f_t[r]) : !f32c_within_bound(res, f_m[r], f_t[r]);
            f_s[r] = 0.f; f_c[r] = 0.f; f_m[r] = 0.f; f_t[r] = 0;
          }
          if (missed) row_flag[i] = 1;
        } else if constexpr (Mode == kModeF64X) {
          for (int r = threadIdx.x; r < ncnt; r += kNumThreads) {
            const double res = fx_to_double(x_l0[r], x_l1[r], x_l2[r], x_lt[r], fx_lsb, &row_bad);
            if (out + r < out_end) static_cast<double*>(cval_)[out + r] = res;
            x_l0[r] = 0u; x_l1[r] = 0u; x_l2[r] = 0u; x_lt[r] = 0;
          }
        } else {
          for (int r = threadIdx.x; r < ncnt; r += kNumThreads) {
            if (out + r < out_end) {
              if constexpr (Mode == kModeF64) static_cast<double*>(cval_)[out + r] = vals[r];
              else static_cast<float*>(cval_)[out + r] = static_cast<float>(vals[r]);
            }
            vals[r] = 0.0;
          }
        }
        __syncthreads();
        if (stored) {
          // the columns of a row with a stored bitmap are written by k_expand_cols
          for (int w = threadIdx.x; w < nwords; w += kNumThreads) bm[w] = 0u;
        } else {
          for (int w = threadIdx.x; w < nwords; w += kNumThreads) {
            uint32_t m = bm[w];
            if (!m) continue;
            bm[w] = 0u;
            int r = pre[w];
            for (; m; m &= m - 1) {
              if (r < kRankCap) colbuf[r] = static_cast<int32_t>(w0 - cb + w * 32 + (__ffs(m) - 1));
              ++r;
            }
          }
          __syncthreads();
          for (int r = threadIdx.x; r < ncnt; r += kNumThreads) {
            if (out + r < out_end) ccol[out + r] = colbuf[r];
            colbuf[r] = 0;
          }
        }
        out += cnt;
        __syncthreads();
      }
    }
    if (threadIdx.x == 0 && out != out_end) set_error(err, kErrCount);
    if (Mode == kModeF64X && row_bad) row_flag[i] = 1;
  }
}

// Columns of the windowed rows with a stored bitmap, straight from that bitmap: a warp per row
// walks the row's blocks 32 at a time (their entry counts scanned across the lanes), in groups of
// kExpandGroup consecutive blocks (lane: kExpandWords consecutive words of a group). A non-empty
// group's nonzero words are listed in shared memory with their running bit counts; its set bits
// are then cut into 32 equal runs of consecutive ranks, so that every lane extracts the same
// number of columns however the bits are spread. Each lane finds its first rank by binary search
// over the list, writes its run into a staging buffer in rank order, and the warp stores the
// buffer out contiguously, kExpandStage at a time.
constexpr int kExpandStage = 512;
constexpr int kExpandWarps = 8;
constexpr int kExpandGroup = 4;                                    // blocks per group
constexpr int kExpandGroupWords = kExpandGroup * kBlockWords;      // 512
constexpr int kExpandWords = kExpandGroupWords / 32;               // words per lane, 16

// Position of the set bit of rank r (0-based, r < popc(m)) in m: a binary search on popcounts of
// the low halves.
__device__ __forceinline__ int select_bit(uint32_t m, int r) {
  int p = 0;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const int c = __popc(m & ((1u << h) - 1u));
    if (r >= c) { r -= c; m >>= h; p += h; }
  }
  return p;
}

struct ExpandWarpSmem {
  alignas(16) int32_t stage[kExpandStage + 4];   // columns of the current run of ranks, shifted so
                                                 // that stage[p] goes to a 16-byte aligned slot p
  uint2 list[kExpandGroupWords];    // nonzero words of the group in column order, with the column
                                    // of their bit 0
  uint16_t pre[kExpandGroupWords];  // set bits before each listed word
};

__global__ void __launch_bounds__(kExpandWarps * 32, 3) k_expand_cols(const int32_t* __restrict__ perm, int64_t count,
                                                     const int32_t* __restrict__ win_slot,
                                                     const int64_t* __restrict__ woff, const uint32_t* __restrict__ wbits,
                                                     const uint16_t* __restrict__ blockcnt, int64_t nblocks,
                                                     const int64_t* __restrict__ c_off,
                                                     const int32_t* __restrict__ awidth, int64_t width_all,
                                                     int32_t* __restrict__ ccol, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char s_expand[];
  const int lane = threadIdx.x & 31;
  ExpandWarpSmem& sw = reinterpret_cast<ExpandWarpSmem*>(s_expand)[threadIdx.x >> 5];
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < count; r += nw) {
    const int32_t i = perm[r];
    const int32_t slot = win_slot[i];
    const int64_t toff = woff[slot];
    if (toff < 0) continue;   // the windowed kernel writes this row's columns
    const int64_t width = awidth ? awidth[i] : width_all;
    const int64_t nb = (width + kBlockCols - 1) / kBlockCols;
    const uint16_t* cnts = blockcnt + int64_t(slot) * nblocks;
    int64_t out = c_off[i];
    const int64_t out_end = c_off[i + 1];
    bool bad = false;
    for (int64_t b0 = 0; b0 < nb; b0 += 32) {
      const int64_t b = b0 + lane;
      const int c = b < nb ? cnts[b] : 0;
      const int incl = warp_incl_scan(c);
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      const unsigned nzb = __ballot_sync(0xffffffffu, c != 0);
      for (int g = 0; g < 32 / kExpandGroup; ++g) {
        if (((nzb >> (g * kExpandGroup)) & ((1u << kExpandGroup) - 1u)) == 0u) continue;
        const int first = g * kExpandGroup, last = first + kExpandGroup - 1;
        const int64_t base = out + __shfl_sync(0xffffffffu, incl - c, first);
        const int gcnt = __shfl_sync(0xffffffffu, incl, last) - __shfl_sync(0xffffffffu, incl - c, first);
        const int64_t gb = b0 + first;                     // the group's first block
        const int32_t col0 = static_cast<int32_t>(gb * kBlockCols);
        // the lane's words: blocks past the row's last are not the row's (read as zero)
        uint32_t wv[kExpandWords];
        if (gb + (lane * kExpandWords) / kBlockWords < nb) {
          const uint4* src = reinterpret_cast<const uint4*>(wbits + toff + gb * kBlockWords + lane * kExpandWords);
#pragma unroll
          for (int q = 0; q < kExpandWords / 4; ++q) {
            const uint4 v = src[q];
            wv[4 * q] = v.x;
            wv[4 * q + 1] = v.y;
            wv[4 * q + 2] = v.z;
            wv[4 * q + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int t = 0; t < kExpandWords; ++t) wv[t] = 0u;
        }
        // one scan gives each lane its first bit rank (low 16 bits) and list slot (high bits)
        int pc = 0, nzw = 0;
#pragma unroll
        for (int t = 0; t < kExpandWords; ++t) { pc += __popc(wv[t]); nzw += wv[t] != 0u; }
        const int packed = (nzw << 16) | pc;
        const int pincl = warp_incl_scan(packed);
        const int ptot = __shfl_sync(0xffffffffu, pincl, 31);
        const int nbits = ptot & 0xffff, nlist = ptot >> 16;
        int rk = (pincl - packed) & 0xffff, pos = (pincl - packed) >> 16;
#pragma unroll
        for (int t = 0; t < kExpandWords; ++t)
          if (wv[t]) {
            sw.list[pos] = make_uint2(wv[t], static_cast<uint32_t>(col0 + (lane * kExpandWords + t) * 32));
            sw.pre[pos] = static_cast<uint16_t>(rk);
            ++pos;
            rk += __popc(wv[t]);
          }
        if (nbits != gcnt) bad = true;
        __syncwarp();
        for (int lo = 0; lo < nbits; lo += kExpandStage) {
          const int n = nbits - lo < kExpandStage ? nbits - lo : kExpandStage;
          const int64_t g0 = base + lo;
          const int sh = static_cast<int>((reinterpret_cast<uintptr_t>(ccol + g0) >> 2) & 3u);
          // an odd run length keeps the lanes' staging writes on distinct banks
          const int q = ((n + 31) >> 5) | 1;
          const int s = lo + q * lane;
          const int e = s + q < lo + n ? s + q : lo + n;
          if (s < e) {
            int j = 0;
#pragma unroll
            for (int h = kExpandGroupWords / 2; h >= 1; h >>= 1)
              if (j + h < nlist && sw.pre[j + h] <= s) j += h;
            uint2 wj = sw.list[j];
            uint32_t m = wj.x & (0xffffffffu << select_bit(wj.x, s - sw.pre[j]));
            int32_t cb = static_cast<int32_t>(wj.y);
            for (int k = s - lo + sh; k < e - lo + sh; ++k) {
              if (m == 0u) {
                ++j;
                wj = sw.list[j];
                m = wj.x;
                cb = static_cast<int32_t>(wj.y);
              }
              sw.stage[k] = cb + __ffs(m) - 1;
              m &= m - 1;
            }
          }
          __syncwarp();
          // stage[p] -> dst[p] for p in [sh, pend): whole 16-byte slots as one vector store
          int lim = n;
          if (out_end - g0 < lim) lim = out_end - g0 < 0 ? 0 : static_cast<int>(out_end - g0);
          const int pend = sh + lim;
          int32_t* dst = ccol + (g0 - sh);
          for (int v = lane; v * 4 < pend; v += 32) {
            const int p0 = v * 4;
            if (p0 >= sh && p0 + 4 <= pend) {
              reinterpret_cast<int4*>(dst)[v] = reinterpret_cast<const int4*>(sw.stage)[v];
            } else {
              for (int p = p0 > sh ? p0 : sh; p < p0 + 4 && p < pend; ++p) dst[p] = sw.stage[p];
            }
          }
          __syncwarp();
        }
        __syncwarp();
      }
      out += tot;
    }
    if (lane == 0 && (out != out_end || bad)) set_error(err, kErrCount);
  }
}

}  // namespace

int launch_expand_cols(const int32_t* perm, int64_t count, const int32_t* win_slot, const int64_t* woff,
                       const uint32_t* wbits, const uint16_t* blockcnt, int64_t nblocks, const int64_t* c_off,
                       const int32_t* awidth, int64_t width, int32_t* ccol, int num_sms, uint32_t* err,
                       cudaStream_t s) {
  if (count <= 0 || !wbits) return 0;
  constexpr int smem = kExpandWarps * static_cast<int>(sizeof(ExpandWarpSmem));
  cudaFuncSetAttribute(k_expand_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int64_t g = (count + kExpandWarps - 1) / kExpandWarps;
  if (g > int64_t(num_sms) * 16) g = int64_t(num_sms) * 16;
  k_expand_cols<<<static_cast<unsigned>(g), kExpandWarps * 32, smem, s>>>(perm, count, win_slot, woff, wbits, blockcnt, nblocks, c_off,
                                                       awidth, width, ccol, err);
  return 1;
}

int64_t split_table_bytes(int64_t brows, int64_t nblocks) { return brows * (nblocks + 1) * 4; }

int launch_bsplit(const DevCsr& B, int64_t nblocks, const int32_t* bbase, int32_t* split, cudaStream_t s) {
  if (B.rows <= 0) return 0;
  int64_t g = (B.rows * 32 + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  k_bsplit<<<static_cast<unsigned>(g), 256, 0, s>>>(B, nblocks, bbase, split);
  return 1;
}

int64_t num_window_blocks(int64_t count, int num_sms) {
  return count < int64_t(2) * num_sms ? count : int64_t(2) * num_sms;
}

int launch_num_window(int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                      int32_t* counter, const int64_t* c_off, const int32_t* win_slot,
                      const uint16_t* blockcnt, int64_t nblocks, int64_t nslots, const int32_t* split,
                      int32_t merge_cap, int32_t* ccol, void* cval, int32_t* row_flag,
                      const int32_t* abase, const int32_t* awidth, int64_t width, const uint32_t* wbits,
                      const int64_t* woff, const uint16_t* bexp, const int32_t* dev_count,
                      const int32_t* negflag, int64_t* list_bs, int32_t* list_len, double* list_av,
                      int64_t list_cap, int num_sms, uint32_t* err, cudaStream_t s) {
  if (count <= 0) return 0;
  cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  auto go = [&](auto kernel, int smem, int per_sm) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int64_t g = count < int64_t(per_sm) * num_sms ? count : int64_t(per_sm) * num_sms;
    kernel<<<static_cast<unsigned>(g), kNumThreads, smem, s>>>(A, B, perm, count, counter, c_off, win_slot,
                                                               blockcnt, nblocks, nslots, split, merge_cap,
                                                               ccol, cval, row_flag, abase, awidth, width, wbits,
                                                               woff, bexp, dev_count, negflag, list_bs, list_len,
                                                               list_av, list_cap, err);
  };
  if (mode == kModeF32C) go(k_num_window<kModeF32C>, WinGeom<kModeF32C>::kSmemBytes, 2);
  else if (mode == kModeF32R) go(k_num_window<kModeF32R>, WinGeom<kModeF32R>::kSmemBytes, 2);
  else if (mode == kModeF64X) go(k_num_window<kModeF64X>, WinGeom<kModeF64X>::kSmemBytes, 2);
  else go(k_num_window<kModeF64>, WinGeom<kModeF64>::kSmemBytes, 2);
  return 1;
}

// flag = 1 if any of the n FP32 values is negative, infinite or NaN (the flag starts at 0).
__global__ void __launch_bounds__(256) k_any_negative(const uint32_t* __restrict__ v, int64_t n,
                                                      int32_t* __restrict__ flag) {
  bool neg = false;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t x = v[i];
    neg |= (x & 0x80000000u) != 0u || (x & 0x7fffffffu) >= 0x7f800000u;   // also infinities
  }
  if (__any_sync(0xffffffffu, neg) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

int launch_negative_check(const void* a, int64_t na, const void* b, int64_t nb, int32_t* flag, int num_sms,
                          cudaStream_t s) {
  cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
  int nl = 0;
  for (int t = 0; t < 2; ++t) {
    const int64_t n = t == 0 ? na : nb;
    if (n <= 0) continue;
    int64_t g = (n + 255) / 256;
    if (g > int64_t(num_sms) * 8) g = int64_t(num_sms) * 8;
    k_any_negative<<<static_cast<unsigned>(g), 256, 0, s>>>(static_cast<const uint32_t*>(t == 0 ? a : b), n, flag);
    ++nl;
  }
  return nl;
}

// Largest biased exponent of the values of every row of B (0 for an empty row): a warp per row.
__global__ void __launch_bounds__(256) k_brow_exponent(DevCsr B, uint16_t* __restrict__ bexp) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const double* bv = static_cast<const double*>(B.val);
  for (int64_t k = gw; k < B.rows; k += nw) {
    int e = 0;
    for (int64_t q = B.rp[k] + lane; q < B.rp[k + 1]; q += 32) e = max(e, fx_exponent(bv[q]));
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) bexp[k] = static_cast<uint16_t>(e);
  }
}

int launch_brow_exponent(const DevCsr& B, uint16_t* bexp, int num_sms, cudaStream_t s) {
  if (B.rows <= 0) return 0;
  int64_t g = (B.rows * 32 + 255) / 256;
  if (g > int64_t(num_sms) * 16) g = int64_t(num_sms) * 16;
  k_brow_exponent<<<static_cast<unsigned>(g), 256, 0, s>>>(B, bexp);
  return 1;
}

}  // namespace spg
