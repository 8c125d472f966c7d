// Windowed numeric pass for rows with more entries of C than a block-wide hash table holds,
// and the column-block split table of B it reads.
//
// The columns of C are cut into blocks of kBlockCols. The symbolic pass counted, for each
// windowed row, the entries of C_i in every block. The numeric pass takes the blocks of a
// row in column order and groups them into windows:
//  * a block holding more than `hash_fill` entries is a dense window: an FP64 array indexed
//    by column minus the window start, plus a bitmap of the columns that received a
//    partial product;
//  * a run of consecutive blocks holding at most `hash_fill` entries together is a hash
//    window: a hash table (column -> FP64 sum) of kHashWinSlots slots; at the end its keys
//    are marked in a bitmap of the window's columns.
// Reading the bitmap word by word gives the row's columns in ascending order, so no sort is
// needed (Algorithm 1 sorts the partial products of a row and emits one entry per column of
// COLB, Sec. III-A; here the order comes from the bitmap).
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

constexpr int kWinRegionBytes = kBlockCols * 8;                   // dense FP64 window
constexpr int kWinBitmapWords = kHashWinBlocks * kBlockWords;     // hash window bitmap
constexpr int kWinEntBytes = kWinThreads * (8 + 8 + 4);           // per-entry chunk state
constexpr int kWinSmemBytes = kWinRegionBytes + kWinBitmapWords * 4 + kWinEntBytes;
constexpr int kHashWinLog2 = 13;
static_assert((1 << kHashWinLog2) == kHashWinSlots, "hash window size");
static_assert(kHashWinSlots * 12 <= kWinRegionBytes, "hash window fits the region");
static_assert(kWinSmemBytes <= 227 * 1024, "shared memory budget");

enum : int { kWinDone = 0, kWinDense = 1, kWinHash = 2 };

// Split table: one warp per row k of B writes split[k * (nblocks + 1) + b] for b in
// [0, nblocks]: the offset within row k of its first entry with column >= b * kBlockCols.
__global__ void __launch_bounds__(256) k_bsplit(DevCsr B, int64_t nblocks, int32_t* __restrict__ split) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  constexpr int kShift = 14;
  static_assert((1 << kShift) == kBlockCols, "block width");
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

__device__ __forceinline__ void win_accumulate(int wtype, double* dense, int32_t* hkeys, double* hvals,
                                               uint32_t* bm, int64_t w0, int64_t w1, int32_t c, double v,
                                               uint32_t* err) {
  if (c < w0 || c >= w1) {        // cannot happen with a consistent split table
    set_error(err, kErrWindowPlan);
    return;
  }
  const int32_t rel = static_cast<int32_t>(c - w0);
  if (wtype == kWinDense) {
    atomicAdd(&dense[rel], v);
    atomicOr(&bm[rel >> 5], 1u << (rel & 31));
  } else {
    const int32_t key = c + 1;
    uint32_t h = hash_slot(key, kHashWinLog2);
    for (int probe = 0; probe < kHashWinSlots; ++probe) {
      const int32_t cur = *reinterpret_cast<volatile int32_t*>(&hkeys[h]);
      if (cur == key) { atomicAdd(&hvals[h], v); return; }
      if (cur == 0) {
        const int32_t old = atomicCAS(&hkeys[h], 0, key);
        if (old == 0 || old == key) { atomicAdd(&hvals[h], v); return; }
      }
      h = (h + 1) & (kHashWinSlots - 1);
    }
    set_error(err, kErrHashFull);
  }
}

// Shared layout (dynamic): [0, 128 KB): dense FP64[kBlockCols] | hash {keys int32[8192] at 0,
// vals FP64[8192] at 32 KB}; the window bitmap; the chunk's per-entry state. Hash keys are
// stored as column + 1 so that all-zero bytes are the clean state of both layouts.
__global__ void __launch_bounds__(kWinThreads, 1) k_num_window(
    DevCsr A, DevCsr B, const int32_t* __restrict__ perm, int64_t count, int32_t* counter,
    const int64_t* __restrict__ c_off, const int32_t* __restrict__ win_slot,
    const uint16_t* __restrict__ blockcnt, int64_t nblocks, int64_t nslots,
    const int32_t* __restrict__ split, int32_t hash_fill, int32_t* __restrict__ ccol,
    double* __restrict__ cval, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char win_smem[];
  double* dense = reinterpret_cast<double*>(win_smem);
  int32_t* hkeys = reinterpret_cast<int32_t*>(win_smem);
  double* hvals = reinterpret_cast<double*>(win_smem + kHashWinSlots * 4);
  uint32_t* bm = reinterpret_cast<uint32_t*>(win_smem + kWinRegionBytes);
  int64_t* e_bs = reinterpret_cast<int64_t*>(win_smem + kWinRegionBytes + kWinBitmapWords * 4);
  double* e_av = reinterpret_cast<double*>(e_bs + kWinThreads);
  int32_t* e_excl = reinterpret_cast<int32_t*>(e_av + kWinThreads);
  __shared__ int64_t s_scan64[33];
  __shared__ int32_t s_scan32[33];
  __shared__ int32_t s_ctl[6];
  const int64_t n = B.cols;
  const double* av_ = static_cast<const double*>(A.val);
  const double* bv_ = static_cast<const double*>(B.val);
  constexpr int kClearBytes = kWinRegionBytes + kWinBitmapWords * 4;

  for (int t = threadIdx.x; t < kClearBytes / 16; t += kWinThreads)
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
    const uint16_t* cnts = blockcnt + slot * nblocks;
    const int64_t a0 = A.rp[i];
    const int64_t na = A.rp[i + 1] - a0;
    int64_t out = c_off[i];
    const int64_t out_end = c_off[i + 1];
    int64_t next_b = 0;   // meaningful in thread 0 only
    for (;;) {
      if (threadIdx.x == 0) {
        int64_t b = next_b;
        while (b < nblocks && cnts[b] == 0) ++b;
        if (b >= nblocks) {
          s_ctl[1] = kWinDone;
        } else if (cnts[b] > hash_fill) {
          s_ctl[1] = kWinDense; s_ctl[2] = static_cast<int32_t>(b); s_ctl[3] = static_cast<int32_t>(b + 1);
          s_ctl[4] = cnts[b];
          next_b = b + 1;
        } else {
          int64_t e = b;
          int32_t sum = 0;
          while (e < nblocks && e - b < kHashWinBlocks && sum + cnts[e] <= hash_fill) { sum += cnts[e]; ++e; }
          s_ctl[1] = kWinHash; s_ctl[2] = static_cast<int32_t>(b); s_ctl[3] = static_cast<int32_t>(e);
          s_ctl[4] = sum;
          next_b = e;
        }
      }
      __syncthreads();
      const int wtype = s_ctl[1];
      if (wtype == kWinDone) break;
      const int64_t b0 = s_ctl[2], b1 = s_ctl[3];
      const int64_t w0 = b0 * kBlockCols;
      const int64_t w1 = b1 * kBlockCols < n ? b1 * kBlockCols : n;
      const int32_t expect = s_ctl[4];
      // accumulate, one chunk of A entries at a time
      for (int64_t base = 0; base < na; base += kWinThreads) {
        const int64_t e = base + threadIdx.x;
        int32_t len = 0;
        int64_t bs = 0;
        double av = 0.0;
        if (e < na) {
          const int32_t k = A.col[a0 + e];
          const int64_t rs = B.rp[k];
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
          len = s1 - s0;
          bs = rs + s0;
          av = av_[a0 + e];
        }
        int32_t total;
        const int32_t ex = block_excl_scan<int32_t>(len, s_scan32, &total);
        e_excl[threadIdx.x] = ex;
        e_bs[threadIdx.x] = bs;
        e_av[threadIdx.x] = av;
        const int nvalid = static_cast<int>(na - base < kWinThreads ? na - base : kWinThreads);
        __syncthreads();
        int owner = 0;
        for (int32_t p = threadIdx.x; p < total; p += 2 * kWinThreads) {
          const int o1 = find_owner(e_excl, nvalid, p, owner);
          const int64_t j1 = e_bs[o1] + (p - e_excl[o1]);
          const int32_t p2 = p + kWinThreads;
          const bool two = p2 < total;
          const int o2 = two ? find_owner(e_excl, nvalid, p2, o1) : o1;
          const int64_t j2 = e_bs[o2] + (p2 - e_excl[o2]);
          const int32_t c1 = B.col[j1];
          const double b1v = bv_[j1];
          int32_t c2 = 0;
          double b2v = 0.0;
          if (two) { c2 = B.col[j2]; b2v = bv_[j2]; }
          win_accumulate(wtype, dense, hkeys, hvals, bm, w0, w1, c1, e_av[o1] * b1v, err);
          if (two) win_accumulate(wtype, dense, hkeys, hvals, bm, w0, w1, c2, e_av[o2] * b2v, err);
          owner = o2;
        }
        __syncthreads();
      }
      int64_t tot = 0;
      if (wtype == kWinDense) {
        const int nwords = static_cast<int>((w1 - w0 + 31) >> 5);
        const uint32_t word = threadIdx.x < nwords ? bm[threadIdx.x] : 0u;
        const int64_t pos = block_excl_scan<int64_t>(__popc(word), s_scan64, &tot);
        if (word) {
          int64_t o = out + pos;
          for (uint32_t m = word; m; m &= m - 1) {
            const int rel = threadIdx.x * 32 + (__ffs(m) - 1);
            if (o < out_end) {
              ccol[o] = static_cast<int32_t>(w0 + rel);
              cval[o] = dense[rel];
            }
            dense[rel] = 0.0;
            ++o;
          }
          bm[threadIdx.x] = 0u;
        }
      } else {
        for (int s = threadIdx.x; s < kHashWinSlots; s += kWinThreads) {
          const int32_t key = hkeys[s];
          if (key) {
            const int32_t rel = static_cast<int32_t>(key - 1 - w0);
            atomicOr(&bm[rel >> 5], 1u << (rel & 31));
          }
        }
        __syncthreads();
        const int nwords = static_cast<int>((w1 - w0 + 31) >> 5);
        constexpr int kPer = kWinBitmapWords / kWinThreads;
        const int wlo = threadIdx.x * kPer;
        int c = 0;
#pragma unroll
        for (int t = 0; t < kPer; ++t) c += (wlo + t < nwords) ? __popc(bm[wlo + t]) : 0;
        const int64_t pos = block_excl_scan<int64_t>(c, s_scan64, &tot);
        int64_t o = out + pos;
        for (int t = 0; t < kPer; ++t) {
          if (wlo + t >= nwords) break;
          uint32_t m = bm[wlo + t];
          if (!m) continue;
          bm[wlo + t] = 0u;
          for (; m; m &= m - 1) {
            const int rel = (wlo + t) * 32 + (__ffs(m) - 1);
            const int32_t key = static_cast<int32_t>(w0 + rel) + 1;
            uint32_t h = hash_slot(key, kHashWinLog2);
            double v = 0.0;
            for (int probe = 0; probe < kHashWinSlots; ++probe) {
              if (hkeys[h] == key) { v = hvals[h]; break; }
              h = (h + 1) & (kHashWinSlots - 1);
            }
            if (o < out_end) {
              ccol[o] = key - 1;
              cval[o] = v;
            }
            ++o;
          }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < kHashWinSlots; s += kWinThreads) { hkeys[s] = 0; hvals[s] = 0.0; }
      }
      if (threadIdx.x == 0 && tot != expect) set_error(err, kErrCount);
      out += tot;
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
  k_num_window<<<static_cast<unsigned>(g), kWinThreads, kWinSmemBytes, s>>>(
      A, B, perm, count, counter, c_off, win_slot, blockcnt, nblocks, nslots, split, hash_fill, ccol, cval,
      err);
  return 1;
}

}  // namespace spg
