// Small products of narrow matrices: one warp per row in both passes, the warp holding a bitmap
// of all n columns of C, so the whole product takes two kernels around one host read of the
// summary (nnz(C), sum P_i, the longest row of C, error bits).
//
// Row i of C is the union of the named B rows (Algorithm 1, Sec. III-A): the symbolic kernel
// marks every column a partial product reaches (shared atomicOr) and counts the set bits; the
// numeric kernel marks them again, turns the bitmap into each column's rank (a prefix count over
// the words: the columns in ascending order), adds a_ik * b_kj into a rank-indexed FP64 array and
// writes the row out in column order, so no sort is needed (the order of Algorithm 1's sorted
// PP comes from the bitmap).
//
// The bitmap is laid out for conflict-free vector access: lane l owns the vectors l, l + 32, ...
// of VW words (VW = 4, or 1 for n <= 3,072), PER words in all, so a pass over it is PER / VW
// vector loads per lane and the ranks take one warp scan per vector. It stays zero between rows:
// the pass that reads a row's bits last (the count, or the write-out) clears them.
//
// Each block of the symbolic kernel takes a contiguous run of rows and ends with their offsets
// within the run; the last block to finish scans the runs' totals. The kernel also checks both
// inputs (A row by row as it counts; B in the warps' second loop) and clamps every row range it
// reads. Row pointers are read as the caller stores them (int32 or int64). A row of C with more
// than kSmallCap entries sends the plan to the general path.
#include <mutex>
#include <vector>

#include "runtime.h"

namespace spg {

namespace {

constexpr int kSymWarps = 8;     // warps per block, symbolic kernel
constexpr int kNumWarpsB = 4;    // warps per block, numeric kernel
constexpr int kSlots = 4;        // partial products per lane in one step (loads in flight)
constexpr int kRunShared = 512;  // symbolic runs of up to this many rows keep their counts in shared memory
constexpr int kSymWarpBytes = 4096;       // bitmap bytes per symbolic warp (all its row slots)
constexpr int kNumSmemMax = 64 * 1024;   // numeric: 4 warps x (192 B x 32 + 8 B x 1,024) = 57,344 B at most
constexpr unsigned kFull = 0xffffffffu;
enum : uint32_t { kSmallTooLong = 1u };   // summary->small_flags bit: a row needs the general path

__device__ __forceinline__ int64_t rp_at(const SmallCsr& M, int64_t i) {
  return M.rp64 ? static_cast<const int64_t*>(M.rp)[i] : static_cast<const int32_t*>(M.rp)[i];
}

// Row r's entry range, clamped to [0, nnz] and to at most `cols` entries (a longer row cannot be
// canonical); *bad is set for any violation when check is on.
__device__ __forceinline__ void row_range(const SmallCsr& M, int64_t r, bool check, bool& bad, int64_t& s,
                                          int32_t& len) {
  int64_t a = rp_at(M, r), b = rp_at(M, r + 1);
  if (check && (a < 0 || b < a || b > M.nnz || (r == 0 && a != 0) || (r == M.rows - 1 && b != M.nnz))) bad = true;
  a = a < 0 ? 0 : (a > M.nnz ? M.nnz : a);
  b = b < a ? a : (b > M.nnz ? M.nnz : b);
  if (b - a > M.cols) {
    if (check) bad = true;
    b = a + M.cols;
  }
  s = a;
  len = static_cast<int32_t>(b - a);
}

// The warp's 32 ranges [bs_l, bs_l + len_l) (with a payload a_l), flattened over the lanes,
// kSlots * 32 entries per step: f(ok, j, pos, a, own) gets, for each of the lane's kSlots
// slots, whether it holds an entry, the entry, its position in its range, its range's payload
// and the lane that owns the range. f runs on every lane; groups of 32 slots past the end are
// skipped as a whole.
template <typename F>
__device__ __forceinline__ void for_slots(int32_t len, int64_t bs, double a, F&& f) {
  const int lane = threadIdx.x & 31;
  const int32_t incl = warp_incl_scan(len);
  const int32_t excl = incl - len;
  const int32_t total = __shfl_sync(kFull, incl, 31);
  for (int32_t p0 = 0; p0 < total; p0 += kSlots * 32) {
    bool ok[kSlots];
    int64_t j[kSlots];
    int32_t pos[kSlots];
    double av[kSlots];
    int own[kSlots];
#pragma unroll
    for (int u = 0; u < kSlots; ++u) {
      ok[u] = false;
      j[u] = 0;
      pos[u] = 0;
      av[u] = 0.0;
      own[u] = 0;
      if (p0 + u * 32 < total) {
        const int32_t p = p0 + u * 32 + lane;
        int o = 0;   // the first lane whose inclusive end exceeds p
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (__shfl_sync(kFull, incl, o + step - 1) <= p) o += step;
        const int32_t st = __shfl_sync(kFull, excl, o);
        j[u] = __shfl_sync(kFull, bs, o) + (p - st);
        pos[u] = p - st;
        av[u] = __shfl_sync(kFull, a, o);
        own[u] = o;
        ok[u] = p < total;
      }
    }
    f(ok, j, pos, av, own);
  }
}

// Shared bytes of one numeric warp: bitmap (128 PER), ranks (64 PER) and values (8 cap, rounded
// up to 16 so that every warp's bitmap starts 16-byte aligned for its vector accesses).
__host__ __device__ __forceinline__ size_t num_warp_bytes(int per, int cap) {
  return static_cast<size_t>(192) * per + ((sizeof(double) * cap + 15) & ~size_t(15));
}

// The lane's share of a bitmap of 32 * PER words: NV vectors of VW words, vector q at lane + 32 q.
template <int PER>
struct Lanes {
  static constexpr int VW = PER >= 4 ? 4 : 1;
  static constexpr int NV = PER / VW;
  static __device__ __forceinline__ int vec(int q) { return (threadIdx.x & 31) + 32 * q; }
  static __device__ __forceinline__ void load(const uint32_t* bm, int q, uint32_t (&w)[VW]) {
    if constexpr (VW == 4) {
      const uint4 t = reinterpret_cast<const uint4*>(bm)[vec(q)];
      w[0] = t.x;
      w[1] = t.y;
      w[2] = t.z;
      w[3] = t.w;
    } else {
      w[0] = bm[vec(q)];
    }
  }
  static __device__ __forceinline__ void zero(uint32_t* bm, int q) {
    if constexpr (VW == 4) reinterpret_cast<uint4*>(bm)[vec(q)] = make_uint4(0u, 0u, 0u, 0u);
    else bm[vec(q)] = 0u;
  }
  static __device__ __forceinline__ void zero_all(uint32_t* bm) {
#pragma unroll
    for (int q = 0; q < NV; ++q) zero(bm, q);
  }
};

// Exclusive scan of n values by one block, thread t taking a run of consecutive values: ld(i)
// reads value i, st(i, offset) writes its offset; returns the total. Up to kScanRegs values per
// thread are loaded once, together, before the block scan.
constexpr int kScanRegs = 8;
template <typename Ld, typename St>
__device__ __forceinline__ int64_t block_scan_chunks(int64_t n, int64_t* s_scan, Ld&& ld, St&& st) {
  const int64_t k = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = threadIdx.x * k < n ? threadIdx.x * k : n;
  const int64_t hi = lo + k < n ? lo + k : n;
  int64_t v[kScanRegs];
  int64_t mine = 0;
  if (k <= kScanRegs) {
#pragma unroll
    for (int t = 0; t < kScanRegs; ++t) v[t] = lo + t < hi ? ld(lo + t) : 0;
#pragma unroll
    for (int t = 0; t < kScanRegs; ++t) mine += v[t];
  } else {
    for (int64_t i = lo; i < hi; ++i) mine += ld(i);
  }
  int64_t total;
  int64_t off = block_excl_scan<int64_t>(mine, s_scan, &total);
  if (k <= kScanRegs) {
#pragma unroll
    for (int t = 0; t < kScanRegs; ++t)
      if (lo + t < hi) {
        st(lo + t, off);
        off += v[t];
      }
  } else {
    for (int64_t i = lo; i < hi; ++i) {
      const int64_t x = ld(i);
      st(i, off);
      off += x;
    }
  }
  return total;
}

// A warp's group of ng consecutive rows of A, seen as one flat list of their entries: lane l < ng
// holds row l's entry range [a, a + na) and q, the flat position of its first entry; E is the
// number of entries in all (the same on every lane).
struct RowGroup {
  int ng;
  int64_t a;
  int32_t na, q, E;
};

__device__ __forceinline__ RowGroup group_rows(const SmallCsr& A, int64_t gs, int ng, bool check, bool& bad) {
  const int lane = threadIdx.x & 31;
  RowGroup gr;
  gr.ng = ng;
  gr.a = 0;
  gr.na = 0;
  if (lane < ng) row_range(A, gs + lane, check, bad, gr.a, gr.na);
  const int32_t incl = warp_incl_scan(gr.na);
  gr.q = incl - gr.na;
  gr.E = __shfl_sync(kFull, incl, 31);
  return gr;
}

// Flat position p of a group (lanes may differ): its row g (0..ng-1), the row's first entry a_g
// and the entry e. Every lane must call it.
__device__ __forceinline__ void group_entry(const RowGroup& gr, int32_t p, int& g, int64_t& a_g, int64_t& e) {
  g = 0;
#pragma unroll
  for (int t = 1; t < 4; ++t) {
    const int32_t qt = __shfl_sync(kFull, gr.q, t);
    if (t < gr.ng && qt <= p) g = t;
  }
  a_g = __shfl_sync(kFull, gr.a, g);
  e = a_g + (p - __shfl_sync(kFull, gr.q, g));
}

// Lane's share of the flat entries [c0, c0 + 32) of a group: row g, B row range, A value.
__device__ __forceinline__ void group_chunk(const SmallCsr& A, const SmallCsr& B, const RowGroup& gr, int32_t c0,
                                            bool check, bool& bad, int& g, int64_t& bs, int32_t& len, double& a) {
  const int32_t p = c0 + (threadIdx.x & 31);
  int64_t a_g, e;
  group_entry(gr, p, g, a_g, e);
  bs = 0;
  len = 0;
  a = 0.0;
  if (p < gr.E) {
    const int32_t k = A.col[e];
    if (check && (k < 0 || k >= B.rows || (e > a_g && A.col[e - 1] >= k))) bad = true;
    if (k >= 0 && k < B.rows) {
      row_range(B, k, false, bad, bs, len);
      a = static_cast<const double*>(A.val)[e];
    }
  }
}

// Bits set in the warp's bitmap (this lane's share), clearing them.
template <int PER>
__device__ __forceinline__ int count_clear(uint32_t* bm) {
  using L = Lanes<PER>;
  int c = 0;
#pragma unroll
  for (int q = 0; q < L::NV; ++q) {
    uint32_t w[L::VW];
    L::load(bm, q, w);
#pragma unroll
    for (int t = 0; t < L::VW; ++t) c += __popc(w[t]);
    L::zero(bm, q);
  }
  return c;
}

// pre[w] = bits set in the bitmap before word w (the per-vector warp scans run side by side);
// returns the number of bits set.
template <int PER>
__device__ __forceinline__ int rank_words(const uint32_t* bm, uint16_t* pre) {
  using L = Lanes<PER>;
  constexpr int VW = L::VW;
  const int lane = threadIdx.x & 31;
  int cq[L::NV], iq[L::NV];
#pragma unroll
  for (int q = 0; q < L::NV; ++q) {
    uint32_t w[VW];
    L::load(bm, q, w);
    cq[q] = 0;
#pragma unroll
    for (int t = 0; t < VW; ++t) cq[q] += __popc(w[t]);
    iq[q] = cq[q];
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int q = 0; q < L::NV; ++q) {
      const int t = __shfl_up_sync(kFull, iq[q], d);
      if (lane >= d) iq[q] += t;
    }
  }
  int carry = 0;
#pragma unroll
  for (int q = 0; q < L::NV; ++q) {
    uint32_t w[VW];
    L::load(bm, q, w);
    const int b0 = carry + iq[q] - cq[q];
    if constexpr (VW == 4) {
      const int p1 = b0 + __popc(w[0]), p2 = p1 + __popc(w[1]), p3 = p2 + __popc(w[2]);
      const uint32_t lo = static_cast<uint32_t>(b0) | (static_cast<uint32_t>(p1) << 16);
      const uint32_t hi = static_cast<uint32_t>(p2) | (static_cast<uint32_t>(p3) << 16);
      reinterpret_cast<uint2*>(pre)[L::vec(q)] = make_uint2(lo, hi);
    } else {
      pre[L::vec(q)] = static_cast<uint16_t>(b0);
    }
    carry += __shfl_sync(kFull, iq[q], 31);
  }
  return carry;
}

// Rank of column `col` in a row whose bits and word ranks are set.
__device__ __forceinline__ int rank_of(const uint32_t* bm, const uint16_t* pre, int32_t col) {
  const int w = col >> 5;
  return pre[w] + __popc(bm[w] & ((1u << (col & 31)) - 1u));
}

// Row of C out in column order (each lane its vectors' columns at their ranks), clearing the bits.
template <int PER>
__device__ __forceinline__ void write_row(uint32_t* bm, const uint16_t* pre, const double* vals, int n_out,
                                          int64_t len, int64_t off, int32_t* __restrict__ ccol,
                                          double* __restrict__ cval) {
  using L = Lanes<PER>;
  constexpr int VW = L::VW;
#pragma unroll
  for (int q = 0; q < L::NV; ++q) {
    uint32_t w[VW];
    L::load(bm, q, w);
    const int v = L::vec(q);
#pragma unroll
    for (int t = 0; t < VW; ++t) {
      uint32_t mk = w[t];
      int r = pre[v * VW + t];
      for (; mk; mk &= mk - 1, ++r) {
        if (r < n_out && r < len) {
          ccol[off + r] = (v * VW + t) * 32 + (__ffs(mk) - 1);
          cval[off + r] = vals[r];
        }
      }
    }
    L::zero(bm, q);
  }
}

// A warp takes G consecutive rows at a time (G = 1 to 4), each with a bitmap of its own, and
// enumerates their partial products as one flat list, 32 entries of A at a time, so the memory
// round trips of the group's rows overlap.
template <int PER>
__global__ void __launch_bounds__(kSymWarps * 32) k_small_sym(SmallCsr A, SmallCsr B, int32_t width, int check,
                                                              int64_t run, int G, int32_t* __restrict__ nnz_row,
                                                              int32_t* __restrict__ loc,
                                                              int64_t* __restrict__ blk, Summary* sum,
                                                              Summary* hsum) {
  extern __shared__ __align__(16) unsigned char small_smem[];
  __shared__ int64_t s_scan[33];
  __shared__ int32_t s_cnt[kRunShared];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* bm0 = reinterpret_cast<uint32_t*>(small_smem) + static_cast<size_t>(wid) * G * 32 * PER;
  for (int g = 0; g < G; ++g) Lanes<PER>::zero_all(bm0 + g * 32 * PER);
  __syncwarp();
  const int64_t m = A.rows;
  const int64_t r0 = blockIdx.x * run < m ? blockIdx.x * run : m;
  const int64_t r1 = r0 + run < m ? r0 + run : m;
  const bool chk = check != 0;
  bool bad = false;
  int64_t prod = 0;
  int max_cnt = 0;
  for (int64_t gs = r0 + wid * G; gs < r1; gs += int64_t(kSymWarps) * G) {
    const int ng = r1 - gs < G ? static_cast<int>(r1 - gs) : G;
    const RowGroup gr = group_rows(A, gs, ng, chk, bad);
    // lane g < ng: the first column of row gs + g's column space (a stacked batch's job)
    const int32_t cb_lane = A.cbase && lane < ng ? A.cbase[gs + lane] : 0;
    for (int32_t c0 = 0; c0 < gr.E; c0 += 32) {
      int g;
      int64_t bs;
      int32_t len;
      double a;
      group_chunk(A, B, gr, c0, chk, bad, g, bs, len, a);
      prod += len;
      for_slots(len, bs, a, [&](const bool* ok, const int64_t* j, const int32_t*, const double*, const int* own) {
        int32_t c[kSlots];
        int go[kSlots];
#pragma unroll
        for (int u = 0; u < kSlots; ++u) {
          c[u] = ok[u] ? B.col[j[u]] : -1;
          go[u] = __shfl_sync(kFull, g, own[u]);
          const int32_t cb = __shfl_sync(kFull, cb_lane, go[u]);
          c[u] = c[u] >= 0 ? c[u] - cb : -1;
        }
#pragma unroll
        for (int u = 0; u < kSlots; ++u)
          if (c[u] >= 0 && c[u] < width) atomicOr(&bm0[go[u] * 32 * PER + (c[u] >> 5)], 1u << (c[u] & 31));
          else if (ok[u] && chk) bad = true;   // a column outside its row's column space
      });
    }
    __syncwarp();
    int cg[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) cg[g] = g < ng ? count_clear<PER>(bm0 + g * 32 * PER) : 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g < ng) {
        const int cnt = warp_sum(cg[g]);
        if (lane == 0) {
          nnz_row[gs + g] = cnt;
          if (run <= kRunShared) s_cnt[gs + g - r0] = cnt;
        }
        max_cnt = cnt > max_cnt ? cnt : max_cnt;
      }
    }
    __syncwarp();
  }
  if (chk) {
    // B: row pointers, columns in range and strictly increasing, 32 rows per warp at a time
    const int64_t gw = blockIdx.x * int64_t(kSymWarps) + wid;
    const int64_t nw = int64_t(gridDim.x) * kSymWarps;
    for (int64_t g = gw * 32; g < B.rows; g += nw * 32) {
      const int64_t r = g + lane;
      int64_t s = 0;
      int32_t len = 0;
      if (r < B.rows) row_range(B, r, true, bad, s, len);
      for_slots(len, s, 0.0, [&](const bool* ok, const int64_t* j, const int32_t* pos, const double*, const int*) {
#pragma unroll
        for (int u = 0; u < kSlots; ++u) {
          if (!ok[u]) continue;
          const int32_t c = B.col[j[u]];
          if (c < 0 || c >= B.cols || (pos[u] > 0 && B.col[j[u] - 1] >= c)) bad = true;
        }
      });
    }
    if (B.rows == 0 && gw == 0 && lane == 0 && (rp_at(B, 0) != 0 || B.nnz != 0)) bad = true;
  }
  prod = warp_sum(prod);
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(&sum->err, kErrInvalidCsr);
  if (lane == 0) {
    if (prod) atomicAdd(&sum->small_products, static_cast<unsigned long long>(prod));
    if (max_cnt > 0)
      atomicMax(reinterpret_cast<unsigned long long*>(&sum->max_row), static_cast<unsigned long long>(max_cnt));
    if (max_cnt > kSmallCap) atomicOr(&sum->small_flags, kSmallTooLong);
  }
  // offsets within this block's run of rows, and the run's total
  __syncthreads();
  const int64_t carry = block_scan_chunks(
      r1 - r0, s_scan,
      [&](int64_t t) -> int64_t { return run <= kRunShared ? s_cnt[t] : nnz_row[r0 + t]; },
      [&](int64_t t, int64_t off) { loc[r0 + t] = static_cast<int32_t>(off); });
  if (threadIdx.x == 0) blk[blockIdx.x] = carry;
  // the last block to finish turns the runs' totals into their offsets (blk[0..grid], in place)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&sum->small_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int64_t total = block_scan_chunks(
      gridDim.x, s_scan, [&](int64_t b) -> int64_t { return __ldcg(blk + b); },
      [&](int64_t b, int64_t off) { blk[b] = off; });
  if (threadIdx.x == 0) {
    blk[gridDim.x] = total;
    sum->total = total;
    if (hsum) {
      // every other block's updates of the summary came before its ticket (and this block's fence
      // after it): read them from L2, where the atomics ran, as independent loads, and store what
      // the host reads into mapped page-locked memory, so the host needs no copy after the kernel
      const uint32_t e = __ldcg(&sum->err);
      const uint32_t f = __ldcg(&sum->small_flags);
      const unsigned long long pr = __ldcg(&sum->small_products);
      const long long mr = __ldcg(reinterpret_cast<const long long*>(&sum->max_row));
      hsum->err = e;
      hsum->small_flags = f;
      hsum->small_products = pr;
      hsum->max_row = mr;
      hsum->total = total;
    }
  }
}

// Lane's share of the A entries [a0 + base, a0 + base + 32): its B row range and A value.
__device__ __forceinline__ void a_entry(const SmallCsr& A, const SmallCsr& B, int64_t a0, int64_t na, int64_t base,
                                        int64_t& bs, int32_t& len, double& a) {
  const int64_t e = base + (threadIdx.x & 31);
  bool unused = false;
  len = 0;
  bs = 0;
  a = 0.0;
  if (e < na) {
    const int32_t k = A.col[a0 + e];
    if (k >= 0 && k < B.rows) {
      row_range(B, k, false, unused, bs, len);
      a = static_cast<const double*>(A.val)[a0 + e];
    }
  }
}

// Numeric pass, one warp per row. A row of at most 32 entries of A and kSlots * 32 partial
// products keeps the loads of its marking step in registers for the accumulation; longer rows
// enumerate their products twice.
template <int PER>
__global__ void __launch_bounds__(kNumWarpsB * 32) k_small_num(SmallCsr A, SmallCsr B, int32_t width, int cap,
                                                               int64_t run,
                                                               const int32_t* __restrict__ nnz_row,
                                                               const int32_t* __restrict__ loc,
                                                               const int64_t* __restrict__ blk, int64_t nblk,
                                                               void* crp, int crp64, int32_t* __restrict__ ccol,
                                                               double* __restrict__ cval, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char small_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* base = small_smem + static_cast<size_t>(wid) * num_warp_bytes(PER, cap);
  uint32_t* bm = reinterpret_cast<uint32_t*>(base);
  uint16_t* pre = reinterpret_cast<uint16_t*>(base + 128 * PER);
  double* vals = reinterpret_cast<double*>(base + 192 * PER);
  Lanes<PER>::zero_all(bm);
  __syncwarp();
  const int64_t gw = blockIdx.x * int64_t(kNumWarpsB) + wid;
  const int64_t nw = int64_t(gridDim.x) * kNumWarpsB;
  const double* bv = static_cast<const double*>(B.val);
  const int64_t m = A.rows;
  bool bad = false;
  for (int64_t i = gw; i < m; i += nw) {
    int64_t a0;
    int32_t na;
    row_range(A, i, false, bad, a0, na);
    const int64_t off = blk[i / run] + loc[i];
    const int64_t len = nnz_row[i];
    if (lane == 0) {
      if (crp64) static_cast<int64_t*>(crp)[i] = off;
      else static_cast<int32_t*>(crp)[i] = static_cast<int32_t>(off);
      if (i == m - 1) {
        const int64_t total = blk[nblk];
        if (crp64) static_cast<int64_t*>(crp)[m] = total;
        else static_cast<int32_t*>(crp)[m] = static_cast<int32_t>(total);
      }
    }
    const int32_t cb = A.cbase ? A.cbase[i] : 0;   // the row's column space (a stacked batch's job)
    int64_t bs;
    int32_t blen;
    double a;
    a_entry(A, B, a0, na, 0, bs, blen, a);
    const int32_t ptot = __shfl_sync(kFull, warp_incl_scan(blen), 31);
    const bool fast = na <= 32 && ptot <= kSlots * 32;
    int32_t fc[kSlots];
    double fv[kSlots];
#pragma unroll
    for (int u = 0; u < kSlots; ++u) {
      fc[u] = -1;
      fv[u] = 0.0;
    }
    if (fast) {
      for_slots(blen, bs, a, [&](const bool* ok, const int64_t* j, const int32_t*, const double* av, const int*) {
#pragma unroll
        for (int u = 0; u < kSlots; ++u) {
          fc[u] = ok[u] ? B.col[j[u]] - cb : -1;
          fv[u] = ok[u] ? av[u] * bv[j[u]] : 0.0;
        }
      });
#pragma unroll
      for (int u = 0; u < kSlots; ++u)
        if (fc[u] >= 0 && fc[u] < width) atomicOr(&bm[fc[u] >> 5], 1u << (fc[u] & 31));
    } else {
      for (int64_t b0 = 0; b0 < na; b0 += 32) {
        a_entry(A, B, a0, na, b0, bs, blen, a);
        for_slots(blen, bs, a, [&](const bool* ok, const int64_t* j, const int32_t*, const double*, const int*) {
          int32_t c[kSlots];
#pragma unroll
          for (int u = 0; u < kSlots; ++u) c[u] = ok[u] ? B.col[j[u]] - cb : -1;
#pragma unroll
          for (int u = 0; u < kSlots; ++u)
            if (c[u] >= 0 && c[u] < width) atomicOr(&bm[c[u] >> 5], 1u << (c[u] & 31));
        });
      }
    }
    __syncwarp();
    const int cnt = rank_words<PER>(bm, pre);
    if (cnt != len || cnt > cap) bad = true;
    const int n_out = cnt < cap ? cnt : cap;
    for (int r = lane; r < n_out; r += 32) vals[r] = 0.0;
    __syncwarp();
    auto add = [&](int32_t col, double v) {
      if (col < 0 || col >= width) return;
      const int r = rank_of(bm, pre, col);
      if (r < n_out) atomicAdd(&vals[r], v);
    };
    if (fast) {
#pragma unroll
      for (int u = 0; u < kSlots; ++u) add(fc[u], fv[u]);
    } else {
      for (int64_t b0 = 0; b0 < na; b0 += 32) {
        a_entry(A, B, a0, na, b0, bs, blen, a);
        for_slots(blen, bs, a, [&](const bool* ok, const int64_t* j, const int32_t*, const double* av, const int*) {
          int32_t cc[kSlots];
          double vv[kSlots];
#pragma unroll
          for (int u = 0; u < kSlots; ++u) {
            cc[u] = ok[u] ? B.col[j[u]] - cb : -1;
            vv[u] = ok[u] ? av[u] * bv[j[u]] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < kSlots; ++u) add(cc[u], vv[u]);
        });
      }
    }
    __syncwarp();
    write_row<PER>(bm, pre, vals, n_out, len, off, ccol, cval);
    __syncwarp();
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(err, kErrCount);
}

// Words of the bitmap per lane for n columns: the power of two >= ceil(n / 1024) (1..32).
int small_per(int64_t n) {
  int per = 1;
  while (per * 1024 < n) per *= 2;
  return per;
}

// Kernel instances by words per lane (1, 2, 4, 8, 16, 32).
constexpr int kPerCount = 6;
int per_index(int per) { return __builtin_ctz(static_cast<unsigned>(per)); }

template <int PER>
void sym_launch(dim3 g, size_t smem, cudaStream_t s, const SmallCsr& A, const SmallCsr& B, int32_t width, int check,
                int64_t run, int G, int32_t* nnz_row, int32_t* loc, int64_t* blk, Summary* sum, Summary* hsum) {
  k_small_sym<PER><<<g, kSymWarps * 32, smem, s>>>(A, B, width, check, run, G, nnz_row, loc, blk, sum, hsum);
}

template <int PER>
void num_launch(dim3 g, size_t smem, cudaStream_t s, const SmallCsr& A, const SmallCsr& B, int32_t width, int cap,
                int64_t run, const int32_t* nnz_row, const int32_t* loc, const int64_t* blk, int64_t nblk, void* crp,
                int crp64, int32_t* ccol, double* cval, uint32_t* err) {
  k_small_num<PER><<<g, kNumWarpsB * 32, smem, s>>>(A, B, width, cap, run, nnz_row, loc, blk, nblk, crp, crp64, ccol,
                                                     cval, err);
}

// c_off[i] = blk[i / run] + loc[i]; c_off[m] = blk[blocks].
__global__ void __launch_bounds__(256) k_small_offsets(const int32_t* __restrict__ loc, const int64_t* __restrict__ blk,
                                                       int64_t run, int64_t nblk, int64_t m, int64_t* __restrict__ c_off) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i <= m; i += int64_t(gridDim.x) * blockDim.x)
    c_off[i] = i < m ? blk[i / run] + loc[i] : blk[nblk];
}

const void* sym_fn(int k) {
  switch (k) {
    case 0: return reinterpret_cast<const void*>(k_small_sym<1>);
    case 1: return reinterpret_cast<const void*>(k_small_sym<2>);
    case 2: return reinterpret_cast<const void*>(k_small_sym<4>);
    case 3: return reinterpret_cast<const void*>(k_small_sym<8>);
    case 4: return reinterpret_cast<const void*>(k_small_sym<16>);
    default: return reinterpret_cast<const void*>(k_small_sym<32>);
  }
}

const void* num_fn(int k) {
  switch (k) {
    case 0: return reinterpret_cast<const void*>(k_small_num<1>);
    case 1: return reinterpret_cast<const void*>(k_small_num<2>);
    case 2: return reinterpret_cast<const void*>(k_small_num<4>);
    case 3: return reinterpret_cast<const void*>(k_small_num<8>);
    case 4: return reinterpret_cast<const void*>(k_small_num<16>);
    default: return reinterpret_cast<const void*>(k_small_num<32>);
  }
}

// Per device, once: the registers a thread of each kernel instance holds, and the numeric
// kernels' dynamic shared memory limit raised to kNumSmemMax.
struct SmallKernelInfo {
  int sym_regs[kPerCount] = {}, num_regs[kPerCount] = {};
  bool ready = false;
};

std::mutex g_small_mu;
std::vector<SmallKernelInfo> g_small_info;

const SmallKernelInfo& small_info() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_small_mu);
  if (static_cast<int>(g_small_info.size()) <= dev) g_small_info.resize(dev + 1);
  SmallKernelInfo& k = g_small_info[dev];
  if (!k.ready) {
    for (int i = 0; i < kPerCount; ++i) {
      cudaFuncAttributes fa{};
      k.sym_regs[i] = cudaFuncGetAttributes(&fa, sym_fn(i)) == cudaSuccess && fa.numRegs > 0 ? fa.numRegs : 64;
      k.num_regs[i] = cudaFuncGetAttributes(&fa, num_fn(i)) == cudaSuccess && fa.numRegs > 0 ? fa.numRegs : 64;
      cudaFuncSetAttribute(num_fn(i), cudaFuncAttributeMaxDynamicSharedMemorySize, kNumSmemMax);
    }
    cudaGetLastError();
    k.ready = true;
  }
  return k;
}

// Blocks of `threads` threads, `regs` registers each and `smem` shared bytes resident per SM
// (register file 64K, 2,048 threads, about 228 KB of shared memory with 1 KB reserved per
// block), at most max_per_sm.
int resident(int regs, int threads, size_t smem, int max_per_sm) {
  const int warps = threads / 32;
  const int warp_regs = (regs * 32 + 255) / 256 * 256;
  int nb = 2048 / threads;
  const int by_regs = 65536 / warp_regs / warps;
  const int by_smem = static_cast<int>((228 * 1024) / (smem + 1024));
  nb = nb < by_regs ? nb : by_regs;
  nb = nb < by_smem ? nb : by_smem;
  nb = nb < 1 ? 1 : nb;
  return nb < max_per_sm ? nb : max_per_sm;
}

// Rows per group (1 to 4): about 24 entries of A per group on average (one chunk of 32 for most
// groups), while G row slots of `slot_bytes` stay within `budget` bytes per warp.
int small_groups(double avg, size_t slot_bytes, size_t budget) {
  int g = avg > 0.0 ? static_cast<int>(24.0 / avg) : 4;
  g = g < 1 ? 1 : (g > 4 ? 4 : g);
  while (g > 1 && slot_bytes * g > budget) --g;
  return g;
}

double avg_row(const SmallCsr& A) { return A.rows > 0 ? static_cast<double>(A.nnz) / A.rows : 0.0; }

size_t sym_smem(int per, int G) { return static_cast<size_t>(128) * per * G * kSymWarps; }
size_t num_smem(int per, int cap) { return num_warp_bytes(per, cap) * kNumWarpsB; }

}  // namespace

bool small_path_fits(int64_t m, int64_t n) { return m <= kSmallMaxRows && n <= kSmallMaxCols && n > 0; }

SmallGrid small_sym_grid(const SmallCsr& A, int64_t width, int num_sms) {
  const int per = small_per(width);
  const int G = small_groups(avg_row(A), static_cast<size_t>(128) * per, kSymWarpBytes);
  const int regs = small_info().sym_regs[per_index(per)];
  const int64_t m = A.rows;
  const int64_t cap = int64_t(num_sms) * resident(regs, kSymWarps * 32, sym_smem(per, G), 8);
  int64_t g = (m + int64_t(kSymWarps) * G - 1) / (int64_t(kSymWarps) * G);
  g = g < cap ? g : cap;
  g = g > 0 ? g : 1;
  const int64_t run = (m + g - 1) / g;
  return SmallGrid{(m + run - 1) / run, run, G};
}

int launch_small_symbolic(const SmallCsr& A, const SmallCsr& B, int64_t width, SmallGrid g, int check,
                          int32_t* nnz_row, int32_t* loc, int64_t* blk, Summary* sum, Summary* hsum,
                          cudaStream_t s) {
  const int per = small_per(width);
  const dim3 grid(static_cast<unsigned>(g.blocks));
  const size_t smem = sym_smem(per, g.groups);
  const int G = g.groups;
  const int32_t w = static_cast<int32_t>(width);
#define SPG_SYM(P) sym_launch<P>(grid, smem, s, A, B, w, check, g.run, G, nnz_row, loc, blk, sum, hsum)
  switch (per) {
    case 1: SPG_SYM(1); break;
    case 2: SPG_SYM(2); break;
    case 4: SPG_SYM(4); break;
    case 8: SPG_SYM(8); break;
    case 16: SPG_SYM(16); break;
    default: SPG_SYM(32); break;
  }
#undef SPG_SYM
  return 1;
}

int launch_small_offsets(const int32_t* loc, const int64_t* blk, SmallGrid g, int64_t m, int64_t* c_off,
                         cudaStream_t s) {
  int64_t nb = (m + 1 + 255) / 256;
  nb = nb < 4096 ? nb : 4096;
  k_small_offsets<<<static_cast<unsigned>(nb), 256, 0, s>>>(loc, blk, g.run, g.blocks, m, c_off);
  return 1;
}

int launch_small_numeric(const SmallCsr& A, const SmallCsr& B, int64_t width, SmallGrid g, int cap,
                         const int32_t* nnz_row, const int32_t* loc, const int64_t* blk, void* crp, int crp64,
                         int32_t* ccol, double* cval, uint32_t* err, int num_sms, cudaStream_t s) {
  if (A.rows <= 0) return 0;
  const int per = small_per(width);
  cap = cap < 1 ? 1 : (cap > kSmallCap ? kSmallCap : cap);
  const size_t smem = num_smem(per, cap);
  const int regs = small_info().num_regs[per_index(per)];
  const int64_t most = int64_t(num_sms) * resident(regs, kNumWarpsB * 32, smem, 16);
  int64_t nb = (A.rows + kNumWarpsB - 1) / kNumWarpsB;
  nb = nb < most ? nb : most;
  const dim3 grid(static_cast<unsigned>(nb > 0 ? nb : 1));
  const int32_t w = static_cast<int32_t>(width);
#define SPG_NUM(P) \
  num_launch<P>(grid, smem, s, A, B, w, cap, g.run, nnz_row, loc, blk, g.blocks, crp, crp64, ccol, cval, err)
  switch (per) {
    case 1: SPG_NUM(1); break;
    case 2: SPG_NUM(2); break;
    case 4: SPG_NUM(4); break;
    case 8: SPG_NUM(8); break;
    case 16: SPG_NUM(16); break;
    default: SPG_NUM(32); break;
  }
#undef SPG_NUM
  return 1;
}

}  // namespace spg
