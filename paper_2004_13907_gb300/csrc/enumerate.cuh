// Enumeration of the partial products of one row of C = A*B (internal).
//
// Algorithm 1 (Sec. III-A) forms, for row i, one partial product for every pair of a
// stored (k, a_ik) of row i of A and a stored (j, b_kj) of row k of B. These helpers hand
// those pairs out to the lanes of a warp or the threads of a block "flattened": the pairs
// of consecutive A entries are numbered consecutively, so short B rows do not leave lanes
// idle. A chunk of up to 32 (warp) or NT (block) A entries is loaded, the lengths of their
// B rows are scanned, and each lane finds the A entry that owns its pair number.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace spg {

// Largest o in [hint, nvalid) with excl[o] <= p, given excl[hint] <= p (excl is
// non-decreasing). A few linear steps first (owners change slowly when B rows are long),
// then binary search.
__device__ __forceinline__ int find_owner(const int32_t* excl, int nvalid, int32_t p, int hint) {
  int o = hint;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (o + 1 < nvalid && excl[o + 1] <= p) ++o;
    else return o;
  }
  int lo = o, hi = nvalid - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (excl[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Warp-flattened enumeration over all A entries of row [a0, a0+na). For every partial
// product, f(j, a_val_index) is called on the lane that owns it, with j the index into
// B.col / B.val and e the index of the A entry (0-based within the row). All 32 lanes must
// call this together. The per-chunk product count must fit int32 (true when each of the
// row's B rows, times 32, fits; the callers' classes guarantee it).
template <typename F>
__device__ __forceinline__ void warp_for_each_product(const DevCsr& A, const DevCsr& B, int64_t a0,
                                                      int64_t na, F&& f) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = 0; base < na; base += 32) {
    const int64_t e = base + lane;
    int32_t len = 0;
    int64_t bs = 0;
    if (e < na) {
      const int32_t k = A.col[a0 + e];
      bs = B.rp[k];
      len = static_cast<int32_t>(B.rp[k + 1] - bs);
    }
    const int32_t incl = warp_incl_scan(len);
    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
    for (int32_t p0 = 0; p0 < total; p0 += 32) {
      const int32_t p = p0 + lane;
      // owner = number of entries whose inclusive end is <= p
      int o = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int32_t v = __shfl_sync(0xffffffffu, incl, o + step - 1);
        if (v <= p) o += step;
      }
      const int32_t incl_o = __shfl_sync(0xffffffffu, incl, o & 31);
      const int32_t len_o = __shfl_sync(0xffffffffu, len, o & 31);
      const int64_t bs_o = __shfl_sync(0xffffffffu, bs, o & 31);
      if (p < total) f(bs_o + (p - (incl_o - len_o)), base + o);
    }
  }
}

// Block-flattened enumeration (NT threads). Shared scratch: s_excl[NT], s_bs[NT],
// scan[33] (int32). All threads of the block must call this together; it ends with
// __syncthreads.
template <int NT, typename F>
__device__ __forceinline__ void block_for_each_product(const DevCsr& A, const DevCsr& B, int64_t a0,
                                                       int64_t na, int32_t* s_excl, int64_t* s_bs,
                                                       int32_t* scan, F&& f) {
  for (int64_t base = 0; base < na; base += NT) {
    const int64_t e = base + threadIdx.x;
    int32_t len = 0;
    int64_t bs = 0;
    if (e < na) {
      const int32_t k = A.col[a0 + e];
      bs = B.rp[k];
      len = static_cast<int32_t>(B.rp[k + 1] - bs);
    }
    int32_t total;
    const int32_t ex = block_excl_scan<int32_t>(len, scan, &total);
    s_excl[threadIdx.x] = ex;
    s_bs[threadIdx.x] = bs;
    const int nvalid = static_cast<int>(na - base < NT ? na - base : NT);
    __syncthreads();
    int owner = 0;
    for (int32_t p = threadIdx.x; p < total; p += NT) {
      owner = find_owner(s_excl, nvalid, p, owner);
      f(s_bs[owner] + (p - s_excl[owner]), base + owner);
    }
    __syncthreads();
  }
}

}  // namespace spg
