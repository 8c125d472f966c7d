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

// Owner of each lane's partial product in a warp-contiguous range. The non-empty segments of a
// chunk of A entries are numbered 0..nent-1 with exclusive prefix c_excl (c_excl[nent] = total).
// For the 32 consecutive products p0..p0+31 whose first owner is `o`, lane t looks at the
// boundary c_excl[o + 1 + t]; the boundaries inside the group form a bit mask, and lane l's owner
// is o plus the number of boundaries at or before position l. Segments are non-empty, so at most
// 31 boundaries fall inside a group of 32 products.
__device__ __forceinline__ int group_owner(const int32_t* c_excl, int nent, int o, int32_t p0) {
  const int lane = threadIdx.x & 31;
  const int t = o + 1 + lane;
  const int32_t rel = (t <= nent ? c_excl[t] : 0x7fffffff) - p0;
  const unsigned bit = (rel >= 0 && rel < 32) ? (1u << rel) : 0u;
  const unsigned q = __reduce_or_sync(0xffffffffu, bit);
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  return o + __popc(q & upto);
}

// Hands out a warp's contiguous range of product numbers 32 at a time (lane l takes g0 + l). The
// segment owning the current group stays in registers: its start in B, its first product number,
// the next boundary, and a value the caller attaches to it (load(segment), e.g. its a_ik). A group
// that lies inside that segment (the next boundary 32 or more products on; o and g0 are the same on
// every lane, so the test is warp-uniform) touches no shared memory; a group across boundaries
// takes group_owner, and the segment of its last lane becomes the cached one. Segments past the
// last (the last lane beyond the range's end) are never asked for, so the cache is clamped.
template <typename T, typename Load>
struct GroupWalker {
  const int32_t* c_excl;
  const int64_t* c_bs;
  int nent;
  Load load;
  int o;
  int32_t oex, onext;
  int64_t obs;
  T oval;

  __device__ __forceinline__ GroupWalker(const int32_t* ce, const int64_t* cb, int n, int o0, Load ld)
      : c_excl(ce), c_bs(cb), nent(n), load(ld) {
    set(o0);
  }
  __device__ __forceinline__ void set(int o0) {
    o = o0 < nent ? o0 : nent - 1;
    oex = c_excl[o];
    onext = c_excl[o + 1];
    obs = c_bs[o];
    oval = load(o);
  }
  // The n products from p0 (same on every lane) all lie in the cached segment and below hi: the
  // lane's product p0 + l + 32 u then has index first(p0) + 32 u into B.
  __device__ __forceinline__ bool whole(int32_t p0, int32_t n, int32_t hi) const {
    return onext - p0 >= n && hi - p0 >= n;
  }
  __device__ __forceinline__ int64_t first(int32_t p0) const {
    return obs + (p0 + static_cast<int32_t>(threadIdx.x & 31) - oex);
  }
  // U consecutive groups from p0 (< hi, same on every lane) at once: lane l of group u gets the
  // index into B of product p0 + 32u + l (-1 at or past hi) and its segment's value. When at most
  // 32 segment boundaries fall among the 32U products, one load of the next 32 boundaries gives U
  // masks (one per group) and every group's owners follow from them without waiting on the
  // previous group; otherwise the groups are stepped one after the other.
  template <int U>
  __device__ __forceinline__ void step_many(int32_t p0, int32_t hi, int64_t (&j)[U], T (&val)[U]) {
    static_assert(U >= 1 && U <= 8, "groups per step");
    const int lane = static_cast<int>(threadIdx.x & 31);
    const int t = o + 1 + lane;
    const int32_t rel = (t <= nent ? c_excl[t] : 0x7fffffff) - p0;   // >= 0: o owns p0 or p0 - 1
    const bool more = __shfl_sync(0xffffffffu, rel, 31) < 32 * U;  // a 33rd boundary may lie inside
    if (more) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t g0 = p0 + 32 * u;
        j[u] = -1;
        val[u] = T(0);
        if (g0 < hi) step(g0, hi, j[u], val[u]);
      }
      return;
    }
    int before = 0;   // boundaries in the earlier groups
    int last = o;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned bit = (rel >= 32 * u && rel < 32 * (u + 1)) ? (1u << (rel - 32 * u)) : 0u;
      const unsigned q = __reduce_or_sync(0xffffffffu, bit);
      const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
      const int my = o + before + __popc(q & upto);
      const int32_t p = p0 + 32 * u + lane;
      j[u] = p < hi ? c_bs[my] + (p - c_excl[my]) : -1;
      val[u] = p < hi ? load(my) : T(0);
      before += __popc(q);
      last = o + before;
    }
    // the owner of the last product of the last group becomes the cached segment
    set(last);
  }
  // Group g0 (< hi, same on every lane): the lane's index into B (-1 at or past hi) and the
  // value of its segment (T(0) at or past hi). A product below hi has its owner below nent.
  __device__ __forceinline__ void step(int32_t g0, int32_t hi, int64_t& j, T& val) {
    const int32_t p = g0 + static_cast<int32_t>(threadIdx.x & 31);
    if (onext - g0 >= 32) {
      j = p < hi ? obs + (p - oex) : -1;
      val = oval;
    } else {
      // a lane past the range's end may be past the last segment (my == nent): no load for it
      const int my = group_owner(c_excl, nent, o, g0);
      j = p < hi ? c_bs[my] + (p - c_excl[my]) : -1;
      val = p < hi ? load(my) : T(0);
      set(__shfl_sync(0xffffffffu, my, 31));
    }
  }
};

template <typename T, typename Load>
__device__ __forceinline__ GroupWalker<T, Load> make_walker(const int32_t* c_excl, const int64_t* c_bs, int nent,
                                                            int o0, Load ld) {
  return GroupWalker<T, Load>(c_excl, c_bs, nent, o0, ld);
}

// Largest o in [0, nent) with c_excl[o] <= p.
__device__ __forceinline__ int search_owner(const int32_t* c_excl, int nent, int32_t p) {
  int lo = 0, hi = nent - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (c_excl[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Block-wide enumeration by contiguous ranges (NT threads): for each chunk of NT A entries the
// non-empty B rows are compacted and their products numbered; each warp takes one contiguous
// range of the numbers and walks it 32 at a time (lane l takes number p0 + l), finding the lanes'
// B rows with group_owner, so loads of B are coalesced along each row. f is called with U
// indices into B (-1: none) per step, so a caller can issue its loads before using them.
// Shared scratch: s_excl[NT + 1], s_bs[NT], s_scan64[33], s_ctl[2]. All threads call this
// together; it ends with __syncthreads. The products of one chunk must fit int32.
template <int NT, int U, typename F>
__device__ __forceinline__ void block_range_for_each_product(const DevCsr& A, const DevCsr& B, int64_t a0,
                                                             int64_t na, int32_t* s_excl, int64_t* s_bs,
                                                             long long* s_scan64, int32_t* s_ctl, F&& f) {
  const int wid = threadIdx.x >> 5;
  constexpr int kWarps = NT / 32;
  for (int64_t base = 0; base < na; base += NT) {
    const int64_t e = base + threadIdx.x;
    int64_t bs = 0;
    int32_t len = 0;
    if (e < na) {
      const int32_t k = A.col[a0 + e];
      bs = B.rp[k];
      len = static_cast<int32_t>(B.rp[k + 1] - bs);
    }
    const long long packed = (static_cast<long long>(len > 0) << 32) | static_cast<long long>(len);
    long long tot;
    const long long ex = block_excl_scan<long long>(packed, s_scan64, &tot);
    if (len > 0) {
      const int pos = static_cast<int>(ex >> 32);
      s_bs[pos] = bs;
      s_excl[pos] = static_cast<int32_t>(ex & 0xffffffffLL);
    }
    if (threadIdx.x == 0) {
      const int nent = static_cast<int>(tot >> 32);
      s_excl[nent] = static_cast<int32_t>(tot & 0xffffffffLL);
      s_ctl[0] = nent;
      s_ctl[1] = static_cast<int32_t>(tot & 0xffffffffLL);
    }
    __syncthreads();
    const int nent = s_ctl[0];
    const int32_t total = s_ctl[1];
    int32_t per = (total + kWarps - 1) / kWarps;
    per = (per + 31) & ~31;
    const int32_t lo = wid * per;
    const int32_t hi = total < lo + per ? total : lo + per;
    if (lo < hi) {
      auto walk = make_walker<int>(s_excl, s_bs, nent, search_owner(s_excl, nent, lo), [](int) { return 0; });
      for (int32_t p0 = lo; p0 < hi; p0 += 32 * U) {
        int64_t j[U];
        if (walk.whole(p0, 32 * U, hi)) {
          const int64_t j0 = walk.first(p0);
#pragma unroll
          for (int u = 0; u < U; ++u) j[u] = j0 + 32 * u;
        } else {
          int unused[U];
          walk.template step_many<U>(p0, hi, j, unused);
        }
        f(j);
      }
    }
    __syncthreads();
  }
}

}  // namespace spg
