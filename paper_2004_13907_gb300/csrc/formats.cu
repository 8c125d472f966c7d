// Format front-ends: COO to canonical CSR, and CSR transposition (a CSR matrix's CSC form is
// the CSR of its transpose), both on the device.
//
// The paper's CPU side turns the input matrices into its streamed row bundles (RIR, Sec. II)
// and back; here the host hands the library COO or CSC arrays and the conversion runs on the GPU.
// Both conversions are a stable sort of the entries by a key (the column for a transposition,
// (row, column) for COO), done by a least-significant-digit radix sort of 32-bit keys with 8-bit
// digits:
//   1. per tile of kSortTile keys, a histogram of the current digit (shared atomics);
//   2. per digit, an exclusive scan of its tile counts (one block per digit), and a scan of the
//      digit totals;
//   3. per tile, each key's position: its digit's base + the tile's offset in that digit + the
//      number of equal digits before it in the tile, counted in tile order (each warp takes 32
//      consecutive keys at a time: a match mask gives the rank among the warp's 32, per-warp
//      digit counters the rest), so equal keys keep their order.
// The sort carries a 32-bit index; the entries are gathered by it at the end.
#include <cstring>

#include "runtime.h"

namespace spg {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                        // keys per thread of a tile
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kRadix = 256;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                          int64_t ntiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t = blockIdx.x;
  const int64_t base = t * kSortTile;
  for (int q = threadIdx.x; q < kSortTile; q += kSortThreads) {
    const int64_t i = base + q;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  hist[int64_t(threadIdx.x) * ntiles + t] = h[threadIdx.x];
}

// One block per digit: exclusive scan of the digit's tile counts (in place), total to tot[d].
__global__ void __launch_bounds__(1024) k_rs_scan_tiles(uint32_t* __restrict__ hist, int64_t ntiles,
                                                        uint32_t* __restrict__ tot) {
  __shared__ uint32_t s_scan[33];
  uint32_t* row = hist + int64_t(blockIdx.x) * ntiles;
  uint32_t carry = 0;
  for (int64_t b = 0; b < ntiles; b += 1024) {
    const int64_t i = b + threadIdx.x;
    const uint32_t v = i < ntiles ? row[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan<uint32_t>(v, s_scan, &total);
    if (i < ntiles) row[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// One block of 256: exclusive scan of the digit totals.
__global__ void __launch_bounds__(kRadix) k_rs_scan_digits(const uint32_t* __restrict__ tot,
                                                           uint32_t* __restrict__ base) {
  __shared__ uint32_t s_scan[33];
  uint32_t total;
  base[threadIdx.x] = block_excl_scan<uint32_t>(tot[threadIdx.x], s_scan, &total);
}

__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ idx, int64_t n, int shift,
                                                             int64_t ntiles, const uint32_t* __restrict__ tile_off,
                                                             const uint32_t* __restrict__ dbase,
                                                             uint32_t* __restrict__ keys_out,
                                                             uint32_t* __restrict__ idx_out) {
  __shared__ uint32_t cnt[kSortWarps][kRadix];   // per warp: its keys of each digit, then its base
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t t = blockIdx.x;
  // warp w takes the tile's keys [w * 512, (w + 1) * 512), 32 at a time, in order
  const int64_t wbase = t * kSortTile + int64_t(w) * (kSortTile / kSortWarps);
  for (int d = lane; d < kRadix; d += 32) cnt[w][d] = 0;
  __syncwarp();
  for (int r = 0; r < kSortTile / kSortWarps / 32; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool ok = i < n;
    const uint32_t dg = ok ? (keys[i] >> shift) & (kRadix - 1) : 0u;
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? dg : kRadix + static_cast<uint32_t>(lane));
    if (ok && lane == __ffs(peers) - 1) cnt[w][dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: the warps' bases within the tile, added to the digit's base and the tile's offset
  {
    const int d = threadIdx.x;   // kSortThreads == kRadix
    uint32_t run = dbase[d] + tile_off[int64_t(d) * ntiles + t];
    for (int ww = 0; ww < kSortWarps; ++ww) {
      const uint32_t c = cnt[ww][d];
      cnt[ww][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int r = 0; r < kSortTile / kSortWarps / 32; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool ok = i < n;
    const uint32_t key = ok ? keys[i] : 0u;
    const uint32_t dg = (key >> shift) & (kRadix - 1);
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? dg : kRadix + static_cast<uint32_t>(lane));
    const uint32_t before = __popc(peers & ((1u << lane) - 1u));
    const uint32_t pos = cnt[w][dg] + before;
    __syncwarp();
    if (ok) {
      keys_out[pos] = key;
      idx_out[pos] = idx ? idx[i] : static_cast<uint32_t>(i);
      if (lane == __ffs(peers) - 1) cnt[w][dg] += __popc(peers);
    }
    __syncwarp();
  }
}

// Stable sort of n 32-bit keys whose values lie below 2^key_bits, carrying a 32-bit index (the
// identity when idx_in is NULL; idx_in is only read). keys_a holds the input keys on entry; the
// passes alternate between (keys_a, idx_a) and (keys_b, idx_b), and *result_in_b tells which pair
// holds the sorted keys and indices at the end. Returns the launches made.
int stable_sort(uint32_t* keys_a, uint32_t* idx_a, const uint32_t* idx_in, uint32_t* keys_b, uint32_t* idx_b,
                int64_t n, int key_bits, uint32_t* hist, uint32_t* tot, uint32_t* dbase, cudaStream_t s,
                bool* result_in_b) {
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  int launches = 0;
  uint32_t* ki = keys_a;
  const uint32_t* ii = idx_in;
  uint32_t* ko = keys_b;
  uint32_t* io = idx_b;
  uint32_t* spare_k = keys_a;
  uint32_t* spare_i = idx_a;
  bool in_b = false;
  for (int shift = 0; shift < (key_bits > 0 ? key_bits : 1); shift += 8) {
    k_rs_hist<<<static_cast<unsigned>(ntiles), kSortThreads, 0, s>>>(ki, n, shift, ntiles, hist);
    k_rs_scan_tiles<<<kRadix, 1024, 0, s>>>(hist, ntiles, tot);
    k_rs_scan_digits<<<1, kRadix, 0, s>>>(tot, dbase);
    k_rs_scatter<<<static_cast<unsigned>(ntiles), kSortThreads, 0, s>>>(ki, ii, n, shift, ntiles, hist, dbase, ko,
                                                                         io);
    launches += 4;
    // the next pass reads what this one wrote
    uint32_t* nk = (ko == keys_b) ? spare_k : keys_b;
    uint32_t* ni = (io == idx_b) ? spare_i : idx_b;
    in_b = ko == keys_b;
    ki = ko;
    ii = io;
    ko = nk;
    io = ni;
  }
  *result_in_b = in_b;
  return launches;
}

int bits_for(int64_t v) {
  int b = 0;
  while (b < 32 && (int64_t(1) << b) < v) ++b;
  return b;
}

// Row index of every stored entry of M (one thread per row writes its entries).
__global__ void k_expand_rows(const int64_t* __restrict__ rp, int64_t m, uint32_t* __restrict__ row_of) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x)
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) row_of[q] = static_cast<uint32_t>(i);
}

__global__ void k_keys_from_col(const int32_t* __restrict__ col, int64_t n, uint32_t* __restrict__ keys) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x)
    keys[q] = static_cast<uint32_t>(col[q]);
}

// Counts of each key (row of the output) into cnt[0..m) (zeroed), with a range check.
__global__ void k_count_keys(const uint32_t* __restrict__ keys, int64_t n, int64_t m, int64_t* __restrict__ cnt,
                             uint32_t* err) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = keys[q];
    if (k < m) atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[k]), 1ull);
    else atomicOr(err, kErrInvalidCsr);
  }
}

__global__ void __launch_bounds__(1024) k_scan_counts(const int64_t* __restrict__ cnt, int64_t m,
                                                      int64_t* __restrict__ rp) {
  __shared__ int64_t s_scan[33];
  int64_t carry = 0;
  for (int64_t b = 0; b < m; b += 1024) {
    const int64_t i = b + threadIdx.x;
    const int64_t v = i < m ? cnt[i] : 0;
    int64_t total;
    const int64_t ex = block_excl_scan<int64_t>(v, s_scan, &total);
    if (i < m) rp[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) rp[m] = carry;
}

// out row pointers (int32 or int64) from the int64 scan
__global__ void k_store_rowptr(const int64_t* __restrict__ rp, int64_t m1, void* out, int idx64) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m1; i += int64_t(gridDim.x) * blockDim.x) {
    if (idx64) static_cast<int64_t*>(out)[i] = rp[i];
    else static_cast<int32_t*>(out)[i] = static_cast<int32_t>(rp[i]);
  }
}

// The entries in sorted order: out_col[q] = new_col[perm[q]], out_val[q] = val[perm[q]] (8 or 4
// bytes per value).
__global__ void k_gather_entries(const uint32_t* __restrict__ perm, int64_t n, const uint32_t* __restrict__ new_col,
                                 const void* __restrict__ val, int vbytes, int32_t* __restrict__ out_col,
                                 void* __restrict__ out_val) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t p = perm[q];
    out_col[q] = static_cast<int32_t>(new_col[p]);
    if (vbytes == 8) static_cast<double*>(out_val)[q] = static_cast<const double*>(val)[p];
    else static_cast<float*>(out_val)[q] = static_cast<const float*>(val)[p];
  }
}

// COO inputs: keys = columns with a range check; row keys gathered through the first sort's order.
__global__ void k_coo_keys(const int32_t* __restrict__ col, int64_t n, int64_t ncols, uint32_t* __restrict__ keys,
                           uint32_t* err) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const int32_t c = col[q];
    if (c < 0 || c >= ncols) {
      atomicOr(err, kErrInvalidCsr);
      keys[q] = 0u;
    } else {
      keys[q] = static_cast<uint32_t>(c);
    }
  }
}

__global__ void k_gather_keys(const uint32_t* __restrict__ perm, int64_t n, const int32_t* __restrict__ src,
                              int64_t limit, uint32_t* __restrict__ keys, uint32_t* err) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = src[perm[q]];
    if (v < 0 || v >= limit) {
      atomicOr(err, kErrInvalidCsr);
      keys[q] = 0u;
    } else {
      keys[q] = static_cast<uint32_t>(v);
    }
  }
}

// Sorted COO entries: a repeated (row, column) pair is an error (the output must be canonical).
__global__ void k_check_unique(const uint32_t* __restrict__ perm, int64_t n, const int32_t* __restrict__ row,
                               const int32_t* __restrict__ col, uint32_t* err) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x + 1; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t a = perm[q - 1], b = perm[q];
    if (row[a] == row[b] && col[a] == col[b]) atomicOr(err, kErrInvalidCsr);
  }
}

unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

// Device scratch of one conversion, from the caller's allocator or the stream-ordered pool.
struct Scratch {
  Workspace ws;
  spgemm_status st = SPGEMM_OK;
  template <typename T>
  T* get(int64_t count) {
    if (st != SPGEMM_OK) return nullptr;
    void* p = ws.get(static_cast<size_t>(count < 1 ? 1 : count) * sizeof(T));
    if (!p) st = set_error_msg(SPGEMM_ERR_OOM, "conversion scratch of %lld bytes", (long long)(count * sizeof(T)));
    return static_cast<T*>(p);
  }
};

spgemm_status finish(Scratch& sc, uint32_t* err, cudaStream_t s, const char* what) {
  uint32_t h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  sc.ws.release_all();
  if (e != cudaSuccess) return cuda_status(e, what);
  if (h & kErrInvalidCsr)
    return set_error_msg(SPGEMM_ERR_INVALID_CSR, "%s: an index is out of range or a (row, column) pair repeats", what);
  if (h) return set_error_msg(SPGEMM_ERR_INTERNAL, "%s: device check failed (0x%x)", what, h);
  return SPGEMM_OK;
}

void init_scratch(Scratch& sc, const spgemm_allocator* alloc, void* stream) {
  sc.ws.stream = stream;
  if (alloc && alloc->alloc && alloc->free) {
    sc.ws.alloc = *alloc;
    sc.ws.has_alloc = true;
  }
}

}  // namespace

}  // namespace spg

using namespace spg;

extern "C" spgemm_status spgemm_csr_transpose(const spgemm_csr_in* M, int32_t value_bytes, spgemm_csr_out* T,
                                              const spgemm_allocator* alloc, void* stream) {
  clear_error_msg();
  if (!M || !T) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  if (value_bytes != 8 && value_bytes != 4) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "value_bytes is 8 or 4");
  spgemm_status st = check_csr_in(M, "M", value_bytes == 8 ? SPGEMM_F64 : SPGEMM_F32_COMPENSATED);
  if (st != SPGEMM_OK) return st;
  const int vbytes = value_bytes;
  const int64_t m = M->rows, n = M->cols, nnz = M->nnz;
  if (nnz > 0xffffffffLL) return set_error_msg(SPGEMM_ERR_UNSUPPORTED, "transposition takes fewer than 2^32 entries");
  if (!T->row_ptr || (nnz > 0 && (!T->col || !T->val)))
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "T's arrays are NULL");
  if (!T->idx64_rowptr && nnz > 0x7fffffffLL) return set_error_msg(SPGEMM_ERR_INDEX_OVERFLOW, "T needs an int64 row_ptr");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc;
  init_scratch(sc, alloc, stream);
  uint32_t* err = sc.get<uint32_t>(4);
  int64_t* rp64 = nullptr;
  if (!M->idx64_rowptr) rp64 = sc.get<int64_t>(m + 1);
  const int64_t ntiles = (nnz + kSortTile - 1) / kSortTile;
  uint32_t* keys_a = sc.get<uint32_t>(nnz);
  uint32_t* idx_a = sc.get<uint32_t>(nnz);
  uint32_t* keys_b = sc.get<uint32_t>(nnz);
  uint32_t* idx_b = sc.get<uint32_t>(nnz);
  uint32_t* row_of = sc.get<uint32_t>(nnz);
  uint32_t* hist = sc.get<uint32_t>(kRadix * (ntiles > 0 ? ntiles : 1));
  uint32_t* tot = sc.get<uint32_t>(kRadix);
  uint32_t* dbase = sc.get<uint32_t>(kRadix);
  int64_t* cnt = sc.get<int64_t>(n + 1);
  int64_t* trp = sc.get<int64_t>(n + 1);
  if (sc.st != SPGEMM_OK) {
    sc.ws.release_all();
    return sc.st;
  }
  cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
  const int64_t* rp = static_cast<const int64_t*>(M->row_ptr);
  if (!M->idx64_rowptr) {
    launch_rowptr_to64(static_cast<const int32_t*>(M->row_ptr), rp64, m + 1, s);
    rp = rp64;
  }
  cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (n + 1), s);
  if (nnz > 0) {
    k_keys_from_col<<<grid_for(nnz), 256, 0, s>>>(M->col, nnz, keys_a);
    k_count_keys<<<grid_for(nnz), 256, 0, s>>>(keys_a, nnz, n, cnt, err);
    if (m > 0) k_expand_rows<<<grid_for(m), 256, 0, s>>>(rp, m, row_of);
    bool in_b = false;
    stable_sort(keys_a, idx_a, nullptr, keys_b, idx_b, nnz, bits_for(n), hist, tot, dbase, s, &in_b);
    const uint32_t* perm = in_b ? idx_b : idx_a;
    k_gather_entries<<<grid_for(nnz), 256, 0, s>>>(perm, nnz, row_of, M->val, vbytes, T->col, T->val);
  }
  k_scan_counts<<<1, 1024, 0, s>>>(cnt, n, trp);
  k_store_rowptr<<<grid_for(n + 1), 256, 0, s>>>(trp, n + 1, T->row_ptr, T->idx64_rowptr);
  st = finish(sc, err, s, "transposing");
  if (st != SPGEMM_OK) return st;
  T->rows = n;
  T->cols = m;
  T->nnz = nnz;
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_coo_to_csr(int64_t rows, int64_t cols, int64_t nnz, const int32_t* row,
                                           const int32_t* col, const void* val, int32_t value_bytes,
                                           spgemm_csr_out* C, const spgemm_allocator* alloc, void* stream) {
  clear_error_msg();
  if (rows < 0 || cols < 0 || nnz < 0) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "negative size");
  if (rows > 0x7fffffffLL || cols > 0x7fffffffLL)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "row and column indices are int32");
  if (value_bytes != 8 && value_bytes != 4) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "value_bytes is 8 or 4");
  if (nnz > 0xffffffffLL) return set_error_msg(SPGEMM_ERR_UNSUPPORTED, "conversion takes fewer than 2^32 entries");
  if (!C || !C->row_ptr || (nnz > 0 && (!row || !col || !val || !C->col || !C->val)))
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL array");
  if (!C->idx64_rowptr && nnz > 0x7fffffffLL) return set_error_msg(SPGEMM_ERR_INDEX_OVERFLOW, "C needs an int64 row_ptr");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc;
  init_scratch(sc, alloc, stream);
  uint32_t* err = sc.get<uint32_t>(4);
  const int64_t ntiles = (nnz + kSortTile - 1) / kSortTile;
  uint32_t* keys_a = sc.get<uint32_t>(nnz);
  uint32_t* idx_a = sc.get<uint32_t>(nnz);
  uint32_t* keys_b = sc.get<uint32_t>(nnz);
  uint32_t* idx_b = sc.get<uint32_t>(nnz);
  uint32_t* keys_c = sc.get<uint32_t>(nnz);
  uint32_t* idx_c = sc.get<uint32_t>(nnz);
  uint32_t* hist = sc.get<uint32_t>(kRadix * (ntiles > 0 ? ntiles : 1));
  uint32_t* tot = sc.get<uint32_t>(kRadix);
  uint32_t* dbase = sc.get<uint32_t>(kRadix);
  int64_t* cnt = sc.get<int64_t>(rows + 1);
  int64_t* crp = sc.get<int64_t>(rows + 1);
  if (sc.st != SPGEMM_OK) {
    sc.ws.release_all();
    return sc.st;
  }
  cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
  cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (rows + 1), s);
  if (nnz > 0) {
    // sort by column, then (stably) by row: the entries end in (row, column) order
    k_coo_keys<<<grid_for(nnz), 256, 0, s>>>(col, nnz, cols, keys_a, err);
    bool in_b = false;
    stable_sort(keys_a, idx_a, nullptr, keys_b, idx_b, nnz, bits_for(cols), hist, tot, dbase, s, &in_b);
    const uint32_t* perm1 = in_b ? idx_b : idx_a;
    uint32_t* idx_keep = in_b ? idx_b : idx_a;        // the first order, read by the second sort
    uint32_t* idx_free = in_b ? idx_a : idx_b;
    k_gather_keys<<<grid_for(nnz), 256, 0, s>>>(perm1, nnz, row, rows, keys_c, err);
    bool in_c = false;
    stable_sort(keys_c, idx_free, idx_keep, keys_a, idx_c, nnz, bits_for(rows), hist, tot, dbase, s, &in_c);
    const uint32_t* keys_sorted = in_c ? keys_a : keys_c;
    const uint32_t* perm = in_c ? idx_c : idx_free;
    k_count_keys<<<grid_for(nnz), 256, 0, s>>>(keys_sorted, nnz, rows, cnt, err);
    k_check_unique<<<grid_for(nnz), 256, 0, s>>>(perm, nnz, row, col, err);
    // the column of each sorted entry: gather the input columns (as keys) through the order
    k_coo_keys<<<grid_for(nnz), 256, 0, s>>>(col, nnz, cols, keys_b, err);
    k_gather_entries<<<grid_for(nnz), 256, 0, s>>>(perm, nnz, keys_b, val, value_bytes, C->col, C->val);
  }
  k_scan_counts<<<1, 1024, 0, s>>>(cnt, rows, crp);
  k_store_rowptr<<<grid_for(rows + 1), 256, 0, s>>>(crp, rows + 1, C->row_ptr, C->idx64_rowptr);
  spgemm_status st = finish(sc, err, s, "converting COO to CSR");
  if (st != SPGEMM_OK) return st;
  C->rows = rows;
  C->cols = cols;
  C->nnz = nnz;
  return SPGEMM_OK;
}
