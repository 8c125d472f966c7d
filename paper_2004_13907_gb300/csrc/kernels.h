// Host-side launch wrappers of the SpGEMM kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace spg {

constexpr int kTileRows = 1024;    // rows per tile in the counting / scan kernels
constexpr int kMaxClasses = 16;

struct DevCsr {
  int64_t rows, cols, nnz;
  const int64_t* rp;     // int64 row pointers (converted when the caller gave int32)
  const int32_t* col;
  const void* val;
};

// Summary the host reads back after the plan and after the symbolic pass.
struct Summary {
  int64_t class_off[kMaxClasses + 1];
  int64_t total;          // sum of P_i (plan) or of nnz(C_i) (symbolic)
  int64_t max_row;        // max P_i
  unsigned long long cls_sums[kMaxClasses][3];  // per numeric class: sum P_i, sum nnz(A_i), sum nnz(C_i)
  uint32_t err;
  uint32_t small_flags;   // small-product path: bit 0 = a row of C exceeds kSmallCap entries
  unsigned long long small_products;   // small-product path: sum of P_i
  uint32_t small_done;    // small-product path: blocks of the symbolic kernel that have finished
};

// ---- small products of narrow matrices (k_small.cu): a warp per row with a bitmap of all the
// row's columns (n, or a stacked batch's widest job); taken for F64 plans with m <=
// kSmallMaxRows (kSmallMaxBatchRows for batches) and a width <= kSmallMaxCols, left for the
// general path when a row of C has more than kSmallCap entries.
constexpr int64_t kSmallMaxRows = 65536;
constexpr int64_t kSmallMaxCols = 32768;
constexpr int64_t kSmallMaxBatchRows = int64_t(1) << 24;
constexpr int kSmallCap = 1024;
constexpr uint32_t kSmallUnwritten = 0x80000000u;   // small_flags of a host summary no kernel stored
// A CSR input with its row pointers as the caller stores them.
struct SmallCsr {
  int64_t rows, cols, nnz;
  const void* rp;        // int32 or int64 row pointers
  int32_t rp64;
  const int32_t* col;
  const void* val;
  const int32_t* cbase;  // A of a stacked batch: the first column of each row's job (else null)
};
bool small_path_fits(int64_t m, int64_t n);
// The symbolic kernel's grid: `blocks` blocks, each a contiguous run of `run` rows, its warps
// taking `groups` rows at a time.
struct SmallGrid {
  int64_t blocks, run;
  int groups;
};
SmallGrid small_sym_grid(const SmallCsr& A, int64_t width, int num_sms);
// Symbolic pass, validation of A and B (when `check`) and the offsets of C's rows, in one kernel:
// nnz_row[i], loc[i] (row i's offset within its block's run), blk[b] (run b's offset, b <= blocks,
// blk[blocks] = nnz(C)), summary->total (nnz(C)), max_row (longest row of C), small_products,
// small_flags, err. The summary must start zeroed. hsum (may be null): mapped page-locked memory
// (as a device pointer) that receives err, small_flags, small_products, max_row and total once
// the kernel ends.
int launch_small_symbolic(const SmallCsr& A, const SmallCsr& B, int64_t width, SmallGrid g, int check,
                          int32_t* nnz_row, int32_t* loc, int64_t* blk, Summary* sum, Summary* hsum,
                          cudaStream_t s);
// c_off[i] = offset of row i of C (i <= m) from the symbolic kernel's runs (a stacked batch reads them).
int launch_small_offsets(const int32_t* loc, const int64_t* blk, SmallGrid g, int64_t m, int64_t* c_off,
                         cudaStream_t s);
// Numeric pass: the row pointers (int32 or int64), columns and values of C; `cap` = the longest
// row of C (at most kSmallCap).
int launch_small_numeric(const SmallCsr& A, const SmallCsr& B, int64_t width, SmallGrid g, int cap,
                         const int32_t* nnz_row,
                         const int32_t* loc, const int64_t* blk, void* crp, int crp64, int32_t* ccol, double* cval,
                         uint32_t* err, int num_sms, cudaStream_t s);

// ---- setup / scan kernels (k_setup.cu)
int launch_rowptr_to64(const int32_t* in, int64_t* out, int64_t n1, cudaStream_t s);
// dst (mapped page-locked host memory, as a device pointer) = src[0 .. bytes), bytes a multiple of 4.
int launch_fetch(const void* src, void* dst, int64_t bytes, cudaStream_t s);
// out[t] = in[r0 + t] - base for t < n1 (in: int32 or int64 row pointers).
int launch_rowptr_rebase(const void* in, int idx64, int64_t r0, int64_t n1, int64_t base, int64_t* out,
                         cudaStream_t s);
// starts: scratch of validate_words(M.nnz) words (the row-start bitmap).
int64_t validate_words(int64_t nnz);
int launch_validate(const DevCsr& M, uint32_t* starts, uint32_t* err, cudaStream_t s);
int launch_count(const DevCsr& A, const DevCsr& B, ClassParams cp, int64_t* P, int32_t* nnz_row,
                  int32_t* tile_hist, int64_t* tile_sum, int64_t* tile_max, cudaStream_t s);
int launch_class_scan(int64_t ntiles, int nclasses, int32_t* tile_hist, const int64_t* tile_sum,
                       const int64_t* tile_max, int64_t* tile_sum_off, Summary* summary,
                       cudaStream_t s);
int launch_scatter_sym(const DevCsr& A, ClassParams cp, const int64_t* P, const int32_t* tile_hist,
                        int32_t* perm, cudaStream_t s);
int launch_num_tiles(const DevCsr& A, ClassParams cp, const int64_t* P, const int32_t* nnz_row,
                      int32_t* tile_hist, int64_t* tile_sum, unsigned long long* cls_sums,
                      cudaStream_t s);
int launch_scatter_num(const DevCsr& A, ClassParams cp, const int64_t* P, const int32_t* nnz_row,
                        const int32_t* tile_hist, const int64_t* tile_sum_off, int32_t* perm,
                        int64_t* c_off, cudaStream_t s);
int launch_write_rowptr(const int64_t* c_off, int64_t m1, void* out, int idx64, cudaStream_t s);

// ---- symbolic kernels (k_symbolic.cu). Each handles perm[start, start+count).
int launch_sym_tiny(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     int32_t* nnz_row, int num_sms, cudaStream_t s);
// Micro rows (nnz(A_i) <= kMicroNa): one thread per row merges the B rows.
int launch_sym_micro(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     int32_t* nnz_row, int num_sms, cudaStream_t s);
int launch_sym_warp(int log2S, const DevCsr& A, const DevCsr& B, const int32_t* perm,
                     int64_t count, int32_t* nnz_row, uint32_t* err, int num_sms, cudaStream_t s);
int launch_sym_block(int log2S, const DevCsr& A, const DevCsr& B, const int32_t* perm,
                      int64_t count, int32_t* nnz_row, uint32_t* err, int num_sms, cudaStream_t s);
// abase (per row of A, may be NULL = 0) and awidth (per row, may be NULL = width) give each
// row's column space [abase[i], abase[i] + awidth[i]); blocks are counted from abase[i]. nblocks
// (the block-count stride of a row) covers the widest row. wbits (may be NULL) receives, for each
// row no wider than one symbolic window, its column bitmap (128 words per block of the row) at
// word woff[slot], reserved from the cursor *wcur; -1 when the wcap words are used up or the row
// is wider.
int launch_sym_window(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                       int32_t* counter, int32_t* nnz_row, int32_t* win_slot, uint16_t* blockcnt,
                       int64_t nblocks, int32_t* cursor, const int32_t* abase, const int32_t* awidth,
                       int64_t width, uint32_t* wbits, int64_t wcap, unsigned long long* wcur, int64_t* woff,
                       int num_sms, uint32_t* err, cudaStream_t s);

// ---- numeric kernels, FP64 (k_numeric.cu)
int launch_num_tiny(int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                    const int64_t* c_off, int32_t* ccol, void* cval, int32_t* row_flag, const int32_t* abase,
                    uint32_t* err, int num_sms, cudaStream_t s);
int launch_num_micro(const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     const int64_t* c_off, int32_t* ccol, double* cval, const int32_t* abase, uint32_t* err,
                     int num_sms, cudaStream_t s);
// Warp and block hash kernels, kModeF64 or kModeF32C (row_flag lists kModeF32C rows for the FP64
// recomputation; negflag is the device flag of launch_negative_check).
int launch_num_warp(int log2S, int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                    const int64_t* c_off, int32_t* ccol, void* cval, const int32_t* abase, int32_t* row_flag,
                    const int32_t* negflag, uint32_t* err, int num_sms, cudaStream_t s);
int launch_num_block(int log2S, int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                     const int64_t* c_off, int32_t* ccol, void* cval, const int32_t* abase, int32_t* row_flag,
                     const int32_t* negflag, uint32_t* err, int num_sms, cudaStream_t s);

// ---- windowed numeric pass and the column-block split table of B (k_window.cu)
// Columns of C for the windowed rows with a stored bitmap (k_window.cu); rows without one get
// theirs from the windowed numeric kernel.
int launch_expand_cols(const int32_t* perm, int64_t count, const int32_t* win_slot, const int64_t* woff,
                       const uint32_t* wbits, const uint16_t* blockcnt, int64_t nblocks, const int64_t* c_off,
                       const int32_t* awidth, int64_t width, int32_t* ccol, int num_sms, uint32_t* err,
                       cudaStream_t s);

// ---- FP64 recomputation of flagged windowed FP32 rows (k_rerun.cu): groups of group_rows rows
// share `dense` (group_rows * width FP64), every partial product added with a global atomic.
int64_t rerun_group_rows(int64_t width, int64_t budget_bytes);
int launch_rerun_dense(const DevCsr& A, const DevCsr& B, const int32_t* rows, int64_t nrows, const int64_t* c_off,
                       int32_t* ccol, float* cval, const int32_t* abase, int64_t width, double* dense,
                       int64_t group_rows, int num_sms, uint32_t* err, cudaStream_t s);

int64_t split_table_bytes(int64_t brows, int64_t nblocks);
int launch_bsplit(const DevCsr& B, int64_t nblocks, const int32_t* bbase, int32_t* split, cudaStream_t s);
int launch_num_window(int mode, const DevCsr& A, const DevCsr& B, const int32_t* perm, int64_t count,
                      int32_t* counter, const int64_t* c_off, const int32_t* win_slot,
                      const uint16_t* blockcnt, int64_t nblocks, int64_t nslots, const int32_t* split,
                      int32_t merge_cap, int32_t* ccol, void* cval, int32_t* row_flag,
                      const int32_t* abase, const int32_t* awidth, int64_t width, const uint32_t* wbits,
                      const int64_t* woff, const uint16_t* bexp, const int32_t* dev_count,
                      const int32_t* negflag, int64_t* list_bs, int32_t* list_len, double* list_av,
                      int64_t list_cap, int num_sms, uint32_t* err, cudaStream_t s);
// Blocks of k_num_window for `count` rows (its grid), and the entries each block's window lists of
// a row with more than 512 A entries can hold (list_cap; 0 turns the lists off).
int64_t num_window_blocks(int64_t count, int num_sms);
// *flag = 1 if a value of the FP32 arrays a[na] or b[nb] is negative, infinite or NaN, else 0.
int launch_negative_check(const void* a, int64_t na, const void* b, int64_t nb, int32_t* flag, int num_sms,
                          cudaStream_t s);
// Largest biased exponent of the values of every row of B (FP64), for the exact accumulation mode
int launch_brow_exponent(const DevCsr& B, uint16_t* bexp, int num_sms, cudaStream_t s);
// F32-compensated rerun lists: the rows of perm[0, count) whose flag is set (all rows when
// `all`), appended to list at list_count (a device counter)
int launch_collect_flagged(const int32_t* perm, int64_t count, const int32_t* row_flag, int all,
                           int32_t* list, int32_t* list_count, cudaStream_t s);

}  // namespace spg
