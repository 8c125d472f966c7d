/* spgemm.h: C ABI of the GB300 sparse matrix-matrix product C = A*B (CSR in, CSR out).
 *
 * The operation is the row-by-row (Gustavson) product of the paper's Algorithm 1
 * (Sec. III-A, "A row-by-row formulation of SpGEMM"): row i of C is the merge, by column,
 * of the rows of B named by the column indices of row i of A, each scaled by the
 * matching value of A. Every column that receives a partial product is an entry of C,
 * even when its sum is exactly zero (Algorithm 1 emits every column of COLB), and each
 * row of C is sorted by column (Algorithm 1 sorts the partial products before merging;
 * the sort unit of Sec. III-A keeps them in column order).
 *
 * The call sequence splits the product the way the method does: a plan that counts the
 * partial products of each row (the B rows "streamed" for row i, Sec. III-A) and groups
 * rows by work (the device-side counterpart of the CPU scheduling of RIR bundles,
 * Sec. II and III-A), a symbolic pass that sizes every row of C, and a numeric pass that
 * multiplies, merges and writes the sorted rows (the match/multiply, sort and merge units
 * of Sec. III-A).
 *
 * Conventions for every entry point:
 *  - Pointers documented as "device" must be CUDA device pointers on the current device;
 *    "host" pointers are ordinary (pageable or pinned) host memory.
 *  - A CSR matrix has row_ptr[rows+1] (int32 or int64, chosen by idx64_rowptr), col[nnz]
 *    (int32) and val[nnz] (double for SPGEMM_F64, float for SPGEMM_F32_COMPENSATED).
 *    Inputs must be canonical: row_ptr[0] == 0, row_ptr non-decreasing, row_ptr[rows] ==
 *    nnz, and within each row the columns strictly increasing in [0, cols). Stored zeros
 *    are allowed and are structural.
 *  - Streams are cudaStream_t passed as void*; NULL means the legacy default stream.
 *  - Functions return a status and never throw or abort. On failure the thread-local
 *    message from spgemm_last_error() says what went wrong. A plan that returned an error
 *    other than SPGEMM_ERR_NOT_READY or SPGEMM_ERR_TIMEOUT must only be destroyed.
 *  - No entry point falls back to the CPU: every step of the product runs in the CUDA
 *    kernels of this library.
 */
#ifndef SPGEMM_H_
#define SPGEMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spgemm_status {
  SPGEMM_OK = 0,
  SPGEMM_ERR_INVALID_ARG = 1,     /* bad pointer, size, shape or call order */
  SPGEMM_ERR_INVALID_CSR = 2,     /* an input violates the canonical-CSR rules above */
  SPGEMM_ERR_OOM = 3,             /* the allocator returned NULL */
  SPGEMM_ERR_INDEX_OVERFLOW = 4,  /* nnz(C) needs an int64 row_ptr but int32 was requested */
  SPGEMM_ERR_CUDA = 5,            /* a CUDA runtime call failed (message has the CUDA error) */
  SPGEMM_ERR_TIMEOUT = 6,         /* a bounded wait gave up */
  SPGEMM_ERR_REJECTED = 7,        /* the server refused the job (over the memory cap) */
  SPGEMM_ERR_NOT_READY = 8,       /* a polled server job has not finished */
  SPGEMM_ERR_UNSUPPORTED = 9,     /* a size or combination this build does not handle */
  SPGEMM_ERR_INTERNAL = 10        /* a device-side consistency check failed */
} spgemm_status;

typedef enum spgemm_prec {
  SPGEMM_F64 = 0,              /* FP64 values, FP64 products and sums */
  SPGEMM_F32_COMPENSATED = 1   /* FP32 values; error-free product and compensated (two-sum)
                                  accumulation per entry; rows whose entries exceed the
                                  compensated error bound are recomputed in FP64 and
                                  rounded once to FP32 */
} spgemm_prec;

/* Input matrix (device pointers, caller-owned; must stay valid until the numeric pass's
 * stream work has completed). */
typedef struct spgemm_csr_in {
  int64_t rows, cols, nnz;
  int32_t idx64_rowptr;      /* 0: row_ptr is int32, 1: int64 */
  int32_t reserved_;
  const void* row_ptr;
  const int32_t* col;
  const void* val;
} spgemm_csr_in;

/* Output matrix (caller-allocated arrays: row_ptr[rows+1], col[nnz], val[nnz]). */
typedef struct spgemm_csr_out {
  int64_t rows, cols, nnz;
  int32_t idx64_rowptr;      /* 0: int32 row_ptr (only when nnz(C) < 2^31), 1: int64 */
  int32_t reserved_;
  void* row_ptr;
  int32_t* col;
  void* val;
} spgemm_csr_out;

/* Device workspace allocator. alloc returns device memory usable on `stream` (or NULL);
 * free releases it in stream order. When the allocator pointer passed to an entry point is
 * NULL the library allocates in stream order (cudaMallocFromPoolAsync / cudaFreeAsync) from a
 * memory pool of its own on the current device, which keeps freed memory reserved for reuse
 * by later calls until the process exits. */
typedef struct spgemm_allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} spgemm_allocator;

/* Tuning and test knobs. Fill with spgemm_opts_default() and change what you need. */
typedef struct spgemm_opts {
  int32_t validate;           /* 1 (default): check the canonical-CSR rules of A and B */
  int32_t tiny_max;           /* rows with <= this many products (<= 32) use one warp and no
                                 shared table (default 32; 0 disables the class) */
  int32_t warp_max;           /* symbolic: rows with min(P_i, n) <= this use a warp table;
                                 numeric: rows with nnz(C_i) <= warp_max/2 (default 1024) */
  int32_t block_max;          /* rows up to this size use a block-wide hash table; larger
                                 rows take the windowed path (default 2048, at most 4096) */
  int32_t window_hash_fill;   /* windowed rows: consecutive column blocks are merged into one
                                 window while it holds at most this many entries of C (default
                                 and maximum 4096; a single block is always one window) */
  int32_t force_window;       /* 1: every non-empty row takes the windowed path (tests) */
  int64_t rowptr32_limit;     /* nnz(C) >= this requires an int64 row_ptr (default 2^31-1;
                                 tests lower it) */
  int32_t f32c_rerun_all;     /* 1: recompute every F32 row in FP64 (tests) */
  int32_t f32c_rerun_none;    /* 1: never recompute (tests measure the bound alone) */
  int32_t num_streams;        /* unused (kept for the layout; default 4) */
  int32_t record_timings;     /* 1: record CUDA events around every stage of the passes
                                 (read them with spgemm_plan_get_timings); default 0 */
  int32_t window_split_max_mb;/* device memory budget (MiB) of the column-block split table
                                 of B used by the windowed rows (default 4096); when the table
                                 would be larger, those rows binary-search B instead (0: always) */
  int32_t max_sms;            /* grids of the persistent and grid-stride kernels are sized for
                                 this many SMs (0, default: all), leaving room on the device for
                                 work on other streams */
  int32_t window_cols_max_mb; /* device memory budget (MiB) in which the symbolic pass stores the
                                 column bitmaps of windowed rows (those within 2^20 columns; 512
                                 bytes per 4096 columns of the row), so the numeric pass copies
                                 them instead of marking every partial product again; rows beyond
                                 the budget are marked again (default 49152; 0: never store) */
  int32_t fp64_accumulate;    /* how FP64 sums are formed (F64 plans):
                                 0 (default): FP64 shared-memory atomics (fastest; the order of
                                   the additions, so the last bits, may vary from run to run);
                                 1: rows of the windowed path (more entries of C than a block
                                   table) sum every entry exactly in integer fixed point and round
                                   it once: the correctly rounded sum of the entry's products;
                                 2: deterministic: every non-empty row takes the windowed path
                                   with that exact sum, so every value of C is the correctly
                                   rounded sum of its FP64 partial products and repeats bit for
                                   bit. In 1 and 2 a row whose products span more than about 2^40
                                   in magnitude, or hold subnormal or non-finite values, is redone
                                   with FP64 atomics (counted in f32c_rerun_rows) */
  int32_t general_path;       /* 1: never take the small-product path. By default an F64 product
                                 with at most 65,536 rows and 32,768 columns of C and the default
                                 class options runs as a warp per row over a bitmap of all columns
                                 (one symbolic kernel, a scan, one numeric kernel around the single
                                 host read of nnz(C)); a row of C with more than 1,024 entries, or
                                 this flag, sends it through the general row classes */
  int32_t host_panels;        /* spgemm_multiply_host: row panels of A multiplied one after another
                                 while the previous panels' C is copied to the host, each with an
                                 equal share of the partial products. 0: 4 panels when A's entries
                                 times B's mean row length reach 1e8, else one; N >= 1: N panels
                                 (at most 64) */
  int32_t reserved[8];
} spgemm_opts;

/* Opaque plan: the work description of one product (row counts, row classes, row
 * offsets of C) and its device workspace. */
typedef struct spgemm_plan_s spgemm_plan_t;

/* Counters describing a plan (host values).
 * Row classes, in the order of the class arrays:
 *   symbolic: 0-3 windowed (P_i >= 2^22, >= 2^20, >= 2^17, rest), 4 block table,
 *             5-7 warp tables (2048, 512, 128 keys), 8 tiny (<= 32 products), 9 empty;
 *   numeric:  0-3 windowed (same split), 4-5 block tables (8192, 2048 slots),
 *             6-8 warp tables (1024, 256, 64 slots), 9 tiny, 10 empty. */
typedef struct spgemm_plan_info {
  int64_t rows, inner, cols;
  int64_t products;            /* sum_i P_i = number of partial products (flops = 2x) */
  int64_t nnz_c;               /* -1 before spgemm_symbolic */
  int64_t max_row_products;
  int64_t sym_class_rows[16];  /* rows per symbolic row class */
  int64_t num_class_rows[16];  /* rows per numeric row class (after spgemm_symbolic) */
  int64_t num_class_products[16];  /* sum of P_i over each numeric class */
  int64_t num_class_annz[16];      /* sum of nnz(A_i) over each numeric class */
  int64_t num_class_cnnz[16];      /* sum of nnz(C_i) over each numeric class */
  int64_t workspace_bytes;     /* device workspace held by the plan */
  int64_t f32c_rerun_rows;     /* rows recomputed in FP64 by the last numeric pass: F32 rows over
                                  the compensated bound; FP64 windowed rows outside the exact
                                  fixed-point range (read by spgemm_plan_check) */
  int64_t kernel_launches;     /* CUDA kernels this plan has launched so far */
  int32_t needs_rowptr64;
  int32_t state;               /* 0 planned, 1 symbolic done, 2 numeric done */
} spgemm_plan_info;

/* Stages timed when spgemm_opts.record_timings is set. */
typedef enum spgemm_stage {
  SPGEMM_STAGE_VALIDATE = 0,
  SPGEMM_STAGE_COUNT = 1,        /* product count, class scan, class scatter */
  SPGEMM_STAGE_SYM_WINDOW = 2,
  SPGEMM_STAGE_SYM_BLOCK = 3,
  SPGEMM_STAGE_SYM_WARP = 4,
  SPGEMM_STAGE_SYM_TINY = 5,
  SPGEMM_STAGE_SYM_SCAN = 6,     /* row offsets of C and numeric classes */
  SPGEMM_STAGE_NUM_ROWPTR = 7,
  SPGEMM_STAGE_NUM_WINDOW = 8,
  SPGEMM_STAGE_NUM_BLOCK = 9,
  SPGEMM_STAGE_NUM_WARP = 10,
  SPGEMM_STAGE_NUM_TINY = 11,
  SPGEMM_STAGE_NUM_RERUN = 12,   /* FP64 recomputation of flagged FP32 rows */
  SPGEMM_STAGE_NUM_EXPAND = 13,  /* columns of the windowed rows whose bitmap the symbolic pass stored */
  SPGEMM_NUM_STAGES = 14
} spgemm_stage;

typedef struct spgemm_timings {
  double ms[16];          /* device time of each stage's last run (CUDA events on its stream) */
  int32_t launches[16];   /* kernels launched by that run of the stage */
} spgemm_timings;

void spgemm_opts_default(spgemm_opts* opts);

/* The plan: validate A and B (if opts->validate), count P_i for every row of A
 * (the partial products of Algorithm 1's inner loops), and group the rows into classes by
 * work on the device. A and B are read on `stream`; the plan keeps their pointers.
 * Blocks `stream` once to read back the class sizes and sum_i P_i.
 * Small products take a path of their own: F64, 1 <= A.rows <= 65,536, B.cols <= 32,768, the
 * default class options (tiny_max 32, warp_max 1024, block_max 2048, window_hash_fill 4096,
 * force_window 0, fp64_accumulate 0) and general_path 0. There the plan does not block and
 * already launches the symbolic kernel on `stream` (one warp per row of A counts its row over a
 * bitmap of all columns of C; the numeric kernel later computes it the same way); INVALID_CSR in
 * A or B, sum_i P_i and the class counters (every row in the 1024-slot warp class) come with
 * spgemm_symbolic, which reads them back in its one host read (waiting for the plan's stream).
 * A row of C over 1,024 entries sends spgemm_symbolic back through the general plan (one more
 * host read).
 * Errors: INVALID_ARG (NULL pointers, A.cols != B.rows, negative sizes, prec mismatch),
 * INVALID_CSR, OOM, CUDA, UNSUPPORTED (sizes beyond int32 column indices). */
spgemm_status spgemm_plan(const spgemm_csr_in* A, const spgemm_csr_in* B, spgemm_prec prec,
                          const spgemm_opts* opts, const spgemm_allocator* alloc,
                          void* stream, spgemm_plan_t** out_plan);

/* The symbolic pass. Computes nnz(C_i) for every row (the size of Algorithm 1's
 * COLB set for row i), the row offsets of C, and the numeric row classes. Blocks `stream`
 * once and returns nnz(C) in *nnz_c and, in *needs_rowptr64, 1 when nnz(C) does not fit an
 * int32 row_ptr. Either output pointer may be NULL. Errors: INVALID_ARG (wrong state),
 * OOM, CUDA, INTERNAL. */
spgemm_status spgemm_symbolic(spgemm_plan_t* plan, void* stream, int64_t* nnz_c,
                              int32_t* needs_rowptr64);

/* The numeric pass. Writes C.row_ptr, C.col (sorted per row) and C.val into the
 * caller's device arrays, asynchronously on `stream` (no host synchronisation, except for
 * SPGEMM_F32_COMPENSATED, which reads back the number of rows to recompute in FP64).
 * C->rows/cols/nnz must equal A.rows/B.cols/nnz(C). May be called again on the same plan
 * (for example after the values of A or B changed but not their patterns).
 * Errors: INVALID_ARG (wrong state or shape, NULL arrays), INDEX_OVERFLOW, CUDA, INTERNAL. */
spgemm_status spgemm_numeric(spgemm_plan_t* plan, spgemm_csr_out* C, void* stream);

spgemm_status spgemm_plan_get_info(const spgemm_plan_t* plan, spgemm_plan_info* info);

/* Waits for `stream` and reports the device-side consistency checks latched by the passes
 * run so far on this plan (a row that wrote a different number of entries than the
 * symbolic pass counted, a full hash table): INTERNAL when any fired, else OK.
 * spgemm_numeric itself does not wait, so call this to check a numeric pass. */
spgemm_status spgemm_plan_check(spgemm_plan_t* plan, void* stream);

/* Waits for the recorded events and returns the per-stage times of the last run of each
 * stage (zero for stages that did not run or when record_timings was not set). */
spgemm_status spgemm_plan_get_timings(spgemm_plan_t* plan, spgemm_timings* timings);

/* Releases the workspace (in order on the stream given at plan time) and the plan.
 * NULL is accepted. */
spgemm_status spgemm_plan_destroy(spgemm_plan_t* plan);

/* One product through HOST buffers: copies A and B (host pointers) to the device, runs
 * plan, symbolic and numeric, and copies C back into the caller's host arrays C->row_ptr
 * (rows+1), C->col and C->val, which must hold nnz_capacity entries. When nnz(C) exceeds
 * nnz_capacity, *nnz_c is set and INVALID_ARG is returned (the host arrays' contents are then
 * unspecified), so the caller can grow its buffers and call again. Large products run in row
 * panels of A (opts->host_panels): each panel is planned and multiplied while the previous ones'
 * rows of C are copied to the host on a second stream. Synchronous. C->idx64_rowptr selects the
 * row_ptr type (INDEX_OVERFLOW when nnz(C) needs int64 and it is int32). Device staging comes
 * from `alloc` (cudaMallocAsync when NULL); panels of C come from the library's pool. */
spgemm_status spgemm_multiply_host(const spgemm_csr_in* A_host, const spgemm_csr_in* B_host,
                                   spgemm_prec prec, const spgemm_opts* opts,
                                   const spgemm_allocator* alloc, void* stream,
                                   spgemm_csr_out* C_host, int64_t nnz_capacity,
                                   int64_t* nnz_c);

/* ---- Batched products: C_j = A_j * B_j for n_jobs independent jobs, run as one product.
 * The jobs are stacked into one block-diagonal product, so the whole batch takes the launches of
 * a single product (plan, symbolic, numeric) instead of a set per job. A[j], B[j]: host arrays of
 * descriptors of device CSR matrices (as for spgemm_plan; same precision for all jobs), which must
 * stay valid while the batch is used. The call blocks `stream` (two reads, as plan and symbolic)
 * and returns with the numeric pass enqueued; results are valid once `stream` reaches that point.
 * The results are owned by the batch until spgemm_batch_destroy. Errors as spgemm_plan, plus
 * INVALID_CSR when a job's column index exceeds its own matrix and UNSUPPORTED when the stacked
 * batch has 2^31 or more rows or columns. */
typedef struct spgemm_batch_s spgemm_batch_t;

spgemm_status spgemm_batch(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B,
                           spgemm_prec prec, const spgemm_opts* opts, const spgemm_allocator* alloc,
                           void* stream, spgemm_batch_t** out_batch);

/* Job j's result as a standalone CSR view into the batch's arrays (device pointers, int64
 * row_ptr starting at 0, job-local column indices). */
spgemm_status spgemm_batch_result(const spgemm_batch_t* batch, int64_t job, spgemm_csr_out* C);

/* Counters of the stacked product (as spgemm_plan_get_info). */
spgemm_status spgemm_batch_get_info(const spgemm_batch_t* batch, spgemm_plan_info* info);

/* Waits for `stream` and reports the device-side consistency checks (as spgemm_plan_check). */
spgemm_status spgemm_batch_check(spgemm_batch_t* batch, void* stream);

/* Re-reads the jobs' current values (patterns unchanged) and recomputes every job's values, as
 * one CUDA graph launch on `stream`: the first call captures the value refresh and the numeric
 * pass into a graph, later calls launch it. FP64 batches only (UNSUPPORTED otherwise). */
spgemm_status spgemm_batch_replay(spgemm_batch_t* batch, void* stream);

spgemm_status spgemm_batch_destroy(spgemm_batch_t* batch);

/* ---- Autotuning of the batched form. Times the caller's batch (spgemm_batch with the same
 * arguments) under candidate row-class thresholds and window merge caps and returns the fastest
 * options. Coordinate descent from `base` (library defaults when NULL): window_hash_fill in
 * {1024, 2048, 4096}, block_max in {1024, 2048, 4096}, warp_max in {64, 256, 1024}, tiny_max in
 * {0, 16, 32}, each trial the best of `reps` (>= 1) runs of the whole batch, timed with CUDA events
 * on `stream`. Every candidate gives the same exact pattern and in-tolerance values; only the time
 * differs. Blocks until done (about 12 trials). *best receives the chosen options; report (may be
 * NULL) the trials in order. The paper has no counterpart: it chooses the thresholds of this
 * library's row classes. */
#define SPGEMM_TUNE_MAX_TRIALS 32
typedef struct {
  int32_t trials;             /* trials timed (the first is the starting options) */
  int32_t reps;
  double default_ms;          /* time of the starting options */
  double best_ms;             /* time of the chosen options */
  double trial_ms[SPGEMM_TUNE_MAX_TRIALS];
  int32_t trial_tiny_max[SPGEMM_TUNE_MAX_TRIALS];
  int32_t trial_warp_max[SPGEMM_TUNE_MAX_TRIALS];
  int32_t trial_block_max[SPGEMM_TUNE_MAX_TRIALS];
  int32_t trial_window_fill[SPGEMM_TUNE_MAX_TRIALS];
} spgemm_tune_report;

spgemm_status spgemm_autotune_batch(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B,
                                    spgemm_prec prec, const spgemm_opts* base, int32_t reps,
                                    void* stream, spgemm_opts* best, spgemm_tune_report* report);

/* ---- Format front-ends. The paper's CPU side reorganises the input matrices into its streamed
 * row bundles and back (Sec. II); here the reorganisation between formats runs on the device, as
 * a stable radix sort of the entries by their new row (see formats.cu). CSC is the CSR of the
 * transpose, so a product of CSC matrices needs no conversion: C = A*B in CSC is
 * C^T = B^T * A^T in CSR, i.e. spgemm_plan(B_csc viewed as CSR, A_csc viewed as CSR).
 *
 * spgemm_csr_transpose: T = M^T in CSR (= M in CSC). M: device CSR (int32 or int64 row_ptr),
 * values of value_bytes bytes (8: FP64, 4: FP32) copied as they are. T: caller-allocated device
 * arrays, row_ptr[M.cols + 1] (T->idx64_rowptr selects its type), col/val[M.nnz]; T->rows, cols
 * and nnz are set on return. Rows of T list their entries in ascending column (the order of M's
 * rows). Scratch (about 24 bytes per entry) comes from `alloc` (NULL: the library pool) on
 * `stream` and is freed before return; the call waits for `stream`. Errors: INVALID_ARG (NULL
 * arrays, bad value_bytes), INVALID_CSR (a column of M outside [0, M.cols)), UNSUPPORTED
 * (nnz >= 2^32), INDEX_OVERFLOW (int32 row_ptr too small).
 *
 * spgemm_coo_to_csr: canonical CSR from nnz (row, col, val) triples in any order (device arrays,
 * int32 indices, values of value_bytes bytes). C: caller-allocated, row_ptr[rows + 1], col/val[nnz];
 * columns come out sorted within each row. A repeated (row, col) pair or an index out of range
 * returns INVALID_CSR (the output of this library's products must be canonical). Scratch, waiting
 * and the other errors as for spgemm_csr_transpose. */
spgemm_status spgemm_csr_transpose(const spgemm_csr_in* M, int32_t value_bytes, spgemm_csr_out* T,
                                   const spgemm_allocator* alloc, void* stream);
spgemm_status spgemm_coo_to_csr(int64_t rows, int64_t cols, int64_t nnz, const int32_t* row, const int32_t* col,
                                const void* val, int32_t value_bytes, spgemm_csr_out* C,
                                const spgemm_allocator* alloc, void* stream);

/* C = A*B without allocating any device memory, for callers that cannot allocate while they
 * call: services that reserve the whole device up front and hand out fixed buffers (an
 * allocation would fail or take memory promised to someone else), and real-time loops that
 * must not block in an allocator or risk its failure. The paper has no counterpart; it is an
 * interface convenience of this library.
 * A and B: device CSR (int32 or int64 row_ptr), FP64 values, canonical. C: caller-allocated
 * device arrays, row_ptr[A.rows + 1] (C->idx64_rowptr selects its type) and col/val with room
 * for nnz_capacity entries. *nnz_c receives nnz(C). Limits: A.rows <= 65536 and every row of C
 * has at most 4096 entries (else SPGEMM_ERR_UNSUPPORTED); nnz(C) > nnz_capacity returns
 * SPGEMM_ERR_INVALID_ARG with *nnz_c set and nothing written to C. A column of A outside
 * [0, B.rows) or of B outside [0, B.cols) returns SPGEMM_ERR_INVALID_CSR (other CSR invariants
 * are not checked here).
 * Scratch: one fixed device array of about 770 KB inside the library, which every GPU that
 * loads the library holds until the process exits. The first call on a device looks up that
 * array's address (cudaGetSymbolAddress, with the device current). Every call uses the same
 * array: calls whose work overlaps on the GPU (from several threads or streams) race and must
 * be serialised by the caller. The call waits for `stream` twice (to read nnz(C) and the device
 * error word) and returns with C written. */
spgemm_status spgemm_multiply_noalloc(const spgemm_csr_in* A, const spgemm_csr_in* B,
                                      spgemm_csr_out* C, int64_t nnz_capacity, int64_t* nnz_c,
                                      void* stream);

/* ---- Serving: a long-lived server that takes products one at a time, from any host thread, and
 * runs them in fused batches (continuous batching). The paper has no counterpart; this is the
 * library's serving layer over the batched product above. A scheduler thread gathers queued jobs
 * in arrival order (up to max_batch_jobs, or until the jobs' input entries reach
 * max_batch_entries; it waits up to batch_window_us after the oldest queued job arrived for more
 * to come; small jobs may overtake a large one for up to max_defer_ms), stacks them as
 * spgemm_batch does and runs the plan and symbolic pass. That pass gives the EXACT device bytes of
 * the batch (stacked inputs, plan workspace, numeric tables and output); the numeric pass starts
 * only when the bytes held by the server plus that figure fit mem_cap_bytes, else it waits for
 * running batches to finish or for results to be released. A batch that does not fit the cap even
 * alone is split in halves; a single job that does not fit alone runs as row panels into a pinned
 * host result (host_panels), or is REJECTED when host_panels is 0 or a single row does not fit. A
 * batch whose preparation fails is retried job by job, so one bad job fails alone. Up to
 * num_streams batches are in flight, each on a stream of its own, so one batch's symbolic pass
 * overlaps another's numeric pass. Completion is signalled by a host callback on the batch's
 * stream; a job's latency runs from its submit call until it is marked done. Results stay in
 * device memory, counted against the cap, until spgemm_server_release. Every call is thread-safe. */
typedef struct spgemm_server_s spgemm_server_t;

typedef struct {
  int64_t mem_cap_bytes;       /* device bytes the server's batches and results may hold
                                  (default 32 GiB) */
  int64_t max_batch_entries;   /* a batch stops growing once its jobs' nnz(A)+nnz(B) reach
                                  this (default 2^24); a bigger job runs alone */
  int32_t max_batch_jobs;      /* jobs per batch at most (default 1024) */
  int32_t batch_window_us;     /* fill window after the oldest queued job (default 200) */
  int32_t num_streams;         /* batches in flight, 1..8 (default 2) */
  int32_t start_paused;        /* queue jobs but start none until spgemm_server_resume */
  int32_t prec;                /* spgemm_prec of every job (default SPGEMM_F64) */
  int32_t reserve_sms;         /* with 2+ streams, a batch holding at least half of
                                  max_batch_entries runs its kernels on all SMs but this many
                                  (opts.max_sms), so a batch of small jobs on another stream is not
                                  held behind it (default 0: off) */
  int32_t small_products;      /* jobs whose expected partial products, nnz(A)*nnz(B)/B.rows,
                                  are at most this are small: while the oldest queued job is larger
                                  and has waited less than max_defer_ms, batches take only small
                                  jobs, which so overtake it (default 2^26; 0: strict arrival
                                  order) */
  int32_t max_defer_ms;        /* longest a large job at the head of the queue is overtaken
                                  (default 250) */
  int32_t host_panels;         /* 1 (default): a single job over the cap runs as row panels, each
                                  under a quarter of the cap, into a result in pinned host memory;
                                  0: such a job is REJECTED */
  int32_t reserved_[3];
  spgemm_opts opts;            /* options of each batch's plan */
} spgemm_server_cfg;

typedef enum {
  SPGEMM_JOB_QUEUED = 0,
  SPGEMM_JOB_RUNNING = 1,      /* in a batch being prepared, admitted or computed */
  SPGEMM_JOB_DONE = 2,
  SPGEMM_JOB_FAILED = 3,       /* status says why (spgemm_server_poll sets the message) */
  SPGEMM_JOB_REJECTED = 4      /* needs more than mem_cap_bytes on its own */
} spgemm_job_state;

typedef struct {
  int32_t state;               /* spgemm_job_state */
  int32_t status;              /* spgemm_status of a finished job */
  int64_t batch;               /* id of the batch it ran in (-1 if none) */
  int64_t batch_jobs;          /* jobs in that batch */
  int64_t rows, cols, nnz;     /* shape and nnz of C */
  int64_t bytes;               /* device bytes of the job's result (row_ptr, col, val) */
  int64_t needed_bytes;        /* exact bytes of the smallest batch that held it (for a
                                  REJECTED job: what it alone would need) */
  double queue_ms;             /* submit -> its batch started preparing */
  double run_ms;               /* batch start -> done */
  double latency_ms;           /* submit -> done */
  int64_t panels;              /* row panels of a job run over the cap (0: none) */
  int64_t result_on_host;      /* 1: spgemm_server_result gives host pointers (row panels) */
} spgemm_job_info;

typedef struct {
  int64_t submitted, completed, failed, rejected, queued, running;
  int64_t batches;             /* batches completed */
  int64_t splits;              /* batches split for the memory cap */
  int64_t products;            /* partial products of completed batches */
  int64_t nnz_out;             /* entries of completed results */
  int64_t bytes_in_use;        /* device bytes held now (batches in flight + unreleased results) */
  int64_t bytes_peak;          /* most bytes held at once */
  int64_t mem_cap_bytes;
  double latency_p50_ms, latency_p99_ms, latency_max_ms, latency_mean_ms;
  double mean_batch_jobs;      /* jobs per completed batch */
  double elapsed_s;            /* first submit to last completion */
  double jobs_per_s;           /* completed jobs / elapsed_s */
  double products_per_s;       /* products / elapsed_s */
  int64_t kernel_launches;     /* kernels launched by completed batches */
  int64_t reserved_[7];
} spgemm_server_stats;

spgemm_status spgemm_server_cfg_default(spgemm_server_cfg* cfg);

/* Starts a server on the current device (its threads and num_streams streams). */
spgemm_status spgemm_server_create(const spgemm_server_cfg* cfg, spgemm_server_t** out_server);

/* Queues C = A*B. A, B: device CSR descriptors (as for spgemm_plan), in the server's precision;
 * the arrays must stay valid and unchanged until the job reaches a final state. *job receives
 * the job id. The server reads them on its own streams, which are not ordered after the caller's:
 * the arrays must already be written (synchronize the stream that produced them). Shape errors
 * are returned here (INVALID_ARG); errors found on the device fail the job. */
spgemm_status spgemm_server_submit(spgemm_server_t* server, const spgemm_csr_in* A,
                                   const spgemm_csr_in* B, int64_t* job);

/* Job state now: OK when done, NOT_READY while queued or running, the job's status when it
 * failed or was rejected (with its message in spgemm_last_error). info may be NULL. */
spgemm_status spgemm_server_poll(spgemm_server_t* server, int64_t job, spgemm_job_info* info);

/* As poll, but waits up to timeout_s seconds (< 0: no limit) for a final state; TIMEOUT if the
 * job is still queued or running then. */
spgemm_status spgemm_server_wait(spgemm_server_t* server, int64_t job, double timeout_s,
                                 spgemm_job_info* info);

/* Completion queue: waits up to timeout_s seconds (< 0: no limit, 0: no wait) for a job that
 * reached a final state (done, failed or rejected) and that this call has not returned yet, and
 * writes its id to *job. Jobs come out in the order they finished, each once; a job released
 * before it comes out is skipped. TIMEOUT when none finished in time (or the server is being
 * destroyed). Lets a client consume results as they finish without polling every job. */
spgemm_status spgemm_server_wait_any(spgemm_server_t* server, double timeout_s, int64_t* job);

/* A done job's result as a standalone CSR view (int64 row_ptr from 0), valid until
 * spgemm_server_release of that job: device pointers, or pinned host pointers for a job that ran
 * as row panels (spgemm_job_info.result_on_host). NOT_READY before it is done. */
spgemm_status spgemm_server_result(spgemm_server_t* server, int64_t job, spgemm_csr_out* C);

/* Forgets a finished job. Its result memory returns to the budget once every job of its batch
 * has been released. NOT_READY for a job not yet finished, INVALID_ARG for an unknown id. */
spgemm_status spgemm_server_release(spgemm_server_t* server, int64_t job);

/* Stop / restart starting new batches (queued and submitted jobs wait). */
spgemm_status spgemm_server_pause(spgemm_server_t* server);
spgemm_status spgemm_server_resume(spgemm_server_t* server);

/* Counters and latency percentiles since creation or the last reset. */
spgemm_status spgemm_server_get_stats(spgemm_server_t* server, spgemm_server_stats* stats);
spgemm_status spgemm_server_reset_stats(spgemm_server_t* server);

/* Stops the scheduler, waits for the batches in flight, fails jobs still queued and frees every
 * result. NULL is accepted. */
spgemm_status spgemm_server_destroy(spgemm_server_t* server);

/* Thread-local description of the last error on this thread ("" if none). */
const char* spgemm_last_error(void);

/* Library version string. */
const char* spgemm_version(void);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif /* SPGEMM_H_ */
