// Internal interface of the batched product, used by the C ABI and by the server (internal).
#pragma once

#include "runtime.h"

namespace spg {

// Stacks the jobs, plans and runs the symbolic pass (blocks `stream`); the output is not yet
// allocated. On failure nothing is left allocated.
spgemm_status batch_prepare(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B, spgemm_prec prec,
                            const spgemm_opts* opts, const spgemm_allocator* alloc, void* stream,
                            spgemm_batch_t** out);
// Bounds, from the jobs' sizes alone, on the device bytes batch_prepare allocates: *lo is always
// allocated, *hi never exceeded.
void batch_prepare_bounds(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B, spgemm_prec prec,
                          const spgemm_opts* opts, int64_t* lo, int64_t* hi);
// Device bytes the prepared batch holds now, and the bytes its output will take.
int64_t batch_device_bytes(const spgemm_batch_t* b);
int64_t batch_output_bytes(const spgemm_batch_t* b);
// Exact device bytes of the whole batch once its numeric pass has run: what it holds now, the
// numeric pass's own tables and the output.
int64_t batch_needed_bytes(const spgemm_batch_t* b);
int64_t batch_products(const spgemm_batch_t* b);
int64_t batch_rows(const spgemm_batch_t* b);
// Row offsets of the stacked C (rows + 1 int64) after the symbolic pass, read to the host.
spgemm_status batch_row_offsets(const spgemm_batch_t* b, int64_t* host_off, void* stream);
int64_t batch_nnz(const spgemm_batch_t* b);
// Stream on which the batch's memory is handed back to the pool when it is destroyed.
void batch_set_release_stream(spgemm_batch_t* b, void* stream);
int64_t batch_jobs(const spgemm_batch_t* b);
// Allocates the output and enqueues the numeric pass and the per-job row pointers on `stream`.
spgemm_status batch_execute(spgemm_batch_t* b, void* stream);

}  // namespace spg
