// Autotuner of the batched product: chooses the row-class thresholds (which rows take a thread
// merge, a warp, a block or the windowed kernels, and so the table size each row gets) and the
// window merge cap by timing the caller's own batch.
//
// Coordinate descent from the given options: for each parameter in turn, every candidate value
// is timed with the others fixed and the fastest is kept. A trial is one whole batch (stacking,
// plan, symbolic and numeric passes) timed with CUDA events on the caller's stream; the best of
// `reps` repetitions counts. Every candidate is a valid configuration, so the results of any
// trial are exact; only the time differs.
#include <cstring>
#include <string>

#include "batch.h"

namespace spg {
namespace {

struct Param {
  int32_t spgemm_opts::*field;
  int32_t values[4];
  int nvalues;
};

// Candidate values; the library defaults are among them.
const Param kParams[] = {
    {&spgemm_opts::window_hash_fill, {1024, 2048, 4096, 0}, 3},
    {&spgemm_opts::block_max, {1024, 2048, 4096, 0}, 3},
    {&spgemm_opts::warp_max, {64, 256, 1024, 0}, 3},
    {&spgemm_opts::tiny_max, {0, 16, 32, 0}, 3},
};

}  // namespace
}  // namespace spg

using namespace spg;

extern "C" spgemm_status spgemm_autotune_batch(int64_t n_jobs, const spgemm_csr_in* A, const spgemm_csr_in* B,
                                               spgemm_prec prec, const spgemm_opts* base, int32_t reps,
                                               void* stream, spgemm_opts* best, spgemm_tune_report* report) {
  clear_error_msg();
  if (!best) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "best is NULL");
  if (reps < 1) reps = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spgemm_opts cur;
  spgemm_opts_default(&cur);
  if (base) cur = *base;
  cur.record_timings = 0;
  spgemm_tune_report rep{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_status(ce, "creating the autotuner's events");
  }
  // one timed batch with options o (best of reps); returns a negative time on error
  auto trial = [&](const spgemm_opts& o, spgemm_status* st) -> double {
    double bestms = -1.0;
    for (int r = 0; r < reps; ++r) {
      spgemm_batch_t* b = nullptr;
      cudaEventRecord(e0, s);
      *st = spgemm_batch(n_jobs, A, B, prec, &o, nullptr, stream, &b);
      if (*st != SPGEMM_OK) return -1.0;
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess) *st = spgemm_batch_check(b, stream);
      spgemm_batch_destroy(b);
      if (e != cudaSuccess) {
        *st = cuda_status(e, "timing an autotuner trial");
        return -1.0;
      }
      if (*st != SPGEMM_OK) return -1.0;
      if (bestms < 0 || ms < bestms) bestms = ms;
    }
    return bestms;
  };
  auto record = [&](const spgemm_opts& o, double ms) {
    if (rep.trials < SPGEMM_TUNE_MAX_TRIALS) {
      rep.trial_ms[rep.trials] = ms;
      rep.trial_tiny_max[rep.trials] = o.tiny_max;
      rep.trial_warp_max[rep.trials] = o.warp_max;
      rep.trial_block_max[rep.trials] = o.block_max;
      rep.trial_window_fill[rep.trials] = o.window_hash_fill;
    }
    ++rep.trials;
  };
  spgemm_status st = SPGEMM_OK;
  trial(cur, &st);   // warm-up: first-touch of the memory pool and the kernels
  double best_ms = st == SPGEMM_OK ? trial(cur, &st) : -1.0;
  if (st == SPGEMM_OK) {
    record(cur, best_ms);
    rep.default_ms = best_ms;
    for (const Param& prm : kParams) {
      const int32_t start = cur.*prm.field;
      int32_t chosen = start;
      for (int v = 0; v < prm.nvalues && st == SPGEMM_OK; ++v) {
        if (prm.values[v] == start) continue;
        spgemm_opts o = cur;
        o.*prm.field = prm.values[v];
        const double ms = trial(o, &st);
        if (st != SPGEMM_OK) break;
        record(o, ms);
        if (ms < best_ms) {
          best_ms = ms;
          chosen = prm.values[v];
        }
      }
      if (st != SPGEMM_OK) break;
      cur.*prm.field = chosen;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SPGEMM_OK) return st;
  rep.best_ms = best_ms;
  rep.reps = reps;
  *best = cur;
  if (report) *report = rep;
  return SPGEMM_OK;
}
