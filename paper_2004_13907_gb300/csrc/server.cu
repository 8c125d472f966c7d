// Serving layer: independent products submitted one at a time run in fused batches
// (continuous batching) over the stacked product of batch.cu.
//
// Two host threads per server. The scheduler gathers queued jobs into a batch, prepares it
// (stacking, plan, symbolic pass) on a free stream, admits it against the memory cap with the
// exact byte count the symbolic pass gives, and enqueues its numeric pass followed by a host
// callback. The completer takes batches whose callback fired, reads the device error word and
// marks their jobs done. With several streams, the next batch's symbolic pass runs while the
// previous batch's numeric pass is on the GPU.
//
// Locking: one mutex guards all server state. No CUDA call that can wait for a stream is made
// while holding it, because the stream callbacks take the same mutex.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.h"

namespace spg {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxStreams = 8;
constexpr int64_t kIndexLimit = 0x7fffffffLL;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

bool is_final(int32_t state) {
  return state == SPGEMM_JOB_DONE || state == SPGEMM_JOB_FAILED || state == SPGEMM_JOB_REJECTED;
}

struct Job {
  spgemm_csr_in A{}, B{};
  int32_t state = SPGEMM_JOB_QUEUED;
  spgemm_status status = SPGEMM_OK;
  std::string msg;
  int64_t entries = 0;     // nnz(A) + nnz(B)
  double work = 0.0;       // expected partial products, nnz(A) * nnz(B) / B.rows
  int64_t max_group = 1;   // largest batch it may join; halved when a batch is split for memory
  int64_t batch = -1;
  int64_t index = 0;       // position within its batch
  int64_t batch_jobs = 0;
  int64_t nnz = 0, bytes = 0, needed = 0;
  Clock::time_point t_submit, t_start, t_done;
  // a job over the cap runs as row panels and its result lives in pinned host memory
  int64_t panels = 0;
  int64_t* host_rp = nullptr;
  int32_t* host_col = nullptr;
  void* host_val = nullptr;
};

void free_host_result(Job& j) {
  if (j.host_rp) cudaFreeHost(j.host_rp);
  if (j.host_col) cudaFreeHost(j.host_col);
  if (j.host_val) cudaFreeHost(j.host_val);
  j.host_rp = nullptr;
  j.host_col = nullptr;
  j.host_val = nullptr;
}

struct BatchRec {
  spgemm_batch_t* b = nullptr;
  std::vector<int64_t> jobs;
  int slot = -1;
  int64_t bytes = 0;      // exact bytes charged to the budget
  int64_t live = 0;       // jobs not yet released
  int64_t products = 0;
  int64_t launches = 0;   // kernels the batch launched
  bool done = false;
};

}  // namespace
}  // namespace spg

using namespace spg;

struct spgemm_server_s {
  spgemm_server_cfg cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_sched;   // scheduler: new jobs, free slots, freed memory, resume, stop
  std::condition_variable cv_done;    // completer: batches whose stream passed the callback
  std::condition_variable cv_wait;    // callers of spgemm_server_wait
  bool stop = false, paused = false;
  std::deque<int64_t> pending;
  std::unordered_map<int64_t, Job> jobs;
  std::unordered_map<int64_t, BatchRec> batches;
  std::deque<int64_t> finished;
  std::deque<int64_t> final_q;        // jobs in a final state, not yet returned by wait_any
  int64_t next_job = 1, next_batch = 1;
  int num_streams = 1;
  int sm_count = 0;
  cudaStream_t streams[kMaxStreams]{};
  bool slot_busy[kMaxStreams]{};
  cudaStream_t release_stream = nullptr;
  int64_t in_use = 0, peak = 0;
  int64_t inflight = 0;               // batches prepared or running, not yet completed
  int64_t running = 0;                // jobs in those batches
  // statistics since creation or the last reset
  int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_rejected = 0;
  int64_t n_batches = 0, n_splits = 0, n_products = 0, n_nnz = 0, n_batch_jobs = 0, n_launches = 0;
  bool have_first = false;
  Clock::time_point first_submit, last_done;
  std::vector<double> latencies;
  std::thread scheduler, completer;

  int free_slot() const {
    for (int i = 0; i < num_streams; ++i)
      if (!slot_busy[i]) return i;
    return -1;
  }

  void charge(int64_t bytes) {
    in_use += bytes;
    peak = std::max(peak, in_use);
  }

  bool is_small(const Job& j) const { return j.work <= static_cast<double>(cfg.small_products); }

  // Positions in the queue of the jobs the next batch takes, in queue order; *limited is set when
  // a limit (rather than the end of the queue) stops it. Jobs are taken in arrival order, except
  // that while the oldest job is large (over small_products) and has waited less than
  // max_defer_ms, only small jobs are taken (they overtake it), so a burst of small requests does
  // not wait behind a long product.
  std::vector<size_t> pick_group(bool* limited) {
    std::vector<size_t> pos;
    *limited = false;
    if (pending.empty()) return pos;
    bool small_only = false;
    if (cfg.small_products > 0) {
      const Job& front = jobs.at(pending.front());
      const double waited = ms_between(front.t_submit, Clock::now());
      if (!is_small(front) && waited < cfg.max_defer_ms)
        for (int64_t id : pending)
          if (is_small(jobs.at(id))) { small_only = true; break; }
    }
    int64_t entries = 0, rows = 0, inner = 0, cols = 0;
    int64_t cap = cfg.max_batch_jobs;
    for (size_t q = 0; q < pending.size(); ++q) {
      const Job& j = jobs.at(pending[q]);
      if (small_only && !is_small(j)) continue;
      cap = std::min(cap, j.max_group);
      const bool over = !pos.empty() && (entries + j.entries > cfg.max_batch_entries || rows + j.A.rows >= kIndexLimit ||
                                         inner + j.B.rows >= kIndexLimit || cols + j.B.cols >= kIndexLimit);
      if (static_cast<int64_t>(pos.size()) >= cap || over) {
        *limited = true;
        break;
      }
      pos.push_back(q);
      entries += j.entries;
      rows += j.A.rows;
      inner += j.B.rows;
      cols += j.B.cols;
    }
    return pos;
  }

  void finish_job(int64_t id, int32_t state, spgemm_status st, const std::string& msg, Clock::time_point now) {
    Job& j = jobs.at(id);
    if (j.state == SPGEMM_JOB_RUNNING) --running;
    j.state = state;
    j.status = st;
    j.msg = msg;
    j.t_done = now;
    final_q.push_back(id);
    if (state == SPGEMM_JOB_DONE) {
      ++n_completed;
      latencies.push_back(ms_between(j.t_submit, now));
      n_nnz += j.nnz;
    } else if (state == SPGEMM_JOB_REJECTED) {
      ++n_rejected;
    } else {
      ++n_failed;
    }
  }

  // Puts a group back at the front of the queue, each job limited to batches of `max_group`.
  void requeue_front(const std::vector<int64_t>& group, int64_t max_group) {
    for (auto it = group.rbegin(); it != group.rend(); ++it) {
      Job& j = jobs.at(*it);
      if (j.state == SPGEMM_JOB_RUNNING) --running;
      j.state = SPGEMM_JOB_QUEUED;
      j.max_group = std::max<int64_t>(1, std::min(j.max_group, max_group));
      pending.push_front(*it);
    }
  }
};

namespace {

struct CallbackArg {
  spgemm_server_s* S;
  int64_t batch;
};

void CUDART_CB on_batch_done(void* p) {
  CallbackArg* a = static_cast<CallbackArg*>(p);
  {
    // notify under the lock: once it is released the server may be destroyed
    std::lock_guard<std::mutex> g(a->S->mu);
    a->S->finished.push_back(a->batch);
    a->S->cv_done.notify_all();
  }
  delete a;
}

// Frees a batch whose device work has finished, on the server's idle release stream, so the
// memory goes back to the pool at once rather than behind another batch's work.
void destroy_batch(spgemm_server_s* S, spgemm_batch_t* b) {
  batch_set_release_stream(b, S->release_stream);
  spgemm_batch_destroy(b);
}

// Device bytes of one panel: its plan's workspace and its output.
int64_t charged_need(spgemm_plan_t* p, int64_t prow, int64_t pnnz, int vb) {
  spgemm_plan_info info{};
  spgemm_plan_get_info(p, &info);
  return info.workspace_bytes + ws_rounded(8 * (prow + 1)) + ws_rounded(4 * pnnz) + ws_rounded(int64_t(vb) * pnnz);
}

// Runs a single job whose exact bytes exceed the cap as row panels: rows are cut where a panel's
// output (known exactly from the job's symbolic pass, `off`) reaches a quarter of the cap; each
// panel is its own product on A's rows [r0, r1) (row pointers rebased on the device) and B, charged
// to the cap while it runs, and copied into a pinned host result. Called and returns with the
// lock held; finishes the job.
void run_panels(spgemm_server_s* S, int64_t id, const std::vector<int64_t>& off, cudaStream_t stream,
                std::unique_lock<std::mutex>& lk) {
  Job& j = S->jobs.at(id);
  const spgemm_csr_in A = j.A, B = j.B;
  const spgemm_prec prec = static_cast<spgemm_prec>(S->cfg.prec);
  const spgemm_opts opts = S->cfg.opts;
  const int64_t cap = S->cfg.mem_cap_bytes;
  const int vb = prec == SPGEMM_F64 ? 8 : 4;
  const int64_t rows = A.rows, nnz = off[rows];
  lk.unlock();
  spgemm_status st = SPGEMM_OK;
  std::string msg;
  auto fail = [&](spgemm_status code, const char* what) {
    if (st == SPGEMM_OK) {
      st = code;
      msg = std::string(what) + ": " + spgemm_last_error();
    }
  };
  int64_t* hrp = nullptr;
  int32_t* hcol = nullptr;
  void* hval = nullptr;
  if (cudaMallocHost(&hrp, sizeof(int64_t) * (rows + 1)) != cudaSuccess ||
      cudaMallocHost(&hcol, sizeof(int32_t) * (nnz > 0 ? nnz : 1)) != cudaSuccess ||
      cudaMallocHost(&hval, size_t(vb) * (nnz > 0 ? nnz : 1)) != cudaSuccess) {
    cudaGetLastError();
    set_error_msg(SPGEMM_ERR_OOM, "pinned host memory for the result (%lld entries)", (long long)nnz);
    fail(SPGEMM_ERR_OOM, "row panels");
  }
  std::vector<int64_t> arp(static_cast<size_t>(rows) + 1);
  if (st == SPGEMM_OK) {
    std::memcpy(hrp, off.data(), sizeof(int64_t) * (rows + 1));
    cudaError_t e;
    if (A.idx64_rowptr) {
      e = cudaMemcpyAsync(arp.data(), A.row_ptr, sizeof(int64_t) * (rows + 1), cudaMemcpyDeviceToHost, stream);
    } else {
      std::vector<int32_t> t(static_cast<size_t>(rows) + 1);
      e = cudaMemcpyAsync(t.data(), A.row_ptr, sizeof(int32_t) * (rows + 1), cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      for (int64_t r = 0; r <= rows; ++r) arp[r] = t[r];
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) fail(cuda_status(e, "reading A's row pointers"), "row panels");
  }
  const int64_t budget = cap / 4;
  int64_t npanels = 0;
  for (int64_t r0 = 0; r0 < rows && st == SPGEMM_OK; ++npanels) {
    int64_t r1 = r0 + 1;
    while (r1 < rows && (off[r1 + 1] - off[r0]) * (4 + vb) + 8 * (r1 + 1 - r0) <= budget) ++r1;
    const int64_t prow = r1 - r0, base = arp[r0], pnnz = off[r1] - off[r0];
    int64_t* drp = nullptr;
    int64_t* dout_rp = nullptr;
    int32_t* dcol = nullptr;
    void* dval = nullptr;
    spgemm_plan_t* p = nullptr;
    int64_t charged = 0;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&drp), sizeof(int64_t) * (prow + 1), stream);
    if (e == cudaSuccess) {
      launch_rowptr_rebase(A.row_ptr, A.idx64_rowptr, r0, prow + 1, base, drp, stream);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) fail(cuda_status(e, "rebasing a panel's row pointers"), "row panels");
    spgemm_csr_in Ap{prow, A.cols, arp[r1] - base, 1, 0, drp, A.col + base,
                     static_cast<const unsigned char*>(A.val) + size_t(vb) * base};
    if (st == SPGEMM_OK && spgemm_plan(&Ap, &B, prec, &opts, nullptr, stream, &p) != SPGEMM_OK)
      fail(SPGEMM_ERR_INVALID_CSR, "panel plan");
    int64_t got = 0;
    if (st == SPGEMM_OK && spgemm_symbolic(p, stream, &got, nullptr) != SPGEMM_OK)
      fail(SPGEMM_ERR_INTERNAL, "panel symbolic");
    if (st == SPGEMM_OK && got != pnnz) {
      set_error_msg(SPGEMM_ERR_INTERNAL, "panel rows [%lld, %lld) have %lld entries, expected %lld", (long long)r0,
                    (long long)r1, (long long)got, (long long)pnnz);
      fail(SPGEMM_ERR_INTERNAL, "row panels");
    }
    if (st == SPGEMM_OK && charged_need(p, prow, pnnz, vb) > cap) {
      {   // a panel (a single row, since panels stop at a quarter of the cap) does not fit the cap
        const int64_t need = charged_need(p, prow, pnnz, vb);
        set_error_msg(SPGEMM_ERR_REJECTED, "rows [%lld, %lld) need %lld device bytes, over the server's cap of %lld",
                      (long long)r0, (long long)r1, (long long)need, (long long)cap);
        fail(SPGEMM_ERR_REJECTED, "row panels");
      }
    }
    if (st == SPGEMM_OK) {
      const int64_t need = charged_need(p, prow, pnnz, vb);
      lk.lock();
      S->cv_sched.wait(lk, [&] { return S->stop || S->in_use == 0 || S->in_use + need <= cap; });
      const bool stopped = S->stop;
      if (!stopped) {
        S->charge(need);
        charged = need;
      }
      lk.unlock();
      if (stopped) {
        set_error_msg(SPGEMM_ERR_INVALID_ARG, "server stopped");
        fail(SPGEMM_ERR_INVALID_ARG, "row panels");
      }
    }
    if (st == SPGEMM_OK) {
      e = cudaMallocAsync(reinterpret_cast<void**>(&dout_rp), sizeof(int64_t) * (prow + 1), stream);
      if (e == cudaSuccess)
        e = cudaMallocAsync(reinterpret_cast<void**>(&dcol), sizeof(int32_t) * (pnnz > 0 ? pnnz : 1), stream);
      if (e == cudaSuccess) e = cudaMallocAsync(&dval, size_t(vb) * (pnnz > 0 ? pnnz : 1), stream);
      if (e != cudaSuccess) fail(cuda_status(e, "allocating a panel's output"), "row panels");
    }
    if (st == SPGEMM_OK) {
      spgemm_csr_out Cp{prow, B.cols, pnnz, 1, 0, dout_rp, dcol, dval};
      if (spgemm_numeric(p, &Cp, stream) != SPGEMM_OK || spgemm_plan_check(p, stream) != SPGEMM_OK)
        fail(SPGEMM_ERR_INTERNAL, "panel numeric");
    }
    if (st == SPGEMM_OK && pnnz > 0) {
      e = cudaMemcpyAsync(hcol + off[r0], dcol, sizeof(int32_t) * pnnz, cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<unsigned char*>(hval) + size_t(vb) * off[r0], dval, size_t(vb) * pnnz,
                            cudaMemcpyDeviceToHost, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) fail(cuda_status(e, "copying a panel to the host"), "row panels");
    }
    cudaStreamSynchronize(stream);
    if (p) spgemm_plan_destroy(p);
    if (dval) cudaFreeAsync(dval, stream);
    if (dcol) cudaFreeAsync(dcol, stream);
    if (dout_rp) cudaFreeAsync(dout_rp, stream);
    if (drp) cudaFreeAsync(drp, stream);
    cudaStreamSynchronize(stream);
    if (charged) {
      lk.lock();
      S->in_use -= charged;
      lk.unlock();
      S->cv_sched.notify_all();
    }
    r0 = r1;
  }
  lk.lock();
  if (st != SPGEMM_OK) {
    if (hrp) cudaFreeHost(hrp);
    if (hcol) cudaFreeHost(hcol);
    if (hval) cudaFreeHost(hval);
    S->finish_job(id, st == SPGEMM_ERR_REJECTED ? SPGEMM_JOB_REJECTED : SPGEMM_JOB_FAILED, st, msg, Clock::now());
    return;
  }
  j.host_rp = hrp;
  j.host_col = hcol;
  j.host_val = hval;
  j.panels = npanels;
  j.nnz = nnz;
  j.bytes = 0;   // the result holds no device memory
  S->finish_job(id, SPGEMM_JOB_DONE, SPGEMM_OK, "", Clock::now());
}

void scheduler_main(spgemm_server_s* S) {
  cudaSetDevice(S->device);
  const spgemm_prec prec = static_cast<spgemm_prec>(S->cfg.prec);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_sched.wait(lk, [&] { return S->stop || (!S->paused && !S->pending.empty() && S->free_slot() >= 0); });
    if (S->stop) break;
    // fill window: wait for more jobs until the oldest queued one has waited batch_window_us
    const auto deadline = S->jobs.at(S->pending.front()).t_submit + std::chrono::microseconds(S->cfg.batch_window_us);
    bool limited = false;
    S->pick_group(&limited);
    while (!S->stop && !S->paused && !limited && Clock::now() < deadline) {
      S->cv_sched.wait_until(lk, deadline);
      if (S->pending.empty()) break;
      S->pick_group(&limited);
    }
    if (S->stop) break;
    if (S->paused || S->pending.empty()) continue;
    const std::vector<size_t> picked = S->pick_group(&limited);
    const int64_t n = static_cast<int64_t>(picked.size());
    std::vector<int64_t> group;
    group.reserve(picked.size());
    {
      std::deque<int64_t> rest;
      size_t k = 0;
      for (size_t q = 0; q < S->pending.size(); ++q) {
        if (k < picked.size() && picked[k] == q) {
          group.push_back(S->pending[q]);
          ++k;
        } else {
          rest.push_back(S->pending[q]);
        }
      }
      S->pending.swap(rest);
    }
    std::vector<spgemm_csr_in> As(n), Bs(n);
    for (int64_t k = 0; k < n; ++k) {
      As[k] = S->jobs.at(group[k]).A;
      Bs[k] = S->jobs.at(group[k]).B;
    }
    // bytes of the preparation from the sizes: split a group whose preparation could not fit
    // the cap, reject a job whose preparation alone is over it
    int64_t lo = 0, hi = 0;
    batch_prepare_bounds(n, As.data(), Bs.data(), prec, &S->cfg.opts, &lo, &hi);
    if (n > 1 && hi > S->cfg.mem_cap_bytes) {
      S->requeue_front(group, n / 2);
      ++S->n_splits;
      continue;
    }
    if (lo > S->cfg.mem_cap_bytes) {
      char buf[160];
      std::snprintf(buf, sizeof(buf), "the job needs at least %lld device bytes, over the server's cap of %lld",
                    (long long)lo, (long long)S->cfg.mem_cap_bytes);
      S->jobs.at(group[0]).needed = lo;
      S->finish_job(group[0], SPGEMM_JOB_REJECTED, SPGEMM_ERR_REJECTED, buf, Clock::now());
      S->cv_wait.notify_all();
      continue;
    }
    const auto t0 = Clock::now();
    for (int64_t id : group) {
      Job& j = S->jobs.at(id);
      j.state = SPGEMM_JOB_RUNNING;
      j.t_start = t0;
    }
    S->running += n;
    // hold the preparation back until its bytes fit beside what the server holds (a lone
    // oversized job goes ahead once nothing else is held, to learn its exact size)
    S->cv_sched.wait(lk, [&] { return S->stop || S->in_use == 0 || S->in_use + hi <= S->cfg.mem_cap_bytes; });
    if (S->stop) {
      for (int64_t id : group) S->finish_job(id, SPGEMM_JOB_FAILED, SPGEMM_ERR_INVALID_ARG, "server stopped", Clock::now());
      break;
    }
    const int slot = S->free_slot();
    S->slot_busy[slot] = true;
    ++S->inflight;
    const cudaStream_t stream = S->streams[slot];
    spgemm_opts opts = S->cfg.opts;
    {
      // a large batch leaves reserve_sms SMs to the batches on the other streams
      int64_t entries = 0;
      for (int64_t k = 0; k < n; ++k) entries += As[k].nnz + Bs[k].nnz;
      if (S->num_streams > 1 && S->cfg.reserve_sms > 0 && 2 * entries >= S->cfg.max_batch_entries &&
          S->sm_count > S->cfg.reserve_sms) {
        const int cap = S->sm_count - S->cfg.reserve_sms;
        if (opts.max_sms <= 0 || opts.max_sms > cap) opts.max_sms = cap;
      }
    }
    lk.unlock();

    spgemm_batch_t* b = nullptr;
    spgemm_status st = batch_prepare(n, As.data(), Bs.data(), prec, &opts, nullptr, stream, &b);
    std::string msg = st != SPGEMM_OK ? spgemm_last_error() : "";
    int64_t dev = 0, need = 0;
    if (st == SPGEMM_OK) {
      dev = batch_device_bytes(b);
      need = batch_needed_bytes(b);
    }

    lk.lock();
    auto give_up_slot = [&] {
      S->slot_busy[slot] = false;
      --S->inflight;
      S->cv_done.notify_all();
    };
    if (st != SPGEMM_OK) {
      give_up_slot();
      if (n > 1 && st != SPGEMM_ERR_CUDA) {
        // retry: halves after running out of memory, else one job at a time to find the bad job
        S->requeue_front(group, st == SPGEMM_ERR_OOM ? n / 2 : 1);
        if (st == SPGEMM_ERR_OOM) ++S->n_splits;
      } else {
        for (int64_t id : group) S->finish_job(id, SPGEMM_JOB_FAILED, st, msg, Clock::now());
        S->cv_wait.notify_all();
      }
      continue;
    }
    S->charge(dev);
    for (int64_t id : group) S->jobs.at(id).needed = need;
    if (need > S->cfg.mem_cap_bytes) {
      // does not fit even alone: split, run a single job as row panels, or reject it
      const bool paneled = n == 1 && S->cfg.host_panels != 0;
      std::vector<int64_t> off;
      spgemm_status ost = SPGEMM_OK;
      if (paneled) {
        off.resize(static_cast<size_t>(batch_rows(b)) + 1);
        lk.unlock();
        ost = batch_row_offsets(b, off.data(), stream);
        lk.lock();
      }
      S->in_use -= dev;
      if (!paneled) give_up_slot();
      lk.unlock();
      destroy_batch(S, b);
      lk.lock();
      if (n > 1) {
        S->requeue_front(group, n / 2);
        ++S->n_splits;
      } else if (paneled) {
        if (ost == SPGEMM_OK) run_panels(S, group[0], off, stream, lk);
        else S->finish_job(group[0], SPGEMM_JOB_FAILED, ost, spgemm_last_error(), Clock::now());
        give_up_slot();
        S->cv_wait.notify_all();
      } else {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "the job needs %lld device bytes, over the server's cap of %lld",
                      (long long)need, (long long)S->cfg.mem_cap_bytes);
        S->finish_job(group[0], SPGEMM_JOB_REJECTED, SPGEMM_ERR_REJECTED, buf, Clock::now());
        S->cv_wait.notify_all();
      }
      continue;
    }
    // exact admission: wait for completions or releases until the rest of the batch fits
    S->cv_sched.wait(lk, [&] { return S->stop || S->in_use + (need - dev) <= S->cfg.mem_cap_bytes; });
    if (S->stop) {
      S->in_use -= dev;
      give_up_slot();
      for (int64_t id : group) S->finish_job(id, SPGEMM_JOB_FAILED, SPGEMM_ERR_INVALID_ARG, "server stopped", Clock::now());
      lk.unlock();
      destroy_batch(S, b);
      lk.lock();
      break;
    }
    S->charge(need - dev);
    const int64_t bid = S->next_batch++;
    BatchRec& rec = S->batches[bid];
    rec.b = b;
    rec.jobs = group;
    rec.slot = slot;
    rec.bytes = need;
    rec.live = n;
    rec.products = batch_products(b);
    for (int64_t k = 0; k < n; ++k) {
      Job& j = S->jobs.at(group[k]);
      j.batch = bid;
      j.index = k;
      j.batch_jobs = n;
    }
    lk.unlock();

    st = batch_execute(b, stream);
    if (st == SPGEMM_OK) {
      CallbackArg* arg = new CallbackArg{S, bid};
      cudaError_t e = cudaLaunchHostFunc(stream, on_batch_done, arg);
      if (e != cudaSuccess) {
        delete arg;
        st = cuda_status(e, "enqueueing the completion callback");
      }
    }
    if (st != SPGEMM_OK) {
      msg = spgemm_last_error();
      cudaStreamSynchronize(stream);
      destroy_batch(S, b);
      lk.lock();
      S->batches.erase(bid);
      S->in_use -= need;
      give_up_slot();
      if (n > 1 && st == SPGEMM_ERR_OOM) {
        S->requeue_front(group, n / 2);
        ++S->n_splits;
      } else {
        for (int64_t id : group) {
          S->jobs.at(id).batch = -1;
          S->finish_job(id, SPGEMM_JOB_FAILED, st, msg, Clock::now());
        }
        S->cv_wait.notify_all();
      }
      continue;
    }
    lk.lock();
  }
}

void completer_main(spgemm_server_s* S) {
  cudaSetDevice(S->device);
  const int vb = S->cfg.prec == SPGEMM_F64 ? 8 : 4;
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_done.wait(lk, [&] { return !S->finished.empty() || (S->stop && S->inflight == 0); });
    if (S->finished.empty()) break;
    const int64_t bid = S->finished.front();
    S->finished.pop_front();
    BatchRec& rec = S->batches.at(bid);
    spgemm_batch_t* b = rec.b;
    const cudaStream_t stream = S->streams[rec.slot];
    const int64_t n = static_cast<int64_t>(rec.jobs.size());
    lk.unlock();

    spgemm_status st = spgemm_batch_check(b, stream);
    const std::string msg = st != SPGEMM_OK ? spgemm_last_error() : "";
    std::vector<spgemm_csr_out> outs(static_cast<size_t>(n));
    for (int64_t k = 0; k < n; ++k) spgemm_batch_result(b, k, &outs[k]);
    spgemm_plan_info pinfo{};
    spgemm_batch_get_info(b, &pinfo);

    lk.lock();
    const auto now = Clock::now();
    for (int64_t k = 0; k < n; ++k) {
      Job& j = S->jobs.at(rec.jobs[k]);
      j.nnz = outs[k].nnz;
      j.bytes = (outs[k].rows + 1) * 8 + outs[k].nnz * (4 + vb);
      S->finish_job(rec.jobs[k], st == SPGEMM_OK ? SPGEMM_JOB_DONE : SPGEMM_JOB_FAILED, st, msg, now);
    }
    rec.done = true;
    S->slot_busy[rec.slot] = false;
    --S->inflight;
    ++S->n_batches;
    S->n_products += rec.products;
    S->n_launches += pinfo.kernel_launches;
    S->n_batch_jobs += n;
    S->last_done = now;
    S->cv_sched.notify_all();
    S->cv_wait.notify_all();
  }
}

void fill_info(const spgemm_server_s* S, const Job& j, spgemm_job_info* info) {
  if (!info) return;
  *info = spgemm_job_info{};
  info->state = j.state;
  info->status = j.status;
  info->batch = j.batch;
  info->batch_jobs = j.batch_jobs;
  info->rows = j.A.rows;
  info->cols = j.B.cols;
  info->nnz = j.nnz;
  info->bytes = j.bytes;
  info->needed_bytes = j.needed;
  const auto now = Clock::now();
  const bool started = j.state != SPGEMM_JOB_QUEUED && j.t_start.time_since_epoch().count() != 0;
  info->queue_ms = ms_between(j.t_submit, started ? j.t_start : now);
  info->run_ms = started ? ms_between(j.t_start, is_final(j.state) ? j.t_done : now) : 0.0;
  info->latency_ms = ms_between(j.t_submit, is_final(j.state) ? j.t_done : now);
  info->panels = j.panels;
  info->result_on_host = j.host_rp != nullptr;
  (void)S;
}

spgemm_status final_status(const Job& j) {
  if (j.state == SPGEMM_JOB_DONE) return SPGEMM_OK;
  if (j.state == SPGEMM_JOB_FAILED || j.state == SPGEMM_JOB_REJECTED) return set_error_msg(j.status, "%s", j.msg.c_str());
  return set_error_msg(SPGEMM_ERR_NOT_READY, "job is %s", j.state == SPGEMM_JOB_QUEUED ? "queued" : "running");
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" spgemm_status spgemm_server_cfg_default(spgemm_server_cfg* cfg) {
  clear_error_msg();
  if (!cfg) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "cfg is NULL");
  *cfg = spgemm_server_cfg{};
  cfg->mem_cap_bytes = int64_t(32) << 30;
  cfg->max_batch_entries = int64_t(1) << 24;
  cfg->max_batch_jobs = 1024;
  cfg->batch_window_us = 200;
  cfg->num_streams = 2;
  cfg->start_paused = 0;
  cfg->prec = SPGEMM_F64;
  cfg->reserve_sms = 0;
  cfg->small_products = 1 << 26;
  cfg->max_defer_ms = 250;
  cfg->host_panels = 1;
  spgemm_opts_default(&cfg->opts);
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_create(const spgemm_server_cfg* cfg, spgemm_server_t** out) {
  clear_error_msg();
  if (!out) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  spgemm_server_cfg c{};
  spgemm_server_cfg_default(&c);
  if (cfg) c = *cfg;
  if (c.prec != SPGEMM_F64 && c.prec != SPGEMM_F32_COMPENSATED)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "unknown precision %d", int(c.prec));
  if (c.mem_cap_bytes <= 0 || c.max_batch_jobs < 1 || c.max_batch_entries < 1 || c.batch_window_us < 0 ||
      c.num_streams < 1 || c.num_streams > kMaxStreams || c.reserve_sms < 0 || c.small_products < 0 ||
      c.max_defer_ms < 0)
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "bad server configuration");
  spgemm_server_s* S = new (std::nothrow) spgemm_server_s();
  if (!S) return set_error_msg(SPGEMM_ERR_OOM, "host allocation of the server failed");
  // the stored-column workspace of a batch counts against the cap: at most an eighth of it
  const int64_t cols_mb = (c.mem_cap_bytes >> 20) / 8;
  if (c.opts.window_cols_max_mb > cols_mb) c.opts.window_cols_max_mb = static_cast<int32_t>(cols_mb);
  S->cfg = c;
  S->paused = c.start_paused != 0;
  S->num_streams = c.num_streams;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device);
  for (int i = 0; e == cudaSuccess && i < S->num_streams; ++i)
    e = cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->release_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    spgemm_status st = cuda_status(e, "creating the server streams");
    for (int i = 0; i < kMaxStreams; ++i)
      if (S->streams[i]) cudaStreamDestroy(S->streams[i]);
    if (S->release_stream) cudaStreamDestroy(S->release_stream);
    delete S;
    return st;
  }
  S->scheduler = std::thread(scheduler_main, S);
  S->completer = std::thread(completer_main, S);
  *out = S;
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_submit(spgemm_server_t* S, const spgemm_csr_in* A, const spgemm_csr_in* B,
                                              int64_t* job) {
  clear_error_msg();
  if (!S || !A || !B || !job) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  const spgemm_prec prec = static_cast<spgemm_prec>(S->cfg.prec);
  spgemm_status st;
  if ((st = check_csr_in(A, "A", prec)) != SPGEMM_OK) return st;
  if ((st = check_csr_in(B, "B", prec)) != SPGEMM_OK) return st;
  if (A->cols != B->rows) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "A.cols != B.rows");
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "the server is stopping");
    const int64_t id = S->next_job++;
    Job& j = S->jobs[id];
    j.A = *A;
    j.B = *B;
    j.entries = A->nnz + B->nnz;
    j.work = B->rows > 0 ? static_cast<double>(A->nnz) * static_cast<double>(B->nnz) / static_cast<double>(B->rows) : 0.0;
    j.max_group = S->cfg.max_batch_jobs;
    j.t_submit = Clock::now();
    if (!S->have_first) {
      S->have_first = true;
      S->first_submit = j.t_submit;
    }
    ++S->n_submitted;
    S->pending.push_back(id);
    *job = id;
  }
  S->cv_sched.notify_all();
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_poll(spgemm_server_t* S, int64_t job, spgemm_job_info* info) {
  clear_error_msg();
  if (!S) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->jobs.find(job);
  if (it == S->jobs.end()) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "unknown job %lld", (long long)job);
  fill_info(S, it->second, info);
  return final_status(it->second);
}

extern "C" spgemm_status spgemm_server_wait(spgemm_server_t* S, int64_t job, double timeout_s,
                                            spgemm_job_info* info) {
  clear_error_msg();
  if (!S) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->jobs.find(job) == S->jobs.end())
    return set_error_msg(SPGEMM_ERR_INVALID_ARG, "unknown job %lld", (long long)job);
  auto ready = [&] {
    auto it = S->jobs.find(job);
    return it == S->jobs.end() || is_final(it->second.state);
  };
  bool ok = true;
  if (timeout_s < 0 || !std::isfinite(timeout_s)) {
    S->cv_wait.wait(lk, ready);
  } else {
    ok = S->cv_wait.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
  }
  auto it = S->jobs.find(job);
  if (it == S->jobs.end()) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "job %lld was released", (long long)job);
  fill_info(S, it->second, info);
  if (!ok)
    return set_error_msg(SPGEMM_ERR_TIMEOUT, "job %lld still %s after %g s", (long long)job,
                         it->second.state == SPGEMM_JOB_QUEUED ? "queued" : "running", timeout_s);
  return final_status(it->second);
}

extern "C" spgemm_status spgemm_server_wait_any(spgemm_server_t* S, double timeout_s, int64_t* job) {
  clear_error_msg();
  if (!S || !job) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&] {
    while (!S->final_q.empty() && S->jobs.find(S->final_q.front()) == S->jobs.end()) S->final_q.pop_front();
    return S->stop || !S->final_q.empty();
  };
  bool ok = true;
  if (timeout_s < 0 || !std::isfinite(timeout_s)) {
    S->cv_wait.wait(lk, ready);
  } else {
    ok = S->cv_wait.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
  }
  if (!ok || S->final_q.empty())
    return set_error_msg(SPGEMM_ERR_TIMEOUT, "no job finished within %g s", timeout_s);
  *job = S->final_q.front();
  S->final_q.pop_front();
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_result(spgemm_server_t* S, int64_t job, spgemm_csr_out* C) {
  clear_error_msg();
  if (!S || !C) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->jobs.find(job);
  if (it == S->jobs.end()) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "unknown job %lld", (long long)job);
  const Job& j = it->second;
  if (j.state != SPGEMM_JOB_DONE) return final_status(j);
  if (j.host_rp) {   // row-paneled job: the result is in pinned host memory
    *C = spgemm_csr_out{j.A.rows, j.B.cols, j.nnz, 1, 0, j.host_rp, j.host_col, j.host_val};
    return SPGEMM_OK;
  }
  return spgemm_batch_result(S->batches.at(j.batch).b, j.index, C);
}

extern "C" spgemm_status spgemm_server_release(spgemm_server_t* S, int64_t job) {
  clear_error_msg();
  if (!S) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "server is NULL");
  spgemm_batch_t* dead = nullptr;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(job);
    if (it == S->jobs.end()) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "unknown job %lld", (long long)job);
    if (!is_final(it->second.state)) return set_error_msg(SPGEMM_ERR_NOT_READY, "job %lld has not finished", (long long)job);
    const int64_t bid = it->second.batch;
    free_host_result(it->second);
    S->jobs.erase(it);
    if (bid >= 0) {
      BatchRec& rec = S->batches.at(bid);
      if (--rec.live == 0) {
        dead = rec.b;
        S->in_use -= rec.bytes;
        S->batches.erase(bid);
      }
    }
  }
  if (dead) {
    DeviceGuard dg(S->device);
    destroy_batch(S, dead);
    S->cv_sched.notify_all();
  }
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_pause(spgemm_server_t* S) {
  clear_error_msg();
  if (!S) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(S->mu);
  S->paused = true;
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_resume(spgemm_server_t* S) {
  clear_error_msg();
  if (!S) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->paused = false;
  }
  S->cv_sched.notify_all();
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_get_stats(spgemm_server_t* S, spgemm_server_stats* out) {
  clear_error_msg();
  if (!S || !out) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "NULL argument");
  std::vector<double> lat;
  spgemm_server_stats st{};
  {
    std::lock_guard<std::mutex> g(S->mu);
    st.submitted = S->n_submitted;
    st.completed = S->n_completed;
    st.failed = S->n_failed;
    st.rejected = S->n_rejected;
    st.queued = static_cast<int64_t>(S->pending.size());
    st.running = S->running;
    st.batches = S->n_batches;
    st.splits = S->n_splits;
    st.products = S->n_products;
    st.nnz_out = S->n_nnz;
    st.bytes_in_use = S->in_use;
    st.bytes_peak = S->peak;
    st.mem_cap_bytes = S->cfg.mem_cap_bytes;
    st.kernel_launches = S->n_launches;
    st.mean_batch_jobs = S->n_batches ? double(S->n_batch_jobs) / double(S->n_batches) : 0.0;
    if (S->have_first && S->n_batches > 0 && S->last_done > S->first_submit)
      st.elapsed_s = std::chrono::duration<double>(S->last_done - S->first_submit).count();
    lat = S->latencies;
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto rank = [&](double q) {   // nearest-rank percentile
      size_t k = static_cast<size_t>(std::ceil(q * double(lat.size())));
      return lat[k == 0 ? 0 : k - 1];
    };
    st.latency_p50_ms = rank(0.50);
    st.latency_p99_ms = rank(0.99);
    st.latency_max_ms = lat.back();
    double sum = 0;
    for (double v : lat) sum += v;
    st.latency_mean_ms = sum / double(lat.size());
  }
  if (st.elapsed_s > 0) {
    st.jobs_per_s = double(st.completed) / st.elapsed_s;
    st.products_per_s = double(st.products) / st.elapsed_s;
  }
  *out = st;
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_reset_stats(spgemm_server_t* S) {
  clear_error_msg();
  if (!S) return set_error_msg(SPGEMM_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(S->mu);
  S->n_submitted = S->n_completed = S->n_failed = S->n_rejected = 0;
  S->n_batches = S->n_splits = S->n_products = S->n_nnz = S->n_batch_jobs = S->n_launches = 0;
  S->have_first = false;
  S->latencies.clear();
  S->peak = S->in_use;
  return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_server_destroy(spgemm_server_t* S) {
  if (!S) return SPGEMM_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
  S->cv_wait.notify_all();
  if (S->scheduler.joinable()) S->scheduler.join();
  S->cv_done.notify_all();
  if (S->completer.joinable()) S->completer.join();
  DeviceGuard dg(S->device);
  {
    std::lock_guard<std::mutex> g(S->mu);
    for (auto& kv : S->batches) destroy_batch(S, kv.second.b);
    S->batches.clear();
    for (auto& kv : S->jobs) free_host_result(kv.second);
    S->jobs.clear();
    S->pending.clear();
  }
  S->cv_wait.notify_all();
  cudaStreamSynchronize(S->release_stream);
  for (int i = 0; i < S->num_streams; ++i) cudaStreamDestroy(S->streams[i]);
  cudaStreamDestroy(S->release_stream);
  delete S;
  return SPGEMM_OK;
}
