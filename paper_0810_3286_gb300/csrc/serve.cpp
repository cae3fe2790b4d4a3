// Serving runtime: first-in first-out admission of completion jobs by worker slots and device
// memory, one svt context and CUDA stream per job in flight, per-job arrival / start / end times.
// See include/svt_serve.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/svt.h"
#include "../../include/svt_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t id = 0;
  svt_job spec{};
  std::vector<int32_t> rows, cols;
  std::vector<double> vals;
  size_t bytes = 0;
  svt_job_result res{};
  std::vector<double> U, d, V;
  bool done = false;
};

}  // namespace

struct svt_server {
  svt_server_options opt{};
  int device = 0;
  int orth_grid = 0;   // cooperative-grid cap of a job that leaves svt_options.orth_grid at 0
  size_t budget = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::map<int64_t, std::unique_ptr<Job>> jobs;   // submitted and not yet collected
  size_t in_use = 0, peak_bytes = 0;
  int running = 0, peak_running = 0;
  int64_t next_id = 1, submitted = 0, completed = 0, failed = 0;
  double first_submit_ms = -1.0, last_end_ms = 0.0;
  std::vector<double> latencies_ms;
  bool stopping = false;
  std::vector<std::thread> workers;

  double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

  // head of the queue admissible now (strict FIFO)
  bool head_fits() const {
    if (queue.empty() || running >= opt.slots) return false;
    return in_use + queue.front()->bytes <= budget;
  }

  void run_job(Job* j, cudaStream_t st) {
    svt_job_result& r = j->res;
    if (opt.dry_run) {
      std::this_thread::sleep_for(std::chrono::microseconds(std::max<int64_t>(0, j->spec.dry_run_us)));
      r.status = SVT_OK;
      return;
    }
    svt_options o = j->spec.opt;
    o.stream = st;
    o.indices_on_device = 0;
    if (o.orth_grid == 0) o.orth_grid = orth_grid;
    svt_ctx* ctx = nullptr;
    svt_status s = svt_create(j->spec.m, j->spec.n, j->spec.nnz, j->rows.data(), j->cols.data(), j->vals.data(), &o,
                              &ctx);
    if (s == SVT_OK && j->spec.noise_sigma > 0.0) s = svt_set_noise_stop(ctx, j->spec.noise_sigma, j->spec.noise_eps);
    if (s == SVT_OK) {
      svt_result out{};
      s = svt_solve(ctx, j->spec.tau, j->spec.delta, j->spec.eps, j->spec.max_rank, &out);
      r.iterations = out.iterations;
      r.rank = (int)out.rank;
      r.residual = out.residual;
      if ((s == SVT_OK || s == SVT_ERR_NOT_CONVERGED) && opt.keep_factors && out.rank > 0) {
        const int rk = (int)out.rank;
        j->U.assign((size_t)j->spec.m * rk, 0.0);
        j->d.assign(rk, 0.0);
        j->V.assign((size_t)j->spec.n * rk, 0.0);
        const svt_status s2 = svt_get_factors(ctx, j->U.data(), j->d.data(), j->V.data(), rk);
        if (s2 != SVT_OK) s = s2;
      }
    }
    r.status = s;
    if (ctx) svt_destroy(ctx);
  }

  void worker() {
    cudaStream_t st = nullptr;
    if (!opt.dry_run) {
      cudaSetDevice(device);
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    }
    for (;;) {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return head_fits() || (stopping && queue.empty()); });
      if (queue.empty()) break;   // stopping and nothing left
      Job* j = queue.front();
      queue.pop_front();
      in_use += j->bytes;
      ++running;
      peak_bytes = std::max(peak_bytes, in_use);
      peak_running = std::max(peak_running, running);
      j->res.t_start_ms = now_ms();
      lk.unlock();
      run_job(j, st);
      lk.lock();
      in_use -= j->bytes;
      --running;
      j->res.t_end_ms = now_ms();
      j->done = true;
      if (j->res.status == SVT_OK) {
        ++completed;
        latencies_ms.push_back(j->res.t_end_ms - j->res.t_submit_ms);
        last_end_ms = std::max(last_end_ms, j->res.t_end_ms);
      } else {
        ++failed;
      }
      lk.unlock();
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  }
};

extern "C" void svt_server_default_options(svt_server_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->slots = 8;
}

extern "C" svt_status svt_server_create(const svt_server_options* opt, svt_server** out) {
  if (!out) return SVT_ERR_ARG;
  *out = nullptr;
  svt_server_options o;
  svt_server_default_options(&o);
  if (opt) o = *opt;
  if (o.slots < 1) return SVT_ERR_ARG;
  svt_server* s = new (std::nothrow) svt_server();
  if (!s) return SVT_ERR_OOM;
  s->opt = o;
  s->t0 = Clock::now();
  if (o.dry_run) {
    s->budget = o.device_budget ? o.device_budget : (size_t)-1;
  } else {
    size_t free_b = 0, total_b = 0;
    if (cudaGetDevice(&s->device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      (void)cudaGetLastError();
      delete s;
      return SVT_ERR_CUDA;
    }
    s->budget = o.device_budget ? o.device_budget : (size_t)(0.9 * (double)free_b);
    // the slots' cooperative orthonormalisations share the GPU: each gets an equal part of two
    // CTAs per SM (at least 16), so that all of them can be resident at once
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
      (void)cudaGetLastError();
      delete s;
      return SVT_ERR_CUDA;
    }
    s->orth_grid = std::max(16, 2 * sms / o.slots);
  }
  try {
    for (int i = 0; i < o.slots; ++i) s->workers.emplace_back([s] { s->worker(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
    return SVT_ERR_INTERNAL;
  }
  *out = s;
  return SVT_OK;
}

extern "C" svt_status svt_server_submit(svt_server* s, const svt_job* job, int64_t* job_id) {
  if (!s || !job || !job_id) return SVT_ERR_ARG;
  *job_id = 0;
  if (job->m < 1 || job->n < 1 || job->nnz < 1 || job->nnz > job->m * job->n) return SVT_ERR_ARG;
  if (!s->opt.dry_run && (!job->rows || !job->cols || !job->vals)) return SVT_ERR_ARG;
  std::unique_ptr<Job> j(new (std::nothrow) Job());
  if (!j) return SVT_ERR_OOM;
  j->spec = *job;
  if (s->opt.dry_run) {
    j->bytes = job->dry_run_bytes;
  } else {
    j->bytes = svt_estimate_device_bytes(job->m, job->n, job->nnz, &job->opt);
    if (j->bytes == 0) return SVT_ERR_ARG;
  }
  if (j->bytes > s->budget) return SVT_ERR_OOM;
  j->res.device_bytes = j->bytes;
  if (job->rows) j->rows.assign(job->rows, job->rows + job->nnz);
  if (job->cols) j->cols.assign(job->cols, job->cols + job->nnz);
  if (job->vals) j->vals.assign(job->vals, job->vals + job->nnz);
  j->spec.rows = nullptr;
  j->spec.cols = nullptr;
  j->spec.vals = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return SVT_ERR_ARG;
    j->id = s->next_id++;
    j->res.t_submit_ms = s->now_ms();
    if (s->first_submit_ms < 0) s->first_submit_ms = j->res.t_submit_ms;
    ++s->submitted;
    *job_id = j->id;
    s->queue.push_back(j.get());
    s->jobs[j->id] = std::move(j);
  }
  s->cv_work.notify_all();
  return SVT_OK;
}

extern "C" svt_status svt_server_wait(svt_server* s, int64_t job_id, svt_job_result* out, double* U, double* d,
                                      double* V, int capacity_r) {
  if (!s) return SVT_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return SVT_ERR_ARG;
  Job* j = it->second.get();
  s->cv_done.wait(lk, [&] { return j->done; });
  const int rk = (int)j->d.size();
  if ((U || d || V) && rk > capacity_r) return SVT_ERR_ARG;
  if (out) *out = j->res;
  for (int64_t i = 0; U && i < j->spec.m; ++i)
    for (int t = 0; t < rk; ++t) U[i * capacity_r + t] = j->U[(size_t)i * rk + t];
  for (int64_t i = 0; V && i < j->spec.n; ++i)
    for (int t = 0; t < rk; ++t) V[i * capacity_r + t] = j->V[(size_t)i * rk + t];
  for (int t = 0; d && t < rk; ++t) d[t] = j->d[t];
  s->jobs.erase(it);
  return SVT_OK;
}

extern "C" svt_status svt_server_drain(svt_server* s) {
  if (!s) return SVT_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->queue.empty() && s->running == 0; });
  return SVT_OK;
}

extern "C" svt_status svt_server_stats_get(svt_server* s, svt_server_stats* out) {
  if (!s || !out) return SVT_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof *out);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = (int64_t)s->queue.size();
  out->running = s->running;
  out->peak_bytes = s->peak_bytes;
  out->peak_running = s->peak_running;
  if (!s->latencies_ms.empty()) {
    std::vector<double> l = s->latencies_ms;
    std::sort(l.begin(), l.end());
    // nearest-rank percentiles
    auto pct = [&](double q) {
      size_t k = (size_t)std::ceil(q * (double)l.size());
      if (k < 1) k = 1;
      return l[std::min(k, l.size()) - 1];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0.0;
    for (double v : l) sum += v;
    out->mean_ms = sum / (double)l.size();
    const double span = s->last_end_ms - s->first_submit_ms;
    out->solves_per_s = span > 0 ? 1000.0 * (double)s->completed / span : 0.0;
  }
  return SVT_OK;
}

extern "C" void svt_server_destroy(svt_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}
