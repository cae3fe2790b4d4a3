/*
 * svt_serve.h: serving runtime of libsvt.  A server takes a stream of matrix completion jobs
 * (each one Algorithm 1 of Sec. 5.1.5 on its own Omega, sampled values and parameters), admits
 * them in arrival order as worker slots and device memory free up, and runs every admitted job on
 * its own svt context and CUDA stream from its own worker thread, so that the work of jobs that
 * are in flight together overlaps on the GPU.  Each job's dual iterate, factors and Lanczos state
 * stay resident in its context from admission to completion.  The paper has no serving layer;
 * the latency it reports is the time of one solve (Table 1), which this measures per job from
 * arrival.
 *
 * Admission: a job is admitted when a slot is free and its device footprint (an upper estimate,
 * svt_estimate_device_bytes) fits into the budget next to the jobs in flight; the queue is strict
 * first-in first-out (a job that does not fit yet holds back the later ones, so large jobs cannot
 * starve).  A job larger than the whole budget is refused at submission (SVT_ERR_OOM).
 *
 * Results: the same contexts, kernels and launch shapes run a job alone or in a mix, and every
 * reduction has a fixed order, so a job's result does not depend on what runs beside it.  A job
 * whose options leave orth_grid at 0 gets max(16, 2 SMs / slots): its result is that of an svt
 * context with that orth_grid (the same for every job of a server, whatever else is running).
 *
 * Threading: the server's calls are thread-safe.  Dry-run servers (options.dry_run) touch no
 * device: a job sleeps for its dry_run_us and occupies dry_run_bytes, for exercising admission and
 * latency accounting without a GPU.
 */
#ifndef SVT_SERVE_H
#define SVT_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "svt.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct svt_server svt_server;

typedef struct svt_server_options {
  int slots;                  /* jobs in flight at once (one worker thread each); default 8 */
  size_t device_budget;       /* admission budget in bytes; 0 = 90 % of the free device memory at
                                 creation (dry run: 0 = unlimited) */
  int keep_factors;           /* 1: keep each finished job's factors until svt_server_wait collects them */
  int dry_run;                /* 1: no device work (see above) */
} svt_server_options;

typedef struct svt_job {
  int64_t m, n, nnz;          /* sizes; rows / cols / vals: nnz host entries, copied at submission */
  const int32_t* rows;
  const int32_t* cols;
  const double* vals;
  double tau, delta, eps;     /* as svt_solve (<= 0 selects the defaults) */
  int max_rank;
  double noise_sigma;         /* > 0: the noisy-data stop eq. (5.10) (svt_set_noise_stop) */
  double noise_eps;
  svt_options opt;            /* context options (the stream field is ignored: each worker has one) */
  int64_t dry_run_us;         /* dry run: duration of the job */
  size_t dry_run_bytes;       /* dry run: its footprint */
} svt_job;

typedef struct svt_job_result {
  int status;                 /* svt_status of the solve */
  int64_t iterations;
  int rank;
  double residual;
  double t_submit_ms, t_start_ms, t_end_ms;   /* since server creation */
  size_t device_bytes;        /* footprint charged at admission */
} svt_job_result;

typedef struct svt_server_stats {
  int64_t submitted, completed, failed, queued, running;
  double p50_ms, p99_ms, mean_ms;   /* time from arrival (submission) to completion, completed jobs */
  double solves_per_s;              /* completed jobs / (last completion - first submission) */
  size_t peak_bytes;                /* largest sum of footprints in flight */
  int peak_running;                 /* largest number of jobs in flight */
} svt_server_stats;

void svt_server_default_options(svt_server_options* opt);
/* Errors: SVT_ERR_ARG (slots < 1), SVT_ERR_CUDA (no device, unless dry run). */
svt_status svt_server_create(const svt_server_options* opt, svt_server** out);
/* Queues a job (its arrays are copied); *job_id receives its id.  Errors: SVT_ERR_ARG (sizes,
 * NULL arrays), SVT_ERR_OOM (footprint above the whole budget; the job is not queued). */
svt_status svt_server_submit(svt_server* srv, const svt_job* job, int64_t* job_id);
/* Blocks until the job has finished, writes its result and, when the server keeps factors and the
 * pointers are given, U (m x r), d (sigma - tau) and V (n x r) (row-major, capacity_r columns), then
 * forgets the job.  Errors: SVT_ERR_ARG (unknown id, capacity_r < rank). */
svt_status svt_server_wait(svt_server* srv, int64_t job_id, svt_job_result* out, double* U, double* d, double* V,
                           int capacity_r);
/* Blocks until every submitted job has finished. */
svt_status svt_server_drain(svt_server* srv);
svt_status svt_server_stats_get(svt_server* srv, svt_server_stats* out);
/* Stops accepting jobs, finishes the queued ones, joins the workers and frees everything. */
void svt_server_destroy(svt_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* SVT_SERVE_H */
