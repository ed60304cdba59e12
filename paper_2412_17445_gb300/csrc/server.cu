// Serving layer of librve: a continuous-batching server for crack-increment requests.
//
// Requests (an RVE description, its notch and a number of crack-length increments) queue
// in arrival order.  The scheduler admits a request as soon as its device footprint fits in
// the HBM budget next to the RVEs already resident and a slot is free.  It takes the oldest
// request that fits, so a large request at the head does not block smaller ones behind it;
// a request can be overtaken this way by at most max_active later ones, after which nothing
// is admitted until it fits (no starvation).  A fixed pool of max_active worker threads,
// each with its own CUDA stream, runs the admitted requests, so requests that arrive while
// others are on the GPU overlap with them on the device.  Resident RVEs of equal shape join a
// launch group of the library (rve_internal.h), so their BiCGStab chunks run as single
// launches per pass, as in a batch (RVE_SERVER_GROUPS=0 runs each on its own).  An RVE's fields
// and Krylov state stay resident on the device from admission to completion; its memory is
// returned when it completes.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rve.h"
#include "rve_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id;
  rve_desc desc;
  std::vector<uint8_t> phase, notch;
  std::vector<double> E, nu, Gc;
  int n_inc;
  double da;
  long long footprint;
  double t_submit;
  int overtaken = 0;       // later requests admitted while this one waited
};

}  // namespace

struct rve_server {
  long long budget;
  int max_active;
  int device;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> queue;                       // submitted, not yet admitted
  std::deque<std::pair<Request, double>> ready;    // admitted (with the admission time)
  std::vector<rve_result> done;
  long long in_use = 0;
  int active = 0;                                  // admitted and not yet completed
  long long next_id = 1;
  long long submitted = 0, completed = 0;
  bool stop = false;
  void *groups = nullptr;                          // launch groups of the resident RVEs
  std::thread scheduler;
  std::vector<std::thread> workers;                // max_active threads for the server's life
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

static void run_request(rve_server *s, cudaStream_t st, Request &r, double t_start) {
  rve_result res;
  memset(&res, 0, sizeof res);
  res.id = r.id;
  res.t_submit = r.t_submit;
  res.t_start = t_start;
  res.footprint = r.footprint;
  rve_t *h = nullptr;
  int rc = st ? RVE_OK : RVE_E_CUDA;
  r.desc.phase = r.phase.data();
  r.desc.E = r.E.data();
  r.desc.nu = r.nu.data();
  r.desc.Gc = r.Gc.data();
  if (rc == RVE_OK) rc = rve_create(&r.desc, &h);
  if (rc == RVE_OK) rc = rve_set_stream(h, st);
  if (rc == RVE_OK && !r.notch.empty()) rc = rve_set_notch(h, r.notch.data());
  if (rc == RVE_OK && s->groups) rc = rve_group_pool_join(s->groups, h);
  rve_step step;
  memset(&step, 0, sizeof step);
  if (rc == RVE_OK) rc = rve_startup(h, 0.25, nullptr);
  for (int k = 0; rc == RVE_OK && k < r.n_inc; ++k) {
    rc = rve_crack_increment(h, r.da, &step);
    if (rc == RVE_OK) res.n_increments = k + 1;
  }
  res.status = rc;
  res.E = step.E;
  for (int k = 0; k < 6; ++k) res.sigma[k] = step.sigma[k];
  res.gamma = step.gamma;
  if (rc != RVE_OK) snprintf(res.error, sizeof res.error, "%s", rve_last_error(h));
  if (h && s->groups) rve_group_pool_leave(s->groups, h);
  if (h) rve_destroy(h);
  res.t_end = s->now();
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_use -= r.footprint;
  s->active -= 1;
  s->completed += 1;
  s->done.push_back(res);
  s->cv.notify_all();
}

// One of the max_active pool threads: runs admitted requests until the server stops.
static void worker_loop(rve_server *s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] { return s->stop || !s->ready.empty(); });
    if (s->ready.empty()) break;  // stop requested and nothing left to run
    std::pair<Request, double> job = std::move(s->ready.front());
    s->ready.pop_front();
    lk.unlock();
    run_request(s, st, job.first, job.second);
    lk.lock();
  }
  lk.unlock();
  if (st) cudaStreamDestroy(st);
}

// Index of the request to admit next, or -1: the oldest queued request that fits beside
// the resident ones (any request when nothing is resident), unless a request has already
// been overtaken max_active times, in which case only that one may be admitted.
static int pick_admissible(const rve_server *s) {
  if (s->active >= s->max_active) return -1;
  for (size_t i = 0; i < s->queue.size(); ++i) {
    const Request &q = s->queue[i];
    const bool fits = s->in_use + q.footprint <= s->budget || s->active == 0;
    if (fits) return (int)i;
    if (q.overtaken >= s->max_active) return -1;  // it waits for room; nobody passes it
  }
  return -1;
}

static void schedule_loop(rve_server *s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    int i = -1;
    s->cv.wait(lk, [&] { return s->stop || (i = pick_admissible(s)) >= 0; });
    if (s->stop) return;
    for (int j = 0; j < i; ++j) s->queue[j].overtaken += 1;
    Request r = std::move(s->queue[i]);
    s->queue.erase(s->queue.begin() + i);
    s->in_use += r.footprint;
    s->active += 1;
    s->ready.emplace_back(std::move(r), s->now());
    s->cv.notify_all();
  }
}

extern "C" {

int rve_server_create(long long hbm_budget, int max_active, rve_server_t **out) {
  if (!out || hbm_budget <= 0 || max_active < 1) return RVE_E_ARG;
  rve_server *s = new rve_server();
  s->budget = hbm_budget;
  s->max_active = max_active;
  cudaGetDevice(&s->device);
  {
    const char *e = getenv("RVE_SERVER_GROUPS");
    if (!(e && e[0] == '0')) s->groups = rve_group_pool_create();
  }
  s->t0 = Clock::now();
  for (int k = 0; k < max_active; ++k) s->workers.emplace_back(worker_loop, s);
  s->scheduler = std::thread(schedule_loop, s);
  *out = s;
  return RVE_OK;
}

int rve_server_submit(rve_server_t *s, const rve_desc *desc, const uint8_t *notch, int n_increments,
                      double da, long long *id) {
  if (!s || !desc || !desc->phase || !desc->E || !desc->nu || !desc->Gc || n_increments < 0) return RVE_E_ARG;
  if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1 || desc->n_phases < 1 || desc->n_phases > RVE_MAX_PHASES)
    return RVE_E_ARG;
  Request r;
  r.desc = *desc;
  const size_t n = (size_t)desc->nx * desc->ny * desc->nz;
  r.phase.assign(desc->phase, desc->phase + n);
  if (notch) r.notch.assign(notch, notch + n);
  r.E.assign(desc->E, desc->E + desc->n_phases);
  r.nu.assign(desc->nu, desc->nu + desc->n_phases);
  r.Gc.assign(desc->Gc, desc->Gc + desc->n_phases);
  r.n_inc = n_increments;
  r.da = da;
  if (rve_footprint(desc, &r.footprint) != RVE_OK) return RVE_E_ARG;
  if (r.footprint > s->budget) return RVE_E_OOM;
  std::lock_guard<std::mutex> lk(s->mu);
  r.id = s->next_id++;
  r.t_submit = s->now();
  if (id) *id = r.id;
  s->queue.push_back(std::move(r));
  s->submitted += 1;
  s->cv.notify_all();
  return RVE_OK;
}

int rve_server_poll(rve_server_t *s, rve_result *res, int max, int *n) {
  if (!s || !n || (max > 0 && !res)) return RVE_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max && !s->done.empty()) {
    res[k++] = s->done.front();
    s->done.erase(s->done.begin());
  }
  *n = k;
  return RVE_OK;
}

int rve_server_drain(rve_server_t *s) {
  if (!s) return RVE_E_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait(lk, [&] { return s->completed == s->submitted; });
  return RVE_OK;
}

int rve_server_stats(rve_server_t *s, long long *hbm_in_use, int *active, int *queued) {
  if (!s) return RVE_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (hbm_in_use) *hbm_in_use = s->in_use;
  if (active) *active = s->active;
  if (queued) *queued = (int)s->queue.size();
  return RVE_OK;
}

void rve_server_destroy(rve_server_t *s) {
  if (!s) return;
  rve_server_drain(s);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->scheduler.join();
  for (auto &t : s->workers) t.join();
  rve_group_pool_destroy(s->groups);
  delete s;
}

}  // extern "C"
