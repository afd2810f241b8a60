// Serving runtime: admission of control problems against a device-memory
// budget, and either concurrent solves on per-problem CUDA streams (worker
// threads, mode 0) or steps in which the NSO V-cycles of every resident
// problem run as one batched CUDA graph launch (mode 1).  Host code; the
// device work is the library's own kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <future>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/stc.h"
#include "../../include/stc_server.h"
#include "stc_kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long ticket = 0;
  stc_params prm{};
  std::vector<double> rho0, v0, stars, cs;
  std::vector<int> steps;
  double tol = 1e-4;
  int max_admm = 50;
  double sim_seconds = 0.0;
  int sim_status = 0;
  size_t bytes = 0;
  int bypassed = 0;
  stc_ticket_info info{};
  std::vector<double> forces;
  stc_problem* p = nullptr;   // stepped mode: the resident problem
  bool owned = true;          // false: submitted by the caller (stc_server_submit_problem)
  cudaStream_t st = nullptr;  // stepped mode: the stream of a server-created problem
  std::future<stc_status> job;  // stepped mode: a head or tail running in the background
};

}  // namespace

struct stc_server {
  stc_server_params sp{};
  std::mutex mu;
  std::condition_variable cv_work;   // workers: a request may be admissible
  std::condition_variable cv_done;   // waiters: a ticket changed state
  std::deque<Request*> queue;        // arrival order
  std::map<long long, std::unique_ptr<Request>> all;
  size_t in_use = 0, peak = 0;
  int running = 0;
  long long next_ticket = 1;
  bool stopping = false;
  Clock::time_point t0 = Clock::now();
  std::vector<std::thread> workers;
  // stepped mode (sp.mode == 1)
  std::mutex step_mu;                 // one step at a time
  std::vector<Request*> resident;     // admitted, solving (touched by the stepping thread only)
  stc_batch* batch = nullptr;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

bool finished(int state) {
  return state == STC_TICKET_DONE || state == STC_TICKET_FAILED || state == STC_TICKET_CANCELLED;
}

// First fit in arrival order, except that a request passed over max_bypass
// times must be admitted before anything behind it.  Called with mu held.
Request* pick(stc_server* s) {
  const size_t free_bytes = s->sp.budget_bytes - s->in_use;
  for (size_t k = 0; k < s->queue.size(); ++k) {
    Request* r = s->queue[k];
    if (r->bytes <= free_bytes) {
      for (size_t j = 0; j < k; ++j) s->queue[j]->bypassed++;
      s->queue.erase(s->queue.begin() + (long)k);
      return r;
    }
    if (r->bypassed >= s->sp.max_bypass) return nullptr;   // holds the line until it fits
  }
  return nullptr;
}

void set_error(Request* r, const char* msg) {
  std::strncpy(r->info.error, msg ? msg : "", sizeof(r->info.error) - 1);
  r->info.error[sizeof(r->info.error) - 1] = 0;
}

// The solve of one admitted request (no lock held).
void solve(stc_server* s, Request* r) {
  if (s->sp.backend == 1) {   // simulated: no CUDA call
    if (r->sim_seconds > 0) std::this_thread::sleep_for(std::chrono::duration<double>(r->sim_seconds));
    r->info.status = r->sim_status;
    const size_t F = (size_t)r->prm.ny * (r->prm.nx + 1) + (size_t)(r->prm.ny + 1) * r->prm.nx;
    if (r->sim_status == STC_OK || r->sim_status == STC_ERR_NOT_CONVERGED)
      r->forces.assign((size_t)r->prm.num_steps * F, 0.0);
    else
      set_error(r, "simulated failure");
    return;
  }
  cudaStream_t st = nullptr;
  stc_problem* p = nullptr;
  stc_status status = STC_OK;
  if (cudaSetDevice(s->sp.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    r->info.status = STC_ERR_CUDA;
    set_error(r, "could not create a stream for the request");
    return;
  }
  status = stc_create_problem(&r->prm, r->rho0.data(), r->v0.empty() ? nullptr : r->v0.data(), st, &p);
  if (status == STC_OK && !r->steps.empty())
    status = stc_set_keyframes(p, (int)r->steps.size(), r->steps.data(), r->stars.data(), r->cs.data());
  if (status == STC_OK) {
    status = stc_solve(p, r->tol, r->max_admm, &r->info.report);
    if (status == STC_OK || status == STC_ERR_NOT_CONVERGED) {
      const size_t F = (size_t)r->prm.ny * (r->prm.nx + 1) + (size_t)(r->prm.ny + 1) * r->prm.nx;
      r->forces.resize((size_t)r->prm.num_steps * F);
      const stc_status g = stc_get_forces(p, r->forces.data(), r->forces.size());
      if (g != STC_OK) status = g;
    }
  }
  r->info.status = status;
  if (status != STC_OK && status != STC_ERR_NOT_CONVERGED) set_error(r, stc_last_error());
  if (p) stc_destroy_problem(p);
  cudaStreamDestroy(st);
}

void worker(stc_server* s) {
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    Request* r = nullptr;
    s->cv_work.wait(lock, [&] { return s->stopping || (r = pick(s)) != nullptr; });
    if (!r) return;   // stopping
    s->in_use += r->bytes;
    s->peak = std::max(s->peak, s->in_use);
    s->running++;
    r->info.state = STC_TICKET_RUNNING;
    r->info.t_admit = s->now();
    s->cv_done.notify_all();
    lock.unlock();
    solve(s, r);
    lock.lock();
    s->in_use -= r->bytes;
    s->running--;
    r->info.t_done = s->now();
    r->info.state = (r->info.status == STC_OK || r->info.status == STC_ERR_NOT_CONVERGED) ? STC_TICKET_DONE
                                                                                          : STC_TICKET_FAILED;
    s->cv_done.notify_all();
    s->cv_work.notify_all();   // memory came back: another request may fit
  }
}

stc_status fail_arg(const char* msg, stc_status code = STC_ERR_INVALID_ARG) {
  stc::set_last_error(msg);
  return code;
}

Request* find(stc_server* s, long long ticket) {
  auto it = s->all.find(ticket);
  return it == s->all.end() ? nullptr : it->second.get();
}

// stepped mode: a resident request ends (its memory returns to the budget)
void finish_stepped(stc_server* s, Request* r, stc_status status) {
  r->info.status = status;
  if (status != STC_OK && status != STC_ERR_NOT_CONVERGED) set_error(r, stc_last_error());
  if (r->p) {
    stc_solve_report(r->p, &r->info.report, nullptr);
    if (r->owned) stc_destroy_problem(r->p);
    r->p = nullptr;
  }
  if (r->st) {
    cudaStreamDestroy(r->st);
    r->st = nullptr;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  s->in_use -= r->bytes;
  s->running--;
  r->info.t_done = s->now();
  r->info.state = (status == STC_OK || status == STC_ERR_NOT_CONVERGED) ? STC_TICKET_DONE : STC_TICKET_FAILED;
  s->cv_done.notify_all();
}

size_t face_count(const stc_params& prm) {
  if (prm.nz > 0)
    return (size_t)prm.nz * prm.ny * (prm.nx + 1) + (size_t)prm.nz * (prm.ny + 1) * prm.nx +
           (size_t)(prm.nz + 1) * prm.ny * prm.nx;
  return (size_t)prm.ny * (prm.nx + 1) + (size_t)(prm.ny + 1) * prm.nx;
}

// One serving step: admission; background jobs (one host thread and the
// problem's own stream each) for the set-up of admitted problems, the heads
// (Alg. 1) of problems whose ADMM iteration begins and the tails (KKT metric,
// multiplier update, stopping tests) of problems whose NSO solve ended; one
// batched launch of the next NSO V-cycle of every idle problem that wants one
// (or, when none does, a wait for a job to finish); retirement of finished
// problems.  A problem in a job does not hold up the others' V-cycles.
stc_status step_stepped(stc_server* s, int* active) {
  std::lock_guard<std::mutex> step_lock(s->step_mu);
  std::vector<Request*> admitted;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    while ((int)(s->resident.size() + admitted.size()) < s->sp.max_resident) {
      Request* r = pick(s);
      if (!r) break;
      s->in_use += r->bytes;
      s->peak = std::max(s->peak, s->in_use);
      s->running++;
      r->info.state = STC_TICKET_RUNNING;
      r->info.t_admit = s->now();
      admitted.push_back(r);
    }
    if (!admitted.empty()) s->cv_done.notify_all();
  }
  // an admitted request's set-up (problem creation, keyframes, stc_solve_begin)
  // runs as its first background job
  for (Request* r : admitted) {
    r->job = std::async(std::launch::async, [r] {
      stc_status st = STC_OK;
      if (!r->p) {
        // each server-created problem has its own stream, so that the heads
        // and tails of different problems overlap on the device
        if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess) {
          cudaGetLastError();
          r->st = nullptr;
          stc::set_last_error("could not create a stream for the request");
          return STC_ERR_CUDA;
        }
        st = stc_create_problem(&r->prm, r->rho0.data(), r->v0.empty() ? nullptr : r->v0.data(), r->st, &r->p);
        if (st == STC_OK && !r->steps.empty())
          st = stc_set_keyframes(r->p, (int)r->steps.size(), r->steps.data(), r->stars.data(), r->cs.data());
      }
      if (st == STC_OK) st = stc_solve_begin(r->p, r->tol, r->max_admm);
      return st;
    });
    s->resident.push_back(r);
  }
  // background jobs that have finished: their problems are idle again
  std::vector<std::pair<Request*, stc_status>> failed;
  auto collect = [&](Request* r) {
    const stc_status st = r->job.get();
    if (st != STC_OK) failed.emplace_back(r, st);
  };
  for (Request* r : s->resident)
    if (r->job.valid() && r->job.wait_for(std::chrono::seconds(0)) == std::future_status::ready) collect(r);
  auto failed_status = [&](Request* r) {
    for (auto& f : failed)
      if (f.first == r) return f.second;
    return STC_OK;
  };
  // (the solve state of a problem is read only while no job of it runs)
  auto phase = [](Request* r, int* wants) {
    int ph = 2;
    stc_solve_phase(r->p, &ph, wants);
    return ph;
  };
  // idle problems whose ADMM iteration begins (Alg. 1), or whose NSO solve
  // ended (KKT metric, multiplier update, stopping tests, then the next head),
  // get a background job on their own stream
  for (Request* r : s->resident) {
    if (r->job.valid() || failed_status(r) != STC_OK || !r->p) continue;
    int w = 0;
    const int ph = phase(r, &w);
    if (ph == 0) {
      r->job = std::async(std::launch::async, [r] { return stc_solve_head(r->p); });
    } else if (ph == 1 && !w) {
      r->job = std::async(std::launch::async, [r] {
        stc_status st = stc_solve_tail(r->p);
        int ph2 = 2, w2 = 0;
        if (st == STC_OK) stc_solve_phase(r->p, &ph2, &w2);
        if (st == STC_OK && ph2 == 0) st = stc_solve_head(r->p);
        return st;
      });
    }
  }
  // one batched launch: the next NSO V-cycle of every idle problem that wants one
  std::vector<stc_problem*> probs;
  std::vector<Request*> owners;
  for (Request* r : s->resident) {
    int w = 0;
    if (!r->job.valid() && failed_status(r) == STC_OK && r->p && phase(r, &w) == 1 && w) {
      probs.push_back(r->p);
      owners.push_back(r);
    }
  }
  if (!probs.empty()) {
    std::vector<stc_status> sts(probs.size(), STC_OK);
    const stc_status b = stc_batch_nso_cycle(s->batch, probs.data(), (int)probs.size(), nullptr, sts.data());
    for (size_t k = 0; k < probs.size(); ++k)
      if (b != STC_OK || sts[k] != STC_OK) failed.emplace_back(owners[k], b != STC_OK ? b : sts[k]);
  } else {
    // nothing to cycle: wait until some background job finishes
    bool any = false, done = false;
    while (!done) {
      any = false;
      for (Request* r : s->resident)
        if (r->job.valid()) {
          any = true;
          if (r->job.wait_for(std::chrono::microseconds(200)) == std::future_status::ready) {
            collect(r);
            done = true;
            break;
          }
        }
      if (!any) break;
    }
  }
  // retire idle problems that failed or finished
  std::vector<Request*> keep;
  for (Request* r : s->resident) {
    if (r->job.valid()) {
      keep.push_back(r);
      continue;
    }
    if (failed_status(r) != STC_OK) {
      finish_stepped(s, r, failed_status(r));
      continue;
    }
    int w = 0;
    if (phase(r, &w) == 2) {
      int conv = 0;
      stc_solve_report(r->p, &r->info.report, &conv);
      stc_status st = conv ? STC_OK : STC_ERR_NOT_CONVERGED;
      r->forces.resize((size_t)r->prm.num_steps * face_count(r->prm));
      const stc_status g = stc_get_forces(r->p, r->forces.data(), r->forces.size());
      if (g != STC_OK) st = g;
      finish_stepped(s, r, st);
      continue;
    }
    keep.push_back(r);
  }
  s->resident.swap(keep);
  if (active) {
    std::lock_guard<std::mutex> lock(s->mu);
    *active = (int)(s->resident.size() + s->queue.size());
  }
  return STC_OK;
}

}  // namespace

extern "C" {

void stc_server_default_params(stc_server_params* sp, size_t budget_bytes) {
  if (!sp) return;
  std::memset(sp, 0, sizeof(*sp));
  sp->budget_bytes = budget_bytes;
  sp->workers = 8;
  sp->backend = 0;
  sp->device = 0;
  sp->max_bypass = 8;
  sp->mode = 0;
  sp->stream = nullptr;
  sp->max_resident = 16;
  sp->kkt_rel_tol = 1e-4;
  sp->max_admm = 50;
}

stc_status stc_server_create(const stc_server_params* sp, stc_server** out) {
  if (!sp || !out || sp->workers < 1 || sp->workers > 256 || sp->budget_bytes == 0 || sp->backend < 0 ||
      sp->backend > 1 || sp->max_bypass < 0 || sp->mode < 0 || sp->mode > 1 ||
      (sp->mode == 1 && (sp->backend != 0 || sp->max_resident < 1 || sp->max_admm < 0)))
    return fail_arg("invalid server parameters");
  *out = nullptr;
  stc_server* s = new (std::nothrow) stc_server();
  if (!s) return fail_arg("host allocation failed", STC_ERR_OOM);
  s->sp = *sp;
  if (sp->mode == 1) {   // stepped: no worker threads; the caller's steps do the work
    if (cudaSetDevice(sp->device) != cudaSuccess || stc_batch_create(sp->stream, &s->batch) != STC_OK) {
      cudaGetLastError();
      delete s;
      return fail_arg("could not set up the batched stepping", STC_ERR_CUDA);
    }
    *out = s;
    return STC_OK;
  }
  try {
    for (int k = 0; k < sp->workers; ++k) s->workers.emplace_back(worker, s);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
    return fail_arg("could not start the worker threads", STC_ERR_OOM);
  }
  *out = s;
  return STC_OK;
}

stc_status stc_server_submit(stc_server* s, const stc_request* rq, long long* ticket) {
  if (!s || !rq || !rq->params || !rq->rho0 || !ticket || rq->nkeys < 0 ||
      (rq->nkeys > 0 && (!rq->key_steps || !rq->key_rho)) || rq->max_admm < 0)
    return fail_arg("invalid request");
  size_t bytes = 0;
  if (stc_problem_bytes(rq->params, rq->nkeys, &bytes) != STC_OK) return fail_arg("invalid problem parameters");
  const stc_params& prm = *rq->params;
  for (int k = 0; k < rq->nkeys; ++k)
    if (rq->key_steps[k] < 1 || rq->key_steps[k] > prm.num_steps) return fail_arg("keyframe step outside 1..N");
  if (bytes > s->sp.budget_bytes) return fail_arg("request exceeds the server's memory budget", STC_ERR_OOM);
  auto r = std::make_unique<Request>();
  try {
    const size_t C = (size_t)prm.nx * prm.ny;
    const size_t F = (size_t)prm.ny * (prm.nx + 1) + (size_t)(prm.ny + 1) * prm.nx;
    r->prm = prm;
    r->rho0.assign(rq->rho0, rq->rho0 + C);
    if (rq->v0) r->v0.assign(rq->v0, rq->v0 + F);
    r->steps.assign(rq->key_steps, rq->key_steps + rq->nkeys);
    if (rq->nkeys > 0) r->stars.assign(rq->key_rho, rq->key_rho + (size_t)rq->nkeys * C);
    r->cs.assign(rq->nkeys, 1.0);
    if (rq->key_c)
      for (int k = 0; k < rq->nkeys; ++k) r->cs[k] = rq->key_c[k];
  } catch (const std::bad_alloc&) {
    return fail_arg("host allocation failed", STC_ERR_OOM);
  }
  r->tol = rq->kkt_rel_tol;
  r->max_admm = rq->max_admm;
  r->sim_seconds = rq->sim_seconds;
  r->sim_status = rq->sim_status;
  r->bytes = bytes;
  r->info.state = STC_TICKET_QUEUED;
  r->info.bytes = bytes;
  r->info.t_admit = r->info.t_done = -1.0;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) return fail_arg("server is shutting down", STC_ERR_BUSY);
    r->ticket = s->next_ticket++;
    r->info.t_submit = s->now();
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->all[r->ticket] = std::move(r);
  }
  s->cv_work.notify_all();
  return STC_OK;
}

stc_status stc_server_submit_problem(stc_server* s, stc_problem* p, long long* ticket) {
  if (!s || !p || !ticket) return fail_arg("null argument");
  if (s->sp.mode != 1) return fail_arg("problem submits need a stepped server (mode 1)");
  size_t bytes = 0;
  if (stc_memory_bytes(p, &bytes) != STC_OK) return fail_arg("invalid problem");
  if (bytes > s->sp.budget_bytes) return fail_arg("problem exceeds the server's memory budget", STC_ERR_OOM);
  auto r = std::make_unique<Request>();
  r->p = p;
  r->owned = false;
  r->tol = s->sp.kkt_rel_tol;
  r->max_admm = s->sp.max_admm;
  int nx = 0, ny = 0, nz = 0, N = 0;
  double dt = 0.0;
  stc_level_dims(p, 0, &nx, &ny, &nz);
  stc_level_steps(p, 0, &N, &dt);
  r->prm.nx = nx;
  r->prm.ny = ny;
  r->prm.nz = nz > 1 ? nz : 0;
  r->prm.num_steps = N;
  r->bytes = bytes;
  r->info.state = STC_TICKET_QUEUED;
  r->info.bytes = bytes;
  r->info.t_admit = r->info.t_done = -1.0;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) return fail_arg("server is shutting down", STC_ERR_BUSY);
    r->ticket = s->next_ticket++;
    r->info.t_submit = s->now();
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->all[r->ticket] = std::move(r);
  }
  return STC_OK;
}

stc_status stc_server_step(stc_server* s, int* active) {
  if (!s) return fail_arg("null argument");
  if (s->sp.mode != 1) return fail_arg("stc_server_step needs a stepped server (mode 1)");
  return step_stepped(s, active);
}

stc_status stc_server_poll(stc_server* s, long long ticket, stc_ticket_info* info) {
  if (!s || !info) return fail_arg("null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  Request* r = find(s, ticket);
  if (!r) return fail_arg("unknown ticket");
  *info = r->info;
  return STC_OK;
}

stc_status stc_server_wait(stc_server* s, long long ticket, double timeout_s, stc_ticket_info* info) {
  if (!s) return fail_arg("null argument");
  std::unique_lock<std::mutex> lock(s->mu);
  Request* r = find(s, ticket);
  if (!r) return fail_arg("unknown ticket");
  auto done = [&] { return finished(r->info.state); };
  if (s->sp.mode == 1) {   // stepped: the waiting thread drives the steps
    const double until = timeout_s < 0 ? -1.0 : s->now() + timeout_s;
    while (!done() && (until < 0 || s->now() < until)) {
      lock.unlock();
      int active = 0;
      const stc_status st = step_stepped(s, &active);
      lock.lock();
      if (st != STC_OK || active == 0) break;
    }
    if (info) *info = r->info;
    return STC_OK;
  }
  if (timeout_s < 0)
    s->cv_done.wait(lock, done);
  else
    s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), done);
  if (info) *info = r->info;
  return STC_OK;
}

stc_status stc_server_cancel(stc_server* s, long long ticket) {
  if (!s) return fail_arg("null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  Request* r = find(s, ticket);
  if (!r) return fail_arg("unknown ticket");
  if (r->info.state == STC_TICKET_RUNNING) return fail_arg("request is running", STC_ERR_BUSY);
  if (r->info.state != STC_TICKET_QUEUED) return STC_OK;
  s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
  r->info.state = STC_TICKET_CANCELLED;
  r->info.t_done = s->now();
  s->cv_done.notify_all();
  s->cv_work.notify_all();   // a request held behind this one may now be admissible
  return STC_OK;
}

stc_status stc_server_get_forces(stc_server* s, long long ticket, double* u, size_t len) {
  if (!s || !u) return fail_arg("null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  Request* r = find(s, ticket);
  if (!r) return fail_arg("unknown ticket");
  if (r->info.state != STC_TICKET_DONE) return fail_arg("ticket has no result", STC_ERR_BUSY);
  if (len != r->forces.size()) return fail_arg("length does not match the force field");
  std::copy(r->forces.begin(), r->forces.end(), u);
  return STC_OK;
}

stc_status stc_server_release(stc_server* s, long long ticket) {
  if (!s) return fail_arg("null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  Request* r = find(s, ticket);
  if (!r) return fail_arg("unknown ticket");
  if (!finished(r->info.state)) return fail_arg("ticket is not finished", STC_ERR_BUSY);
  s->all.erase(ticket);
  return STC_OK;
}

stc_status stc_server_stats_get(stc_server* s, stc_server_stats* out) {
  if (!s || !out) return fail_arg("null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof(*out));
  for (auto& kv : s->all) {
    switch (kv.second->info.state) {
      case STC_TICKET_QUEUED: out->queued++; break;
      case STC_TICKET_RUNNING: out->running++; break;
      case STC_TICKET_DONE: out->done++; break;
      case STC_TICKET_FAILED: out->failed++; break;
      default: out->cancelled++; break;
    }
  }
  out->bytes_in_use = s->in_use;
  out->peak_bytes = s->peak;
  return STC_OK;
}

stc_status stc_server_destroy(stc_server* s) {
  if (!s) return STC_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
    for (Request* r : s->queue) {
      r->info.state = STC_TICKET_CANCELLED;
      r->info.t_done = s->now();
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto& t : s->workers) t.join();
  {
    std::lock_guard<std::mutex> step_lock(s->step_mu);
    for (Request* r : s->resident)     // background jobs finish first
      if (r->job.valid()) r->job.wait();
    for (Request* r : s->resident) {   // stepped mode: solves still in flight end here
      if (r->p && r->owned) stc_destroy_problem(r->p);
      r->p = nullptr;
      if (r->st) cudaStreamDestroy(r->st);
      r->st = nullptr;
      r->info.state = STC_TICKET_CANCELLED;
    }
    s->resident.clear();
    if (s->batch) stc_batch_destroy(s->batch);
  }
  delete s;
  return STC_OK;
}

}  // extern "C"
