// Continuous-batching slab-solve server (stdg_server_* in include/stdg.h).
//
// A worker thread owns one batch (engine.cuh) and its CUDA stream.  Requests
// (a problem description and its initial state, copied at submission) wait in
// a FIFO queue.  Between groups of ticks the worker admits queued requests in
// arrival order while the batch's arena and slot table have room (admission
// by device memory; the head of the queue blocks the ones behind it so that
// admission stays in arrival order), runs ticks over all admitted slots, and
// retires finished slots: result copied to the request, slot memory released.
// A request admitted while others are running joins their launches at the
// next tick.  Timestamps (submit, admit, done) give queueing and service
// latency per request.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "stdg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  stdg_config_desc d;
  std::vector<double> u;  // initial state, then the result
  int slot = -1;
  int status = STDG_OK;
  bool done = false;
  stdg_slab_stats stats;
  Clock::time_point t_submit, t_admit, t_done;
};

size_t state_len(const stdg_config_desc& d) {
  size_t n = d.equation == STDG_EULER ? (size_t)(d.dim + 2) : 1;
  for (int a = 0; a < d.dim; ++a) n *= (size_t)d.cells[a] * (d.N + 1);
  return n;
}

double slab_dof(const stdg_config_desc& d) { return (double)state_len(d) * d.s; }

}  // namespace

struct stdg_server {
  stdg_batch_desc bd;
  int device = 0;
  int ticks_per_round = 4;
  stdg_batch* batch = nullptr;
  cudaStream_t st = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  stdg_status fatal = STDG_OK;
  std::string err;
  unsigned long long next_ticket = 1;
  std::map<unsigned long long, Request> reqs;
  std::deque<unsigned long long> queue;            // submitted, not admitted
  std::map<int, unsigned long long> running;       // slot -> ticket
  // counters
  unsigned long long n_admitted = 0, n_done = 0, ticks = 0;
  int max_running = 0;
  // batch scheduling knobs (applied by the worker before its next round)
  bool cfg_dirty = false;
  double share_quantum = 0.0;
  int share_max_stride = 16, use_graphs = 1, autotune = 0;
  size_t max_queue = 0;                          // 0: unbounded submission queue
  // admission policy (stdg_server_set_policy): order 0 = arrival (FIFO), 1 = smallest space-time
  // problem first (ties in arrival order); max_running_dof > 0 caps the space-time DOF admitted
  // at once (a request larger than the cap runs alone)
  int order = 0;
  double max_running_dof = 0.0;
  double running_dof = 0.0;
  std::vector<int> cancel_slots;                 // slots of cancelled requests, released by the worker
};

namespace {

void fail_all(stdg_server* s, stdg_status st, const std::string& msg) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->fatal = st;
  s->err = msg;
  for (auto& kv : s->reqs)
    if (!kv.second.done) {
      kv.second.done = true;
      kv.second.status = st;
      kv.second.t_done = Clock::now();
    }
  s->queue.clear();
  s->running.clear();
  s->cv.notify_all();
}

void worker_main(stdg_server* s) {
  if (cudaSetDevice(s->device) != cudaSuccess) {
    fail_all(s, STDG_ERR_CUDA, "cudaSetDevice failed in the server thread");
    return;
  }
  if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
    fail_all(s, STDG_ERR_CUDA, "cudaStreamCreate failed in the server thread");
    return;
  }
  stdg_status cs = stdg_batch_create(&s->bd, s->st, &s->batch);
  if (cs != STDG_OK) {
    fail_all(s, cs, "stdg_batch_create failed in the server thread");
    return;
  }
  for (;;) {
    // ---- admission (arrival order, while memory allows)
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      if (s->cfg_dirty) {
        stdg_batch_configure(s->batch, s->share_quantum, s->share_max_stride, s->use_graphs, s->autotune);
        s->cfg_dirty = false;
      }
      // slots of cancelled requests: release them (between ticks, before any new admission can
      // reuse the slot id)
      for (int slot : s->cancel_slots) stdg_batch_remove(s->batch, slot);
      s->cancel_slots.clear();
      if (s->running.empty() && s->queue.empty())
        s->cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
      while (!s->queue.empty()) {
        // next candidate: the head of the queue, or its smallest problem
        auto pick = s->queue.begin();
        if (s->order == 1) {
          for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
            if (slab_dof(s->reqs[*it].d) < slab_dof(s->reqs[*pick].d)) pick = it;
        }
        const unsigned long long t = *pick;
        Request& r = s->reqs[t];
        const double dof = slab_dof(r.d);
        if (s->max_running_dof > 0.0 && !s->running.empty() && s->running_dof + dof > s->max_running_dof) break;
        int slot = -1;
        const stdg_status as = stdg_batch_add(s->batch, &r.d, r.u.data(), STDG_HOST, &slot);
        if (as == STDG_ERR_OOM) {
          if (s->running.empty()) {  // can never fit: refuse it rather than wait forever
            r.done = true;
            r.status = STDG_ERR_OOM;
            r.t_admit = r.t_done = Clock::now();
            s->queue.erase(pick);
            s->cv.notify_all();
            continue;
          }
          break;
        }
        s->queue.erase(pick);
        if (as != STDG_OK) {
          r.done = true;
          r.status = as;
          r.t_admit = r.t_done = Clock::now();
          s->cv.notify_all();
          continue;
        }
        r.slot = slot;
        r.t_admit = Clock::now();
        s->running[slot] = t;
        s->running_dof += dof;
        ++s->n_admitted;
      }
      if ((int)s->running.size() > s->max_running) s->max_running = (int)s->running.size();
    }
    if (s->running.empty()) continue;
    // ---- ticks (no lock held: submitters only touch the queue)
    int working = 0;
    stdg_status ss = stdg_batch_step(s->batch, s->ticks_per_round, &working);
    if (ss != STDG_OK) {
      fail_all(s, ss, std::string("stdg_batch_step: ") + stdg_batch_last_error(s->batch));
      break;
    }
    s->ticks += s->ticks_per_round;
    // ---- retire finished slots
    std::vector<int> fin(s->bd.max_slots);
    const int nfin = stdg_batch_done_slots(s->batch, fin.data(), (int)fin.size());
    std::vector<std::pair<int, unsigned long long>> run;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int i = 0; i < nfin && i < (int)fin.size(); ++i) {
        auto it = s->running.find(fin[i]);
        if (it != s->running.end()) run.push_back(*it);
      }
    }
    bool failed = false;
    for (auto& sr : run) {
      int done = 0, status = 0;
      stdg_slab_stats stats;
      if (stdg_batch_query(s->batch, sr.first, &done, &status, &stats) != STDG_OK) {
        fail_all(s, STDG_ERR_CUDA, "stdg_batch_query failed");
        failed = true;
        break;
      }
      if (!done) continue;
      std::vector<double> out;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(sr.second);
        if (it == s->reqs.end() || it->second.done || s->running.count(sr.first) == 0) continue;  // cancelled
        out.resize(it->second.u.size());
      }
      const stdg_status gs = stdg_batch_get_state(s->batch, sr.first, out.data(), STDG_HOST);
      std::lock_guard<std::mutex> lk(s->mu);
      auto it = s->reqs.find(sr.second);
      if (it == s->reqs.end() || it->second.done || s->running.count(sr.first) == 0) continue;  // cancelled meanwhile
      stdg_batch_remove(s->batch, sr.first);
      Request& r = it->second;
      s->running_dof -= slab_dof(r.d);
      r.slot = -1;
      r.u.swap(out);
      r.status = gs == STDG_OK ? status : gs;
      r.stats = stats;
      r.t_done = Clock::now();
      r.done = true;
      s->running.erase(sr.first);
      ++s->n_done;
      s->cv.notify_all();
    }
    if (failed) break;
  }
  if (s->batch) stdg_batch_destroy(s->batch);
  s->batch = nullptr;
  if (s->st) cudaStreamDestroy(s->st);
  s->st = nullptr;
}

double seconds(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

}  // namespace

extern "C" {

stdg_status stdg_server_create(const stdg_batch_desc* desc, int ticks_per_round, stdg_server** out) {
  if (!out) return STDG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || desc->max_slots < 1 || desc->hbm_budget_bytes == 0 || ticks_per_round < 1) return STDG_ERR_INVALID_ARG;
  if (!((desc->equation == STDG_ADVECTION && (desc->dim == 1 || desc->dim == 2)) ||
        (desc->equation == STDG_BURGERS && desc->dim == 2) || (desc->equation == STDG_EULER && desc->dim == 2)))
    return STDG_ERR_INVALID_ARG;
  stdg_server* s = new stdg_server();
  s->bd = *desc;
  s->ticks_per_round = ticks_per_round;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return STDG_ERR_CUDA;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return STDG_OK;
}

stdg_status stdg_server_destroy(stdg_server* s) {
  if (!s) return STDG_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
  return STDG_OK;
}

stdg_status stdg_server_submit(stdg_server* s, const stdg_config_desc* d, const double* u0,
                               unsigned long long* ticket) {
  if (!s || !d || !u0 || !ticket) return STDG_ERR_INVALID_ARG;
  if (d->dim != s->bd.dim || d->equation != s->bd.equation || d->dim < 1 || d->dim > 2 || d->N < 1 || d->N > 7)
    return STDG_ERR_INVALID_ARG;
  for (int a = 0; a < d->dim; ++a)
    if (d->cells[a] < 1) return STDG_ERR_INVALID_ARG;
  Request r;
  r.d = *d;
  r.u.assign(u0, u0 + state_len(*d));
  std::memset(&r.stats, 0, sizeof(r.stats));
  r.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != STDG_OK) return s->fatal;
  if (s->max_queue && s->queue.size() >= s->max_queue) return STDG_ERR_OOM;  // queue full: refused
  const unsigned long long t = s->next_ticket++;
  s->reqs.emplace(t, std::move(r));
  s->queue.push_back(t);
  *ticket = t;
  s->cv.notify_all();
  return STDG_OK;
}

stdg_status stdg_server_poll(stdg_server* s, unsigned long long ticket, double wait_s, int* done, int* status,
                             stdg_slab_stats* stats, double* u, double* times) {
  if (!s || !done) return STDG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return STDG_ERR_INVALID_ARG;
  if (!it->second.done && wait_s > 0.0)
    s->cv.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return it->second.done; });
  Request& r = it->second;
  *done = r.done ? 1 : 0;
  if (!r.done) return STDG_OK;
  if (status) *status = r.status;
  if (stats) *stats = r.stats;
  if (u) std::memcpy(u, r.u.data(), r.u.size() * sizeof(double));
  if (times) {
    times[0] = seconds(r.t_submit, r.t_admit);
    times[1] = seconds(r.t_admit, r.t_done);
    times[2] = seconds(r.t_submit, r.t_done);
  }
  s->reqs.erase(it);
  return STDG_OK;
}

stdg_status stdg_server_cancel(stdg_server* s, unsigned long long ticket) {
  if (!s) return STDG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return STDG_ERR_INVALID_ARG;
  Request& r = it->second;
  if (r.done) return STDG_OK;  // finished first: the result stands
  auto q = std::find(s->queue.begin(), s->queue.end(), ticket);
  if (q != s->queue.end()) {
    s->queue.erase(q);
  } else if (r.slot >= 0) {
    s->running.erase(r.slot);
    s->running_dof -= slab_dof(r.d);
    s->cancel_slots.push_back(r.slot);
    r.slot = -1;
  }
  r.done = true;
  r.status = STDG_ERR_CANCELLED;
  r.t_done = Clock::now();
  if (r.t_admit.time_since_epoch().count() == 0) r.t_admit = r.t_done;
  s->cv.notify_all();
  return STDG_OK;
}

stdg_status stdg_server_set_queue_limit(stdg_server* s, size_t max_queued) {
  if (!s) return STDG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_queue = max_queued;
  return STDG_OK;
}

stdg_status stdg_server_configure(stdg_server* s, double share_quantum, int share_max_stride, int use_graphs,
                                  int autotune) {
  if (!s || !(share_quantum >= 0.0) || share_max_stride < 1) return STDG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->share_quantum = share_quantum;
  s->share_max_stride = share_max_stride;
  s->use_graphs = use_graphs;
  s->autotune = autotune;
  s->cfg_dirty = true;
  return STDG_OK;
}

stdg_status stdg_server_set_policy(stdg_server* s, int order, double max_running_dof) {
  if (!s || (order != 0 && order != 1) || !(max_running_dof >= 0.0)) return STDG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->order = order;
  s->max_running_dof = max_running_dof;
  return STDG_OK;
}

stdg_status stdg_server_counters(stdg_server* s, unsigned long long* admitted, unsigned long long* completed,
                                 unsigned long long* ticks, int* queued, int* running, int* max_running) {
  if (!s) return STDG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (admitted) *admitted = s->n_admitted;
  if (completed) *completed = s->n_done;
  if (ticks) *ticks = s->ticks;
  if (queued) *queued = (int)s->queue.size();
  if (running) *running = (int)s->running.size();
  if (max_running) *max_running = s->max_running;
  return s->fatal;
}

}  // extern "C"
