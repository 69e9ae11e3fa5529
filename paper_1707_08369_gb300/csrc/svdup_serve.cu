// svdup_serve.cu -- the serving engine: resident SVDs and continuously admitted
// rank-one updates (svdup_server_* in include/svdup.h).
//
// One scheduler thread owns every CUDA call of the engine.  Its loop:
//   1. completions: a busy lane whose completion event has fired finishes its request
//      (status from the lane's handle, latency from the submission time);
//   2. admissions, in submission order: a request is admitted when its matrix has no
//      update in flight, a lane is free, and the free-HBM ledger allows the workspace
//      the update needs.  The ledger counts the workspace every lane holds (a lane
//      keeps the largest workspace it has needed); when a request does not fit, idle
//      lanes give their workspace back (their handle is recreated) before it waits.
// Requests of one matrix therefore apply in submission order, requests of different
// matrices overlap on the device, and a request that arrives while others run is
// admitted as soon as a lane and memory free up (continuous batching).
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/svdup.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  long long ticket;
  int id;
  std::vector<double> a, b;
  double t_submit;
};

struct Result {
  int status;
  double latency_ms;
};

struct Matrix {
  int m, n, ldu, ldv;
  double *U, *S, *V;
  bool busy;
};

struct Lane {
  svdup_t h = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  double* da = nullptr;     // device copies of a, b
  double* db = nullptr;
  double* ha = nullptr;     // pinned staging
  double* hb = nullptr;
  int cap = 0;              // capacity (entries) of the four vectors
  size_t ws = 0;            // workspace bytes the lane's handle holds
  bool busy = false;
  long long ticket = 0;
  int id = -1;
  double t_submit = 0.0;
};

}  // namespace

struct svdup_server {
  int device = 0;
  int mode = 0;
  double eps = 1e-12;
  size_t budget = 0;
  std::vector<Lane> lanes;
  std::vector<Matrix> mats;
  std::deque<Request> pending;
  std::unordered_map<long long, Result> results;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
  bool stop = false;
  bool started = false;
  long long next_ticket = 1;
  long long submitted = 0, completed = 0;
  std::vector<double> lat;
  int in_flight = 0, max_in_flight = 0;
  size_t held = 0, max_held = 0;
};

namespace {

int lane_open(svdup_server* s, Lane& l) {
  if (cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return SVDUP_ECUDA;
  }
  return svdup_create(&l.h, s->device, (void*)l.st, 0);
}

void lane_vectors_free(Lane& l) {
  if (l.da) cudaFree(l.da);
  if (l.db) cudaFree(l.db);
  if (l.ha) cudaFreeHost(l.ha);
  if (l.hb) cudaFreeHost(l.hb);
  l.da = l.db = l.ha = l.hb = nullptr;
  l.cap = 0;
}

int lane_vectors(Lane& l, int n) {
  if (n <= l.cap) return SVDUP_OK;
  lane_vectors_free(l);
  if (cudaMalloc(&l.da, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&l.db, n * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&l.ha, n * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&l.hb, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lane_vectors_free(l);
    return SVDUP_ENOMEM;
  }
  l.cap = n;
  return SVDUP_OK;
}

// Give an idle lane's workspace back to the device (a fresh handle holds none).
void lane_release_ws(svdup_server* s, Lane& l) {
  if (l.ws == 0) return;
  svdup_destroy(l.h);
  l.h = nullptr;
  svdup_create(&l.h, s->device, (void*)l.st, 0);
  s->held -= l.ws;
  l.ws = 0;
}

// Pick a free lane for a request needing `need` workspace bytes under the budget, or -1.
int pick_lane(svdup_server* s, size_t need) {
  int best = -1;
  for (int i = 0; i < (int)s->lanes.size(); i++) {  // a free lane that already holds enough
    const Lane& l = s->lanes[i];
    if (!l.busy && l.ws >= need && (best < 0 || l.ws < s->lanes[best].ws)) best = i;
  }
  if (best >= 0) return best;
  for (int i = 0; i < (int)s->lanes.size(); i++) {  // else the free lane that grows least
    const Lane& l = s->lanes[i];
    if (!l.busy && (best < 0 || l.ws > s->lanes[best].ws)) best = i;
  }
  if (best < 0) return -1;
  size_t grow = need - s->lanes[best].ws;
  if (s->held + grow <= s->budget) return best;
  // free idle workspaces, largest first, until the growth fits
  std::vector<int> idle;
  for (int i = 0; i < (int)s->lanes.size(); i++)
    if (!s->lanes[i].busy && i != best && s->lanes[i].ws > 0) idle.push_back(i);
  std::sort(idle.begin(), idle.end(),
            [&](int x, int y) { return s->lanes[x].ws > s->lanes[y].ws; });
  for (int i : idle) {
    lane_release_ws(s, s->lanes[i]);
    if (s->held + grow <= s->budget) return best;
  }
  return -1;
}

void finish(svdup_server* s, long long ticket, int status, double t_submit) {
  const double lat = now_ms() - t_submit;
  s->results[ticket] = Result{status, lat};
  s->lat.push_back(lat);
  s->completed++;
}

void scheduler(svdup_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progressed = false;
    // 1. completions
    for (Lane& l : s->lanes) {
      if (!l.busy) continue;
      cudaError_t q = cudaEventQuery(l.done);
      if (q == cudaErrorNotReady) continue;
      int st = (q == cudaSuccess) ? svdup_sync(l.h) : SVDUP_ECUDA;
      if (q != cudaSuccess) cudaGetLastError();
      s->mats[l.id].busy = false;
      l.busy = false;
      s->in_flight--;
      finish(s, l.ticket, st, l.t_submit);
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // 2. admissions in submission order
    for (auto it = s->pending.begin(); it != s->pending.end();) {
      Matrix& M = s->mats[it->id];
      if (M.busy) { ++it; continue; }
      size_t need = 0;
      int rc = svdup_update_workspace(s->lanes[0].h, M.m, M.n, s->eps, s->mode, &need);
      if (rc) {
        finish(s, it->ticket, rc, it->t_submit);
        it = s->pending.erase(it);
        s->cv_done.notify_all();
        continue;
      }
      const int li = pick_lane(s, need);
      if (li < 0) { ++it; continue; }
      Lane& l = s->lanes[li];
      rc = lane_vectors(l, M.n);
      if (!rc) {
        memcpy(l.ha, it->a.data(), M.m * sizeof(double));
        memcpy(l.hb, it->b.data(), M.n * sizeof(double));
        if (cudaMemcpyAsync(l.da, l.ha, M.m * sizeof(double), cudaMemcpyHostToDevice, l.st) !=
                cudaSuccess ||
            cudaMemcpyAsync(l.db, l.hb, M.n * sizeof(double), cudaMemcpyHostToDevice, l.st) !=
                cudaSuccess)
          rc = SVDUP_ECUDA;
      }
      if (!rc) rc = svdup_update(l.h, M.m, M.n, M.U, M.ldu, M.S, M.V, M.ldv, l.da, l.db, s->eps,
                                 s->mode);
      if (!rc && cudaEventRecord(l.done, l.st) != cudaSuccess) rc = SVDUP_ECUDA;
      if (rc) {
        cudaGetLastError();
        finish(s, it->ticket, rc, it->t_submit);
        it = s->pending.erase(it);
        s->cv_done.notify_all();
        continue;
      }
      if (need > l.ws) {
        s->held += need - l.ws;
        l.ws = need;
        s->max_held = std::max(s->max_held, s->held);
      }
      l.busy = true;
      l.ticket = it->ticket;
      l.id = it->id;
      l.t_submit = it->t_submit;
      M.busy = true;
      s->in_flight++;
      s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
      it = s->pending.erase(it);
      progressed = true;
    }
    if (s->stop && s->pending.empty() && s->in_flight == 0) break;
    if (!progressed) {
      // nothing to do right now: wait for a submission, or poll completions shortly
      if (s->in_flight > 0) s->cv_work.wait_for(lk, std::chrono::microseconds(50));
      else s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" {

int svdup_server_create(int device, int lanes, size_t hbm_budget, double eps, int mode,
                        svdup_server_t* out) {
  if (!out || lanes < 0 || lanes > 64 || !(eps > 0.0 && eps < 1.0)) return SVDUP_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return SVDUP_ECUDA;
  svdup_server* s = new (std::nothrow) svdup_server();
  if (!s) return SVDUP_ENOMEM;
  s->device = device;
  s->mode = mode;
  s->eps = eps;
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return SVDUP_ECUDA; }
    hbm_budget = fr / 4 * 3;
  }
  s->budget = hbm_budget;
  s->lanes.resize(lanes == 0 ? 8 : lanes);
  for (Lane& l : s->lanes) {
    int rc = lane_open(s, l);
    if (rc) {
      svdup_server_destroy(s);
      return rc;
    }
  }
  // validate the mode once (an m = n = 1 problem is always valid)
  size_t w = 0;
  if (svdup_update_workspace(s->lanes[0].h, 1, 1, eps, mode, &w) != SVDUP_OK) {
    svdup_server_destroy(s);
    return SVDUP_EINVAL;
  }
  s->th = std::thread(scheduler, s);
  s->started = true;
  *out = s;
  return SVDUP_OK;
}

int svdup_server_register(svdup_server_t s, int m, int n, double* U, int ldu, double* S,
                          double* V, int ldv, int* id) {
  if (!s || !U || !S || !V || !id || m < 1 || n < m || ldu < m || ldv < n) return SVDUP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->mats.push_back(Matrix{m, n, ldu, ldv, U, S, V, false});
  *id = (int)s->mats.size() - 1;
  return SVDUP_OK;
}

int svdup_server_submit(svdup_server_t s, int id, const double* a, const double* b,
                        long long* ticket) {
  if (!s || !a || !b || !ticket) return SVDUP_EINVAL;
  Request r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int)s->mats.size() || s->stop) return SVDUP_EINVAL;
    const Matrix& M = s->mats[id];
    r.a.assign(a, a + M.m);
    r.b.assign(b, b + M.n);
    r.id = id;
    r.ticket = s->next_ticket++;
    r.t_submit = now_ms();
    *ticket = r.ticket;
    s->submitted++;
    s->pending.push_back(std::move(r));
  }
  s->cv_work.notify_one();
  return SVDUP_OK;
}

int svdup_server_wait(svdup_server_t s, long long ticket, double timeout_ms, double* latency_ms) {
  if (!s || ticket < 1) return SVDUP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket >= s->next_ticket) return SVDUP_EINVAL;
  auto ready = [&] { return s->results.count(ticket) > 0; };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready))
    return SVDUP_ETIMEOUT;
  const Result& r = s->results[ticket];
  if (latency_ms) *latency_ms = r.latency_ms;
  return r.status;
}

int svdup_server_drain(svdup_server_t s) {
  if (!s) return SVDUP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->completed >= s->submitted; });
  return SVDUP_OK;
}

int svdup_server_stats(svdup_server_t s, long long* completed, double* p50_ms, double* p99_ms,
                       int* max_in_flight, size_t* max_ws_bytes) {
  if (!s) return SVDUP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  std::vector<double> v = s->lat;
  auto pct = [&](double q) -> double {
    if (v.empty()) return 0.0;
    size_t k = (size_t)(q * (double)(v.size() - 1) + 0.5);
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (max_in_flight) *max_in_flight = s->max_in_flight;
  if (max_ws_bytes) *max_ws_bytes = s->max_held;
  return SVDUP_OK;
}

int svdup_server_destroy(svdup_server_t s) {
  if (!s) return SVDUP_EINVAL;
  if (s->started) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->th.join();
  }
  cudaSetDevice(s->device);
  for (Lane& l : s->lanes) {
    if (l.h) svdup_destroy(l.h);
    lane_vectors_free(l);
    if (l.done) cudaEventDestroy(l.done);
    if (l.st) cudaStreamDestroy(l.st);
  }
  delete s;
  return SVDUP_OK;
}

}  // extern "C"
