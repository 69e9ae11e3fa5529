// svdup_serve.cu -- the serving engine: resident SVDs and continuously admitted
// rank-one updates (svdup_server_* in include/svdup.h).
//
// One scheduler thread owns every CUDA call of the engine.  Its loop:
//   1. completions: a lane whose whole group of requests has completed (every slot's
//      event has fired) finishes them (status from the lane's handle, latency from each
//      submission to the moment the result is posted);
//   2. admissions, in submission order: a request is admitted when its matrix has no
//      update in flight, a lane is free, and the free-HBM ledger allows the workspace
//      the update needs.  The admitted request opens a group: later pending requests of
//      the same size class (n in the same power-of-two range) join it, up to the
//      engine's group size, and the group's updates are queued back to back on the
//      lane's stream (updates of one matrix in submission order).  The ledger counts
//      the workspace every lane holds (a lane keeps the largest workspace it has
//      needed); when a group does not fit, idle lanes give their workspace back (their
//      handle is recreated) before it waits.
// Requests of one matrix therefore apply in submission order, requests of different
// matrices overlap on the device, and a request that arrives while others run is
// admitted as soon as a lane and memory free up (continuous batching).
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <list>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
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
  int inflight;  // updates of this matrix queued on a lane
};

constexpr int kMaxGroup = 16;  // requests one lane takes per cycle (at most)

struct Slot {
  cudaEvent_t done = nullptr;
  double* da = nullptr;     // device copies of a, b
  double* db = nullptr;
  double* ha = nullptr;     // pinned staging
  double* hb = nullptr;
  int cap = 0;              // capacity (entries) of the four vectors
  long long ticket = 0;
  int id = -1;
  double t_submit = 0.0;
};

struct Lane {
  svdup_t h = nullptr;
  cudaStream_t st = nullptr;
  size_t ws = 0;            // workspace bytes the lane's handle holds
  int nbusy = 0;            // requests of the current group (0: free)
  Slot slot[kMaxGroup];
};

// Size class of an m x n update: the power-of-two range of n.
int size_class(int n) {
  int c = 0;
  while ((1 << (c + 1)) <= n && c < 30) c++;
  return c;
}

}  // namespace

struct svdup_server {
  int device = 0;
  int mode = 0;
  double eps = 1e-12;
  size_t budget = 0;
  std::vector<Lane> lanes;
  std::vector<Matrix> mats;
  std::list<Request> pending;
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
  int group_max = 4;                      // requests per lane cycle (same size class)
  long long groups = 0, grouped = 0;      // lane cycles launched, requests in them
  int max_group_seen = 0;
};

namespace {

int lane_open(svdup_server* s, Lane& l) {
  if (cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return SVDUP_ECUDA;
  }
  for (Slot& q : l.slot)
    if (cudaEventCreateWithFlags(&q.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return SVDUP_ECUDA;
    }
  return svdup_create(&l.h, s->device, (void*)l.st, 0);
}

void slot_vectors_free(Slot& q) {
  if (q.da) cudaFree(q.da);
  if (q.db) cudaFree(q.db);
  if (q.ha) cudaFreeHost(q.ha);
  if (q.hb) cudaFreeHost(q.hb);
  q.da = q.db = q.ha = q.hb = nullptr;
  q.cap = 0;
}

int slot_vectors(Slot& q, int n) {
  if (n <= q.cap) return SVDUP_OK;
  slot_vectors_free(q);
  if (cudaMalloc(&q.da, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&q.db, n * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&q.ha, n * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&q.hb, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    slot_vectors_free(q);
    return SVDUP_ENOMEM;
  }
  q.cap = n;
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
    if (l.nbusy == 0 && l.ws >= need && (best < 0 || l.ws < s->lanes[best].ws)) best = i;
  }
  if (best >= 0) return best;
  for (int i = 0; i < (int)s->lanes.size(); i++) {  // else the free lane that grows least
    const Lane& l = s->lanes[i];
    if (l.nbusy == 0 && (best < 0 || l.ws > s->lanes[best].ws)) best = i;
  }
  if (best < 0) return -1;
  size_t grow = need - s->lanes[best].ws;
  if (s->held + grow <= s->budget) return best;
  // free idle workspaces, largest first, until the growth fits
  std::vector<int> idle;
  for (int i = 0; i < (int)s->lanes.size(); i++)
    if (s->lanes[i].nbusy == 0 && i != best && s->lanes[i].ws > 0) idle.push_back(i);
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

// Queues request r on slot q of lane l (its vectors, then the update, then the slot's
// event); returns a status code.
int launch_one(svdup_server* s, Lane& l, Slot& q, const Request& r) {
  const Matrix& M = s->mats[r.id];
  int rc = slot_vectors(q, M.n);
  if (rc) return rc;
  memcpy(q.ha, r.a.data(), M.m * sizeof(double));
  memcpy(q.hb, r.b.data(), M.n * sizeof(double));
  if (cudaMemcpyAsync(q.da, q.ha, M.m * sizeof(double), cudaMemcpyHostToDevice, l.st) !=
          cudaSuccess ||
      cudaMemcpyAsync(q.db, q.hb, M.n * sizeof(double), cudaMemcpyHostToDevice, l.st) !=
          cudaSuccess)
    return SVDUP_ECUDA;
  rc = svdup_update(l.h, M.m, M.n, M.U, M.ldu, M.S, M.V, M.ldv, q.da, q.db, s->eps, s->mode);
  if (rc) return rc;
  return cudaEventRecord(q.done, l.st) == cudaSuccess ? SVDUP_OK : SVDUP_ECUDA;
}

void scheduler(svdup_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progressed = false;
    // 1. completions: a lane's group is finished once its last event has fired (the
    //    handle's status word covers the whole group)
    for (Lane& l : s->lanes) {
      if (l.nbusy == 0) continue;
      cudaError_t q = cudaEventQuery(l.slot[l.nbusy - 1].done);
      if (q == cudaErrorNotReady) continue;
      int st = (q == cudaSuccess) ? svdup_sync(l.h) : SVDUP_ECUDA;
      if (q != cudaSuccess) cudaGetLastError();
      for (int i = 0; i < l.nbusy; i++) {
        Slot& sl = l.slot[i];
        s->mats[sl.id].inflight--;
        s->in_flight--;
        finish(s, sl.ticket, st, sl.t_submit);
      }
      l.nbusy = 0;
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // 2. admissions in submission order; a request whose matrix is busy, or that finds
    //    no lane, blocks its matrix's later requests for this pass (order per matrix)
    std::unordered_set<int> blocked;
    for (auto it = s->pending.begin(); it != s->pending.end();) {
      Matrix& M = s->mats[it->id];
      if (M.inflight > 0 || blocked.count(it->id)) {
        blocked.insert(it->id);
        ++it;
        continue;
      }
      size_t need = 0;
      int rc = svdup_update_workspace(s->lanes[0].h, M.m, M.n, s->eps, s->mode, &need);
      if (rc) {
        finish(s, it->ticket, rc, it->t_submit);
        it = s->pending.erase(it);
        s->cv_done.notify_all();
        continue;
      }
      // the group: this request and later ones of its size class whose matrices are idle
      // (or already in the group, in order), up to group_max
      std::vector<std::list<Request>::iterator> grp{it};
      size_t need_g = need;
      const int cls = size_class(M.n);
      std::unordered_set<int> in_grp{it->id}, skipped;
      for (auto jt = std::next(it); jt != s->pending.end() && (int)grp.size() < s->group_max;
           ++jt) {
        const Matrix& Mj = s->mats[jt->id];
        const bool ok = size_class(Mj.n) == cls && !blocked.count(jt->id) &&
                        !skipped.count(jt->id) && (Mj.inflight == 0 || in_grp.count(jt->id));
        if (!ok) {
          skipped.insert(jt->id);  // its later requests must wait behind it
          continue;
        }
        size_t nj = 0;
        if (svdup_update_workspace(s->lanes[0].h, Mj.m, Mj.n, s->eps, s->mode, &nj)) {
          skipped.insert(jt->id);
          continue;
        }
        need_g = std::max(need_g, nj);
        grp.push_back(jt);
        in_grp.insert(jt->id);
      }
      int li = pick_lane(s, need_g);
      if (li < 0 && grp.size() > 1) {  // the group does not fit: the first request alone
        grp.resize(1);
        need_g = need;
        li = pick_lane(s, need);
      }
      if (li < 0) {
        blocked.insert(it->id);
        ++it;
        continue;
      }
      Lane& l = s->lanes[li];
      if (need_g > l.ws) {
        s->held += need_g - l.ws;
        l.ws = need_g;
        s->max_held = std::max(s->max_held, s->held);
      }
      int launched = 0;
      for (auto& g : grp) {
        Slot& sl = l.slot[launched];
        rc = launch_one(s, l, sl, *g);
        if (rc) {  // this request fails; the ones already queued stay with the lane
          cudaGetLastError();
          finish(s, g->ticket, rc, g->t_submit);
          s->cv_done.notify_all();
          continue;
        }
        sl.ticket = g->ticket;
        sl.id = g->id;
        sl.t_submit = g->t_submit;
        s->mats[g->id].inflight++;
        launched++;
      }
      l.nbusy = launched;
      s->in_flight += launched;
      s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
      if (launched > 0) {
        s->groups++;
        s->grouped += launched;
        s->max_group_seen = std::max(s->max_group_seen, launched);
      }
      // erase the group's requests (list iterators stay valid across erasures)
      for (size_t i = grp.size(); i-- > 1;) s->pending.erase(grp[i]);
      it = s->pending.erase(grp[0]);
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
  s->mats.push_back(Matrix{m, n, ldu, ldv, U, S, V, 0});
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

int svdup_server_set_group(svdup_server_t s, int group_max) {
  if (!s || group_max < 1 || group_max > kMaxGroup) return SVDUP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->group_max = group_max;
  return SVDUP_OK;
}

int svdup_server_group_stats(svdup_server_t s, long long* groups, long long* grouped,
                             int* max_group) {
  if (!s) return SVDUP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (groups) *groups = s->groups;
  if (grouped) *grouped = s->grouped;
  if (max_group) *max_group = s->max_group_seen;
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
    for (Slot& q : l.slot) {
      slot_vectors_free(q);
      if (q.done) cudaEventDestroy(q.done);
    }
    if (l.st) cudaStreamDestroy(l.st);
  }
  delete s;
  return SVDUP_OK;
}

}  // extern "C"
