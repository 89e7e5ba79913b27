// Serving form: a request loop of biharmonic solves (different dimension,
// degree, level and right-hand side) with continuous batching.  The paper has
// no counterpart; this is a deployment form of the same solver.
//
//  - Slots: `slots` worker threads; each runs one solve at a time on its own
//    resident hierarchy (context) and that context's own CUDA stream, so the
//    solves of different slots overlap on the device.
//  - Resident hierarchies: contexts are pooled by (dim, degree, level,
//    precision) and reused by later requests of the same shape, keeping the
//    multigrid hierarchy and its 1D eigendata on the device.
//  - Admission by HBM footprint: a request whose shape has no idle context
//    needs a new one; it is admitted when the footprint estimate fits in the
//    memory budget, after evicting idle contexts (least recently used first);
//    otherwise it waits until running solves release memory.
//  - Continuous batching: a request starts as soon as a slot and its memory
//    are free -- requests that arrive while others run join immediately, not
//    at a batch boundary.
//  - Precision: the FP32 V-cycle with compensated FP32 defects
//    (BH_MIXED_FP32_RC) inside flexible FP64 GMRES for degrees up to
//    mixed_max_degree, FP64 otherwise;
//    GMRES is right-preconditioned (true residual) for every request.
//  - Latency of a request = completion time - submission time.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "biharm.h"

namespace bh {
void set_last_error(const std::string& msg);  // api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

bh_status serr(bh_status s, const std::string& m) {
  bh::set_last_error(m);
  return s;
}

struct Request {
  int64_t ticket = 0;
  int dim = 2, degree = 2, level = 1;
  const double* b = nullptr;  // host, owned by the caller until completion
  double* x = nullptr;
  Clock::time_point submitted;
  Clock::time_point deadline = Clock::time_point::max();  // dropped if not started by then
  // results
  bool done = false;
  int status = BH_OK, iters = 0;
  double relres = 0, latency = 0, service = 0;
};

using Key = std::tuple<int, int, int, int>;  // dim, degree, level, precision

struct Pooled {
  bh_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  Key key;
  double bytes = 0;
  bool busy = false;
  Clock::time_point last_used;
};

double footprint(int d, int k, int L, int precision, int restart) {
  // every level: x, b, r (+ FP32 copies); finest: sweep scratch and two
  // transfer vectors (+ FP32); GMRES basis V (m+1), Z (m), w, t; patch lists
  double total = 0, nL = 0;
  // FP64 x, b, r; + FP32 x, b, r (mixed); + the FP64 right-hand side of the
  // defect (RC), and the FP64 iterate copy (R64)
  const double vb = precision == BH_FP64         ? 8.0
                    : precision == BH_MIXED_FP32    ? 12.0
                    : precision == BH_MIXED_FP32_RC ? 14.67
                                                    : 17.33;
  for (int l = 1; l <= L; ++l) {
    const double n = std::pow((double)k * (1 << l) - 1.0, d);
    total += 3 * vb * n + 4.0 * n / std::pow(k, d);
    nL = n;
  }
  total += ((d == 2 ? 3 : 6) + 2) * vb * nL;
  total += (2.0 * restart + 3.0) * 8.0 * nL;
  total += 64.0 * 1024 * 1024;  // tables, inverses, allocation granularity
  return total;
}

}  // namespace

struct bh_server {
  bh_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_mem;
  std::deque<Request*> queue;
  std::map<int64_t, Request*> reqs;
  std::vector<Pooled*> pool;
  std::vector<std::thread> workers;
  double used = 0;
  bool stop = false;
  int64_t next_ticket = 1;
  int running = 0;
  long long admitted = 0, evictions = 0, created = 0, completed = 0, dropped = 0, cancelled = 0,
            failed = 0;
  double busy_seconds = 0;
  Clock::time_point t0;
};

namespace {

// take an idle context of this shape, or make room and create one (mu held)
Pooled* acquire(bh_server* s, std::unique_lock<std::mutex>& lk, const Request& r, int precision,
                bh_status* st) {
  const Key key{r.dim, r.degree, r.level, precision};
  while (!s->stop) {
    for (Pooled* p : s->pool)
      if (!p->busy && p->key == key) {
        p->busy = true;
        return p;
      }
    const double need = footprint(r.dim, r.degree, r.level, precision, s->cfg.gmres_restart);
    if (need > s->cfg.mem_budget_bytes) {
      *st = serr(BH_ENOMEM, "request footprint exceeds the server's memory budget");
      return nullptr;
    }
    // evict idle contexts, least recently used first, until the request fits
    while (s->used + need > s->cfg.mem_budget_bytes) {
      Pooled* victim = nullptr;
      for (Pooled* p : s->pool)
        if (!p->busy && (!victim || p->last_used < victim->last_used)) victim = p;
      if (!victim) break;
      s->pool.erase(std::find(s->pool.begin(), s->pool.end(), victim));
      s->used -= victim->bytes;
      s->evictions++;
      bh_destroy(victim->ctx);
      cudaStreamDestroy(victim->st);
      delete victim;
    }
    if (s->used + need <= s->cfg.mem_budget_bytes) {
      s->used += need;  // reserve before creating outside the lock
      lk.unlock();
      Pooled* p = new Pooled();
      p->key = key;
      p->bytes = need;
      p->busy = true;
      bh_params prm;
      bh_status cs = bh_default_params(r.dim, r.degree, r.level, &prm);
      if (cs == BH_OK) {
        prm.precision = precision;
        prm.gmres_side = BH_RIGHT;
        prm.gmres_restart = s->cfg.gmres_restart;
        if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess) {
          cudaGetLastError();
          cs = serr(BH_ECUDA, "stream creation failed");
        } else {
          cs = bh_create(&prm, p->st, &p->ctx);
        }
      }
      lk.lock();
      if (cs != BH_OK) {
        s->used -= need;
        if (p->st) cudaStreamDestroy(p->st);
        delete p;
        *st = cs;
        s->cv_mem.notify_all();
        return nullptr;
      }
      s->created++;
      s->pool.push_back(p);
      return p;
    }
    s->cv_mem.wait(lk);  // wait for a running solve to release memory
  }
  *st = serr(BH_EBUSY, "server stopping");
  return nullptr;
}

void worker(bh_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    if (s->queue.empty() && s->stop) return;
    Request* r = s->queue.front();
    s->queue.pop_front();
    if (Clock::now() > r->deadline) {  // not started before its deadline: dropped
      r->status = BH_ETIMEOUT;
      r->done = true;
      r->latency = std::chrono::duration<double>(Clock::now() - r->submitted).count();
      s->completed++;
      s->dropped++;
      s->cv_done.notify_all();
      continue;
    }
    const int precision = (s->cfg.mixed_max_degree >= r->degree) ? BH_MIXED_FP32_RC : BH_FP64;
    bh_status st = BH_OK;
    Pooled* p = acquire(s, lk, *r, precision, &st);
    if (!p) {
      r->status = st;
      s->failed++;
      r->done = true;
      r->latency = std::chrono::duration<double>(Clock::now() - r->submitted).count();
      s->completed++;
      s->cv_done.notify_all();
      continue;
    }
    s->admitted++;
    s->running++;
    lk.unlock();
    const auto t_start = Clock::now();
    int it = 0;
    double rr = 0;
    st = bh_solve_host(p->ctx, r->b, r->x, s->cfg.rtol, s->cfg.maxit, &it, &rr);
    const auto t_end = Clock::now();
    lk.lock();
    s->running--;
    s->busy_seconds += std::chrono::duration<double>(t_end - t_start).count();
    p->busy = false;
    p->last_used = t_end;
    r->status = st;
    if (st != BH_OK) s->failed++;
    r->iters = it;
    r->relres = rr;
    r->service = std::chrono::duration<double>(t_end - t_start).count();
    r->latency = std::chrono::duration<double>(t_end - r->submitted).count();
    r->done = true;
    s->completed++;
    s->cv_done.notify_all();
    s->cv_mem.notify_all();
  }
}

}  // namespace

extern "C" {

bh_status bh_server_default_config(bh_server_config* cfg) {
  if (!cfg) return serr(BH_EINVAL, "null config");
  bh_server_config c{};
  c.slots = 4;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
    c.mem_budget_bytes = 0.8 * (double)free_b;
  else {
    cudaGetLastError();
    c.mem_budget_bytes = 0.0;
  }
  c.mixed_max_degree = 7;
  c.rtol = 1e-8;
  c.maxit = 200;
  c.gmres_restart = 30;
  c.queue_capacity = 100000;
  *cfg = c;
  return BH_OK;
}

bh_status bh_server_create(const bh_server_config* cfg, bh_server** out) {
  if (!cfg || !out || cfg->slots < 1 || cfg->slots > 64 || !(cfg->mem_budget_bytes > 0) ||
      !(cfg->rtol > 0) || cfg->maxit < 1 || cfg->gmres_restart < 1 || cfg->queue_capacity < 1)
    return serr(BH_EINVAL, "bh_server_create: bad configuration");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return serr(BH_ECUDA, "no CUDA device available");
  }
  bh_server* s = new (std::nothrow) bh_server();
  if (!s) return serr(BH_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->t0 = Clock::now();
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < cfg->slots; ++i)
    s->workers.emplace_back([s, dev] {
      cudaSetDevice(dev);
      worker(s);
    });
  *out = s;
  return BH_OK;
}

bh_status bh_server_submit(bh_server* s, int dim, int degree, int level, const double* b_host,
                           double* x_host, int64_t* ticket) {
  return bh_server_submit_deadline(s, dim, degree, level, b_host, x_host, 0.0, ticket);
}

bh_status bh_server_submit_deadline(bh_server* s, int dim, int degree, int level,
                                    const double* b_host, double* x_host, double deadline_s,
                                    int64_t* ticket) {
  if (!s || !b_host || !x_host || !ticket || !(deadline_s >= 0.0))
    return serr(BH_EINVAL, "bh_server_submit: bad arguments");
  bh_params tmp;
  bh_status v = bh_default_params(dim, degree, level, &tmp);
  if (v != BH_OK) return v;
  Request* r = new (std::nothrow) Request();
  if (!r) return serr(BH_ENOMEM, "host allocation failed");
  r->dim = dim;
  r->degree = degree;
  r->level = level;
  r->b = b_host;
  r->x = x_host;
  r->submitted = Clock::now();
  if (deadline_s > 0.0)
    r->deadline = r->submitted +
                  std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(deadline_s));
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) {
      delete r;
      return serr(BH_EBUSY, "server stopping");
    }
    if ((int64_t)s->queue.size() >= s->cfg.queue_capacity) {
      delete r;
      return serr(BH_EBUSY, "request queue full");
    }
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_one();
  return BH_OK;
}

bh_status bh_server_wait(bh_server* s, int64_t ticket, double timeout_s, bh_server_result* res) {
  if (!s || !res) return serr(BH_EINVAL, "bh_server_wait: bad arguments");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return serr(BH_EINVAL, "unknown ticket");
  Request* r = it->second;
  const auto pred = [&] { return r->done; };
  if (timeout_s < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
    return serr(BH_ETIMEOUT, "request still running");
  res->status = r->status;
  res->iters = r->iters;
  res->relres = r->relres;
  res->latency_s = r->latency;
  res->service_s = r->service;
  s->reqs.erase(it);
  delete r;
  return BH_OK;
}

bh_status bh_server_cancel(bh_server* s, int64_t ticket) {
  if (!s) return serr(BH_EINVAL, "null server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return serr(BH_EINVAL, "unknown ticket");
  Request* r = it->second;
  auto q = std::find(s->queue.begin(), s->queue.end(), r);
  if (q == s->queue.end()) return serr(BH_EBUSY, "request already started or finished");
  s->queue.erase(q);
  r->status = BH_ECANCELED;
  r->done = true;
  r->latency = std::chrono::duration<double>(Clock::now() - r->submitted).count();
  s->completed++;
  s->cancelled++;
  s->cv_done.notify_all();
  return BH_OK;
}

bh_status bh_server_stats(bh_server* s, char* buf, size_t len) {
  if (!s || !buf || len == 0) return serr(BH_EINVAL, "bad arguments");
  std::lock_guard<std::mutex> g(s->mu);
  const double up = std::chrono::duration<double>(Clock::now() - s->t0).count();
  std::snprintf(buf, len,
                "{\"slots\": %d, \"queued\": %zu, \"running\": %d, \"admitted\": %lld, "
                "\"completed\": %lld, \"resident_contexts\": %zu, \"created\": %lld, "
                "\"evictions\": %lld, \"reserved_bytes\": %.0f, \"budget_bytes\": %.0f, "
                "\"busy_slot_seconds\": %.6f, \"uptime_s\": %.6f, \"dropped\": %lld, "
                "\"cancelled\": %lld, \"failed\": %lld}",
                s->cfg.slots, s->queue.size(), s->running, s->admitted, s->completed,
                s->pool.size(), s->created, s->evictions, s->used, s->cfg.mem_budget_bytes,
                s->busy_seconds, up, s->dropped, s->cancelled, s->failed);
  return BH_OK;
}

bh_status bh_server_destroy(bh_server* s) {
  if (!s) return serr(BH_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_mem.notify_all();
  for (auto& t : s->workers) t.join();
  for (Pooled* p : s->pool) {
    bh_destroy(p->ctx);
    cudaStreamDestroy(p->st);
    delete p;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return BH_OK;
}

}  // extern "C"
