// dwf_server.cu -- request loop over many solves (dwf_submit / dwf_poll), built on the C-ABI.
//
// Requests are queued first come first served.  Each of max_inflight worker threads admits
// the head of the queue once its device-memory estimate fits the budget, together with the
// queued requests of the same operator and solver settings (up to max_batch of them), which
// then run as the rows of one dwf_solve_batch: the same launches and CUDA graphs serve all
// of them.  Contexts are cached by operator (lattice, Ns, m0, mq, weights, gauge ensemble)
// and reused by whichever worker takes the next request of that operator; an idle context
// is released only when a new one needs its memory (least recently used first), and its
// buffers go back to the library's stream-ordered pool without synchronising the device, so
// the solves running beside it are not stalled.  Each gauge ensemble is uploaded once as a
// shared gauge object (dwf_gauge) to which every context of that lattice attaches; its
// bytes count against the budget once.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <cmath>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dwf.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Gauge {
  int dims[4];
  std::vector<double> host;
  dwf_gauge *dev = nullptr;  // created by the first request that needs it
  size_t bytes = 0;          // device bytes reserved for it once resident
};

struct Job {
  uint64_t ticket = 0;
  dwf_request req;
  std::vector<double> omega, sigma, rhs, sol;
  std::string key;   // operator: lattice, Ns, m0, mq, weights, gauge ensemble
  std::string pkey;  // solver settings; equal keys and settings may share a batch
  bool mergeable = true;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  dwf_result result;
};

// a cached context of one operator
struct Entry {
  std::string key;
  dwf_ctx *ctx = nullptr;
  size_t bytes = 0;   // reserved device bytes
  int rows = 0;       // largest batch it is sized for
  bool busy = false;
  uint64_t last = 0;  // LRU stamp
};

size_t site_bytes(int prec) { return prec == DWF_PREC_F64 ? 192 : prec == DWF_PREC_F32 ? 96 : 52; }

// device memory of a gauge ensemble once resident: the FP64 copy and the doubled link
// forms in FP64, FP32 and 16 bits
size_t gauge_bytes(const int dims[4]) {
  const size_t V4 = (size_t)dims[0] * dims[1] * dims[2] * dims[3], h = V4 / 2;
  return V4 * 72 * 8 + 2 * h * (1152 + 656 + 192);
}

// device memory a context needs for a batch of `rows` solves (tables, solver fields,
// staging of the host arrays), its gauge ensemble excluded
size_t estimate_bytes(const int dims[4], int Ns, int prec, int system, int rows) {
  const size_t V4 = (size_t)dims[0] * dims[1] * dims[2] * dims[3], h = V4 / 2, n = h * Ns;
  size_t b = 2 * h * 32 + std::max<size_t>(h, 8192) * 8;  // neighbours, partial sums
  b += (system == DWF_SYS_FULL ? 18 : 4) * n * 192;         // FP64 fields shared by the rows
  b += (size_t)rows * 3 * n * 192;                          // FP64 fields per row
  b += (size_t)rows * 7 * n * site_bytes(prec);             // inner CG fields per row
  b += (size_t)rows * 2 * V4 * Ns * 24 * 8;                 // staging of the host arrays
  return b + ((size_t)8 << 20);
}

std::string config_key(const dwf_request &r, const std::vector<double> &om, const std::vector<double> &sg) {
  std::string k((const char *)r.dims, sizeof(r.dims));
  k.append((const char *)&r.Ns, sizeof(r.Ns));
  k.append((const char *)&r.m0, sizeof(r.m0));
  k.append((const char *)&r.mq, sizeof(r.mq));
  k.append((const char *)&r.gauge, sizeof(r.gauge));
  k.append((const char *)om.data(), om.size() * sizeof(double));
  k.append((const char *)sg.data(), sg.size() * sizeof(double));
  return k;
}

std::string params_key(const dwf_solve_params &p) {
  dwf_solve_params q = p;
  q.profile = 0;
  q.use_x0 = 0;
  memset(q.reserved, 0, sizeof(q.reserved));
  return std::string((const char *)&q, sizeof(q));
}

}  // namespace

struct dwf_server {
  dwf_server_params prm;
  int device = -1;
  size_t budget = 0;
  int max_batch = 8;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job *> queue;
  std::map<uint64_t, Job *> jobs;
  std::vector<Gauge *> gauges;
  std::vector<Entry *> cache;
  std::vector<std::thread> workers;
  size_t reserved = 0;
  uint64_t next_ticket = 1, lru = 0;
  bool stop = false;
  bool admit = true;  // dwf_server_set_admission: queued requests wait while false
  long long submitted = 0, completed = 0, in_flight = 0, cancelled = 0, batched = 0;
  std::vector<double> latencies;
  Clock::time_point first_submit, last_done;
  bool any_submit = false;

  void worker_loop();
  // with mu held: admits the head of the queue (and the queued requests that may share its
  // batch) into a cached or new context entry, evicting idle contexts if memory is short
  bool try_admit(std::vector<Job *> &batch, Entry *&entry, bool &new_gauge, std::vector<dwf_ctx *> &evict);
};

bool dwf_server::try_admit(std::vector<Job *> &batch, Entry *&entry, bool &new_gauge, std::vector<dwf_ctx *> &evict) {
  Job *head = queue.front();
  // the requests of the head's operator and settings, in queue order
  std::vector<Job *> group{head};
  if (head->mergeable)
    for (Job *j : queue) {
      if ((int)group.size() >= max_batch) break;
      if (j != head && j->mergeable && j->key == head->key && j->pkey == head->pkey) group.push_back(j);
    }
  Gauge *g = gauges[head->req.gauge];
  const size_t gneed = g->dev ? 0 : g->bytes;
  Entry *idle = nullptr;
  for (Entry *e : cache)
    if (!e->busy && e->key == head->key && (!idle || e->rows > idle->rows)) idle = e;
  while (true) {
    const int rows = (int)group.size();
    const size_t want = estimate_bytes(head->req.dims, head->req.Ns, head->req.params.inner_prec,
                                       head->req.params.system, rows);
    const size_t have = idle ? idle->bytes : 0;
    const size_t need = (want > have ? want - have : 0) + gneed;
    // release idle contexts of other operators, least recently used first
    while (reserved + need > budget) {
      Entry *victim = nullptr;
      for (Entry *e : cache)
        if (!e->busy && e != idle && (!victim || e->last < victim->last)) victim = e;
      if (!victim) break;
      cache.erase(std::find(cache.begin(), cache.end(), victim));
      reserved -= victim->bytes;
      if (victim->ctx) evict.push_back(victim->ctx);
      delete victim;
    }
    if (reserved + need <= budget) {
      for (Job *j : group) queue.erase(std::find(queue.begin(), queue.end(), j));
      if (!idle) {
        idle = new Entry();
        idle->key = head->key;
        cache.push_back(idle);
      }
      idle->busy = true;
      idle->bytes = std::max(have, want);
      idle->rows = std::max(idle->rows, rows);
      reserved += need;
      if (gneed) g->dev = reinterpret_cast<dwf_gauge *>(1);  // placeholder: uploaded by this worker
      new_gauge = gneed != 0;
      batch = group;
      entry = idle;
      return true;
    }
    if (group.size() == 1) return false;
    group.resize(1);  // a smaller batch may fit
  }
}

void dwf_server::worker_loop() {
  const bool have_device = device >= 0 && cudaSetDevice(device) == cudaSuccess;
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    std::vector<Job *> batch;
    Entry *entry = nullptr;
    bool new_gauge = false;
    std::vector<dwf_ctx *> evict;
    while (!stop) {
      if (admit && !queue.empty() && try_admit(batch, entry, new_gauge, evict)) break;
      if (!evict.empty()) break;
      cv.wait(lk);
    }
    if (!evict.empty()) {
      // the released contexts' buffers return to the pool in their streams' order
      lk.unlock();
      for (dwf_ctx *c : evict) dwf_destroy(c);
      lk.lock();
      if (batch.empty()) continue;
    }
    if (batch.empty()) break;
    in_flight += (long long)batch.size();
    if (batch.size() > 1) batched += (long long)batch.size();
    const Clock::time_point t_start = Clock::now();
    for (Job *j : batch) j->t_start = t_start;
    Job *head = batch.front();
    Gauge *g = gauges[head->req.gauge];
    lk.unlock();

    dwf_status st = have_device ? DWF_OK : DWF_ECUDA;
    if (new_gauge) {
      dwf_gauge *dg = nullptr;
      const dwf_status gs = st == DWF_OK ? dwf_gauge_create(g->dims, g->host.data(), &dg) : st;
      std::lock_guard<std::mutex> lock(mu);
      g->dev = gs == DWF_OK ? dg : nullptr;
      if (gs != DWF_OK) reserved -= g->bytes;
      st = gs;
      cv.notify_all();
    }
    if (st == DWF_OK && g->dev == reinterpret_cast<dwf_gauge *>(1)) {
      // another worker is uploading this ensemble
      std::unique_lock<std::mutex> lock(mu);
      cv.wait(lock, [&] { return g->dev != reinterpret_cast<dwf_gauge *>(1); });
      if (!g->dev) st = DWF_ENOMEM;
    }
    if (st == DWF_OK && !entry->ctx) {
      dwf_ctx *c = nullptr;
      st = dwf_create(head->req.dims, head->req.Ns, head->req.m0, head->req.mq, head->omega.data(),
                      head->sigma.data(), &c);
      if (st == DWF_OK) st = dwf_attach_gauge(c, g->dev);
      if (st == DWF_OK) entry->ctx = c;
      else if (c) dwf_destroy(c);
    }
    std::vector<dwf_solve_stats> stats(batch.size());
    for (auto &x : stats) memset(&x, 0, sizeof(x));
    if (st == DWF_OK) {
      if (batch.size() == 1) {
        st = dwf_solve(entry->ctx, head->rhs.data(), head->sol.data(), &head->req.params, &stats[0]);
      } else {
        const size_t full = head->rhs.size();
        std::vector<double> rhs(full * batch.size()), sol(full * batch.size());
        for (size_t k = 0; k < batch.size(); ++k) memcpy(&rhs[k * full], batch[k]->rhs.data(), full * sizeof(double));
        st = dwf_solve_batch(entry->ctx, (int)batch.size(), rhs.data(), sol.data(), &head->req.params, stats.data());
        for (size_t k = 0; k < batch.size(); ++k) memcpy(batch[k]->sol.data(), &sol[k * full], full * sizeof(double));
      }
    }
    lk.lock();
    const Clock::time_point t_done = Clock::now();
    for (size_t k = 0; k < batch.size(); ++k) {
      Job *job = batch[k];
      job->t_done = t_done;
      // a batch reports the first failing row's status; each row's own outcome is in its stats
      job->result.status = (batch.size() > 1 && st == DWF_ENOCONV && stats[k].converged) ? DWF_OK : st;
      job->result.stats = stats[k];
      job->result.queue_ms = ms_between(job->t_submit, job->t_start);
      job->result.latency_ms = ms_between(job->t_submit, job->t_done);
      job->done = true;
      latencies.push_back(job->result.latency_ms);
    }
    last_done = t_done;
    completed += (long long)batch.size();
    in_flight -= (long long)batch.size();
    entry->busy = false;
    entry->last = ++lru;
    if ((st != DWF_OK && st != DWF_ENOCONV) || !entry->ctx) {
      // a context that failed is not reused; an entry that never got one releases its share
      cache.erase(std::find(cache.begin(), cache.end(), entry));
      reserved -= entry->bytes;
      dwf_ctx *c = entry->ctx;
      delete entry;
      if (c) {
        lk.unlock();
        dwf_destroy(c);
        lk.lock();
      }
    }
    cv.notify_all();
  }
}

extern "C" {

void dwf_server_params_default(dwf_server_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->hbm_budget_gb = 150.0;
  p->max_inflight = 4;
}

dwf_status dwf_server_create(const dwf_server_params *params, dwf_server **out) {
  if (!out) return DWF_EINVAL;
  *out = nullptr;
  dwf_server_params prm;
  if (params) prm = *params;
  else dwf_server_params_default(&prm);
  if (!(prm.hbm_budget_gb > 0.0) || prm.max_inflight < 1 || prm.max_inflight > 64) return DWF_EINVAL;
  if (prm.max_batch < 0 || prm.max_batch > 64) return DWF_EINVAL;
  dwf_server *srv = new dwf_server();
  srv->prm = prm;
  srv->budget = (size_t)(prm.hbm_budget_gb * 1073741824.0);
  srv->max_batch = prm.max_batch ? prm.max_batch : 8;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  srv->device = dev;
  for (int i = 0; i < prm.max_inflight; ++i) srv->workers.emplace_back([srv] { srv->worker_loop(); });
  *out = srv;
  return DWF_OK;
}

dwf_status dwf_server_destroy(dwf_server *srv) {
  if (!srv) return DWF_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->queue.clear();
  }
  srv->cv.notify_all();
  for (auto &t : srv->workers) t.join();
  for (auto &kv : srv->jobs) delete kv.second;
  for (Entry *e : srv->cache) {
    if (e->ctx) dwf_destroy(e->ctx);
    delete e;
  }
  for (Gauge *g : srv->gauges) {
    if (g->dev) dwf_gauge_release(g->dev);  // freed with the last context released above
    delete g;
  }
  delete srv;
  return DWF_OK;
}

dwf_status dwf_server_add_gauge(dwf_server *srv, const int dims[4], const double *U, int *handle) {
  if (!srv || !dims || !U || !handle) return DWF_EINVAL;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || (dims[i] & 1)) return DWF_EINVAL;
  Gauge *g = new Gauge();
  memcpy(g->dims, dims, sizeof(g->dims));
  const size_t n = (size_t)dims[0] * dims[1] * dims[2] * dims[3] * 72;
  g->host.assign(U, U + n);
  g->bytes = gauge_bytes(dims);
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->gauges.push_back(g);
  *handle = (int)srv->gauges.size() - 1;
  return DWF_OK;
}

dwf_status dwf_submit(dwf_server *srv, const dwf_request *req, uint64_t *ticket) {
  if (!srv || !req || !ticket || !req->omega || !req->sigma || !req->rhs) return DWF_EINVAL;
  if (req->Ns < 1 || req->Ns > 64 || !(req->m0 > 0.0 && req->m0 < 2.0) || !(req->mq >= 0.0)) return DWF_EINVAL;
  for (int s = 0; s < req->Ns; ++s)
    if (!(req->omega[s] > 0.0) || !std::isfinite(req->sigma[s])) return DWF_EINVAL;
  if (req->params.system != DWF_SYS_FULL && req->params.system != DWF_SYS_NORMAL) return DWF_EINVAL;
  if (req->params.inner_prec < DWF_PREC_F64 || req->params.inner_prec > DWF_PREC_BF16) return DWF_EINVAL;
  Job *job = new Job();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (req->gauge < 0 || req->gauge >= (int)srv->gauges.size() ||
        memcmp(srv->gauges[req->gauge]->dims, req->dims, sizeof(req->dims)) != 0) {
      delete job;
      return DWF_EINVAL;
    }
  }
  job->req = *req;
  job->req.params.use_x0 = 0;  // a request carries no initial guess
  job->omega.assign(req->omega, req->omega + req->Ns);
  job->sigma.assign(req->sigma, req->sigma + req->Ns);
  const size_t full = (size_t)req->dims[0] * req->dims[1] * req->dims[2] * req->dims[3] * req->Ns * 24;
  job->rhs.assign(req->rhs, req->rhs + full);
  job->sol.assign(full, 0.0);
  job->req.omega = job->omega.data();
  job->req.sigma = job->sigma.data();
  job->req.rhs = job->rhs.data();
  job->key = config_key(*req, job->omega, job->sigma);
  job->pkey = params_key(job->req.params);
  // a 16-bit solve in AUTO mode may switch to FP32 inner iterations, which only a single
  // solve does: such requests run on their own
  job->mergeable = !(job->req.params.inner_prec >= DWF_PREC_F16 && job->req.params.mode == DWF_MODE_AUTO);
  const size_t est = estimate_bytes(req->dims, req->Ns, req->params.inner_prec, req->params.system, 1);
  std::lock_guard<std::mutex> lk(srv->mu);
  const size_t gbytes = srv->gauges[req->gauge]->bytes;
  if (est + gbytes > srv->budget) {
    delete job;
    return DWF_ENOMEM;
  }
  job->ticket = srv->next_ticket++;
  job->t_submit = Clock::now();
  if (!srv->any_submit) {
    srv->first_submit = job->t_submit;
    srv->any_submit = true;
  }
  srv->jobs[job->ticket] = job;
  srv->queue.push_back(job);
  ++srv->submitted;
  *ticket = job->ticket;
  srv->cv.notify_all();
  return DWF_OK;
}

dwf_status dwf_poll(dwf_server *srv, uint64_t ticket, double *psi_out, dwf_result *result) {
  if (!srv) return DWF_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(ticket);
  if (it == srv->jobs.end()) return DWF_EINVAL;
  Job *job = it->second;
  if (!job->done) return DWF_EAGAIN;
  if (psi_out) memcpy(psi_out, job->sol.data(), job->sol.size() * sizeof(double));
  if (result) *result = job->result;
  srv->jobs.erase(it);
  delete job;
  return DWF_OK;
}

dwf_status dwf_cancel(dwf_server *srv, uint64_t ticket) {
  if (!srv) return DWF_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(ticket);
  if (it == srv->jobs.end()) return DWF_EINVAL;
  Job *job = it->second;
  // a queued job is only ever touched under the lock, so it can go; one that a worker has
  // taken runs to completion
  auto q = std::find(srv->queue.begin(), srv->queue.end(), job);
  if (q == srv->queue.end()) return DWF_EBUSY;
  srv->queue.erase(q);
  srv->jobs.erase(it);
  delete job;
  ++srv->cancelled;
  srv->cv.notify_all();  // the next request may now be admissible
  return DWF_OK;
}

dwf_status dwf_server_set_admission(dwf_server *srv, int open) {
  if (!srv) return DWF_EINVAL;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->admit = open != 0;
  }
  srv->cv.notify_all();
  return DWF_OK;
}

dwf_status dwf_server_get_stats(dwf_server *srv, dwf_server_stats *out) {
  if (!srv || !out) return DWF_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = srv->submitted;
  out->cancelled = srv->cancelled;
  out->completed = srv->completed;
  out->in_flight = srv->in_flight;
  out->queued = (long long)srv->queue.size();
  out->hbm_reserved_gb = srv->reserved / 1073741824.0;
  out->batched = srv->batched;
  if (!srv->latencies.empty()) {
    std::vector<double> l = srv->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
      const double pos = q * (l.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - i;
      return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : l) sum += x;
    out->mean_ms = sum / l.size();
    const double span = ms_between(srv->first_submit, srv->last_done);
    out->solves_per_s = span > 0 ? srv->completed / (span * 1e-3) : 0.0;
  }
  return DWF_OK;
}

}  // extern "C"
