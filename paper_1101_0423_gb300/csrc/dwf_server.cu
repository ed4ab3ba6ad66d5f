// dwf_server.cu -- request loop over many solves (dwf_submit / dwf_poll), built on the C-ABI.
//
// Requests are queued first come first served.  Each of max_inflight worker threads takes
// the head of the queue once the request's device-memory estimate fits the budget, builds
// (or reuses) a context for the request's lattice and fifth-dimension parameters, loads the
// resident gauge ensemble into it and runs dwf_solve on the context's own CUDA stream, so
// solves of different requests overlap on the device.  A worker keeps its context only
// while the next queued request has the same configuration; otherwise the context and its
// reservation are released.  Gauge ensembles are kept on the host until a request first
// needs them and are then uploaded once and shared (their bytes count against the budget).
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
  double *dev = nullptr;
  size_t bytes = 0;
};

struct Job {
  uint64_t ticket = 0;
  dwf_request req;
  std::vector<double> omega, sigma, rhs, sol;
  std::string key;
  size_t est_bytes = 0;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  dwf_result result;
};

size_t site_bytes(int prec) { return prec == DWF_PREC_F64 ? 192 : prec == DWF_PREC_F32 ? 96 : 52; }

// device memory a context needs for one solve (gauge copies, tables, solver fields)
size_t estimate_bytes(const int dims[4], int Ns, int prec, int system) {
  const size_t V4 = (size_t)dims[0] * dims[1] * dims[2] * dims[3], h = V4 / 2, n = h * Ns;
  size_t b = V4 * 72 * 8;                        // FP64 host-layout gauge copy
  b += 2 * h * (1152 + 656);                     // doubled FP64 and FP32 gauges
  if (prec >= DWF_PREC_F16) b += 2 * h * 192;    // doubled 16-bit gauge
  b += 2 * h * 32 + std::max<size_t>(h, 8192) * 8;
  b += (system == DWF_SYS_FULL ? 21 : 7) * n * 192;  // FP64 solver and reconstruction fields
  b += 7 * n * site_bytes(prec);                 // inner CG fields
  b += 2 * V4 * Ns * 24 * 8;                     // staging of the host arrays
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

}  // namespace

struct dwf_server {
  dwf_server_params prm;
  int device = -1;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job *> queue;
  std::map<uint64_t, Job *> jobs;
  std::vector<Gauge *> gauges;
  std::vector<std::thread> workers;
  size_t reserved = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool admit = true;  // dwf_server_set_admission: queued requests wait while false
  long long submitted = 0, completed = 0, in_flight = 0, cancelled = 0;
  std::vector<double> latencies;
  Clock::time_point first_submit, last_done;
  bool any_submit = false;

  void worker_loop();
};

void dwf_server::worker_loop() {
  bool have_device = device >= 0 && cudaSetDevice(device) == cudaSuccess;
  dwf_ctx *ctx = nullptr;
  std::string ctx_key;
  size_t ctx_bytes = 0;
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    Job *job = nullptr;
    while (!stop) {
      if (admit && !queue.empty()) {
        Job *head = queue.front();
        const bool reuse = ctx && head->key == ctx_key;
        // a context not reused by the head request is released before admission
        if (!reuse && ctx) {
          lk.unlock();
          dwf_destroy(ctx);
          lk.lock();
          ctx = nullptr;
          reserved -= ctx_bytes;
          ctx_bytes = 0;
          ctx_key.clear();
          cv.notify_all();
          continue;
        }
        Gauge *g = gauges[head->req.gauge];
        const size_t gauge_extra = (have_device && !g->dev) ? g->bytes : 0;
        const size_t need = (reuse ? 0 : head->est_bytes) + gauge_extra;
        if (reserved + need <= budget) {
          queue.pop_front();
          job = head;
          if (!reuse) {
            reserved += head->est_bytes;
            ctx_bytes = head->est_bytes;
          }
          if (gauge_extra) reserved += gauge_extra;
          break;
        }
      }
      cv.wait(lk);
    }
    if (!job) break;
    ++in_flight;
    job->t_start = Clock::now();
    Gauge *g = gauges[job->req.gauge];
    // upload the ensemble once, under the lock (other workers may need it too)
    dwf_status st = DWF_OK;
    if (!have_device) {
      st = DWF_ECUDA;
    } else if (!g->dev) {
      if (cudaMalloc((void **)&g->dev, g->bytes) != cudaSuccess ||
          cudaMemcpy(g->dev, g->host.data(), g->bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        if (g->dev) cudaFree(g->dev);
        g->dev = nullptr;
        reserved -= g->bytes;
        st = DWF_ENOMEM;
      }
    }
    lk.unlock();
    dwf_solve_stats stats;
    memset(&stats, 0, sizeof(stats));
    if (st == DWF_OK && !ctx) {
      st = dwf_create(job->req.dims, job->req.Ns, job->req.m0, job->req.mq, job->omega.data(), job->sigma.data(),
                      &ctx);
      if (st == DWF_OK) st = dwf_load_gauge_dev(ctx, g->dev, nullptr);
      if (st == DWF_OK) ctx_key = job->key;
    }
    if (st == DWF_OK) st = dwf_solve(ctx, job->rhs.data(), job->sol.data(), &job->req.params, &stats);
    lk.lock();
    job->t_done = Clock::now();
    job->result.status = st;
    job->result.stats = stats;
    job->result.queue_ms = ms_between(job->t_submit, job->t_start);
    job->result.latency_ms = ms_between(job->t_submit, job->t_done);
    job->done = true;
    latencies.push_back(job->result.latency_ms);
    last_done = job->t_done;
    ++completed;
    --in_flight;
    if ((st != DWF_OK && st != DWF_ENOCONV) || !ctx) {
      // a context that failed is not reused; a job that never got one releases its share
      if (ctx) {
        lk.unlock();
        dwf_destroy(ctx);
        lk.lock();
      }
      ctx = nullptr;
      ctx_key.clear();
      reserved -= ctx_bytes;
      ctx_bytes = 0;
    }
    cv.notify_all();
  }
  if (ctx) {
    lk.unlock();
    dwf_destroy(ctx);
    lk.lock();
    reserved -= ctx_bytes;
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
  dwf_server *srv = new dwf_server();
  srv->prm = prm;
  srv->budget = (size_t)(prm.hbm_budget_gb * 1073741824.0);
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
  for (Gauge *g : srv->gauges) {
    if (g->dev) cudaFree(g->dev);
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
  g->bytes = n * sizeof(double);
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
  job->est_bytes = estimate_bytes(req->dims, req->Ns, req->params.inner_prec, req->params.system);
  std::lock_guard<std::mutex> lk(srv->mu);
  const size_t gbytes = srv->gauges[req->gauge]->bytes;
  if (job->est_bytes + gbytes > srv->budget) {
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
