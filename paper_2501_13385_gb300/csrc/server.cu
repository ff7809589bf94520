// Serving: continuous batching of completion requests.
//
// ttc_submit copies a request and queues it; an engine thread admits queued
// requests into slots while their estimated device memory fits the budget
// (each becomes a context: observations uploaded, layout built, starting
// cores set), steps all active slots together as one batch (one CUDA graph
// launch per iteration), checks every slot's stop rule after each iteration,
// retires finished slots (cores copied out, context destroyed) and admits
// the next requests while the others keep running.  A slot computes exactly
// what its request computes alone (same kernels and block decomposition), so
// results do not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  uint64_t ticket = 0;
  int d = 0;
  std::vector<int64_t> n;
  std::vector<int32_t> r;
  int64_t N = 0;
  std::vector<int32_t> idx;
  std::vector<double> y;
  std::vector<std::vector<double>> init;
  std::vector<int32_t> truth_r;
  std::vector<std::vector<double>> truth;
  ttc_options opt;
  Clock::time_point t_submit, t_admit, t_done;
  // result
  int status = TTC_OK;
  ttc_solve_info info;
  std::vector<std::vector<double>> cores;
  bool done = false;
  size_t est_bytes = 0;
  char detail[128] = "";
};

struct Slot {
  std::shared_ptr<Request> req;
  ttc_ctx* ctx = nullptr;
  SolveState st;
  size_t bytes = 0;
};

}  // namespace

struct ttc_server {
  size_t budget = 0;
  int max_slots = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread engine;

  // engine-owned
  std::vector<Slot> slots;
  size_t used = 0;
  ttc_batch* batch = nullptr;
  bool batch_stale = true;

  // statistics (under mu)
  std::vector<double> latencies;
  long long completed = 0, failed = 0;
  double entry_iters = 0.0;   // sum over iterations of |Omega| of the stepped slots
  long long iterations = 0;
  long long launches = 0;     // kernels launched by the engine's ticks
  double busy_ms = 0.0;
  long long rebuilds = 0;     // batch (re)captures
  double rebuild_ms = 0.0;    // engine time spent in them
  double admit_ms = 0.0;      // engine time spent admitting requests
  Clock::time_point t0;
};

namespace {

// Device bytes a request will hold: per-mode layout copies of Omega, the
// residual, chunk partials, cores (master, padded mirrors, C, previous,
// scatter), and the interface tables (bounded by 2^17 rows per table).
size_t estimate_bytes(const Request& q) {
  const int m = q.d;
  int bits = 0;
  int rmax = 1;
  for (int k = 0; k <= m; ++k) rmax = std::max(rmax, (int)q.r[k]);
  int R = rmax <= 4 ? 4 : rmax <= 8 ? 8 : rmax <= 16 ? 16 : 32;
  for (int k = 0; k < m; ++k) {
    int b = 0;
    while ((1LL << b) < q.n[k]) ++b;
    bits += b;
  }
  size_t W = (size_t)std::max(1, (bits + 31) / 32);
  if (W == 3) W = 4;
  size_t N = (size_t)q.N;
  size_t bytes = (size_t)m * N * (4 * W + 4 + 8 + 4) + N * 8;
  size_t chunks = 0;
  for (int k = 0; k < m; ++k) chunks += N / 1024 + (size_t)q.n[k];
  bytes += chunks * (size_t)(1 + rmax * rmax) * 8;
  for (int k = 0; k < m; ++k) {
    size_t nk = (size_t)q.n[k];
    bytes += nk * (size_t)q.r[k] * q.r[k + 1] * 8 * 3;   // master, previous, scatter
    bytes += nk * (size_t)R * R * 12;                   // padded mirrors
    bytes += nk * (size_t)(2 * q.r[k]) * (2 * q.r[k + 1]) * 8;   // rank-2r cores
    bytes += nk * 8 * 2;
  }
  bytes += (size_t)2 * m * (1 << 17) * R * 12 / 4;   // tables (typical bound)
  bytes += (size_t)64 << 20;                          // reduction partials and small matrices
  return bytes;
}

void finish(ttc_server* S, Slot& sl, int status) {
  Request& q = *sl.req;
  q.status = status;
  q.info = sl.st.info;
  if (status == TTC_ECUDA) snprintf(q.detail, sizeof(q.detail), "%s", ttc_last_cuda_error());
  if (sl.ctx && (status == TTC_OK || status == TTC_ENOTCONV)) {
    q.cores.assign(q.d, {});
    std::vector<double*> ptrs(q.d);
    for (int k = 0; k < q.d; ++k) {
      q.cores[k].resize((size_t)q.r[k] * q.n[k] * q.r[k + 1]);
      ptrs[k] = q.cores[k].data();
    }
    int s = ttc_get_cores(sl.ctx, ptrs.data());
    if (s != TTC_OK && q.status == TTC_OK) q.status = s;
  }
  if (sl.ctx) ttc_destroy(sl.ctx);
  sl.ctx = nullptr;
  q.t_done = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  q.done = true;
  S->used -= sl.bytes;
  if (q.status == TTC_OK || q.status == TTC_ENOTCONV) {
    S->completed += 1;
    S->latencies.push_back(ms_between(q.t_submit, q.t_done));
  } else {
    S->failed += 1;
  }
  S->cv_done.notify_all();
}

int admit(ttc_server* S, std::shared_ptr<Request> rq, Slot& sl) {
  Request& q = *rq;
  sl.req = rq;
  sl.bytes = q.est_bytes;
  q.t_admit = Clock::now();
  int s = ttc_create(&sl.ctx, q.d, q.n.data(), q.r.data(), &q.opt, nullptr);
  if (s == TTC_OK) s = ttc_set_observations(sl.ctx, q.N, q.idx.data(), q.y.data());
  if (s == TTC_OK) {
    std::vector<const double*> p(q.d);
    for (int k = 0; k < q.d; ++k) p[k] = q.init[k].data();
    s = ttc_set_cores(sl.ctx, p.data());
  }
  if (s == TTC_OK && !q.truth.empty()) {
    std::vector<const double*> p(q.d);
    for (int k = 0; k < q.d; ++k) p[k] = q.truth[k].data();
    s = ttc_set_truth(sl.ctx, q.truth_r.data(), p.data());
  }
  if (s == TTC_OK && q.opt.stop_rule == TTC_STOP_RELERR && q.truth.empty()) s = TTC_EINVAL;
  if (s == TTC_OK) {
    ttc_solve_begin(sl.ctx, sl.st);
    // the step-size override is off for served requests
    double zero = 0.0;
    cudaError_t e = cudaMemcpy(sl.ctx->hp.scal + SC_ALPHA_OVR, &zero, sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      ttc_record_cuda_error(e);
      s = TTC_ECUDA;
    }
  }
  if (s == TTC_OK) {
    // account what the context really holds
    std::lock_guard<std::mutex> lk(S->mu);
    S->used = S->used - sl.bytes + sl.ctx->device_bytes;
    sl.bytes = sl.ctx->device_bytes;
  }
  return s;
}

void engine_loop(ttc_server* S) {
  cudaSetDevice(S->device);
  while (true) {
    // admission
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->slots.empty())
        S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->stop && S->slots.empty() && S->queue.empty()) break;
    }
    while (true) {
      std::shared_ptr<Request> rq;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.empty() || (int)S->slots.size() >= S->max_slots) break;
        auto& front = S->queue.front();
        if (!S->slots.empty() && S->used + front->est_bytes > S->budget) break;   // wait for memory
        rq = front;
        S->queue.pop_front();
        S->used += rq->est_bytes;
      }
      Slot sl;
      const auto ta = Clock::now();
      int s = admit(S, rq, sl);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->admit_ms += ms_between(ta, Clock::now());
      }
      if (s != TTC_OK) {
        finish(S, sl, s);
        continue;
      }
      S->slots.push_back(std::move(sl));
      S->batch_stale = true;
    }
    if (S->slots.empty()) continue;
    // one iteration of every active slot
    auto t0 = Clock::now();
    if (S->batch_stale) {
      if (S->batch) ttc_batch_destroy(S->batch);
      S->batch = nullptr;
      std::vector<ttc_ctx*> members;
      for (auto& sl : S->slots) members.push_back(sl.ctx);
      const auto tb = Clock::now();
      int s = ttc_batch_create(&S->batch, members.data(), (int)members.size(), S->stream);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->rebuilds += 1;
        S->rebuild_ms += ms_between(tb, Clock::now());
      }
      if (s != TTC_OK) {
        for (auto& sl : S->slots) finish(S, sl, s);
        S->slots.clear();
        continue;
      }
      S->batch_stale = false;
    }
    int64_t k0 = 0, k1 = 0;
    ttc_batch_launch_count(S->batch, &k0);
    int s = ttc_batch_step(S->batch);
    ttc_batch_launch_count(S->batch, &k1);
    long long tick_launches = (long long)(k1 - k0);
    double entries = 0.0;
    for (auto& sl : S->slots) {
      ++sl.st.it;
      entries += (double)sl.ctx->N;
    }
    // stop rules: metrics where needed, then all scalars
    std::vector<bool> metric(S->slots.size(), false);
    for (size_t i = 0; i < S->slots.size() && s == TTC_OK; ++i) {
      ttc_ctx* c = S->slots[i].ctx;
      if (ttc_solve_needs_metric(c, S->slots[i].st.it)) {
        cudaStream_t saved = c->stream;
        c->stream = S->stream;   // after the batch's work
        const long long n0 = c->nlaunch;
        s = ttc_launch_metric(c, c->opt.stop_rule == TTC_STOP_RELERR ? 0 : 1);
        tick_launches += c->nlaunch - n0;
        c->stream = saved;
        metric[i] = true;
      }
    }
    std::vector<double> sc(S->slots.size() * SC_COUNT);
    for (size_t i = 0; i < S->slots.size() && s == TTC_OK; ++i) {
      cudaError_t e = cudaMemcpyAsync(&sc[i * SC_COUNT], S->slots[i].ctx->hp.scal, sizeof(double) * SC_COUNT,
                                      cudaMemcpyDeviceToHost, S->stream);
      if (e != cudaSuccess) {
        ttc_record_cuda_error(e);
        s = TTC_ECUDA;
      }
    }
    if (s == TTC_OK) {
      cudaError_t e = cudaStreamSynchronize(S->stream);
      if (e != cudaSuccess) {
        ttc_record_cuda_error(e);
        s = TTC_ECUDA;
      }
    }
    auto t1 = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->busy_ms += ms_between(t0, t1);
      S->entry_iters += entries;
      S->iterations += (long long)S->slots.size();
      S->launches += tick_launches;
    }
    if (s != TTC_OK) {
      for (auto& sl : S->slots) finish(S, sl, s);
      S->slots.clear();
      S->batch_stale = true;
      continue;
    }
    std::vector<Slot> keep;
    for (size_t i = 0; i < S->slots.size(); ++i) {
      Slot& sl = S->slots[i];
      const int prec_before = sl.ctx->cur_prec;
      ttc_solve_after(sl.ctx, sl.st, &sc[i * SC_COUNT], metric[i]);
      if (sl.st.done) {
        finish(S, sl, sl.st.status);
        S->batch_stale = true;
      } else {
        if (sl.ctx->cur_prec != prec_before) S->batch_stale = true;
        keep.push_back(std::move(sl));
      }
    }
    S->slots.swap(keep);
  }
  if (S->batch) ttc_batch_destroy(S->batch);
  S->batch = nullptr;
}

}  // namespace

extern "C" {

int ttc_server_create(ttc_server** out, size_t device_mem_budget, int max_slots, void* cuda_stream) {
  if (!out || max_slots < 1) return TTC_EINVAL;
  *out = nullptr;
  ttc_server* S = new (std::nothrow) ttc_server();
  if (!S) return TTC_ENOMEM;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess && device_mem_budget == 0) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    device_mem_budget = (size_t)(0.8 * (double)fr);
  }
  if (e == cudaSuccess) {
    if (cuda_stream) {
      S->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
      S->own_stream = (e == cudaSuccess);
    }
  }
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    delete S;
    return TTC_ECUDA;
  }
  S->budget = device_mem_budget;
  S->max_slots = max_slots;
  S->t0 = Clock::now();
  S->engine = std::thread(engine_loop, S);
  *out = S;
  return TTC_OK;
}

int ttc_submit(ttc_server* S, const ttc_request* rq, uint64_t* ticket) {
  if (!S || !rq || !ticket) return TTC_EINVAL;
  const int d = rq->d;
  if (d < 2 || !rq->n || !rq->r || !rq->idx || !rq->y || !rq->init || rq->N < 1) return TTC_EINVAL;
  if (d > TTC_MAXM) return TTC_EUNSUPPORTED;
  auto q = std::make_shared<Request>();
  q->d = d;
  q->n.assign(rq->n, rq->n + d);
  q->r.assign(rq->r, rq->r + d + 1);
  for (int k = 0; k < d; ++k)
    if (q->n[k] < 1) return TTC_EINVAL;
  for (int k = 0; k <= d; ++k)
    if (q->r[k] < 1 || q->r[k] > TTC_MAXR) return TTC_EUNSUPPORTED;
  if (q->r[0] != 1 || q->r[d] != 1) return TTC_EINVAL;
  q->N = rq->N;
  q->idx.assign(rq->idx, rq->idx + (size_t)rq->N * d);
  q->y.assign(rq->y, rq->y + rq->N);
  q->init.resize(d);
  for (int k = 0; k < d; ++k) {
    if (!rq->init[k]) return TTC_EINVAL;
    q->init[k].assign(rq->init[k], rq->init[k] + (size_t)q->r[k] * q->n[k] * q->r[k + 1]);
  }
  if (rq->truth && rq->truth_r) {
    q->truth_r.assign(rq->truth_r, rq->truth_r + d + 1);
    q->truth.resize(d);
    for (int k = 0; k < d; ++k)
      q->truth[k].assign(rq->truth[k], rq->truth[k] + (size_t)q->truth_r[k] * q->n[k] * q->truth_r[k + 1]);
  }
  if (rq->opt) {
    q->opt = *rq->opt;
  } else {
    ttc_default_options(&q->opt);
    q->opt.stop_rule = TTC_STOP_RESID;
  }
  q->est_bytes = estimate_bytes(*q);
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return TTC_EBUSY;
    if (q->est_bytes > S->budget) return TTC_ENOMEM;   // could never be admitted
    q->ticket = S->next_ticket++;
    S->all[q->ticket] = q;
    S->queue.push_back(q);
    *ticket = q->ticket;
  }
  S->cv_work.notify_all();
  return TTC_OK;
}

int ttc_poll(ttc_server* S, uint64_t ticket, int64_t timeout_us, ttc_result* out, double* const* cores_out) {
  if (!S) return TTC_EINVAL;
  std::shared_ptr<Request> q;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return TTC_EINVAL;
    q = it->second;
    auto ready = [&] { return q->done; };
    if (timeout_us < 0) {
      S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
      return TTC_ETIMEOUT;
    }
    S->all.erase(ticket);
  }
  if (out) {
    out->status = q->status;
    out->iters = q->info.iters;
    out->converged = q->info.converged;
    out->last_metric = q->info.last_metric;
    out->res_norm = q->info.res_norm;
    out->latency_ms = ms_between(q->t_submit, q->t_done);
    out->queue_ms = ms_between(q->t_submit, q->t_admit);
    memcpy(out->detail, q->detail, sizeof(out->detail));
  }
  if (cores_out && !q->cores.empty())
    for (int k = 0; k < q->d; ++k)
      if (cores_out[k]) memcpy(cores_out[k], q->cores[k].data(), sizeof(double) * q->cores[k].size());
  return TTC_OK;
}

int ttc_server_stats(ttc_server* S, ttc_serving_stats* out) {
  if (!S || !out) return TTC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = (int64_t)S->queue.size();
  out->iterations = S->iterations;
  out->launches = S->launches;
  out->entry_iterations = S->entry_iters;
  out->busy_ms = S->busy_ms;
  out->rebuilds = S->rebuilds;
  out->rebuild_ms = S->rebuild_ms;
  out->admit_ms = S->admit_ms;
  out->wall_ms = ms_between(S->t0, Clock::now());
  out->p50_ms = out->p99_ms = out->max_ms = 0.0;
  if (!S->latencies.empty()) {
    std::vector<double> v = S->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      size_t i = (size_t)std::ceil(p * (double)v.size()) - 1;
      return v[std::min(i, v.size() - 1)];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
  }
  return TTC_OK;
}

void ttc_server_destroy(ttc_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->engine.joinable()) S->engine.join();
  for (auto& sl : S->slots)
    if (sl.ctx) ttc_destroy(sl.ctx);
  if (S->own_stream && S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
