// C ABI of the ttc library (declared in include/ttc.h): context lifetime,
// host<->device copies, one PRGD iteration (Algorithm 2) as a fixed launch
// sequence captured once into a CUDA graph per precision, the solver loop
// and read-back of intermediate results.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.h"

static thread_local char g_last_cuda_error[256] = "";

void ttc_record_cuda_error(cudaError_t e) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

int ttc_fork_create(PassFork& f) {
  for (int i = 0; i < 2; ++i) {
    TTC_CUDA(cudaStreamCreateWithFlags(&f.aux[i], cudaStreamNonBlocking));
    TTC_CUDA(cudaEventCreateWithFlags(&f.join[i], cudaEventDisableTiming));
  }
  TTC_CUDA(cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming));
  return TTC_OK;
}

void ttc_fork_destroy(PassFork& f) {
  for (int i = 0; i < 2; ++i) {
    if (f.aux[i]) cudaStreamDestroy(f.aux[i]);
    if (f.join[i]) cudaEventDestroy(f.join[i]);
    f.aux[i] = nullptr;
    f.join[i] = nullptr;
  }
  if (f.fork) cudaEventDestroy(f.fork);
  f.fork = nullptr;
}

// The library's device memory pool (one per device): stream-ordered
// allocations that stay cached after they are freed (release threshold at
// its maximum), so contexts and layouts built again and again (serving,
// end-to-end solves) neither map nor unmap memory nor synchronise the device.
cudaMemPool_t ttc_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

cudaError_t ttc_pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = ttc_pool();
  if (!pool) return cudaMalloc(p, bytes);
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void ttc_pool_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

int ttc_alloc(ttc_ctx* c, void** p, size_t bytes, bool obs) {
  void* q = nullptr;
  cudaError_t e = ttc_pool_alloc(&q, bytes ? bytes : 16, c->stream);
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TTC_ENOMEM : TTC_ECUDA;
  }
  DevBuf b;
  b.p = q;
  b.bytes = bytes;
  (obs ? c->obs_bufs : c->bufs).push_back(b);
  c->device_bytes += bytes;
  *p = q;
  return TTC_OK;
}

void ttc_free_obs(ttc_ctx* c) {
  for (auto& b : c->obs_bufs) {
    ttc_pool_free(b.p, c->stream);
    c->device_bytes -= b.bytes;
  }
  c->obs_bufs.clear();
}

int ttc_upload_desc(ttc_ctx* c) {
  (void)c;
  return TTC_OK;
}

namespace {

int drop_graphs(ttc_ctx* c) {
  for (int i = 0; i < 2; ++i)
    if (c->graph[i]) {
      cudaGraphExecDestroy(c->graph[i]);
      c->graph[i] = nullptr;
    }
  c->graph_dirty = true;
  return TTC_OK;
}

// the fixed launch sequence of one iteration
int enqueue_iteration(ttc_ctx* c, int prec) {
  c->hp.step_fp64 = (prec == TTC_PREC_FP64) ? 1 : 0;
  c->hp.dense_ff = ttc_dense_ff(c->opt.dense_mode, prec);
  TTC_TRY(ttc_launch_omega_pass(c, prec));
  TTC_TRY(ttc_launch_save_prev(c));   // also the slice weights, which need this step's eps
  TTC_TRY(ttc_launch_dense(c));
  return TTC_OK;
}

int build_graph(ttc_ctx* c, int slot, int prec) {
  cudaGraph_t g = nullptr;
  long long before = c->nlaunch;
  TTC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int s = enqueue_iteration(c, prec);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->graph_kernels[slot] = c->nlaunch - before;   // kernels per replay
  c->nlaunch = before;                             // nothing ran yet
  if (s != TTC_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    return TTC_ECUDA;
  }
  e = cudaGraphInstantiate(&c->graph[slot], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    return TTC_ECUDA;
  }
  return TTC_OK;
}

int set_scalar(ttc_ctx* c, int idx, double v) {
  TTC_CUDA(cudaMemcpyAsync(c->hp.scal + idx, &v, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  return TTC_OK;
}

int read_scalars(ttc_ctx* c, double* out) {
  TTC_CUDA(cudaMemcpyAsync(out, c->hp.scal, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, c->stream));
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  return TTC_OK;
}

int run_iteration(ttc_ctx* c, int prec) {
  const int slot = (prec == TTC_PREC_FP64) ? 1 : 0;
  if (!c->opt.use_graph) {
    TTC_TRY(enqueue_iteration(c, prec));
  } else {
    if (c->graph_dirty) {
      drop_graphs(c);
      c->graph_dirty = false;
    }
    if (!c->graph[slot]) TTC_TRY(build_graph(c, slot, prec));
    TTC_CUDA(cudaGraphLaunch(c->graph[slot], c->stream));
    c->nlaunch += c->graph_kernels[slot];
  }
  if (c->prof) {
    // the Omega pass of this iteration was bracketed by ev_beg / ev_end
    TTC_CUDA(cudaEventSynchronize(c->ev_end));
    float t = 0.f;
    TTC_CUDA(cudaEventElapsedTime(&t, c->ev_beg, c->ev_end));
    c->prof_ms += t;
    c->prof_count += 1;
  }
  return TTC_OK;
}

void host_to_slice_major(const double* src, double* dst, int ra, int n, int rb) {
  // src (ra, n, rb) -> dst (n, ra, rb)
  for (int a = 0; a < ra; ++a)
    for (int x = 0; x < n; ++x)
      for (int b = 0; b < rb; ++b) dst[((size_t)x * ra + a) * rb + b] = src[((size_t)a * n + x) * rb + b];
}

void slice_major_to_host(const double* src, double* dst, int ra, int n, int rb) {
  for (int a = 0; a < ra; ++a)
    for (int x = 0; x < n; ++x)
      for (int b = 0; b < rb; ++b) dst[((size_t)a * n + x) * rb + b] = src[((size_t)x * ra + a) * rb + b];
}

}  // namespace

extern "C" {

void ttc_default_options(ttc_options* o) {
  if (!o) return;
  o->precision = TTC_PREC_MIXED;
  o->eps_rel = 1.0;
  o->alpha_scale = 1.5;
  o->eps_frozen = 0;
  o->tol = 1e-6;
  o->max_iter = 500;
  o->stop_rule = TTC_STOP_RELERR;
  o->check_every = 1;
  o->polish_below = 1e-5;
  o->polish_factor = 10.0;
  o->step_fallback = 1;
  o->dense_mode = TTC_DENSE_AUTO;
  o->use_graph = 1;
  o->step_rule = TTC_STEP_CONSTANT;
  o->metric = TTC_METRIC_PRECOND;
  o->retraction = TTC_RETRACT_PLAIN;
}

const char* ttc_strerror(int s) {
  switch (s) {
    case TTC_OK: return "ok";
    case TTC_EINVAL: return "invalid argument";
    case TTC_ENOMEM: return "out of memory";
    case TTC_ERANGE: return "index coordinate out of range";
    case TTC_EDUP: return "duplicate index in Omega";
    case TTC_ENONFINITE: return "non-finite value";
    case TTC_ENOTCONV: return "not converged";
    case TTC_ETIMEOUT: return "timeout";
    case TTC_ECUDA: return "CUDA error";
    case TTC_EBUSY: return "busy";
    case TTC_EUNSUPPORTED: return "unsupported shape";
    default: return "unknown status";
  }
}

const char* ttc_last_cuda_error(void) { return g_last_cuda_error; }

int ttc_create(ttc_ctx** out, int d, const int64_t* n, const int32_t* r, const ttc_options* opt, void* cuda_stream) {
  if (!out || !n || !r) return TTC_EINVAL;
  *out = nullptr;
  if (d < 2) return TTC_EINVAL;
  if (d > TTC_MAXM) return TTC_EUNSUPPORTED;
  if (r[0] != 1 || r[d] != 1) return TTC_EINVAL;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1) return TTC_EINVAL;
    if (n[k] > (1LL << 30)) return TTC_EUNSUPPORTED;
  }
  int rmax = 1;
  for (int k = 0; k <= d; ++k) {
    if (r[k] < 1) return TTC_EINVAL;
    if (r[k] > TTC_MAXR) return TTC_EUNSUPPORTED;
    rmax = r[k] > rmax ? r[k] : rmax;
  }
  // a TT-rank is at most both dimensions of its unfolding (n_1..n_k rows,
  // n_{k+1}..n_d columns): no tensor has a larger one, so the manifold of
  // that rank is empty (products saturate above the largest rank)
  for (int k = 1; k < d; ++k) {
    long long left = 1, right = 1;
    for (int j = 0; j < k; ++j) left = std::min<long long>(left * n[j], 1 << 20);
    for (int j = k; j < d; ++j) right = std::min<long long>(right * n[j], 1 << 20);
    if (r[k] > left || r[k] > right) return TTC_EINVAL;
  }
  ttc_ctx* c = new (std::nothrow) ttc_ctx();
  if (!c) return TTC_ENOMEM;
  ttc_default_options(&c->opt);
  if (opt) c->opt = *opt;
  if (c->opt.check_every < 1) c->opt.check_every = 1;
  c->m = d;
  for (int k = 0; k < d; ++k) c->n[k] = n[k];
  for (int k = 0; k <= d; ++k) c->r[k] = r[k];
  c->rank_bucket = rmax <= 4 ? 4 : rmax <= 8 ? 8 : rmax <= 16 ? 16 : 32;
  c->rank_max = rmax;
  memset(&c->hp, 0, sizeof(DevProb));
  DevProb& P = c->hp;
  P.m = d;
  double dstar = 1.0;
  long long dl = 1;
  bool ovf = false;
  long long minn = n[0];
  for (int k = 0; k < d; ++k) {
    P.n[k] = (int)n[k];
    dstar *= (double)n[k];
    if (!ovf && dl > (1LL << 62) / n[k]) ovf = true;
    if (!ovf) dl *= n[k];
    if (n[k] < minn) minn = n[k];
  }
  for (int k = 0; k <= d; ++k) P.r[k] = r[k];
  P.R = c->rank_bucket;
  P.dstar = ovf ? 0 : dl;
  P.inv_min_n = 1.0 / (double)minn;
  P.inv_2m = 1.0 / (2.0 * (double)d);
  if (c->opt.step_rule < 0 || c->opt.step_rule > 1 || c->opt.metric < 0 || c->opt.metric > 1 ||
      c->opt.retraction < 0 || c->opt.retraction > 1 || c->opt.precision < 0 || c->opt.precision > 2 ||
      c->opt.dense_mode < 0 || c->opt.dense_mode > 2) {
    delete c;
    return TTC_EINVAL;
  }
  P.steepest = c->opt.step_rule == TTC_STEP_STEEPEST;
  P.uniform = c->opt.metric == TTC_METRIC_UNIFORM;
  P.weighted_retraction = c->opt.retraction == TTC_RETRACT_WEIGHTED;
  (void)dstar;
  int s = TTC_OK;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ttc_record_cuda_error(e);
      delete c;
      return TTC_ECUDA;
    }
    c->own_stream = true;
  }
  for (int k = 0; k < d && s == TTC_OK; ++k) {
    size_t cnt = (size_t)n[k] * r[k] * r[k + 1];
    if ((s = ttc_alloc(c, (void**)&P.core64[k], sizeof(double) * cnt, false)) != TTC_OK) break;
    size_t padcnt = (size_t)n[k] * c->rank_bucket * c->rank_bucket;
    if ((s = ttc_alloc(c, (void**)&P.core32p[k], sizeof(float) * padcnt, false)) != TTC_OK) break;
    if ((s = ttc_alloc(c, (void**)&P.core64p[k], sizeof(double) * padcnt, false)) != TTC_OK) break;
    cudaMemsetAsync(P.core32p[k], 0, sizeof(float) * padcnt, c->stream);
    cudaMemsetAsync(P.core64p[k], 0, sizeof(double) * padcnt, c->stream);
    if ((s = ttc_alloc(c, (void**)&P.s[k], sizeof(double) * (size_t)n[k], false)) != TTC_OK) break;
    if ((s = ttc_alloc(c, (void**)&P.wt[k], sizeof(double) * 2 * (size_t)n[k], false)) != TTC_OK) break;
    if ((s = ttc_alloc(c, (void**)&P.E[k], sizeof(double) * cnt, false)) != TTC_OK) break;
  }
  if (s == TTC_OK) s = ttc_fork_create(c->fork);
  if (s == TTC_OK) s = ttc_prepare_omega_pass();
  if (s == TTC_OK) s = ttc_alloc_dense(c);
  if (s == TTC_OK) {
    double v[2] = {c->opt.eps_rel, c->opt.alpha_scale};
    cudaError_t e = cudaMemcpyAsync(P.scal + SC_EPS_REL, v, sizeof(v), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // allocations ready for every stream
    if (e != cudaSuccess) {
      ttc_record_cuda_error(e);
      s = TTC_ECUDA;
    }
  }
  if (s != TTC_OK) {
    ttc_destroy(c);
    return s;
  }
  c->cur_prec = (c->opt.precision == TTC_PREC_FP64) ? TTC_PREC_FP64 : TTC_PREC_FP32;
  *out = c;
  return TTC_OK;
}

void ttc_destroy(ttc_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->ev_beg) cudaEventDestroy(c->ev_beg);
  if (c->ev_end) cudaEventDestroy(c->ev_end);
  ttc_fork_destroy(c->fork);
  ttc_free_obs(c);
  for (auto& b : c->bufs) ttc_pool_free(b.p, c->stream);
  c->bufs.clear();
  cudaStreamSynchronize(c->stream);
  ttc_free_plan(c);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int ttc_set_observations(ttc_ctx* c, int64_t N, const int32_t* idx, const double* y) {
  if (!c || !idx || !y || N < 1) return TTC_EINVAL;
  if (N >= (1LL << 31) - TTC_CHUNK) return TTC_EUNSUPPORTED;
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  ttc_free_obs(c);
  c->have_obs = false;
  c->N = (int)N;
  DevProb& P = c->hp;
  double dstar = 1.0;
  for (int k = 0; k < c->m; ++k) dstar *= (double)c->n[k];
  P.p = (double)N / dstar;
  int s = ttc_build_layout(c, idx, y);
  if (s != TTC_OK) return s;
  {   // ||y||^2 with four interleaved partial sums (a shorter add chain)
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t e = 0;
    for (; e + 3 < N; e += 4) {
      a0 += y[e] * y[e];
      a1 += y[e + 1] * y[e + 1];
      a2 += y[e + 2] * y[e + 2];
      a3 += y[e + 3] * y[e + 3];
    }
    for (; e < N; ++e) a0 += y[e] * y[e];
    c->ynorm2 = (a0 + a1) + (a2 + a3);
  }
  ttc_plan_tables(c);
  P.tab32 = nullptr;
  P.tab64 = nullptr;
  P.ztab32 = nullptr;
  P.ztab64 = nullptr;
  if (P.tab_total > 0) {
    size_t cnt = (size_t)P.tab_total * c->rank_bucket;
    TTC_TRY(ttc_alloc(c, (void**)&P.tab32, sizeof(float) * cnt, true));
    TTC_TRY(ttc_alloc(c, (void**)&P.tab64, sizeof(double) * cnt, true));
    TTC_TRY(ttc_alloc(c, (void**)&P.ztab32, sizeof(float) * cnt, true));
    TTC_TRY(ttc_alloc(c, (void**)&P.ztab64, sizeof(double) * cnt, true));
    // rows whose coordinates lie outside the mode sizes stand for no entry:
    // zero once here, never written by the per-step builds
    TTC_CUDA(cudaMemsetAsync(P.tab32, 0, sizeof(float) * cnt, c->stream));
    TTC_CUDA(cudaMemsetAsync(P.tab64, 0, sizeof(double) * cnt, c->stream));
    TTC_CUDA(cudaMemsetAsync(P.ztab32, 0, sizeof(float) * cnt, c->stream));
    TTC_CUDA(cudaMemsetAsync(P.ztab64, 0, sizeof(double) * cnt, c->stream));
  }
  c->have_obs = true;
  c->eps_set = false;
  TTC_TRY(set_scalar(c, SC_EPS_FIXED, 0.0));
  return TTC_OK;
}

int ttc_set_cores(ttc_ctx* c, const double* const* cores) {
  if (!c || !cores) return TTC_EINVAL;
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<double> tmp;
  for (int k = 0; k < c->m; ++k) {
    if (!cores[k]) return TTC_EINVAL;
    size_t cnt = (size_t)c->n[k] * c->r[k] * c->r[k + 1];
    tmp.resize(cnt);
    host_to_slice_major(cores[k], tmp.data(), c->r[k], (int)c->n[k], c->r[k + 1]);
    for (size_t i = 0; i < cnt; ++i)
      if (!std::isfinite(tmp[i])) return TTC_ENONFINITE;
    TTC_CUDA(cudaMemcpy(c->hp.core64[k], tmp.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice));
  }
  TTC_TRY(ttc_launch_mirror32(c));
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  c->have_cores = true;
  return TTC_OK;
}

int ttc_get_cores(ttc_ctx* c, double* const* cores_out) {
  if (!c || !cores_out) return TTC_EINVAL;
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<double> tmp;
  for (int k = 0; k < c->m; ++k) {
    if (!cores_out[k]) return TTC_EINVAL;
    size_t cnt = (size_t)c->n[k] * c->r[k] * c->r[k + 1];
    tmp.resize(cnt);
    TTC_CUDA(cudaMemcpy(tmp.data(), c->hp.core64[k], sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    slice_major_to_host(tmp.data(), cores_out[k], c->r[k], (int)c->n[k], c->r[k + 1]);
  }
  return TTC_OK;
}

int ttc_set_truth(ttc_ctx* c, const int32_t* rt, const double* const* cores) {
  if (!c || !rt || !cores) return TTC_EINVAL;
  if (rt[0] != 1 || rt[c->m] != 1) return TTC_EINVAL;
  for (int k = 0; k <= c->m; ++k) {
    if (rt[k] < 1) return TTC_EINVAL;
    if (rt[k] > TTC_MAXR) return TTC_EUNSUPPORTED;
  }
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  DevProb& P = c->hp;
  std::vector<double> tmp;
  for (int k = 0; k < c->m; ++k) {
    size_t cnt = (size_t)c->n[k] * rt[k] * rt[k + 1];
    if (!P.has_truth || P.rt[k] != rt[k] || P.rt[k + 1] != rt[k + 1]) {
      double* p = nullptr;
      TTC_TRY(ttc_alloc(c, (void**)&p, sizeof(double) * cnt, false));
      P.truth[k] = p;
    }
    tmp.resize(cnt);
    host_to_slice_major(cores[k], tmp.data(), rt[k], (int)c->n[k], rt[k + 1]);
    TTC_CUDA(cudaMemcpy(P.truth[k], tmp.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice));
  }
  for (int k = 0; k <= c->m; ++k) P.rt[k] = rt[k];
  P.has_truth = 1;
  drop_graphs(c);
  return TTC_OK;
}

static int step_impl(ttc_ctx* c, double alpha, ttc_step_info* out, bool sync_info) {
  if (!c->have_obs || !c->have_cores) return TTC_EINVAL;
  (void)alpha;   // the step-size override lives in device memory (SC_ALPHA_OVR)
  int prec = c->cur_prec;
  TTC_TRY(run_iteration(c, prec));
  ++c->iter;
  if (c->opt.eps_frozen && !c->eps_set) {
    TTC_CUDA(cudaMemcpyAsync(c->hp.scal + SC_EPS_FIXED, c->hp.scal + SC_EPS, sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
    c->eps_set = true;
  }
  if (sync_info || out) {
    double sc[SC_COUNT];
    TTC_TRY(read_scalars(c, sc));
    unsigned flags;
    memcpy(&flags, &sc[SC_FLAGS], sizeof(flags));
    if (out) {
      out->eps = sc[SC_EPS];
      out->alpha = sc[SC_ALPHA];
      out->res_norm = std::sqrt(sc[SC_G2]);
      out->precision_used = prec;
      out->subspace_iters = (int)sc[SC_SUBIT];
    }
    if (flags & 1) return TTC_ENONFINITE;
  }
  return TTC_OK;
}

int ttc_step(ttc_ctx* c, double alpha, ttc_step_info* out) {
  if (!c) return TTC_EINVAL;
  double a = alpha > 0.0 ? alpha : 0.0;
  if (a != c->alpha_ovr) {
    TTC_TRY(set_scalar(c, SC_ALPHA_OVR, a));
    c->alpha_ovr = a;
  }
  return step_impl(c, alpha, out, out != nullptr);
}

}  // extern "C"

void ttc_solve_begin(ttc_ctx* c, SolveState& st) {
  st.it = 0;
  st.status = TTC_ENOTCONV;
  st.done = false;
  st.info.iters = 0;
  st.info.converged = 0;
  st.info.last_metric = -1.0;
  st.info.res_norm = -1.0;
  st.info.polish_iter = -1;
  st.info.fallback_iter = -1;
  st.prev_res = -1.0;
  // every solve starts with the configured step rule (a previous solve may have fallen back)
  const int steep = c->opt.step_rule == TTC_STEP_STEEPEST ? 1 : 0;
  if (c->hp.steepest != steep) {
    c->hp.steepest = steep;
    c->graph_dirty = true;
  }
  if (c->opt.precision == TTC_PREC_FP64) c->cur_prec = TTC_PREC_FP64;
  if (c->opt.precision == TTC_PREC_FP32 || c->opt.precision == TTC_PREC_MIXED) c->cur_prec = TTC_PREC_FP32;
}

bool ttc_solve_needs_metric(const ttc_ctx* c, int it) {
  const bool check = (it % c->opt.check_every == 0) || it == c->opt.max_iter;
  return check && (c->opt.stop_rule == TTC_STOP_RELERR || c->opt.stop_rule == TTC_STOP_STEP);
}

int ttc_read_scalars(ttc_ctx* c, double* out) { return read_scalars(c, out); }

void ttc_solve_after(ttc_ctx* c, SolveState& st, const double* sc, bool checked) {
  st.info.iters = st.it;
  unsigned flags;
  memcpy(&flags, &sc[SC_FLAGS], sizeof(flags));
  if (flags & 1u) {
    st.status = TTC_ENONFINITE;
    st.done = true;
    return;
  }
  st.info.res_norm = std::sqrt(sc[SC_G2]);
  const double rel_res = std::sqrt(sc[SC_G2] / std::fmax(c->ynorm2, 1e-300));
  if (!std::isfinite(rel_res)) {
    st.status = TTC_ENONFINITE;
    st.done = true;
    return;
  }
  // a constant step whose scale diverges on this problem shows as a growing
  // residual: the remaining iterations take the steepest step (the exact line
  // search of Eq. (PRGD stepsize)), which cannot increase f along the
  // projected direction
  if (c->opt.step_fallback && !c->hp.steepest && st.prev_res > 0.0 && rel_res > 2.0 * st.prev_res) {
    c->hp.steepest = 1;
    c->graph_dirty = true;
    st.info.fallback_iter = st.it + 1;
  }
  st.prev_res = rel_res;
  if (checked && (c->opt.stop_rule == TTC_STOP_RELERR || c->opt.stop_rule == TTC_STOP_STEP) &&
      !(std::isfinite(sc[SC_METRIC]) && std::isfinite(sc[SC_NORM]))) {
    // the new iterate is not finite: never read that as convergence
    st.status = TTC_ENONFINITE;
    st.done = true;
    return;
  }
  double metric = -1.0;
  if (c->opt.stop_rule == TTC_STOP_RESID) {
    metric = rel_res;
  } else if (checked && c->opt.stop_rule == TTC_STOP_RELERR) {
    metric = std::sqrt(std::fmax(sc[SC_METRIC], 0.0) / sc[SC_NORM]);
  } else if (checked && c->opt.stop_rule == TTC_STOP_STEP) {
    // ||T_{l+1} - T_l|| <= tol max(1, ||T_l||): SC_NORM holds ||T_l||^2
    metric = std::sqrt(std::fmax(sc[SC_METRIC], 0.0)) / std::fmax(1.0, std::sqrt(sc[SC_NORM]));
  }
  if (metric >= 0.0) st.info.last_metric = metric;
  // MIXED: the pass switches to FP64 once the relative residual is small
  // (noiseless data) or the stop metric is within polish_factor of its
  // tolerance (near convergence; with noisy data the residual stays at the
  // noise level and only this second test fires)
  if (c->opt.precision == TTC_PREC_MIXED && c->cur_prec != TTC_PREC_FP64 &&
      (rel_res <= c->opt.polish_below || (metric >= 0.0 && metric <= c->opt.polish_factor * c->opt.tol))) {
    c->cur_prec = TTC_PREC_FP64;
    st.info.polish_iter = st.it + 1;
  }
  const bool polishing_done = (c->opt.precision != TTC_PREC_MIXED) || c->cur_prec == TTC_PREC_FP64;
  if (metric >= 0.0 && metric <= c->opt.tol && polishing_done) {
    st.info.converged = 1;
    st.status = TTC_OK;
    st.done = true;
    return;
  }
  if (st.it >= c->opt.max_iter) {
    if (c->opt.stop_rule == TTC_STOP_NONE) {
      st.info.converged = 1;
      st.status = TTC_OK;
    }
    st.done = true;
  }
}

extern "C" {

int ttc_solve(ttc_ctx* c, ttc_solve_info* out) {
  if (!c) return TTC_EINVAL;
  if (!c->have_obs || !c->have_cores) return TTC_EINVAL;
  if (c->opt.stop_rule == TTC_STOP_RELERR && !c->hp.has_truth) return TTC_EINVAL;
  TTC_TRY(set_scalar(c, SC_ALPHA_OVR, 0.0));
  c->alpha_ovr = 0.0;
  SolveState st;
  ttc_solve_begin(c, st);
  // scalars are read back every check, and every iteration in MIXED mode
  // (the FP64 switch) or with the residual rule
  const bool every = c->opt.precision == TTC_PREC_MIXED || c->opt.stop_rule == TTC_STOP_RESID;
  while (!st.done) {
    ++st.it;
    int s = step_impl(c, 0.0, nullptr, false);
    if (s != TTC_OK) {
      st.status = s;
      break;
    }
    const bool check = (st.it % c->opt.check_every == 0) || st.it == c->opt.max_iter;
    if (!check && !every) continue;
    const bool metric = ttc_solve_needs_metric(c, st.it);
    if (metric) TTC_TRY(ttc_launch_metric(c, c->opt.stop_rule == TTC_STOP_RELERR ? 0 : 1));
    double sc[SC_COUNT];
    TTC_TRY(read_scalars(c, sc));
    ttc_solve_after(c, st, sc, metric);
  }
  st.info.iters = st.it;
  if (out) *out = st.info;
  return st.status;
}

int ttc_relerr(ttc_ctx* c, double* out) {
  if (!c || !out) return TTC_EINVAL;
  if (!c->hp.has_truth || !c->have_cores) return TTC_EINVAL;
  TTC_TRY(ttc_launch_metric(c, 0));
  double sc[SC_COUNT];
  TTC_TRY(read_scalars(c, sc));
  *out = std::sqrt(std::fmax(sc[SC_METRIC], 0.0) / sc[SC_NORM]);
  return TTC_OK;
}

int ttc_eval(ttc_ctx* c, int64_t M, const int32_t* idx, int precision, double* out) {
  if (!c || !idx || !out || M < 1 || !c->have_cores) return TTC_EINVAL;
  for (int64_t e = 0; e < M; ++e)
    for (int k = 0; k < c->m; ++k) {
      int x = idx[e * c->m + k];
      if (x < 0 || x >= c->n[k]) return TTC_ERANGE;
    }
  int32_t* di = nullptr;
  double* dout = nullptr;
  cudaError_t e1 = ttc_pool_alloc((void**)&di, sizeof(int32_t) * (size_t)M * c->m, c->stream);
  cudaError_t e2 = ttc_pool_alloc((void**)&dout, sizeof(double) * (size_t)M, c->stream);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    ttc_pool_free(di, c->stream);
    ttc_pool_free(dout, c->stream);
    ttc_record_cuda_error(e1 != cudaSuccess ? e1 : e2);
    return TTC_ENOMEM;
  }
  int s = TTC_OK;
  cudaError_t e = cudaMemcpyAsync(di, idx, sizeof(int32_t) * (size_t)M * c->m, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) s = ttc_launch_eval(c, di, M, precision, dout);
  if (e == cudaSuccess && s == TTC_OK)
    e = cudaMemcpyAsync(out, dout, sizeof(double) * (size_t)M, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  ttc_pool_free(di, c->stream);
  ttc_pool_free(dout, c->stream);
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    return TTC_ECUDA;
  }
  return s;
}

int ttc_get_residual(ttc_ctx* c, double* g_out) {
  if (!c || !g_out || !c->have_obs || !c->have_cores) return TTC_EINVAL;
  // one extra eager pass with the residual write switched on
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  c->hp.keep_residual = 1;
  int s = ttc_launch_omega_pass(c, c->cur_prec == TTC_PREC_FP64 ? TTC_PREC_FP64 : TTC_PREC_FP32);
  c->hp.keep_residual = 0;
  if (s != TTC_OK) return s;
  TTC_CUDA(cudaMemcpyAsync(g_out, c->hp.g, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  return TTC_OK;
}

int ttc_get_slice_energy(ttc_ctx* c, int k, double* s_out) {
  if (!c || !s_out || k < 0 || k >= c->m) return TTC_EINVAL;
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  TTC_CUDA(cudaMemcpy(s_out, c->hp.s[k], sizeof(double) * c->n[k], cudaMemcpyDeviceToHost));
  return TTC_OK;
}

int ttc_get_scatter(ttc_ctx* c, int k, double* E_out) {
  if (!c || !E_out || k < 0 || k >= c->m) return TTC_EINVAL;
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  TTC_CUDA(cudaMemcpy(E_out, c->hp.E[k], sizeof(double) * c->n[k] * c->r[k] * c->r[k + 1], cudaMemcpyDeviceToHost));
  return TTC_OK;
}

int ttc_get_layout(ttc_ctx* c, int k, int32_t* perm_out, int64_t* seg_off_out) {
  if (!c || k < 0 || k >= c->m || !c->have_obs) return TTC_EINVAL;
  TTC_CUDA(cudaStreamSynchronize(c->stream));
  if (perm_out) TTC_CUDA(cudaMemcpy(perm_out, c->hp.perm[k], sizeof(int) * c->N, cudaMemcpyDeviceToHost));
  if (seg_off_out) {
    std::vector<int> tmp(c->n[k] + 1);
    TTC_CUDA(cudaMemcpy(tmp.data(), c->hp.seg[k], sizeof(int) * (c->n[k] + 1), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < tmp.size(); ++i) seg_off_out[i] = tmp[i];
  }
  return TTC_OK;
}

int ttc_profile_enable(ttc_ctx* c, int on) {
  if (!c) return TTC_EINVAL;
  if (on && !c->ev_beg) {
    TTC_CUDA(cudaEventCreate(&c->ev_beg));
    TTC_CUDA(cudaEventCreate(&c->ev_end));
  }
  if ((on != 0) != c->prof) {
    TTC_CUDA(cudaStreamSynchronize(c->stream));
    drop_graphs(c);   // recapture with (or without) the event nodes
  }
  c->prof = on != 0;
  return TTC_OK;
}

int ttc_profile_read(ttc_ctx* c, double* ms, int64_t* count, int reset) {
  if (!c) return TTC_EINVAL;
  if (ms) *ms = c->prof_ms;
  if (count) *count = c->prof_count;
  if (reset) {
    c->prof_ms = 0.0;
    c->prof_count = 0;
  }
  return TTC_OK;
}

int ttc_launch_count(ttc_ctx* c, int64_t* launches) {
  if (!c || !launches) return TTC_EINVAL;
  *launches = c->nlaunch;
  return TTC_OK;
}

int ttc_device_bytes(ttc_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return TTC_EINVAL;
  *bytes = (int64_t)c->device_bytes;
  return TTC_OK;
}

}  // extern "C"
