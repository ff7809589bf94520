// Batches: many independent completion problems stepped by one CUDA graph.
// One PRGD iteration of every member is one graph launch: the sampled pass
// of all members sharing a precision and rank bucket is ONE launch of the
// batched kernel (blocks mapped to (problem, chunk) through a prefix array),
// followed by the batched slice reduction; the dense stages of the members
// then run as parallel branches of the graph, each on its member's stream.
// Every member computes exactly what it computes alone (same kernels, same
// block decomposition), so results are bitwise identical alone or in a batch.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.h"

struct ttc_batch {
  std::vector<ttc_ctx*> members;
  std::vector<int> prec_at_capture;   // per member: 2 x pass precision + steepest-step flag
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  PassFork pfork;              // concurrent mode-class launches of the batched pass
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  struct Group {
    BatchGroup g;
    DevProb* probs = nullptr;
    int* pass_base_c = nullptr;   // three per-class prefix arrays, back to back
    int* seg_base = nullptr;
    long long* tab_base = nullptr;
    std::vector<int> idx;
  };
  std::vector<Group> groups;
  std::vector<DenseGroup*> dense;   // batched dense stages (members grouped by order, then chunked)
  std::vector<int> in_dense;        // per member: its dense group, or -1 (own graph branch)
  std::vector<cudaStream_t> dstreams;   // dense groups after the first run on these, concurrently
  std::vector<cudaEvent_t> djoins;
  cudaGraphExec_t exec = nullptr;
  long long kernels_per_step = 0;
  long long nlaunch = 0;
  bool prof = false;
  // lanes: sub-batches over contiguous member groups, each on its own stream
  std::vector<ttc_batch*> lanes;
  std::vector<cudaEvent_t> lane_join;
  cudaEvent_t lane_fork = nullptr;
  bool forked = false;
  bool stepped = false;
  cudaEvent_t ev_beg = nullptr, ev_end = nullptr;     // the pass
  cudaEvent_t ev_dbeg = nullptr, ev_dend = nullptr;   // the dense part
  double prof_ms = 0.0, prof_dense_ms = 0.0;
  long long prof_count = 0;
};

namespace {

void free_groups(ttc_batch* b) {
  for (auto* d : b->dense) ttc_dense_group_destroy(d);
  b->dense.clear();
  b->in_dense.clear();
  for (auto& G : b->groups) {
    cudaFree(G.probs);
    cudaFree(G.pass_base_c);
    cudaFree(G.seg_base);
    cudaFree(G.tab_base);
  }
  b->groups.clear();
}

int build_groups(ttc_batch* b) {
  free_groups(b);
  std::vector<std::pair<int, int>> keys;   // (prec, R)
  for (auto* c : b->members) {
    int prec = c->cur_prec == TTC_PREC_FP64 ? TTC_PREC_FP64 : TTC_PREC_FP32;
    std::pair<int, int> key(prec, c->rank_bucket);
    if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
  }
  for (auto& key : keys) {
    ttc_batch::Group G;
    std::vector<DevProb> descs;
    std::vector<int> sb(1, 0);
    std::vector<int> pc[3] = {std::vector<int>(1, 0), std::vector<int>(1, 0), std::vector<int>(1, 0)};
    std::vector<long long> tb(1, 0);
    for (int i = 0; i < (int)b->members.size(); ++i) {
      ttc_ctx* c = b->members[i];
      int prec = c->cur_prec == TTC_PREC_FP64 ? TTC_PREC_FP64 : TTC_PREC_FP32;
      if (prec != key.first || c->rank_bucket != key.second) continue;
      G.idx.push_back(i);
      descs.push_back(c->hp);
      for (int cls = 0; cls < 3; ++cls) pc[cls].push_back(pc[cls].back() + ttc_pass_class_blocks(c->hp, cls));
      sb.push_back(sb.back() + ttc_seg_blocks(c->hp));
      tb.push_back(tb.back() + c->hp.tab_total);
    }
    cudaError_t e = cudaMalloc(&G.probs, sizeof(DevProb) * descs.size());
    if (e == cudaSuccess) e = cudaMalloc(&G.seg_base, sizeof(int) * sb.size());
    if (e == cudaSuccess) e = cudaMemcpy(G.probs, descs.data(), sizeof(DevProb) * descs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G.seg_base, sb.data(), sizeof(int) * sb.size(), cudaMemcpyHostToDevice);
    const size_t np1 = pc[0].size();
    if (e == cudaSuccess) e = cudaMalloc(&G.pass_base_c, sizeof(int) * 3 * np1);
    for (int cls = 0; cls < 3 && e == cudaSuccess; ++cls)
      e = cudaMemcpy(G.pass_base_c + cls * np1, pc[cls].data(), sizeof(int) * np1, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&G.tab_base, sizeof(long long) * tb.size());
    if (e == cudaSuccess) e = cudaMemcpy(G.tab_base, tb.data(), sizeof(long long) * tb.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      ttc_record_cuda_error(e);
      b->groups.push_back(G);
      free_groups(b);
      return e == cudaErrorMemoryAllocation ? TTC_ENOMEM : TTC_ECUDA;
    }
    G.g.prec = key.first;
    G.g.R = key.second;
    G.g.RC = 1;
    for (int i : G.idx) G.g.RC = std::max(G.g.RC, b->members[i]->rank_max);
    G.g.nprob = (int)descs.size();
    G.g.probs = G.probs;
    G.g.seg_base = G.seg_base;
    G.g.tab_base = G.tab_base;
    for (int cls = 0; cls < 3; ++cls) {
      G.g.pass_base_c[cls] = G.pass_base_c + cls * np1;
      G.g.pass_blocks_c[cls] = pc[cls].back();
    }
    G.g.seg_blocks = sb.back();
    G.g.tab_rows = tb.back();
    b->groups.push_back(G);
  }
  // members whose dense stages can be batched, grouped by order and split
  // into up to kDenseChunks chunks of at least kDenseChunkMin members whose
  // stage sequences run on concurrent streams: a chunk's single-block
  // retraction steps (latency-bound) then overlap another chunk's
  // slice-parallel FP64 reductions (throughput-bound)
  constexpr int kDenseChunks = 4, kDenseChunkMin = 8;
  b->in_dense.assign(b->members.size(), -1);
  std::vector<int> orders;
  for (auto* c : b->members)
    if (ttc_dense_batchable(c) && std::find(orders.begin(), orders.end(), c->m) == orders.end()) orders.push_back(c->m);
  for (int m : orders) {
    std::vector<ttc_ctx*> mem;
    std::vector<int> at;
    for (int i = 0; i < (int)b->members.size(); ++i)
      if (b->members[i]->m == m && ttc_dense_batchable(b->members[i])) {
        mem.push_back(b->members[i]);
        at.push_back(i);
      }
    const int cnt = (int)mem.size();
    const int nch = std::max(1, std::min(kDenseChunks, cnt / kDenseChunkMin));
    for (int ch = 0; ch < nch; ++ch) {
      const int lo = (int)((long long)cnt * ch / nch), hi = (int)((long long)cnt * (ch + 1) / nch);
      DenseGroup* d = nullptr;
      int s = ttc_dense_group_create(mem.data() + lo, hi - lo, &d);
      if (s != TTC_OK) {
        free_groups(b);
        return s;
      }
      for (int i = lo; i < hi; ++i) b->in_dense[at[i]] = (int)b->dense.size();
      b->dense.push_back(d);
    }
  }
  while (b->dstreams.size() + 1 < b->dense.size()) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      ttc_record_cuda_error(e);
      free_groups(b);
      return TTC_ECUDA;
    }
    b->dstreams.push_back(st);
    b->djoins.push_back(ev);
  }
  return TTC_OK;
}

int capture(ttc_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  // the retraction refines its SVDs to FP64 accuracy in a member's FP64 steps
  for (auto* c : b->members) {
    c->hp.step_fp64 = (c->cur_prec == TTC_PREC_FP64) ? 1 : 0;
    c->hp.dense_ff = ttc_dense_ff(c->opt.dense_mode, c->cur_prec);
  }
  TTC_TRY(build_groups(b));
  b->prec_at_capture.clear();
  for (auto* c : b->members) b->prec_at_capture.push_back(c->cur_prec * 2 + c->hp.steepest);
  std::vector<long long> before;
  for (auto* c : b->members) before.push_back(c->nlaunch);
  cudaGraph_t g = nullptr;
  TTC_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int s = TTC_OK;
  cudaError_t e = cudaSuccess;
  long long batched = 0;
  for (auto& G : b->groups)
    if (s == TTC_OK && G.g.tab_rows > 0) {
      s = ttc_launch_omega_pass_batch(G.g, b->stream, 2);
      ++batched;
    }
  if (b->prof) e = cudaEventRecordWithFlags(b->ev_beg, b->stream, cudaEventRecordExternal);
  for (auto& G : b->groups)
    if (s == TTC_OK && e == cudaSuccess) {
      s = ttc_launch_omega_pass_batch(G.g, b->stream, 0, &b->pfork);
      for (int cls = 0; cls < 3; ++cls) batched += G.g.pass_blocks_c[cls] > 0 ? 1 : 0;   // one launch per class
    }
  if (b->prof && e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev_end, b->stream, cudaEventRecordExternal);
  for (auto& G : b->groups)
    if (s == TTC_OK && e == cudaSuccess) {
      s = ttc_launch_omega_pass_batch(G.g, b->stream, 1);
      ++batched;
    }
  if (s == TTC_OK && e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
  if (b->prof && s == TTC_OK && e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev_dbeg, b->stream, cudaEventRecordExternal);
  long long dense_kernels = 0;
  for (size_t i = 1; i < b->dense.size() && s == TTC_OK && e == cudaSuccess; ++i) {
    cudaStream_t ds = b->dstreams[i - 1];
    e = cudaStreamWaitEvent(ds, b->fork, 0);
    if (e == cudaSuccess) s = ttc_dense_group_launch(b->dense[i], ds, &dense_kernels);
    if (s == TTC_OK && e == cudaSuccess) e = cudaEventRecord(b->djoins[i - 1], ds);
  }
  if (!b->dense.empty() && s == TTC_OK && e == cudaSuccess) s = ttc_dense_group_launch(b->dense[0], b->stream, &dense_kernels);
  for (size_t i = 1; i < b->dense.size() && s == TTC_OK && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(b->stream, b->djoins[i - 1], 0);
  for (size_t i = 0; i < b->members.size() && s == TTC_OK && e == cudaSuccess; ++i) {
    if (b->in_dense[i] >= 0) continue;   // its dense stages ran batched above
    ttc_ctx* c = b->members[i];
    bool own = c->stream != b->stream;
    for (size_t j = 0; j < i && own; ++j)
      if (b->members[j]->stream == c->stream) own = false;
    cudaStream_t saved = c->stream;
    if (!own) c->stream = b->stream;   // shared stream: run this member's branch in line
    if (own) e = cudaStreamWaitEvent(c->stream, b->fork, 0);
    if (e == cudaSuccess) s = ttc_launch_save_prev(c);
    if (s == TTC_OK) s = ttc_launch_dense(c);
    if (s == TTC_OK && own) {
      e = cudaEventRecord(b->joins[i], c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[i], 0);
    }
    c->stream = saved;
  }
  if (b->prof && s == TTC_OK && e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev_dend, b->stream, cudaEventRecordExternal);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  long long kernels = batched + dense_kernels;
  for (size_t i = 0; i < b->members.size(); ++i) {
    kernels += b->members[i]->nlaunch - before[i];
    b->members[i]->nlaunch = before[i];
  }
  if (s != TTC_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) ttc_record_cuda_error(e);
    if (e2 != cudaSuccess) ttc_record_cuda_error(e2);
    return s != TTC_OK ? s : TTC_ECUDA;
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    return TTC_ECUDA;
  }
  b->kernels_per_step = kernels;
  return TTC_OK;
}

}  // namespace

extern "C" {

int ttc_batch_create(ttc_batch** out, ttc_ctx* const* members, int count, void* cuda_stream) {
  if (!out || !members || count < 1) return TTC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!members[i] || !members[i]->have_obs || !members[i]->have_cores) return TTC_EINVAL;
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return TTC_EINVAL;
  }
  ttc_batch* b = new (std::nothrow) ttc_batch();
  if (!b) return TTC_ENOMEM;
  b->members.assign(members, members + count);
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess && ttc_fork_create(b->pfork) != TTC_OK) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  b->joins.assign(count, nullptr);
  for (int i = 0; i < count && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev_beg);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev_end);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev_dbeg);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev_dend);
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    ttc_batch_destroy(b);
    return TTC_ECUDA;
  }
  // members' pending work must be done before the batch reads their state
  for (auto* c : b->members) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      ttc_record_cuda_error(e);
      ttc_batch_destroy(b);
      return TTC_ECUDA;
    }
  }
  *out = b;
  return TTC_OK;
}

int ttc_batch_step(ttc_batch* b) {
  if (!b) return TTC_EINVAL;
  b->stepped = true;
  if (!b->lanes.empty()) {
    if (!b->forked) {   // the lanes start after the work already on the batch's stream
      TTC_CUDA(cudaEventRecord(b->lane_fork, b->stream));
      for (auto* l : b->lanes) TTC_CUDA(cudaStreamWaitEvent(l->stream, b->lane_fork, 0));
      b->forked = true;
    }
    for (auto* l : b->lanes) {
      const long long n0 = l->nlaunch;
      TTC_TRY(ttc_batch_step(l));
      b->nlaunch += l->nlaunch - n0;
    }
    return TTC_OK;
  }
  bool stale = (b->exec == nullptr);
  for (size_t i = 0; i < b->members.size() && !stale; ++i)
    stale = (b->members[i]->cur_prec * 2 + b->members[i]->hp.steepest != b->prec_at_capture[i]);
  if (stale) TTC_TRY(capture(b));
  TTC_CUDA(cudaGraphLaunch(b->exec, b->stream));
  b->nlaunch += b->kernels_per_step;
  for (auto* c : b->members) {
    ++c->iter;
    if (c->opt.eps_frozen && !c->eps_set) {
      // the first iteration's epsilon stays fixed from here on
      TTC_CUDA(cudaMemcpyAsync(c->hp.scal + SC_EPS_FIXED, c->hp.scal + SC_EPS, sizeof(double),
                               cudaMemcpyDeviceToDevice, b->stream));
      c->eps_set = true;
    }
  }
  if (b->prof) {
    TTC_CUDA(cudaEventSynchronize(b->ev_dend));
    float t = 0.f, td = 0.f;
    TTC_CUDA(cudaEventElapsedTime(&t, b->ev_beg, b->ev_end));
    TTC_CUDA(cudaEventElapsedTime(&td, b->ev_dbeg, b->ev_dend));
    b->prof_ms += t;
    b->prof_dense_ms += td;
    b->prof_count += 1;
  }
  return TTC_OK;
}

int ttc_batch_sync(ttc_batch* b) {
  if (!b) return TTC_EINVAL;
  for (auto* l : b->lanes) TTC_TRY(ttc_batch_sync(l));
  b->forked = false;
  TTC_CUDA(cudaStreamSynchronize(b->stream));
  return TTC_OK;
}

int ttc_batch_join(ttc_batch* b) {
  if (!b) return TTC_EINVAL;
  for (size_t i = 0; i < b->lanes.size(); ++i) {
    TTC_CUDA(cudaEventRecord(b->lane_join[i], b->lanes[i]->stream));
    TTC_CUDA(cudaStreamWaitEvent(b->stream, b->lane_join[i], 0));
  }
  b->forked = false;
  return TTC_OK;
}

int ttc_batch_set_lanes(ttc_batch* b, int lanes) {
  if (!b || lanes < 1 || lanes > (int)b->members.size() || b->stepped) return TTC_EINVAL;
  if (lanes == 1 || !b->lanes.empty()) return lanes == 1 && b->lanes.empty() ? TTC_OK : TTC_EINVAL;
  const int cnt = (int)b->members.size();
  cudaError_t e = cudaEventCreateWithFlags(&b->lane_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    return TTC_ECUDA;
  }
  for (int l = 0; l < lanes; ++l) {
    const int lo = (int)((long long)cnt * l / lanes), hi = (int)((long long)cnt * (l + 1) / lanes);
    ttc_batch* sub = nullptr;
    int s = ttc_batch_create(&sub, b->members.data() + lo, hi - lo, nullptr);   // own stream
    cudaEvent_t ev = nullptr;
    if (s == TTC_OK) {
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        ttc_record_cuda_error(e);
        s = TTC_ECUDA;
      }
    }
    if (s != TTC_OK) {
      if (sub) ttc_batch_destroy(sub);
      for (auto* x : b->lanes) ttc_batch_destroy(x);
      for (auto x : b->lane_join) cudaEventDestroy(x);
      b->lanes.clear();
      b->lane_join.clear();
      return s;
    }
    b->lanes.push_back(sub);
    b->lane_join.push_back(ev);
  }
  return TTC_OK;
}

int ttc_batch_profile_enable(ttc_batch* b, int on) {
  if (!b) return TTC_EINVAL;
  for (auto* l : b->lanes) TTC_TRY(ttc_batch_profile_enable(l, on));
  if ((on != 0) != b->prof) {
    TTC_CUDA(cudaStreamSynchronize(b->stream));
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  b->prof = on != 0;
  return TTC_OK;
}

// with lanes: the sums over the lanes (their profiled steps run one after
// another, each waiting on the host)
static int lanes_profile(ttc_batch* b, double* ms, int64_t* count, int reset, bool dense) {
  double tot = 0.0;
  int64_t n = 0;
  for (auto* l : b->lanes) {
    double v = 0.0;
    int64_t c = 0;
    TTC_TRY(dense ? ttc_batch_profile_read_dense(l, &v, &c, reset) : ttc_batch_profile_read(l, &v, &c, reset));
    tot += v;
    n = c;
  }
  if (ms) *ms = tot;
  if (count) *count = n;
  return TTC_OK;
}

int ttc_batch_profile_read(ttc_batch* b, double* ms, int64_t* count, int reset) {
  if (!b) return TTC_EINVAL;
  if (!b->lanes.empty()) return lanes_profile(b, ms, count, reset, false);
  if (ms) *ms = b->prof_ms;
  if (count) *count = b->prof_count;
  if (reset) {
    b->prof_ms = 0.0;
    b->prof_dense_ms = 0.0;
    b->prof_count = 0;
  }
  return TTC_OK;
}

int ttc_batch_profile_read_dense(ttc_batch* b, double* ms, int64_t* count, int reset) {
  if (!b) return TTC_EINVAL;
  if (!b->lanes.empty()) return lanes_profile(b, ms, count, reset, true);
  if (ms) *ms = b->prof_dense_ms;
  if (count) *count = b->prof_count;
  if (reset) {
    b->prof_ms = 0.0;
    b->prof_dense_ms = 0.0;
    b->prof_count = 0;
  }
  return TTC_OK;
}

int ttc_batch_launch_count(ttc_batch* b, int64_t* launches) {
  if (!b || !launches) return TTC_EINVAL;
  *launches = b->nlaunch;
  return TTC_OK;
}

void ttc_batch_destroy(ttc_batch* b) {
  if (!b) return;
  for (auto* l : b->lanes) ttc_batch_destroy(l);   // each waits for its own stream
  for (auto ev : b->lane_join) cudaEventDestroy(ev);
  if (b->lane_fork) cudaEventDestroy(b->lane_fork);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  free_groups(b);
  for (auto st : b->dstreams) cudaStreamDestroy(st);
  for (auto ev : b->djoins) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  ttc_fork_destroy(b->pfork);
  for (auto ev : b->joins)
    if (ev) cudaEventDestroy(ev);
  if (b->ev_beg) cudaEventDestroy(b->ev_beg);
  if (b->ev_end) cudaEventDestroy(b->ev_end);
  if (b->ev_dbeg) cudaEventDestroy(b->ev_dbeg);
  if (b->ev_dend) cudaEventDestroy(b->ev_dend);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
