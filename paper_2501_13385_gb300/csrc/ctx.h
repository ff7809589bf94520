// Host-side context of one completion problem and the internal entry points
// the C ABI (api.cu) calls into.  Device memory is owned through DevBuf and
// released by ttc_destroy.
#pragma once

#include <vector>

#include "common.cuh"

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// streams and events that let the mode-class launches of one pass run
// concurrently (forked from and joined back into the issuing stream; inside
// a stream capture they become parallel graph branches)
struct PassFork {
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[2] = {nullptr, nullptr};
};
int ttc_fork_create(PassFork& f);
void ttc_fork_destroy(PassFork& f);

struct ttc_ctx {
  int m = 0;
  long long n[TTC_MAXM] = {0};
  int r[TTC_MAXM + 1] = {0};
  ttc_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int N = 0;
  bool have_obs = false;
  bool have_cores = false;
  int rank_bucket = 4;             // row stride of the padded core mirrors and tables (4, 8, 16, 32)
  int rank_max = 1;                // largest TT-rank: register size of the small-rank pass

  DevProb hp;                       // host mirror of the descriptor
  DevProb* dp = nullptr;            // device copy
  std::vector<DevBuf> bufs;         // every device allocation (freed on destroy)
  std::vector<DevBuf> obs_bufs;     // allocations that depend on the observations
  size_t device_bytes = 0;

  // graphs of one iteration: [0] Omega pass in FP32, [1] in FP64
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_dirty = true;

  // profiling of the Omega pass
  bool prof = false;
  cudaEvent_t ev_beg = nullptr, ev_end = nullptr;
  double prof_ms = 0.0;
  long long prof_count = 0;

  // kernel launches: enqueued so far (graph replays add their kernel nodes)
  long long nlaunch = 0;
  long long graph_kernels[2] = {0, 0};

  // solver state
  int iter = 0;
  bool eps_set = false;
  int cur_prec = TTC_PREC_FP64;    // precision of the Omega pass for the next step
  double alpha_ovr = 0.0;           // step-size override currently on the device
  double ynorm2 = 0.0;              // ||y||^2 of the observations
  PassFork fork;                    // concurrent mode-class launches of the sampled pass
};

// the solver's per-iteration bookkeeping (shared by ttc_solve and the server)
struct SolveState {
  int it = 0;
  int status = TTC_ENOTCONV;
  bool done = false;
  double prev_res = -1.0;          // relative residual after the previous iteration (-1: none)
  ttc_solve_info info;
};
void ttc_solve_begin(ttc_ctx* c, SolveState& st);
// after iteration st.it (scalars already read into sc, metric computed if the
// rule needed it this iteration): precision switch and stop decision
void ttc_solve_after(ttc_ctx* c, SolveState& st, const double* sc, bool checked);
bool ttc_solve_needs_metric(const ttc_ctx* c, int it);
int ttc_read_scalars(ttc_ctx* c, double* out);

// whether a step of pass precision `prec` runs the block-per-slice dense
// stages' slice products in float-float (TTC_DENSE_*)
inline int ttc_dense_ff(int mode, int prec) {
  return (mode == TTC_DENSE_FF || (mode == TTC_DENSE_AUTO && prec != TTC_PREC_FP64)) ? 1 : 0;
}

// allocation helpers (api.cu): the library's stream-ordered device pool
cudaError_t ttc_pool_alloc(void** p, size_t bytes, cudaStream_t st);
void ttc_pool_free(void* p, cudaStream_t st);
// allocation helpers (api.cu)
int ttc_alloc(ttc_ctx* c, void** p, size_t bytes, bool obs);
void ttc_free_obs(ttc_ctx* c);
int ttc_upload_desc(ttc_ctx* c);

// layout.cu
int ttc_build_layout(ttc_ctx* c, const int32_t* idx_host, const double* y_host);

// one group of a batch: members sharing the sampled-pass precision and rank
// bucket, stepped by one launch of the batched sampled pass
struct BatchGroup {
  int prec;
  int R;
  int nprob;
  const DevProb* probs;      // device array of the members' descriptors
  const int* seg_base;       // device [nprob + 1]: block offsets of the slice reduction
  const long long* tab_base; // device [nprob + 1]: row offsets of the interface tables
  int RC;                    // register size of the pass: the members' largest TT-rank
  const int* pass_base_c[3]; // small ranks: block offsets per mode class (first, interior, last)
  int pass_blocks_c[3];
  int seg_blocks;
  long long tab_rows;
};

// mode classes of the sampled pass (separate launches, each at its own
// register budget): the first mode, the interior modes, the last mode
enum { PC_FIRST = 0, PC_MIDDLE = 1, PC_LAST = 2 };
inline void ttc_pass_class_range(const DevProb& P, int cls, int* c0, int* c1) {
  if (cls == PC_FIRST) {
    *c0 = 0;
    *c1 = P.chunk_base[1];
  } else if (cls == PC_LAST) {
    *c0 = P.chunk_base[P.m - 1];
    *c1 = P.chunk_base[P.m];
  } else {
    *c0 = P.chunk_base[1];
    *c1 = P.chunk_base[P.m - 1];
  }
}
// blocks of one class launch: one chunk per warp, except the interior modes
// at large ranks (R >= 16), one chunk per block
inline int ttc_pass_class_blocks(const DevProb& P, int cls) {
  int c0, c1;
  ttc_pass_class_range(P, cls, &c0, &c1);
  if (c1 <= c0) return 0;
  if (P.R >= 16 && cls == PC_MIDDLE) return c1 - c0;
  return (c1 - c0 + TTC_NT / 32 - 1) / (TTC_NT / 32);
}

// one launch of the sampled-pass kernel: a single problem (g == nullptr)
// or a batch group
struct PassLaunch {
  const DevProb* P;
  const BatchGroup* g;
  cudaStream_t st;
  const PassFork* fork;      // may be null: the class launches then run in sequence
};
// pass_small_f32.cu / pass_small_f64.cu: rank buckets 4 and 8, register size
// RC = the largest TT-rank (1..8); pass_large.cu: buckets 16 and 32, RC 16,
// 24 or 32 (the largest TT-rank rounded up to a multiple of 8)
int ttc_pass_small_f32(int RC, const PassLaunch& L);
int ttc_pass_small_f64(int RC, const PassLaunch& L);
int ttc_pass_small_f32_r4(int RC, const PassLaunch& L);   // pass_small_f32_r4.cu: RC = 1..4
int ttc_pass_small_f64_r4(int RC, const PassLaunch& L);   // pass_small_f64_r4.cu
int ttc_pass_large(bool f32, int R, int RC, const PassLaunch& L);
int ttc_pass_opt_in_large();

// blocks of the slice reduction: one slice per warp, 8 per block
inline int ttc_seg_blocks(const DevProb& P) {
  int nseg = 0;
  for (int k = 0; k < P.m; ++k) nseg += P.n[k];
  return (nseg + 7) / 8;
}

// omega_pass.cu
// phase 0: pass (mode classes forked onto `fork`'s streams when given), 1: slice reduction, 2: tables
int ttc_launch_omega_pass_batch(const BatchGroup& g, cudaStream_t st, int phase, const PassFork* fork = nullptr);
void ttc_plan_tables(ttc_ctx* c);
int ttc_prepare_omega_pass();
int ttc_launch_omega_pass(ttc_ctx* c, int prec);
int ttc_launch_eval(ttc_ctx* c, const int32_t* idx_dev, long long M, int prec, double* out_dev);

// dense.cu
// batched dense stages: members on the warp path without the steepest step
// and of one order run each dense stage as one launch
struct DenseGroup;
bool ttc_dense_batchable(const ttc_ctx* c);
int ttc_dense_group_create(ttc_ctx* const* members, int count, DenseGroup** out);
int ttc_dense_group_launch(const DenseGroup* g, cudaStream_t st, long long* kernels);
void ttc_dense_group_destroy(DenseGroup* g);
int ttc_alloc_dense(ttc_ctx* c);
int ttc_launch_dense(ttc_ctx* c);
int ttc_launch_metric(ttc_ctx* c, int which);   // 0: ||T - T*||^2 , 1: ||T_l - T_{l-1}||^2
int ttc_launch_save_prev(ttc_ctx* c);
int ttc_launch_mirror32(ttc_ctx* c);
void ttc_free_plan(const ttc_ctx* c);
