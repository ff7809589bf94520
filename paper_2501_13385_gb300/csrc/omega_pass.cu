// Host side of the sampled pass over Omega and its companion kernels: the
// interface tables, the per-slice reduction of the chunk partials (with
// eps_l and alpha_l), and the evaluation of T at given indices.  The pass
// kernels themselves live in omega_pass.cuh and are instantiated in
// pass_small_f32.cu, pass_small_f64.cu and pass_large.cu (compiled in
// parallel); this file dispatches to them by precision and rank.
#include <algorithm>

#include "omega_pass.cuh"

namespace {

using namespace ttc_pass;

// 16-byte stores of a padded row (R a multiple of 4)
template <int R>
__device__ __forceinline__ void store_row(float* dst, const float (&v)[R]) {
#pragma unroll
  for (int b = 0; b < R; b += 4) *reinterpret_cast<float4*>(dst + b) = make_float4(v[b], v[b + 1], v[b + 2], v[b + 3]);
}
template <int R>
__device__ __forceinline__ void store_row(double* dst, const double (&v)[R]) {
#pragma unroll
  for (int b = 0; b < R; b += 2) *reinterpret_cast<double2*>(dst + b) = make_double2(v[b], v[b + 1]);
}

// one table row per thread: the chain of core slices it stands for (rows
// whose coordinates are outside the mode sizes stand for no entry: zeroed
// once when the tables are allocated, not written here)
template <typename T, int R>
__device__ __forceinline__ void build_table_row(const DevProb& P, long long g) {
  int t = 0;
  while (t + 1 < P.ntab && g >= P.tab_row0[t + 1]) ++t;
  const unsigned row = (unsigned)(g - P.tab_row0[t]);
  const int jt = P.tab_j[t];
  const bool prefix = P.tab_side[t] == 0;
  const int first = prefix ? 0 : jt, last = prefix ? jt - 1 : P.m - 1;
  int xs[TTC_MAXM];
  bool valid = true;
  for (int j = first; j <= last; ++j) {
    xs[j] = (int)((row >> (P.cshift[j] - P.tab_shift[t])) & ((1u << P.cbits[j]) - 1u));
    valid = valid && xs[j] < P.n[j];
  }
  if (!valid) return;
  T v[R];
  zero(v);
  v[0] = 1;
  if (valid) {
    if (prefix)
      for (int j = first; j <= last; ++j) row_times<T, R, R>(P, j, xs[j], v);
    else
      for (int j = last; j >= first; --j) times_col<T, R, R>(P, j, xs[j], v);
  }
  const int len = valid ? P.r[jt] : 0;
#pragma unroll
  for (int a = 0; a < R; ++a)
    if (a >= len) v[a] = T(0);
  store_row<R>(tab_ptr<T>(P) + g * R, v);
}

// Rows of a two-mode prefix table that share the second mode's coordinate
// x_1 (its bits lie above the first mode's, so a block of consecutive rows
// usually does) read the same slice T_1(x_1): a block whose rows all do
// stages it in shared memory once, and each row is then T_0(x_0) T_1(x_1)
// with the same FMA order as row_times (identical results).  `key` names
// (problem, table, x_1) for that test, -1 when the row cannot take it.
template <typename T, int R>
__device__ __forceinline__ long long prefix2_key(const DevProb& P, long long g, int p, int& x0, int& x1) {
  int t = 0;
  while (t + 1 < P.ntab && g >= P.tab_row0[t + 1]) ++t;
  if (P.tab_side[t] != 0 || P.tab_j[t] != 2) return -1;
  const unsigned row = (unsigned)(g - P.tab_row0[t]);
  x0 = (int)((row >> (P.cshift[0] - P.tab_shift[t])) & ((1u << P.cbits[0]) - 1u));
  x1 = (int)((row >> (P.cshift[1] - P.tab_shift[t])) & ((1u << P.cbits[1]) - 1u));
  if (x1 >= P.n[1]) return -1;
  return ((long long)p * (2 * TTC_MAXM) + t) * (1LL << 32) + x1;
}

template <typename T, int R>
__device__ __forceinline__ void prefix2_row(const DevProb& P, long long g, int x0, const T* sS) {
  const int r1 = P.r[1], r2 = P.r[2];
  const bool valid = x0 < P.n[0];
  if (!valid) return;   // a row that stands for no entry is never read
  const T* S0 = core_ptr<T>(P, 0) + (long long)(valid ? x0 : 0) * R * R;   // a 1 x r_1 slice: row 0
  T l0[R], v[R];
#pragma unroll
  for (int a = 0; a < R; ++a) l0[a] = (valid && a < r1) ? S0[a] : T(0);
#pragma unroll
  for (int b = 0; b < R; ++b) {
    T acc = 0;
    if (valid && b < r2) {
#pragma unroll
      for (int a = 0; a < R; ++a)
        if (a < r1) acc = fma(l0[a], sS[r2 == 1 ? a : a * R + b], acc);
    }
    v[b] = acc;
  }
  store_row<R>(tab_ptr<T>(P) + g * R, v);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_build_tables(const DevProb P) {
  __shared__ __align__(16) T sS[R * R];
  __shared__ long long key0;
  for (long long g0 = blockIdx.x * (long long)blockDim.x; g0 < P.tab_total; g0 += (long long)gridDim.x * blockDim.x) {
    const long long g = g0 + threadIdx.x;
    int x0 = 0, x1 = 0;
    const long long key = g < P.tab_total ? prefix2_key<T, R>(P, g, 0, x0, x1) : -1;
    __syncthreads();   // the previous rows' reads of sS are done
    if (threadIdx.x == 0) key0 = key;
    __syncthreads();
    if (__syncthreads_and(key >= 0 && key == key0)) {
      const T* S1 = core_ptr<T>(P, 1) + (long long)x1 * R * R;
      for (int i = threadIdx.x; i < R * R; i += blockDim.x) sS[i] = S1[i];
      __syncthreads();
      prefix2_row<T, R>(P, g, x0, sS);
    } else if (g < P.tab_total) {
      build_table_row<T, R>(P, g);
    }
  }
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_build_tables_batch(const DevProb* __restrict__ probs,
                                                            const long long* __restrict__ base, int nprob,
                                                            long long total) {
  __shared__ __align__(16) T sS[R * R];
  __shared__ long long key0;
  for (long long g0 = blockIdx.x * (long long)blockDim.x; g0 < total; g0 += (long long)gridDim.x * blockDim.x) {
    const long long g = g0 + threadIdx.x;
    int lo = 0;
    if (g < total) {
      int hi = nprob - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= g) lo = mid; else hi = mid - 1;
      }
    }
    const DevProb& P = probs[lo];
    const long long gl = g - __ldg(base + lo);
    int x0 = 0, x1 = 0;
    const long long key = g < total ? prefix2_key<T, R>(P, gl, lo, x0, x1) : -1;
    __syncthreads();
    if (threadIdx.x == 0) key0 = key;
    __syncthreads();
    if (__syncthreads_and(key >= 0 && key == key0)) {
      const T* S1 = core_ptr<T>(P, 1) + (long long)x1 * R * R;
      for (int i = threadIdx.x; i < R * R; i += blockDim.x) sS[i] = S1[i];
      __syncthreads();
      prefix2_row<T, R>(P, gl, x0, sS);
    } else if (g < total) {
      build_table_row<T, R>(P, gl);
    }
  }
}

inline int table_blocks(long long rows) {
  long long b = (rows + 255) / 256;
  return (int)(b < 64 * 152 ? (b < 1 ? 1 : b) : 64 * 152);
}


// sums the chunk partials of every slice (k, x) in chunk order, in FP64, one
// slice per warp (kSegSlices per block); the last block then forms
// ||G_l||^2 = sum_x s_1(x), eps_l and alpha_l (step-size form of Theorem 4.1;
// eps reading in the options)
constexpr int kSegThreads = 256;
constexpr int kSegSlices = kSegThreads / 32;

template <typename T>
__device__ __forceinline__ void segment_reduce_block(const DevProb& P, int blk, int total_blocks) {
  __shared__ int am_last;
  __shared__ double sh[kSegThreads];
  const int lane = threadIdx.x & 31;
  int g = blk * kSegSlices + (threadIdx.x >> 5);
  int k = 0;
  while (k < P.m - 1 && g >= P.n[k]) {
    g -= P.n[k];
    ++k;
  }
  if (g < P.n[k]) {
    const int x = g;
    const int ra = P.r[k], rb = P.r[k + 1];
    const int nout = 1 + ra * rb;
    const int c0 = P.cfirst[k][x], c1 = P.cfirst[k][x + 1];
    const T* part = reinterpret_cast<const T*>(P.part) + (long long)P.chunk_base[k] * P.part_stride;
    for (int j = lane; j < nout; j += 32) {
      double acc = 0.0;
      for (int cc = c0; cc < c1; ++cc) acc += (double)part[(long long)cc * P.part_stride + j];
      if (j == 0)
        P.s[k][x] = acc;
      else
        P.E[k][(long long)x * ra * rb + (j - 1)] = acc;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(P.counters, 1) == total_blocks - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double a0 = 0.0, a1 = 0.0;
  int i = threadIdx.x;
  for (; i + (int)blockDim.x < P.n[0]; i += 2 * blockDim.x) {
    a0 += __ldcg(P.s[0] + i);
    a1 += __ldcg(P.s[0] + i + blockDim.x);
  }
  if (i < P.n[0]) a0 += __ldcg(P.s[0] + i);
  sh[threadIdx.x] = a0 + a1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double g2 = sh[0];
    const double eps = P.scal[SC_EPS_FIXED] > 0.0 ? P.scal[SC_EPS_FIXED]
                                                  : fmax(P.scal[SC_EPS_REL] * g2 * P.inv_min_n, 1e-300);
    // Theorem 4.1's form; with the uniform metric (RGD) its limit alpha_scale / p.
    // The steepest-step rule overwrites alpha after the dense stage's projection.
    const double alpha = P.scal[SC_ALPHA_OVR] > 0.0 ? P.scal[SC_ALPHA_OVR]
                         : P.uniform            ? P.scal[SC_ALPHA_SCALE] / P.p
                                                : P.scal[SC_ALPHA_SCALE] * sqrt(eps) / P.p;
    P.scal[SC_G2] = g2;
    P.scal[SC_EPS] = eps;
    P.scal[SC_ALPHA] = alpha;
    if (!isfinite(g2)) atomicOr(P.flags, 1u);
    P.counters[0] = 0;
  }
}

template <typename T>
__global__ void k_segment_reduce(const DevProb P, int total_blocks) {
  segment_reduce_block<T>(P, blockIdx.x, total_blocks);
}

template <typename T>
__global__ void k_segment_reduce_batch(const DevProb* __restrict__ probs, const int* __restrict__ base, int nprob) {
  const int p = find_problem(base, nprob, blockIdx.x);
  segment_reduce_block<T>(probs[p], blockIdx.x - __ldg(base + p), __ldg(base + p + 1) - __ldg(base + p));
}

template <typename T, int R>
__global__ void k_eval(const DevProb P, const int32_t* __restrict__ idx, long long M, double* __restrict__ out) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= M) return;
  T v[R];
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = 0;
  v[0] = 1;
  for (int j = 0; j < P.m; ++j) row_times<T, R, R>(P, j, idx[e * P.m + j], v);
  out[e] = (double)v[0];
}

// the pass kernel for (precision, rank bucket R, register size RC)
int launch_pass_kernel(bool f32, int R, int RC, const PassLaunch& L) {
  if (R <= 8) return f32 ? ttc_pass_small_f32(RC, L) : ttc_pass_small_f64(RC, L);
  return ttc_pass_large(f32, R, R == 16 ? 16 : (RC <= 24 ? 24 : 32), L);
}

template <typename T, int R>
int launch_pass(ttc_ctx* c, int RC) {
  const DevProb& P = c->hp;
  if (P.ntab > 0) {
    k_build_tables<T, R><<<table_blocks(P.tab_total), 256, 0, c->stream>>>(P);
    TTC_CUDA(cudaGetLastError());
    c->nlaunch += 1;
  }
  // when profiling, the kernel is bracketed by events; inside a stream capture
  // they become event-record nodes of the graph, so replays are timed too
  unsigned evflags = cudaEventRecordDefault;
  if (c->prof) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TTC_CUDA(cudaStreamIsCapturing(c->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) evflags = cudaEventRecordExternal;
    TTC_CUDA(cudaEventRecordWithFlags(c->ev_beg, c->stream, evflags));
  }
  PassLaunch L{&P, nullptr, c->stream, &c->fork};
  TTC_TRY(launch_pass_kernel(sizeof(T) == 4, R, RC, L));
  if (c->prof) TTC_CUDA(cudaEventRecordWithFlags(c->ev_end, c->stream, evflags));
  const int nsegb = ttc_seg_blocks(P);
  k_segment_reduce<T><<<nsegb, kSegThreads, 0, c->stream>>>(P, nsegb);
  TTC_CUDA(cudaGetLastError());
  int passes = 0;   // one launch per non-empty mode class
  for (int cls = 0; cls < 3; ++cls) passes += ttc_pass_class_blocks(P, cls) > 0 ? 1 : 0;
  c->nlaunch += 1 + passes;
  return TTC_OK;
}

template <typename T, int R>
int launch_eval(ttc_ctx* c, const int32_t* idx_dev, long long M, double* out_dev) {
  k_eval<T, R><<<(int)((M + 127) / 128), 128, 0, c->stream>>>(c->hp, idx_dev, M, out_dev);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  return TTC_OK;
}

template <typename T, int R>
int launch_pass_batch(const BatchGroup& g, cudaStream_t st, int phase, const PassFork* fork) {
  if (phase == 2) {
    if (g.tab_rows > 0)
      k_build_tables_batch<T, R><<<table_blocks(g.tab_rows), 256, 0, st>>>(g.probs, g.tab_base, g.nprob, g.tab_rows);
  } else if (phase == 0) {
    PassLaunch L{nullptr, &g, st, fork};
    return launch_pass_kernel(sizeof(T) == 4, R, g.RC, L);
  } else {
    k_segment_reduce_batch<T><<<g.seg_blocks, kSegThreads, 0, st>>>(g.probs, g.seg_base, g.nprob);
  }
  TTC_CUDA(cudaGetLastError());
  return TTC_OK;
}

}  // namespace

// one-time kernel attributes (outside any stream capture)
int ttc_prepare_omega_pass() { return ttc_pass_opt_in_large(); }

int ttc_launch_omega_pass_batch(const BatchGroup& g, cudaStream_t st, int phase, const PassFork* fork) {
  const bool f32 = (g.prec != TTC_PREC_FP64);
  switch (g.R) {
    case 4: return f32 ? launch_pass_batch<float, 4>(g, st, phase, fork) : launch_pass_batch<double, 4>(g, st, phase, fork);
    case 8: return f32 ? launch_pass_batch<float, 8>(g, st, phase, fork) : launch_pass_batch<double, 8>(g, st, phase, fork);
    case 16: return f32 ? launch_pass_batch<float, 16>(g, st, phase, fork) : launch_pass_batch<double, 16>(g, st, phase, fork);
    default: return f32 ? launch_pass_batch<float, 32>(g, st, phase, fork) : launch_pass_batch<double, 32>(g, st, phase, fork);
  }
}

int ttc_launch_omega_pass(ttc_ctx* c, int prec) {
  const bool f32 = (prec != TTC_PREC_FP64);
  const int RC = c->rank_max;
  switch (c->rank_bucket) {
    case 4: return f32 ? launch_pass<float, 4>(c, RC) : launch_pass<double, 4>(c, RC);
    case 8: return f32 ? launch_pass<float, 8>(c, RC) : launch_pass<double, 8>(c, RC);
    case 16: return f32 ? launch_pass<float, 16>(c, RC) : launch_pass<double, 16>(c, RC);
    default: return f32 ? launch_pass<float, 32>(c, RC) : launch_pass<double, 32>(c, RC);
  }
}

int ttc_launch_eval(ttc_ctx* c, const int32_t* idx_dev, long long M, int prec, double* out_dev) {
  const bool f32 = (prec != TTC_PREC_FP64);
  switch (c->rank_bucket) {
    case 4: return f32 ? launch_eval<float, 4>(c, idx_dev, M, out_dev) : launch_eval<double, 4>(c, idx_dev, M, out_dev);
    case 8: return f32 ? launch_eval<float, 8>(c, idx_dev, M, out_dev) : launch_eval<double, 8>(c, idx_dev, M, out_dev);
    case 16: return f32 ? launch_eval<float, 16>(c, idx_dev, M, out_dev) : launch_eval<double, 16>(c, idx_dev, M, out_dev);
    default: return f32 ? launch_eval<float, 32>(c, idx_dev, M, out_dev) : launch_eval<double, 32>(c, idx_dev, M, out_dev);
  }
}

// Which interface tables a context keeps (sizes depend only on the shape and
// |Omega|): every prefix L_j (2 <= j <= d-1) and suffix R_j (1 <= j <= d-2)
// with at most min(2^17, max(4096, 4|Omega|)) rows.  Mode k then takes the
// longest prefix table inside modes < k and the longest suffix table inside
// modes > k.
void ttc_plan_tables(ttc_ctx* c) {
  DevProb& P = c->hp;
  const int m = c->m;
  const long long cap = std::min<long long>(1LL << 17, std::max<long long>(4096, 4LL * std::max(c->N, 1)));
  P.ntab = 0;
  long long row0 = 0;
  auto add = [&](int side, int j, int first, int last) {
    // modes first..last: one code word, row index = their bit fields
    if (P.cword[first] != P.cword[last]) return false;
    const int bits = P.cshift[last] + P.cbits[last] - P.cshift[first];
    if (bits > 17 || (1LL << bits) > cap) return false;
    const int t = P.ntab++;
    P.tab_side[t] = side;
    P.tab_j[t] = j;
    P.tab_rows[t] = 1LL << bits;
    P.tab_row0[t] = row0;
    P.tab_word[t] = P.cword[first];
    P.tab_shift[t] = P.cshift[first];
    P.tab_bits[t] = bits;
    row0 += 1LL << bits;
    return true;
  };
  for (int j = 2; j <= m - 1; ++j)
    if (!add(0, j, 0, j - 1)) break;
  for (int j = m - 2; j >= 1; --j)
    if (!add(1, j, j, m - 1)) break;
  P.tab_total = row0;
  for (int k = 0; k < m; ++k) {
    P.pre_tab[k] = -1;
    P.suf_tab[k] = -1;
    int bestl = 0, bestr = m;
    for (int t = 0; t < P.ntab; ++t) {
      if (P.tab_side[t] == 0 && P.tab_j[t] <= k && P.tab_j[t] > bestl) {
        bestl = P.tab_j[t];
        P.pre_tab[k] = t;
      }
      if (P.tab_side[t] == 1 && P.tab_j[t] >= k + 1 && P.tab_j[t] < bestr) {
        bestr = P.tab_j[t];
        P.suf_tab[k] = t;
      }
    }
  }
}
