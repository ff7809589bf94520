// The sampled pass over Omega, one pass per mode k (Algorithm 2, first
// lines, with the sparse factor of Lemma 3.5 Eq. (tsp in nm)):
//   v_w  = T_1(x_1) ... T_d(x_d)                   (Eq. (TT Core))
//   g_w  = v_w - y_w                               (entries of G_l = P_Omega(T_l - T*))
//   s_k(x)  = sum_{w : x_k = x} g_w^2              (diag(M_k(G_l) M_k(G_l)^T), Section 3.2)
//   E_k(x)  = sum_{w : x_k = x} g_w l_{k-1}(w)^T r_{k+1}(w)^T
// with l_{k-1} = T^{<=k-1}(x_<k) and r_{k+1} = T^{>=k+1}(x_>k) the interfaces
// of the iterate's own cores.  The weights of the metric are constant on a
// mode-k slice, so they are applied after the reduction (dense stage).
//
// Layout: entries of mode k are stored in mode-k order, so a slice x is a
// contiguous segment; segments are cut into chunks of TTC_CHUNK entries and
// one block reduces one chunk (no atomics); a second kernel sums the chunk
// partials of each slice in chunk order in FP64.  Results are bitwise
// reproducible for a given layout.
#include "ctx.h"

namespace {

template <typename T>
__device__ __forceinline__ T ldg_t(const T* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ const T* core_ptr(const DevProb& P, int k);
template <>
__device__ __forceinline__ const float* core_ptr<float>(const DevProb& P, int k) { return P.core32[k]; }
template <>
__device__ __forceinline__ const double* core_ptr<double>(const DevProb& P, int k) { return P.core64[k]; }

template <typename T>
__device__ __forceinline__ T yval(const DevProb& P, int k, int j);
template <>
__device__ __forceinline__ float yval<float>(const DevProb& P, int k, int j) { return __ldg(P.y32[k] + j); }
template <>
__device__ __forceinline__ double yval<double>(const DevProb& P, int k, int j) { return __ldg(P.y64[k] + j); }

// out[b] = sum_a in[a] M[a][b]  (row vector times an ra x rb slice)
template <typename T, int R>
__device__ __forceinline__ void row_times(const T* __restrict__ M, int ra, int rb, const T (&in)[R], T (&out)[R]) {
#pragma unroll
  for (int b = 0; b < R; ++b) {
    T acc = 0;
#pragma unroll
    for (int a = 0; a < R; ++a)
      if (a < ra && b < rb) acc = fma(in[a], ldg_t(M + a * rb + b), acc);
    out[b] = acc;
  }
}

// out[a] = sum_b M[a][b] in[b]  (an ra x rb slice times a column vector)
template <typename T, int R>
__device__ __forceinline__ void times_col(const T* __restrict__ M, int ra, int rb, const T (&in)[R], T (&out)[R]) {
#pragma unroll
  for (int a = 0; a < R; ++a) {
    T acc = 0;
#pragma unroll
    for (int b = 0; b < R; ++b)
      if (a < ra && b < rb) acc = fma(ldg_t(M + a * rb + b), in[b], acc);
    out[a] = acc;
  }
}

// Evaluates the left interface (modes < k), right interface (modes > k) and
// the entry value for the coordinates held in `words`.
template <typename T, int R>
__device__ __forceinline__ T interfaces(const DevProb& P, int k, const uint32_t* words, T (&lv)[R], T (&rv)[R]) {
  const int m = P.m;
  T tmp[R];
#pragma unroll
  for (int a = 0; a < R; ++a) { lv[a] = 0; rv[a] = 0; }
  lv[0] = 1;
  rv[0] = 1;
  for (int j = 0; j < k; ++j) {
    int x = code_coord(P, words, j);
    const T* M = core_ptr<T>(P, j) + (long long)x * P.r[j] * P.r[j + 1];
    row_times<T, R>(M, P.r[j], P.r[j + 1], lv, tmp);
#pragma unroll
    for (int a = 0; a < R; ++a) lv[a] = tmp[a];
  }
  for (int j = m - 1; j > k; --j) {
    int x = code_coord(P, words, j);
    const T* M = core_ptr<T>(P, j) + (long long)x * P.r[j] * P.r[j + 1];
    times_col<T, R>(M, P.r[j], P.r[j + 1], rv, tmp);
#pragma unroll
    for (int a = 0; a < R; ++a) rv[a] = tmp[a];
  }
  int x = code_coord(P, words, k);
  const T* M = core_ptr<T>(P, k) + (long long)x * P.r[k] * P.r[k + 1];
  times_col<T, R>(M, P.r[k], P.r[k + 1], rv, tmp);
  T v = 0;
#pragma unroll
  for (int a = 0; a < R; ++a) v = fma(lv[a], tmp[a], v);
  return v;
}

template <typename T, int R>
__global__ void __launch_bounds__(TTC_NT) k_sample_project(const DevProb P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Lg = reinterpret_cast<T*>(smraw);     // [TTC_CHUNK][R]: g * l
  T* Rv = Lg + TTC_CHUNK * R;               // [TTC_CHUNK][R]: r
  T* G2 = Rv + TTC_CHUNK * R;               // [TTC_CHUNK]:    g^2

  const int blk = blockIdx.x;
  int k = 0;
  while (k + 1 < P.m && blk >= P.chunk_base[k + 1]) ++k;
  const int c = blk - P.chunk_base[k];
  const int x = P.cseg[k][c];
  const int beg = P.seg[k][x] + (c - P.cfirst[k][x]) * TTC_CHUNK;
  const int end = min(beg + TTC_CHUNK, P.seg[k][x + 1]);
  const int ra = P.r[k], rb = P.r[k + 1];
  const int tid = threadIdx.x;
  const int e = beg + tid;

  T lv[R], rv[R];
  T g = 0;
  if (e < end) {
    uint32_t words[4];
    for (int w = 0; w < P.W; ++w) words[w] = __ldg(P.code[k] + (long long)e * P.W + w);
    T v = interfaces<T, R>(P, k, words, lv, rv);
    g = v - yval<T>(P, k, e);
    if (P.keep_residual && k == 0) P.g[P.perm[0][e]] = (double)g;
  } else {
#pragma unroll
    for (int a = 0; a < R; ++a) { lv[a] = 0; rv[a] = 0; }
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    Lg[tid * R + a] = g * lv[a];
    Rv[tid * R + a] = rv[a];
  }
  G2[tid] = g * g;
  __syncthreads();

  const int nout = 1 + ra * rb;
  const int cnt = end - beg;
  T* out = reinterpret_cast<T*>(P.part) + (long long)(P.chunk_base[k] + c) * P.part_stride;
  for (int j = tid; j < nout; j += TTC_NT) {
    T acc = 0;
    if (j == 0) {
      for (int t = 0; t < cnt; ++t) acc += G2[t];
    } else {
      int a = (j - 1) / rb, b = (j - 1) - ((j - 1) / rb) * rb;
      for (int t = 0; t < cnt; ++t) acc = fma(Lg[t * R + a], Rv[t * R + b], acc);
    }
    out[j] = acc;
  }
}

// sums the chunk partials of every slice (k, x) in chunk order, in FP64
template <typename T>
__global__ void k_segment_reduce(const DevProb P) {
  int blk = blockIdx.x;
  int k = 0;
  while (k < P.m - 1 && blk >= P.n[k]) {
    blk -= P.n[k];
    ++k;
  }
  const int x = blk;
  const int ra = P.r[k], rb = P.r[k + 1];
  const int nout = 1 + ra * rb;
  const int c0 = P.cfirst[k][x], c1 = P.cfirst[k][x + 1];
  const T* part = reinterpret_cast<const T*>(P.part) + (long long)P.chunk_base[k] * P.part_stride;
  for (int j = threadIdx.x; j < nout; j += blockDim.x) {
    double acc = 0.0;
    for (int c = c0; c < c1; ++c) acc += (double)part[(long long)c * P.part_stride + j];
    if (j == 0)
      P.s[k][x] = acc;
    else
      P.E[k][(long long)x * ra * rb + (j - 1)] = acc;
  }
}

template <typename T, int R>
__global__ void k_eval(const DevProb P, const int32_t* __restrict__ idx, long long M, double* __restrict__ out) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= M) return;
  T v[R], tmp[R];
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = 0;
  v[0] = 1;
  for (int j = 0; j < P.m; ++j) {
    int x = idx[e * P.m + j];
    const T* Mj = core_ptr<T>(P, j) + (long long)x * P.r[j] * P.r[j + 1];
    row_times<T, R>(Mj, P.r[j], P.r[j + 1], v, tmp);
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = tmp[a];
  }
  out[e] = (double)v[0];
}

template <typename T, int R>
int launch_pass(ttc_ctx* c) {
  const DevProb& P = c->hp;
  int nblocks = P.chunk_base[P.m];
  size_t smem = sizeof(T) * (2 * TTC_CHUNK * R + TTC_CHUNK);
  auto kern = k_sample_project<T, R>;
  // when profiling, the kernel is bracketed by events; inside a stream capture
  // they become event-record nodes of the graph, so replays are timed too
  unsigned evflags = cudaEventRecordDefault;
  if (c->prof) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TTC_CUDA(cudaStreamIsCapturing(c->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) evflags = cudaEventRecordExternal;
    TTC_CUDA(cudaEventRecordWithFlags(c->ev_beg, c->stream, evflags));
  }
  kern<<<nblocks, TTC_NT, smem, c->stream>>>(P);
  TTC_CUDA(cudaGetLastError());
  if (c->prof) TTC_CUDA(cudaEventRecordWithFlags(c->ev_end, c->stream, evflags));
  c->nlaunch += 2;
  int nseg = 0;
  for (int k = 0; k < P.m; ++k) nseg += P.n[k];
  k_segment_reduce<T><<<nseg, 128, 0, c->stream>>>(P);
  TTC_CUDA(cudaGetLastError());
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
int opt_in() {
  size_t smem = sizeof(T) * (2 * TTC_CHUNK * R + TTC_CHUNK);
  if (smem > 48 * 1024)
    TTC_CUDA(cudaFuncSetAttribute(k_sample_project<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return TTC_OK;
}

}  // namespace

// one-time kernel attributes (outside any stream capture)
int ttc_prepare_omega_pass() {
  TTC_TRY((opt_in<float, 4>()));
  TTC_TRY((opt_in<float, 8>()));
  TTC_TRY((opt_in<float, 16>()));
  TTC_TRY((opt_in<float, 32>()));
  TTC_TRY((opt_in<double, 4>()));
  TTC_TRY((opt_in<double, 8>()));
  TTC_TRY((opt_in<double, 16>()));
  TTC_TRY((opt_in<double, 32>()));
  return TTC_OK;
}

int ttc_launch_omega_pass(ttc_ctx* c, int prec) {
  const bool f32 = (prec != TTC_PREC_FP64);
  switch (c->rank_bucket) {
    case 4: return f32 ? launch_pass<float, 4>(c) : launch_pass<double, 4>(c);
    case 8: return f32 ? launch_pass<float, 8>(c) : launch_pass<double, 8>(c);
    case 16: return f32 ? launch_pass<float, 16>(c) : launch_pass<double, 16>(c);
    default: return f32 ? launch_pass<float, 32>(c) : launch_pass<double, 32>(c);
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
