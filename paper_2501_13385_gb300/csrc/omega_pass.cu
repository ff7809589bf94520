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
// partials of each slice in chunk order in FP64.  Core slices are read from
// padded mirrors (row stride = rank bucket, 16-byte aligned) with 16-byte
// loads; the pass's own slice is constant on the chunk and sits in shared
// memory.  Results are bitwise reproducible for a given layout.
#include "ctx.h"

namespace {

template <typename T>
__device__ __forceinline__ const T* core_ptr(const DevProb& P, int k);
template <>
__device__ __forceinline__ const float* core_ptr<float>(const DevProb& P, int k) { return P.core32p[k]; }
template <>
__device__ __forceinline__ const double* core_ptr<double>(const DevProb& P, int k) { return P.core64p[k]; }

template <typename T>
__device__ __forceinline__ T yval(const DevProb& P, int k, int j);
template <>
__device__ __forceinline__ float yval<float>(const DevProb& P, int k, int j) { return __ldg(P.y32[k] + j); }
template <>
__device__ __forceinline__ double yval<double>(const DevProb& P, int k, int j) { return __ldg(P.y64[k] + j); }

// 16-byte loads of the first `len` entries of a padded row (R a multiple of 4)
template <int R>
__device__ __forceinline__ void load_row(const float* __restrict__ row, int len, float (&out)[R]) {
#pragma unroll
  for (int b = 0; b < R; b += 4) {
    if (b < len) {
      float4 v = __ldg(reinterpret_cast<const float4*>(row + b));
      out[b] = v.x;
      out[b + 1] = v.y;
      out[b + 2] = v.z;
      out[b + 3] = v.w;
    } else {
      out[b] = 0.f;
      out[b + 1] = 0.f;
      out[b + 2] = 0.f;
      out[b + 3] = 0.f;
    }
  }
}
template <int R>
__device__ __forceinline__ void load_row(const double* __restrict__ row, int len, double (&out)[R]) {
#pragma unroll
  for (int b = 0; b < R; b += 2) {
    if (b < len) {
      double2 v = __ldg(reinterpret_cast<const double2*>(row + b));
      out[b] = v.x;
      out[b + 1] = v.y;
    } else {
      out[b] = 0.0;
      out[b + 1] = 0.0;
    }
  }
}

// l <- l T_j(x): row vector times an ra x rb slice (padded layout)
template <typename T, int R>
__device__ __forceinline__ void row_times(const DevProb& P, int j, int x, T (&l)[R]) {
  const int ra = P.r[j], rb = P.r[j + 1];
  const T* S = core_ptr<T>(P, j) + (long long)x * R * R;
  T out[R], row[R];
  if (rb == 1) {   // the slice is one contiguous column
    load_row<R>(S, ra, row);
    T acc = 0;
#pragma unroll
    for (int a = 0; a < R; ++a) acc = fma(l[a], row[a], acc);
#pragma unroll
    for (int b = 0; b < R; ++b) l[b] = (b == 0) ? acc : T(0);
    return;
  }
#pragma unroll
  for (int b = 0; b < R; ++b) out[b] = 0;
#pragma unroll
  for (int a = 0; a < R; ++a) {
    if (a < ra) {
      load_row<R>(S + a * R, rb, row);
#pragma unroll
      for (int b = 0; b < R; ++b) out[b] = fma(l[a], row[b], out[b]);
    }
  }
#pragma unroll
  for (int b = 0; b < R; ++b) l[b] = out[b];
}

// rho <- T_j(x) rho: an ra x rb slice times a column vector (padded layout)
template <typename T, int R>
__device__ __forceinline__ void times_col(const DevProb& P, int j, int x, T (&rho)[R]) {
  const int ra = P.r[j], rb = P.r[j + 1];
  const T* S = core_ptr<T>(P, j) + (long long)x * R * R;
  T out[R], row[R];
  if (rb == 1) {
    load_row<R>(S, ra, row);
#pragma unroll
    for (int a = 0; a < R; ++a) out[a] = row[a] * rho[0];
  } else {
#pragma unroll
    for (int a = 0; a < R; ++a) {
      T acc = 0;
      if (a < ra) {
        load_row<R>(S + a * R, rb, row);
#pragma unroll
        for (int b = 0; b < R; ++b) acc = fma(row[b], rho[b], acc);
      }
      out[a] = acc;
    }
  }
#pragma unroll
  for (int a = 0; a < R; ++a) rho[a] = out[a];
}

// left interface (modes < k), right interface (modes > k) and the entry
// value, with the pass's own slice Ts (row stride R) from shared memory
template <typename T, int R>
__device__ __forceinline__ T interfaces(const DevProb& P, int k, const uint32_t* words, const T* Ts, T (&lv)[R],
                                        T (&rv)[R]) {
#pragma unroll
  for (int a = 0; a < R; ++a) {
    lv[a] = 0;
    rv[a] = 0;
  }
  lv[0] = 1;
  rv[0] = 1;
  for (int j = 0; j < k; ++j) row_times<T, R>(P, j, code_coord(P, words, j), lv);
  for (int j = P.m - 1; j > k; --j) times_col<T, R>(P, j, code_coord(P, words, j), rv);
  const int ra = P.r[k], rb = P.r[k + 1];
  T v = 0;
#pragma unroll
  for (int a = 0; a < R; ++a) {
    if (a < ra) {
      T acc = 0;
#pragma unroll
      for (int b = 0; b < R; ++b)
        if (b < rb) acc = fma(Ts[a * R + b], rv[b], acc);
      v = fma(lv[a], acc, v);
    }
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kEPT = TTC_CHUNK / TTC_NT;   // entries per thread

// Block = one chunk of at most TTC_CHUNK entries of one mode-k slice x.
// Small ranks (R <= 8): per-thread register accumulators, then warp shuffles
// and a fixed-order sum over warps.  Larger ranks: the rank-one terms of 256
// entries at a time are staged in shared memory and every thread owns a tile
// of the r_k x r_{k+1} output.
template <typename T, int R>
__global__ void __launch_bounds__(TTC_NT) k_sample_project(const DevProb P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ts = reinterpret_cast<T*>(smraw);   // R*R: the pass's own slice
  T* wred = Ts + R * R;                   // small ranks: [warps][1 + R*R]
  T* Lg = Ts + R * R;                     // large ranks: [TTC_NT][R]
  T* Rv = Lg + TTC_NT * R;                // large ranks: [TTC_NT][R]

  const int blk = blockIdx.x;
  int k = 0;
  while (k + 1 < P.m && blk >= P.chunk_base[k + 1]) ++k;
  const int c = blk - P.chunk_base[k];
  const int x = P.cseg[k][c];
  const int beg = P.seg[k][x] + (c - P.cfirst[k][x]) * TTC_CHUNK;
  const int end = min(beg + TTC_CHUNK, P.seg[k][x + 1]);
  const int ra = P.r[k], rb = P.r[k + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    const T* S = core_ptr<T>(P, k) + (long long)x * R * R;
    for (int i = tid; i < R * R; i += TTC_NT) {
      int a = i / R, b = i - (i / R) * R;
      Ts[i] = (a < ra && b < rb) ? S[pad_idx(P, k, a, b)] : T(0);
    }
  }
  __syncthreads();
  const int nout = 1 + ra * rb;
  T* out = reinterpret_cast<T*>(P.part) + (long long)(P.chunk_base[k] + c) * P.part_stride;

  if constexpr (R <= 8) {
    T acc[R][R];
    T s2 = 0;
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] = 0;
    for (int it = 0; it < kEPT; ++it) {
      const int e = beg + it * TTC_NT + tid;
      if (e < end) {
        uint32_t words[4];
        for (int w = 0; w < P.W; ++w) words[w] = __ldg(P.code[k] + (long long)e * P.W + w);
        T lv[R], rv[R];
        T v = interfaces<T, R>(P, k, words, Ts, lv, rv);
        T g = v - yval<T>(P, k, e);
        if (P.keep_residual && k == 0) P.g[P.perm[0][e]] = (double)g;
        s2 = fma(g, g, s2);
#pragma unroll
        for (int a = 0; a < R; ++a) {
          T gl = g * lv[a];
#pragma unroll
          for (int b = 0; b < R; ++b) acc[a][b] = fma(gl, rv[b], acc[a][b]);
        }
      }
    }
    T v = warp_sum(s2);
    if (lane == 0) wred[warp * (1 + R * R)] = v;
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) {
        if (a < ra && b < rb) {
          T t = warp_sum(acc[a][b]);
          if (lane == 0) wred[warp * (1 + R * R) + 1 + a * rb + b] = t;
        }
      }
    __syncthreads();
    for (int j = tid; j < nout; j += TTC_NT) {
      T tot = 0;
      for (int w = 0; w < TTC_NT / 32; ++w) tot += wred[w * (1 + R * R) + j];
      out[j] = tot;
    }
  } else {
    // output tiles: R == 16 -> one element per thread, R == 32 -> 2 x 2
    constexpr int TA = (R == 32) ? 2 : 1;
    constexpr int TB = (R == 32) ? 2 : 1;
    const int a0 = (tid / (R / TB)) * TA, b0 = (tid % (R / TB)) * TB;
    T acc[TA][TB];
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
      for (int j = 0; j < TB; ++j) acc[i][j] = 0;
    T s2 = 0;
    for (int it = 0; it < kEPT; ++it) {
      const int e = beg + it * TTC_NT + tid;
      T lv[R], rv[R];
      T g = 0;
      if (e < end) {
        uint32_t words[4];
        for (int w = 0; w < P.W; ++w) words[w] = __ldg(P.code[k] + (long long)e * P.W + w);
        T v = interfaces<T, R>(P, k, words, Ts, lv, rv);
        g = v - yval<T>(P, k, e);
        if (P.keep_residual && k == 0) P.g[P.perm[0][e]] = (double)g;
      } else {
#pragma unroll
        for (int a = 0; a < R; ++a) {
          lv[a] = 0;
          rv[a] = 0;
        }
      }
      s2 = fma(g, g, s2);
      __syncthreads();
#pragma unroll
      for (int a = 0; a < R; ++a) {
        Lg[tid * R + a] = g * lv[a];
        Rv[tid * R + a] = rv[a];
      }
      __syncthreads();
      const int cnt = min(TTC_NT, max(0, end - (beg + it * TTC_NT)));
      for (int t = 0; t < cnt; ++t) {
        T la[TA], rbv[TB];
#pragma unroll
        for (int i = 0; i < TA; ++i) la[i] = Lg[t * R + a0 + i];
#pragma unroll
        for (int j = 0; j < TB; ++j) rbv[j] = Rv[t * R + b0 + j];
#pragma unroll
        for (int i = 0; i < TA; ++i)
#pragma unroll
          for (int j = 0; j < TB; ++j) acc[i][j] = fma(la[i], rbv[j], acc[i][j]);
      }
    }
    T v = warp_sum(s2);
    __syncthreads();
    if (lane == 0) Lg[warp] = v;
    __syncthreads();
    if (tid == 0) {
      T tot = 0;
      for (int w = 0; w < TTC_NT / 32; ++w) tot += Lg[w];
      out[0] = tot;
    }
#pragma unroll
    for (int i = 0; i < TA; ++i)
#pragma unroll
      for (int j = 0; j < TB; ++j) {
        const int a = a0 + i, b = b0 + j;
        if (a < ra && b < rb) out[1 + a * rb + b] = acc[i][j];
      }
  }
}

template <typename T>
size_t pass_smem(int R) {
  if (R <= 8) return sizeof(T) * (size_t)(R * R + (TTC_NT / 32) * (1 + R * R));
  return sizeof(T) * (size_t)(R * R + 2 * TTC_NT * R);
}

// sums the chunk partials of every slice (k, x) in chunk order, in FP64; the
// last block then forms ||G_l||^2 = sum_x s_1(x), eps_l and alpha_l
// (step-size form of Theorem 4.1; eps reading in the options)
template <typename T>
__global__ void k_segment_reduce(const DevProb P, int total_blocks) {
  __shared__ int am_last;
  __shared__ double sh[128];
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
    for (int cc = c0; cc < c1; ++cc) acc += (double)part[(long long)cc * P.part_stride + j];
    if (j == 0)
      P.s[k][x] = acc;
    else
      P.E[k][(long long)x * ra * rb + (j - 1)] = acc;
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
    const double alpha = P.scal[SC_ALPHA_OVR] > 0.0 ? P.scal[SC_ALPHA_OVR] : P.scal[SC_ALPHA_SCALE] * sqrt(eps) / P.p;
    P.scal[SC_G2] = g2;
    P.scal[SC_EPS] = eps;
    P.scal[SC_ALPHA] = alpha;
    if (!isfinite(g2)) atomicOr(P.flags, 1u);
    P.counters[0] = 0;
  }
}

template <typename T, int R>
__global__ void k_eval(const DevProb P, const int32_t* __restrict__ idx, long long M, double* __restrict__ out) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= M) return;
  T v[R];
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = 0;
  v[0] = 1;
  for (int j = 0; j < P.m; ++j) row_times<T, R>(P, j, idx[e * P.m + j], v);
  out[e] = (double)v[0];
}

template <typename T, int R>
int launch_pass(ttc_ctx* c) {
  const DevProb& P = c->hp;
  int nblocks = P.chunk_base[P.m];
  size_t smem = pass_smem<T>(R);
  // when profiling, the kernel is bracketed by events; inside a stream capture
  // they become event-record nodes of the graph, so replays are timed too
  unsigned evflags = cudaEventRecordDefault;
  if (c->prof) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TTC_CUDA(cudaStreamIsCapturing(c->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive) evflags = cudaEventRecordExternal;
    TTC_CUDA(cudaEventRecordWithFlags(c->ev_beg, c->stream, evflags));
  }
  k_sample_project<T, R><<<nblocks, TTC_NT, smem, c->stream>>>(P);
  TTC_CUDA(cudaGetLastError());
  if (c->prof) TTC_CUDA(cudaEventRecordWithFlags(c->ev_end, c->stream, evflags));
  int nseg = 0;
  for (int k = 0; k < P.m; ++k) nseg += P.n[k];
  k_segment_reduce<T><<<nseg, 128, 0, c->stream>>>(P, nseg);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 2;
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
  size_t smem = pass_smem<T>(R);
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
