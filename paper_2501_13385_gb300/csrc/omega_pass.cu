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
#include <algorithm>

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
// (rows are zero-padded, so entries len..round4(len) read as zero; entries
// beyond are left as they are: callers pass zero-initialised arrays)
template <int R>
__device__ __forceinline__ void load_row(const float* __restrict__ row, int len, float (&out)[R]) {
#pragma unroll
  for (int b = 0; b < R; b += 4) {
    if (b >= len) break;
    float4 v = __ldg(reinterpret_cast<const float4*>(row + b));
    out[b] = v.x;
    out[b + 1] = v.y;
    out[b + 2] = v.z;
    out[b + 3] = v.w;
  }
}
template <int R>
__device__ __forceinline__ void load_row(const double* __restrict__ row, int len, double (&out)[R]) {
#pragma unroll
  for (int b = 0; b < R; b += 2) {
    if (b >= len) break;
    double2 v = __ldg(reinterpret_cast<const double2*>(row + b));
    out[b] = v.x;
    out[b + 1] = v.y;
  }
}

// Loops over ranks run to the compile-time bucket R but leave as soon as the
// problem's rank is reached (the bounds are uniform across the block).

// l <- l T_j(x): row vector times an ra x rb slice (padded layout)
template <typename T, int R>
__device__ __forceinline__ void row_times(const DevProb& P, int j, int x, T (&l)[R]) {
  const int ra = P.r[j], rb = P.r[j + 1];
  const T* S = core_ptr<T>(P, j) + (long long)x * R * R;
  T out[R], row[R];
#pragma unroll
  for (int b = 0; b < R; ++b) {
    out[b] = 0;
    row[b] = 0;
  }
  if (rb == 1) {   // the slice is one contiguous column
    load_row<R>(S, ra, row);
    T acc = 0;
#pragma unroll
    for (int a = 0; a < R; ++a) {
      if (a >= ra) break;
      acc = fma(l[a], row[a], acc);
    }
    out[0] = acc;
  } else {
#pragma unroll
    for (int a = 0; a < R; ++a) {
      if (a >= ra) break;
      load_row<R>(S + a * R, rb, row);
#pragma unroll
      for (int b = 0; b < R; ++b) {
        if (b >= rb) break;
        out[b] = fma(l[a], row[b], out[b]);
      }
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
#pragma unroll
  for (int a = 0; a < R; ++a) {
    out[a] = 0;
    row[a] = 0;
  }
  if (rb == 1) {
    load_row<R>(S, ra, row);
#pragma unroll
    for (int a = 0; a < R; ++a) {
      if (a >= ra) break;
      out[a] = row[a] * rho[0];
    }
  } else {
#pragma unroll
    for (int a = 0; a < R; ++a) {
      if (a >= ra) break;
      load_row<R>(S + a * R, rb, row);
      T acc = 0;
#pragma unroll
      for (int b = 0; b < R; ++b) {
        if (b >= rb) break;
        acc = fma(row[b], rho[b], acc);
      }
      out[a] = acc;
    }
  }
#pragma unroll
  for (int a = 0; a < R; ++a) rho[a] = out[a];
}

template <typename T>
__device__ __forceinline__ T* tab_ptr(const DevProb& P);
template <>
__device__ __forceinline__ float* tab_ptr<float>(const DevProb& P) { return P.tab32; }
template <>
__device__ __forceinline__ double* tab_ptr<double>(const DevProb& P) { return P.tab64; }

// left interface (modes < k), right interface (modes > k) and the entry
// value, with the pass's own slice Ts (row stride R) from shared memory.
// Where an interface table covers a run of modes, one table row replaces
// that part of the chain.
template <typename T, int R>
__device__ __forceinline__ T interfaces(const DevProb& P, int k, const Code& words, const T* Ts, T (&lv)[R],
                                        T (&rv)[R]) {
#pragma unroll
  for (int a = 0; a < R; ++a) {
    lv[a] = 0;
    rv[a] = 0;
  }
  lv[0] = 1;
  rv[0] = 1;
  int j0 = 0;
  const int tl = P.pre_tab[k];
  if (tl >= 0) {
    const int jt = P.tab_j[tl];
    int lin = 0;   // table rows are below 2^17
    for (int j = 0; j < jt; ++j) lin = lin * P.n[j] + code_coord(P, words, j);
    load_row<R>(tab_ptr<T>(P) + (P.tab_row0[tl] + lin) * R, P.r[jt], lv);
    j0 = jt;
  }
  for (int j = j0; j < k; ++j) row_times<T, R>(P, j, code_coord(P, words, j), lv);
  int j1 = P.m;
  const int tr = P.suf_tab[k];
  if (tr >= 0) {
    const int jt = P.tab_j[tr];
    int lin = 0;
    for (int j = jt; j < P.m; ++j) lin = lin * P.n[j] + code_coord(P, words, j);
    load_row<R>(tab_ptr<T>(P) + (P.tab_row0[tr] + lin) * R, P.r[jt], rv);
    j1 = jt;
  }
  for (int j = j1 - 1; j > k; --j) times_col<T, R>(P, j, code_coord(P, words, j), rv);
  const int ra = P.r[k], rb = P.r[k + 1];
  T v = 0;
#pragma unroll
  for (int a = 0; a < R; ++a) {
    if (a >= ra) break;
    T acc = 0;
#pragma unroll
    for (int b = 0; b < R; ++b) {
      if (b >= rb) break;
      acc = fma(Ts[a * R + b], rv[b], acc);
    }
    v = fma(lv[a], acc, v);
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
__device__ __forceinline__ void sample_project_block(const DevProb& P, const int blk) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ts = reinterpret_cast<T*>(smraw);   // R*R: the pass's own slice
  T* wred = Ts + R * R;                   // small ranks: [warps][1 + R*R]
  T* Lg = Ts + R * R;                     // large ranks: [TTC_NT][R]
  T* Rv = Lg + TTC_NT * R;                // large ranks: [TTC_NT][R]

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
    // every warp stages its 32 entries' g*l and r (stride R+1: no bank
    // conflicts), then each lane sums its own output elements over them
    constexpr int S = R + 1;
    constexpr int NA = (R * R + 31) / 32;
    T* wl = wred + (TTC_NT / 32) * (1 + R * R) + warp * 2 * 32 * S;
    T* wr = wl + 32 * S;
    T accv[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) accv[i] = 0;
    T s2 = 0;
    const int no = ra * rb;
    for (int it = 0; it < kEPT; ++it) {
      const int e = beg + it * TTC_NT + tid;
      T lv[R], rv[R];
      T g = 0;
      if (e < end) {
        const Code words = load_code(P, k, e);
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
#pragma unroll
      for (int a = 0; a < R; ++a) {
        if (a >= ra) break;
        wl[lane * S + a] = g * lv[a];
      }
#pragma unroll
      for (int b = 0; b < R; ++b) {
        if (b >= rb) break;
        wr[lane * S + b] = rv[b];
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const int o = lane + 32 * i;
        if (o < no) {
          const int a = o / rb, b = o - (o / rb) * rb;
          T acc = 0;
#pragma unroll 8
          for (int t = 0; t < 32; ++t) acc = fma(wl[t * S + a], wr[t * S + b], acc);
          accv[i] += acc;
        }
      }
      __syncwarp();
    }
    T v = warp_sum(s2);
    if (lane == 0) wred[warp * (1 + R * R)] = v;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int o = lane + 32 * i;
      if (o < no) wred[warp * (1 + R * R) + 1 + o] = accv[i];
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
        const Code words = load_code(P, k, e);
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

template <typename T, int R>
__global__ void __launch_bounds__(TTC_NT) k_sample_project(const DevProb P) {
  sample_project_block<T, R>(P, blockIdx.x);
}

// batched form: one launch covers every problem of a batch; blocks
// [base[p], base[p+1]) belong to problem p
__device__ __forceinline__ int find_problem(const int* __restrict__ base, int nprob, int blk) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// copies a problem descriptor into shared memory (16-byte words)
__device__ __forceinline__ void stage_desc(const DevProb* __restrict__ src, DevProb* dst) {
  static_assert(sizeof(DevProb) % 8 == 0, "descriptor size");
  const uint2* s = reinterpret_cast<const uint2*>(src);
  uint2* d = reinterpret_cast<uint2*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(DevProb) / 8); i += blockDim.x) d[i] = __ldg(s + i);
  __syncthreads();
}

template <typename T, int R>
__global__ void __launch_bounds__(TTC_NT) k_sample_project_batch(const DevProb* __restrict__ probs,
                                                                  const int* __restrict__ base, int nprob) {
  __shared__ __align__(16) DevProb Ps;
  const int p = find_problem(base, nprob, blockIdx.x);
  stage_desc(probs + p, &Ps);
  sample_project_block<T, R>(Ps, blockIdx.x - __ldg(base + p));
}

// one table row per thread: the chain of core slices it stands for
template <typename T, int R>
__device__ __forceinline__ void build_table_row(const DevProb& P, long long g) {
  int t = 0;
  while (t + 1 < P.ntab && g >= P.tab_row0[t + 1]) ++t;
  long long row = g - P.tab_row0[t];
  const int jt = P.tab_j[t];
  T v[R];
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = 0;
  v[0] = 1;
  int len;
  if (P.tab_side[t] == 0) {             // prefix over modes 0..jt-1
    int xs[TTC_MAXM];
    for (int j = jt - 1; j >= 0; --j) {
      xs[j] = (int)(row % P.n[j]);
      row /= P.n[j];
    }
    for (int j = 0; j < jt; ++j) row_times<T, R>(P, j, xs[j], v);
    len = P.r[jt];
  } else {                              // suffix over modes jt..m-1
    int xs[TTC_MAXM];
    for (int j = P.m - 1; j >= jt; --j) {
      xs[j] = (int)(row % P.n[j]);
      row /= P.n[j];
    }
    for (int j = P.m - 1; j >= jt; --j) times_col<T, R>(P, j, xs[j], v);
    len = P.r[jt];
  }
  T* dst = tab_ptr<T>(P) + g * R;
#pragma unroll
  for (int a = 0; a < R; ++a) dst[a] = (a < len) ? v[a] : T(0);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_build_tables(const DevProb P) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < P.tab_total;
       g += (long long)gridDim.x * blockDim.x)
    build_table_row<T, R>(P, g);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_build_tables_batch(const DevProb* __restrict__ probs,
                                                            const long long* __restrict__ base, int nprob,
                                                            long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (__ldg(base + mid) <= g) lo = mid; else hi = mid - 1;
    }
    build_table_row<T, R>(probs[lo], g - __ldg(base + lo));
  }
}

inline int table_blocks(long long rows) {
  long long b = (rows + 255) / 256;
  return (int)(b < 4 * 152 ? (b < 1 ? 1 : b) : 4 * 152);
}

template <typename T>
size_t pass_smem(int R) {
  if (R <= 8) return sizeof(T) * (size_t)(R * R + (TTC_NT / 32) * (1 + R * R) + (TTC_NT / 32) * 2 * 32 * (R + 1));
  return sizeof(T) * (size_t)(R * R + 2 * TTC_NT * R);
}

// sums the chunk partials of every slice (k, x) in chunk order, in FP64; the
// last block then forms ||G_l||^2 = sum_x s_1(x), eps_l and alpha_l
// (step-size form of Theorem 4.1; eps reading in the options)
template <typename T>
__device__ __forceinline__ void segment_reduce_block(const DevProb& P, int blk, int total_blocks) {
  __shared__ int am_last;
  __shared__ double sh[128];
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
  for (int j = 0; j < P.m; ++j) row_times<T, R>(P, j, idx[e * P.m + j], v);
  out[e] = (double)v[0];
}

template <typename T, int R>
int launch_pass(ttc_ctx* c) {
  const DevProb& P = c->hp;
  if (P.ntab > 0) {
    k_build_tables<T, R><<<table_blocks(P.tab_total), 256, 0, c->stream>>>(P);
    TTC_CUDA(cudaGetLastError());
    c->nlaunch += 1;
  }
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
int launch_pass_batch(const BatchGroup& g, cudaStream_t st, int phase) {
  if (phase == 2) {
    if (g.tab_rows > 0)
      k_build_tables_batch<T, R><<<table_blocks(g.tab_rows), 256, 0, st>>>(g.probs, g.tab_base, g.nprob, g.tab_rows);
  } else if (phase == 0) {
    k_sample_project_batch<T, R><<<g.pass_blocks, TTC_NT, pass_smem<T>(R), st>>>(g.probs, g.pass_base, g.nprob);
  } else {
    k_segment_reduce_batch<T><<<g.seg_blocks, 128, 0, st>>>(g.probs, g.seg_base, g.nprob);
  }
  TTC_CUDA(cudaGetLastError());
  return TTC_OK;
}

template <typename T, int R>
int opt_in() {
  size_t smem = pass_smem<T>(R);
  if (smem > 48 * 1024) {
    TTC_CUDA(cudaFuncSetAttribute(k_sample_project<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TTC_CUDA(cudaFuncSetAttribute(k_sample_project_batch<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
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

int ttc_launch_omega_pass_batch(const BatchGroup& g, cudaStream_t st, int phase) {
  const bool f32 = (g.prec != TTC_PREC_FP64);
  switch (g.R) {
    case 4: return f32 ? launch_pass_batch<float, 4>(g, st, phase) : launch_pass_batch<double, 4>(g, st, phase);
    case 8: return f32 ? launch_pass_batch<float, 8>(g, st, phase) : launch_pass_batch<double, 8>(g, st, phase);
    case 16: return f32 ? launch_pass_batch<float, 16>(g, st, phase) : launch_pass_batch<double, 16>(g, st, phase);
    default: return f32 ? launch_pass_batch<float, 32>(g, st, phase) : launch_pass_batch<double, 32>(g, st, phase);
  }
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
  for (int j = 2; j <= m - 1; ++j) {
    long long rows = 1;
    bool ok = true;
    for (int i = 0; i < j && ok; ++i) {
      rows *= c->n[i];
      ok = rows <= cap;
    }
    if (!ok) break;
    P.tab_side[P.ntab] = 0;
    P.tab_j[P.ntab] = j;
    P.tab_rows[P.ntab] = rows;
    P.tab_row0[P.ntab] = row0;
    row0 += rows;
    ++P.ntab;
  }
  for (int j = m - 2; j >= 1; --j) {
    long long rows = 1;
    bool ok = true;
    for (int i = j; i < m && ok; ++i) {
      rows *= c->n[i];
      ok = rows <= cap;
    }
    if (!ok) break;
    P.tab_side[P.ntab] = 1;
    P.tab_j[P.ntab] = j;
    P.tab_rows[P.ntab] = rows;
    P.tab_row0[P.ntab] = row0;
    row0 += rows;
    ++P.ntab;
  }
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
