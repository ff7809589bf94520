// Device code of the sampled pass over Omega, one pass per mode k
// (Algorithm 2, first lines, with the sparse factor of Lemma 3.5
// Eq. (tsp in nm)):
//   v_w  = T_1(x_1) ... T_d(x_d)                   (Eq. (TT Core))
//   g_w  = v_w - y_w                               (entries of G_l = P_Omega(T_l - T*))
//   s_k(x)  = sum_{w : x_k = x} g_w^2              (diag(M_k(G_l) M_k(G_l)^T), Section 3.2)
//   E_k(x)  = sum_{w : x_k = x} g_w l_{k-1}(w)^T r_{k+1}(w)^T
// with l_{k-1} = T^{<=k-1}(x_<k) and r_{k+1} = T^{>=k+1}(x_>k) the interfaces
// of the iterate's own cores.  The weights of the metric are constant on a
// mode-k slice, so they are applied after the reduction (dense stage).
//
// Layout: entries of mode k are stored in mode-k order, so a slice x is a
// contiguous segment; segments are cut into chunks of TTC_CHUNK entries, each
// reduced by one warp (small ranks, and the first and last modes at any rank)
// or one block (interior modes at large ranks) without atomics; a second kernel sums the chunk partials of each slice in chunk
// order in FP64.  Core slices are read from padded mirrors (row stride R =
// rank bucket, 16-byte aligned) with 16-byte loads; the pass's own slice is
// constant on a chunk and sits in shared memory.
//
// Two compile-time sizes: R, the row stride of the padded storage (4, 8, 16,
// 32), and RC <= R, the size of the register arrays (the largest TT-rank of
// the problem for small ranks, R for large).  Loops stop at the runtime ranks
// of each mode, so a problem computes the same values, bitwise, with any RC
// at least its largest rank.  Results are reproducible for a given layout.
#pragma once

#include "ctx.h"

namespace ttc_pass {

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

template <typename T>
__device__ __forceinline__ T* tab_ptr(const DevProb& P);
template <>
__device__ __forceinline__ float* tab_ptr<float>(const DevProb& P) { return P.tab32; }
template <>
__device__ __forceinline__ double* tab_ptr<double>(const DevProb& P) { return P.tab64; }

// 32-byte read-only global loads (sm_100 and later); the address must be
// 32-byte aligned
__device__ __forceinline__ void ldg32B(const float* p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void ldg32B(const double* p, double (&v)[4]) {
  asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
               : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
               : "l"(p));
}

// Loads the first min(len, RC) entries of a zero-padded row in vectors:
// 32 bytes at a time from global memory where the row's padded storage
// holds them (RC above 4 floats / 2 doubles: rows are then padded to 8
// floats / 4 doubles and 32-byte aligned), else 16 bytes.  Entries from len
// on are left as they are: callers pass zero-initialised arrays.
template <int RC, bool kGlobal>
__device__ __forceinline__ void load_row(const float* __restrict__ row, int len, float (&out)[RC]) {
  if constexpr (kGlobal && RC > 4) {
#pragma unroll
    for (int b = 0; b < RC; b += 8) {
      if (b >= len) break;
      float v[8];
      ldg32B(row + b, v);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (b + i < RC) out[b + i] = v[i];
    }
  } else {
#pragma unroll
    for (int b = 0; b < RC; b += 4) {
      if (b >= len) break;
      const float4 v = kGlobal ? __ldg(reinterpret_cast<const float4*>(row + b))
                               : *reinterpret_cast<const float4*>(row + b);
      out[b] = v.x;
      if (b + 1 < RC) out[b + 1] = v.y;
      if (b + 2 < RC) out[b + 2] = v.z;
      if (b + 3 < RC) out[b + 3] = v.w;
    }
  }
}
template <int RC, bool kGlobal>
__device__ __forceinline__ void load_row(const double* __restrict__ row, int len, double (&out)[RC]) {
  if constexpr (kGlobal && RC > 2) {
#pragma unroll
    for (int b = 0; b < RC; b += 4) {
      if (b >= len) break;
      double v[4];
      ldg32B(row + b, v);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (b + i < RC) out[b + i] = v[i];
    }
  } else {
#pragma unroll
    for (int b = 0; b < RC; b += 2) {
      if (b >= len) break;
      const double2 v = kGlobal ? __ldg(reinterpret_cast<const double2*>(row + b))
                                : *reinterpret_cast<const double2*>(row + b);
      out[b] = v.x;
      if (b + 1 < RC) out[b + 1] = v.y;
    }
  }
}

// L2 eviction policies: the streamed codes and values are read once per pass
// (evict first, no L1 allocation), the interface rows are gathered many times
// (evict last), so the stream does not push the tables out of L2
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

// load_row for gathered interface rows, with an L2 policy (rows padded and
// aligned as for load_row)
template <int RC>
__device__ __forceinline__ void load_row_hint(const float* row, int len, float (&out)[RC], uint64_t pol) {
  if constexpr (RC > 4) {
#pragma unroll
    for (int b = 0; b < RC; b += 8) {
      if (b >= len) break;
      float v[8];
      asm("ld.global.nc.L2::cache_hint.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
          : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
          : "l"(row + b), "l"(pol));
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (b + i < RC) out[b + i] = v[i];
    }
  } else {
    float v[4];
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
        : "l"(row), "l"(pol));
#pragma unroll
    for (int i = 0; i < RC; ++i) out[i] = v[i];
  }
}
template <int RC>
__device__ __forceinline__ void load_row_hint(const double* row, int len, double (&out)[RC], uint64_t pol) {
  if constexpr (RC > 2) {
#pragma unroll
    for (int b = 0; b < RC; b += 4) {
      if (b >= len) break;
      double v[4];
      asm("ld.global.nc.L2::cache_hint.v4.f64 {%0,%1,%2,%3}, [%4], %5;"
          : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
          : "l"(row + b), "l"(pol));
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (b + i < RC) out[b + i] = v[i];
    }
  } else {
    double v[2];
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(v[0]), "=d"(v[1]) : "l"(row), "l"(pol));
#pragma unroll
    for (int i = 0; i < RC; ++i) out[i] = v[i];
  }
}

template <typename T, int RC>
__device__ __forceinline__ void zero(T (&v)[RC]) {
#pragma unroll
  for (int a = 0; a < RC; ++a) v[a] = 0;
}

// l <- l T_j(x): row vector times an ra x rb slice (padded layout, stride R)
template <typename T, int R, int RC>
__device__ __forceinline__ void row_times(const DevProb& P, int j, int x, T (&l)[RC]) {
  const int ra = P.r[j], rb = P.r[j + 1];
  const T* S = core_ptr<T>(P, j) + (long long)x * R * R;
  T out[RC], row[RC];
  zero(out);
  zero(row);
  if (rb == 1) {   // the slice is one contiguous column
    load_row<RC, true>(S, ra, row);
    T acc = 0;
#pragma unroll
    for (int a = 0; a < RC; ++a) {
      if (a >= ra) break;
      acc = fma(l[a], row[a], acc);
    }
    out[0] = acc;
  } else {
#pragma unroll
    for (int a = 0; a < RC; ++a) {
      if (a >= ra) break;
      load_row<RC, true>(S + a * R, rb, row);
#pragma unroll
      for (int b = 0; b < RC; ++b) {
        if (b >= rb) break;
        out[b] = fma(l[a], row[b], out[b]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < RC; ++b) l[b] = out[b];
}

// rho <- T_j(x) rho: an ra x rb slice times a column vector (padded layout)
template <typename T, int R, int RC>
__device__ __forceinline__ void times_col(const DevProb& P, int j, int x, T (&rho)[RC]) {
  const int ra = P.r[j], rb = P.r[j + 1];
  const T* S = core_ptr<T>(P, j) + (long long)x * R * R;
  T out[RC], row[RC];
  zero(out);
  zero(row);
  if (rb == 1) {
    load_row<RC, true>(S, ra, row);
#pragma unroll
    for (int a = 0; a < RC; ++a) {
      if (a >= ra) break;
      out[a] = row[a] * rho[0];
    }
  } else {
#pragma unroll
    for (int a = 0; a < RC; ++a) {
      if (a >= ra) break;
      load_row<RC, true>(S + a * R, rb, row);
      T acc = 0;
#pragma unroll
      for (int b = 0; b < RC; ++b) {
        if (b >= rb) break;
        acc = fma(row[b], rho[b], acc);
      }
      out[a] = acc;
    }
  }
#pragma unroll
  for (int a = 0; a < RC; ++a) rho[a] = out[a];
}

// l^T Ts r for the pass's own slice Ts (ra x rb, row stride R, zero-padded)
// in shared memory, a row at a time with 16-byte loads (the same rows for
// every lane: broadcasts)
template <typename T, int R, int RC>
__device__ __forceinline__ T slice_value(const T* Ts, int ra, int rb, const T (&lv)[RC], const T (&rv)[RC]) {
  T v = 0;
#pragma unroll
  for (int a = 0; a < RC; ++a) {
    if (a >= ra) break;
    T row[RC];
    zero(row);
    load_row<RC, false>(Ts + a * R, rb, row);
    T acc = 0;
#pragma unroll
    for (int b = 0; b < RC; ++b) {
      if (b >= rb) break;
      acc = fma(row[b], rv[b], acc);
    }
    v = fma(lv[a], acc, v);
  }
  return v;
}

// row of interface table t for an entry: its modes' bit fields
__device__ __forceinline__ int tab_index(const DevProb& P, const Code& words, int t) {
  return (int)((words.word(P.tab_word[t]) >> P.tab_shift[t]) & ((1u << P.tab_bits[t]) - 1u));
}

// left interface (modes < k), right interface (modes > k) and the entry
// value.  Where an interface table covers a run of modes, one table row
// (stride R) replaces that part of the chain.
template <typename T, int R, int RC>
__device__ __forceinline__ T interfaces(const DevProb& P, int k, const Code& words, const T* Ts, T (&lv)[RC],
                                        T (&rv)[RC]) {
  zero(lv);
  zero(rv);
  lv[0] = 1;
  rv[0] = 1;
  int j0 = 0;
  const int tl = P.pre_tab[k];
  if (tl >= 0) {
    const int jt = P.tab_j[tl];
    load_row<RC, true>(tab_ptr<T>(P) + (P.tab_row0[tl] + tab_index(P, words, tl)) * R, P.r[jt], lv);
    j0 = jt;
  }
  for (int j = j0; j < k; ++j) row_times<T, R, RC>(P, j, code_coord(P, words, j), lv);
  int j1 = P.m;
  const int tr = P.suf_tab[k];
  if (tr >= 0) {
    const int jt = P.tab_j[tr];
    load_row<RC, true>(tab_ptr<T>(P) + (P.tab_row0[tr] + tab_index(P, words, tr)) * R, P.r[jt], rv);
    j1 = jt;
  }
  for (int j = j1 - 1; j > k; --j) times_col<T, R, RC>(P, j, code_coord(P, words, j), rv);
  return slice_value<T, R, RC>(Ts, P.r[k], P.r[k + 1], lv, rv);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kEPT = TTC_CHUNK / TTC_NT;   // entries per thread (large ranks)
constexpr int kWarps = TTC_NT / 32;         // chunks per block (small ranks)

__host__ __device__ constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : 2 * pow2_at_least((n + 1) / 2); }
__host__ __device__ constexpr int log2_exact(int n) { return n <= 1 ? 0 : 1 + log2_exact(n / 2); }

// Sum of N = 2^p per-lane values over the 32 lanes of a warp by a halving
// butterfly.  While more than one value is left, the step with offset o has
// every lane keep one half of its values, send the other half to lane ^ o
// and add what it receives; the remaining offsets sum the last value.
// Afterwards v[0] (and v[1] when N = 64) of lane L hold the totals of value
// L >> (5 - p) (N <= 32) or of values 2L and 2L+1 (N = 64).  Every total is
// the same balanced tree over the lanes whatever N is.
template <typename T, int N, int C, int O>
__device__ __forceinline__ void butterfly_step(T (&v)[N], int lane) {
  if constexpr (O >= 1) {
    if constexpr (C >= 2) {
      const bool up = (lane & O) != 0;
      constexpr int h = C / 2;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const T send = up ? v[i] : v[i + h];
        const T keep = up ? v[i + h] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      butterfly_step<T, N, h, O / 2>(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      butterfly_step<T, N, 1, O / 2>(v, lane);
    }
  }
}

// Sums the per-lane accumulators of a warp and writes the chunk partial
// out[1 + a*rb + b].  Accumulator i stands for (a, b) = (0, i) when KIND is 0
// (first mode, r_{k-1} = 1), (i, 0) when KIND is 1 (last mode, r_k = 1) and
// (i / RC, i % RC) otherwise.
template <typename T, int NV, int KIND, int RC>
__device__ __forceinline__ void store_partials(T (&acc)[NV], int lane, T* out, int ra, int rb) {
  butterfly_step<T, NV, NV, 16>(acc, lane);
  auto put = [&](int o, T v) {
    int a, b;
    if constexpr (KIND == 0) {
      a = 0;
      b = o;
    } else if constexpr (KIND == 1) {
      a = o;
      b = 0;
    } else {
      a = o / RC;
      b = o % RC;
    }
    if (a < ra && b < rb) out[1 + a * rb + b] = v;
  };
  if constexpr (NV == 64) {
    put(2 * lane, acc[0]);
    put(2 * lane + 1, acc[1]);
  } else {
    constexpr int sh = 5 - log2_exact(NV);
    if ((lane & ((1 << sh) - 1)) == 0) put(lane >> sh, acc[0]);
  }
}

// where an interface comes from as one padded row: row index = a bit field
// of the entry's code, row at base + index * stride
template <typename T>
struct RowSrc {
  const T* base;
  int word, shift;
  unsigned mask;
  int stride;
};
template <typename T>
__device__ __forceinline__ const T* row_of(const RowSrc<T>& s, const Code& w) {
  return s.base + (long long)((w.word(s.word) >> s.shift) & s.mask) * s.stride;
}

// The left interface of mode k as one row: the prefix table over exactly
// modes 0..k-1, or core 0's slice when k = 1 (a 1 x r_1 row)
template <typename T>
__device__ __forceinline__ bool left_src(const DevProb& P, int k, RowSrc<T>& s) {
  const int t = P.pre_tab[k];
  if (t >= 0 && P.tab_j[t] == k) {
    s = {tab_ptr<T>(P) + P.tab_row0[t] * P.R, P.tab_word[t], P.tab_shift[t], (1u << P.tab_bits[t]) - 1u, P.R};
    return true;
  }
  if (k == 1) {
    s = {core_ptr<T>(P, 0), P.cword[0], P.cshift[0], (1u << P.cbits[0]) - 1u, P.R * P.R};
    return true;
  }
  return false;
}
// The right interface of mode k as one row: the suffix table over exactly
// modes k+1..d-1, or the last core's slice when k = d-2 (an r_{d-1} column,
// stored contiguously)
template <typename T>
__device__ __forceinline__ bool right_src(const DevProb& P, int k, RowSrc<T>& s) {
  const int t = P.suf_tab[k];
  if (t >= 0 && P.tab_j[t] == k + 1) {
    s = {tab_ptr<T>(P) + P.tab_row0[t] * P.R, P.tab_word[t], P.tab_shift[t], (1u << P.tab_bits[t]) - 1u, P.R};
    return true;
  }
  if (k == P.m - 2) {
    const int j = P.m - 1;
    s = {core_ptr<T>(P, j), P.cword[j], P.cshift[j], (1u << P.cbits[j]) - 1u, P.R * P.R};
    return true;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ const T* y_ptr(const DevProb& P, int k);
template <>
__device__ __forceinline__ const float* y_ptr<float>(const DevProb& P, int k) { return P.y32[k]; }
template <>
__device__ __forceinline__ const double* y_ptr<double>(const DevProb& P, int k) { return P.y64[k]; }

__device__ __forceinline__ Code load_code_at(const uint32_t* __restrict__ p, int W, int e, uint64_t pol) {
  Code c;
  p += (long long)e * W;
  c.w0 = ld_stream(p, pol);
  c.w1 = W > 1 ? ld_stream(p + 1, pol) : 0u;
  c.w2 = W > 2 ? ld_stream(p + 2, pol) : 0u;
  c.w3 = W > 3 ? ld_stream(p + 3, pol) : 0u;
  return c;
}

// One chunk whose interfaces are each one row (or the identity at the ends
// of the train).  Loops run over the full register size RC: rows, slices and
// tables are zero-padded, so the extra terms add exact zeros.
// KIND 0: first mode (l = 1), KIND 1: last mode (r = 1), KIND 2: interior.
// Every lane takes U entries per iteration (their row gathers in flight
// together) and fetches the next U codes and observations ahead; a lane
// without an entry for a slot gathers a valid row and contributes g = 0.
// The descriptor's loop-invariant fields are read once into registers.
template <typename T, int R, int RC, int KIND, int U>
__device__ __forceinline__ void warp_chunk_rows(const DevProb& P, int k, int beg, int end, const T* Ts,
                                                const RowSrc<T>& ls, const RowSrc<T>& rs, T* out) {
  const int lane = threadIdx.x & 31;
  const uint32_t* __restrict__ code = P.code[k];
  const int W = P.W;
  const T* __restrict__ yk = y_ptr<T>(P, k);
  const bool keep = P.keep_residual && k == 0;
  double* __restrict__ gout = P.g;
  const int* __restrict__ perm0 = P.perm[0];
  const uint64_t pol_stream = policy_evict_first(), pol_rows = policy_evict_last();
  constexpr int NV = pow2_at_least(KIND == 2 ? RC * RC : RC);
  T acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0;
  T tv[RC];   // KIND 0: the slice's row, KIND 1: its column (registers)
  zero(tv);
  if constexpr (KIND == 0) load_row<RC, false>(Ts, RC, tv);
  if constexpr (KIND == 1) {
#pragma unroll
    for (int a = 0; a < RC; ++a) tv[a] = Ts[a * R];
  }
  T s2 = 0;
  Code nw[U];
  T ny[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int eu = beg + lane + 32 * u;
    nw[u] = {0u, 0u, 0u, 0u};
    ny[u] = 0;
    if (eu < end) {
      nw[u] = load_code_at(code, W, eu, pol_stream);
      ny[u] = ld_stream(yk + eu, pol_stream);
    }
  }
  for (int e = beg + lane; e < end; e += 32 * U) {
    Code w[U];
    T yv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      w[u] = nw[u];
      yv[u] = ny[u];
      const int en = e + 32 * (U + u);
      if (en < end) {
        nw[u] = load_code_at(code, W, en, pol_stream);
        ny[u] = ld_stream(yk + en, pol_stream);
      }
    }
    T lv[U][RC], rv[U][RC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      zero(lv[u]);
      zero(rv[u]);
      if constexpr (KIND != 0) load_row_hint<RC>(row_of(ls, w[u]), RC, lv[u], pol_rows);
      if constexpr (KIND != 1) load_row_hint<RC>(row_of(rs, w[u]), RC, rv[u], pol_rows);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      T v = 0;
      if constexpr (KIND == 0) {
#pragma unroll
        for (int b = 0; b < RC; ++b) v = fma(tv[b], rv[u][b], v);
      } else if constexpr (KIND == 1) {
#pragma unroll
        for (int a = 0; a < RC; ++a) v = fma(lv[u][a], tv[a], v);
      } else {
#pragma unroll
        for (int a = 0; a < RC; ++a) {
          T row[RC];
          zero(row);
          load_row<RC, false>(Ts + a * R, RC, row);
          T t = 0;
#pragma unroll
          for (int b = 0; b < RC; ++b) t = fma(row[b], rv[u][b], t);
          v = fma(lv[u][a], t, v);
        }
      }
      const int eu = e + 32 * u;
      const T g = (eu < end) ? v - yv[u] : T(0);
      if (keep && eu < end) gout[perm0[eu]] = (double)g;
      s2 = fma(g, g, s2);
      if constexpr (KIND == 0) {
#pragma unroll
        for (int b = 0; b < RC; ++b) acc[b] = fma(g, rv[u][b], acc[b]);
      } else if constexpr (KIND == 1) {
#pragma unroll
        for (int a = 0; a < RC; ++a) acc[a] = fma(g, lv[u][a], acc[a]);
      } else {
#pragma unroll
        for (int a = 0; a < RC; ++a) {
          const T gl = g * lv[u][a];
#pragma unroll
          for (int b = 0; b < RC; ++b) acc[a * RC + b] = fma(gl, rv[u][b], acc[a * RC + b]);
        }
      }
    }
  }
  s2 = warp_sum(s2);
  if (lane == 0) out[0] = s2;
  store_partials<T, NV, KIND, RC>(acc, lane, out, P.r[k], P.r[k + 1]);
}

// Any other chunk: interfaces through tables and chains of core slices, with
// loops that stop at the runtime ranks.  KIND shapes the accumulators as in
// warp_chunk_rows (0: first mode, 1: last mode, 2: interior).
template <typename T, int R, int RC, int KIND>
__device__ __forceinline__ void warp_chunk_general(const DevProb& P, int k, int beg, int end, const T* Ts, T* out) {
  const int lane = threadIdx.x & 31;
  const int ra = P.r[k], rb = P.r[k + 1];
  constexpr int NV = pow2_at_least(KIND == 2 ? RC * RC : RC);
  T acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0;
  T s2 = 0;
  const bool keep = P.keep_residual && k == 0;
  int e = beg + lane;
  Code nxt_words = {0u, 0u, 0u, 0u};
  T nxt_y = 0;
  if (e < end) {
    nxt_words = load_code(P, k, e);
    nxt_y = yval<T>(P, k, e);
  }
  for (; e < end; e += 32) {
    const Code words = nxt_words;
    const T yv = nxt_y;
    if (e + 32 < end) {
      nxt_words = load_code(P, k, e + 32);
      nxt_y = yval<T>(P, k, e + 32);
    }
    T lv[RC], rv[RC];
    const T g = interfaces<T, R, RC>(P, k, words, Ts, lv, rv) - yv;
    if (keep) P.g[P.perm[0][e]] = (double)g;
    s2 = fma(g, g, s2);
    if constexpr (KIND == 0) {
#pragma unroll
      for (int b = 0; b < RC; ++b) {
        if (b >= rb) break;
        acc[b] = fma(g, rv[b], acc[b]);
      }
    } else if constexpr (KIND == 1) {
#pragma unroll
      for (int a = 0; a < RC; ++a) {
        if (a >= ra) break;
        acc[a] = fma(g, lv[a], acc[a]);
      }
    } else {
#pragma unroll
      for (int a = 0; a < RC; ++a) {
        if (a >= ra) break;
        const T gl = g * lv[a];
#pragma unroll
        for (int b = 0; b < RC; ++b) {
          if (b >= rb) break;
          acc[a * RC + b] = fma(gl, rv[b], acc[a * RC + b]);
        }
      }
    }
  }
  s2 = warp_sum(s2);
  if (lane == 0) out[0] = s2;
  store_partials<T, NV, KIND, RC>(acc, lane, out, ra, rb);
}

// Small ranks (R <= 8): one warp reduces one chunk of at most TTC_CHUNK
// entries of one mode-k slice x.  Each lane takes every 32nd entry (the next
// entry's code and observation are fetched while the current one is
// processed), forms its interfaces and residual, and accumulates the
// rank-one terms g * l_{k-1} r_{k+1}^T and g^2 in registers; a butterfly then
// sums the lanes.  No shared memory beyond the slice, no block barriers.
template <typename T, int R, int RC, int MC>
__device__ __forceinline__ void sample_project_warp(const DevProb& P, const int call, T* Ts) {
  int k = 0;
  if constexpr (MC == PC_FIRST) {
    k = 0;
  } else if constexpr (MC == PC_LAST) {
    k = P.m - 1;
  } else {
    k = 1;
    while (k + 2 < P.m && call >= P.chunk_base[k + 1]) ++k;
  }
  const int c = call - P.chunk_base[k];
  const int x = P.cseg[k][c];
  const int beg = P.seg[k][x] + (c - P.cfirst[k][x]) * TTC_CHUNK;
  const int end = min(beg + TTC_CHUNK, P.seg[k][x + 1]);
  const int ra = P.r[k], rb = P.r[k + 1];
  const int lane = threadIdx.x & 31;
  {
    const T* S = core_ptr<T>(P, k) + (long long)x * R * R;
    for (int i = lane; i < R * R; i += 32) {
      const int a = i / R, b = i % R;
      Ts[i] = (a < ra && b < rb) ? S[pad_idx(P, k, a, b)] : T(0);
    }
  }
  __syncwarp();
  T* out = reinterpret_cast<T*>(P.part) + (long long)(P.chunk_base[k] + c) * P.part_stride;
  RowSrc<T> ls{}, rs{};
  constexpr int U = sizeof(T) == 4 ? 2 : 1;   // FP64 is bound by its FMA rate
  constexpr int KIND = MC == PC_FIRST ? 0 : MC == PC_LAST ? 1 : 2;
  const bool lrow = (KIND == 0) || left_src<T>(P, k, ls);
  const bool rrow = (KIND == 1) || right_src<T>(P, k, rs);
  if (lrow && rrow)
    warp_chunk_rows<T, R, RC, KIND, U>(P, k, beg, end, Ts, ls, rs, out);
  else
    warp_chunk_general<T, R, RC, KIND>(P, k, beg, end, Ts, out);
}

// Large ranks (R >= 16), interior modes: one block reduces one chunk.  Each
// thread forms one entry's interfaces (one gathered row each, or chains of
// core slices), its value and its residual; the value is one dot product
// with a table row when a table covers exactly modes <= k (a prefix row,
// times r) or modes >= k (l times a suffix row), else l^T T_k(x) r.  The
// block stages g*l and r of NE entries in shared memory and thread t
// accumulates OPT = R*R/256 outputs of the r_{k-1} x r_k partial over them:
// column t mod R, rows OPT*(t div R) ... (threads whose rows or column lie
// beyond the ranks skip the accumulation).
template <typename T, int R, int RC>
__device__ __forceinline__ void sample_project_interior(const DevProb& P, const int call) {
  constexpr int NE = TTC_NT;            // entries staged per round
  constexpr int RS = (RC + 3) & ~3;     // staged row length (16-byte multiple)
  constexpr int OPT = (R * R) / TTC_NT; // outputs per thread
  static_assert(OPT >= 1 && OPT * TTC_NT == R * R && RS % OPT == 0, "output tiling");
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ts = reinterpret_cast<T*>(smraw);  // R*R: the pass's own slice
  T* Lg = Ts + R * R;                    // [NE][RS]: g * l
  T* Rv = Lg + NE * RS;                  // [NE][RS]: r
  int k = 1;
  while (k + 2 < P.m && call >= P.chunk_base[k + 1]) ++k;
  const int c = call - P.chunk_base[k];
  const int x = P.cseg[k][c];
  const int beg = P.seg[k][x] + (c - P.cfirst[k][x]) * TTC_CHUNK;
  const int end = min(beg + TTC_CHUNK, P.seg[k][x + 1]);
  const int ra = P.r[k], rb = P.r[k + 1];
  const int tid = threadIdx.x;
  {
    const T* S = core_ptr<T>(P, k) + (long long)x * R * R;
    for (int i = tid; i < R * R; i += TTC_NT) {
      const int a = i / R, b = i - (i / R) * R;
      Ts[i] = (a < ra && b < rb) ? S[pad_idx(P, k, a, b)] : T(0);
    }
  }
  __syncthreads();
  T* out = reinterpret_cast<T*>(P.part) + (long long)(P.chunk_base[k] + c) * P.part_stride;
  RowSrc<T> ls{}, rs{}, vs{};
  const bool rows = left_src<T>(P, k, ls) && right_src<T>(P, k, rs);
  int vmode = 0;   // 0: l^T T_k(x) r, 1: prefix row . r, 2: l . suffix row
  {
    const int tp = P.pre_tab[k + 1], tq = P.suf_tab[k - 1];
    if (tp >= 0 && P.tab_j[tp] == k + 1) {
      vs = {tab_ptr<T>(P) + P.tab_row0[tp] * P.R, P.tab_word[tp], P.tab_shift[tp], (1u << P.tab_bits[tp]) - 1u, P.R};
      vmode = 1;
    } else if (tq >= 0 && P.tab_j[tq] == k) {
      vs = {tab_ptr<T>(P) + P.tab_row0[tq] * P.R, P.tab_word[tq], P.tab_shift[tq], (1u << P.tab_bits[tq]) - 1u, P.R};
      vmode = 2;
    }
  }
  const uint32_t* __restrict__ code = P.code[k];
  const T* __restrict__ yk = y_ptr<T>(P, k);
  const uint64_t pol_stream = policy_evict_first(), pol_rows = policy_evict_last();
  const int ob = tid % R, oa0 = (tid / R) * OPT;
  const bool owner = oa0 < ra && ob < rb;
  T acc[OPT];
#pragma unroll
  for (int u = 0; u < OPT; ++u) acc[u] = 0;
  T s2 = 0;
  for (int base = beg; base < end; base += NE) {
    const int e = base + tid;
    T lv[RC], rv[RC];
    zero(lv);
    zero(rv);
    T g = 0;
    if (e < end) {
      const Code w = load_code_at(code, P.W, e, pol_stream);
      const T yv = ld_stream(yk + e, pol_stream);
      T v = 0;
      if (rows) {
        load_row_hint<RC>(row_of(ls, w), RC, lv, pol_rows);
        load_row_hint<RC>(row_of(rs, w), RC, rv, pol_rows);
        if (vmode != 0) {
          T vr[RC];
          zero(vr);
          load_row_hint<RC>(row_of(vs, w), RC, vr, pol_rows);
#pragma unroll
          for (int a = 0; a < RC; ++a) v = fma(vr[a], vmode == 1 ? rv[a] : lv[a], v);
        } else {
          v = slice_value<T, R, RC>(Ts, ra, rb, lv, rv);
        }
      } else {
        v = interfaces<T, R, RC>(P, k, w, Ts, lv, rv);
      }
      g = v - yv;
    }
    s2 = fma(g, g, s2);
    __syncthreads();   // the previous round's staged rows are consumed
#pragma unroll
    for (int a = 0; a < RS; ++a) {
      Lg[tid * RS + a] = a < RC ? g * lv[a] : T(0);
      Rv[tid * RS + a] = a < RC ? rv[a] : T(0);
    }
    __syncthreads();
    const int cnt = min(NE, end - base);
    if (owner) {
      for (int i = 0; i < cnt; ++i) {
        const T rvb = Rv[i * RS + ob];
        const T* lrow = Lg + i * RS + oa0;
#pragma unroll
        for (int u = 0; u < OPT; ++u) acc[u] = fma(lrow[u], rvb, acc[u]);
      }
    }
  }
  // block sum of g^2 in warp order (the staged area is free again)
  s2 = warp_sum(s2);
  __syncthreads();
  if ((tid & 31) == 0) Lg[tid >> 5] = s2;
  __syncthreads();
  if (tid == 0) {
    T tot = 0;
    for (int wi = 0; wi < TTC_NT / 32; ++wi) tot += Lg[wi];
    out[0] = tot;
  }
  if (owner) {
#pragma unroll
    for (int u = 0; u < OPT; ++u)
      if (oa0 + u < ra) out[1 + (oa0 + u) * rb + ob] = acc[u];
  }
}

// chunks [c0, c1) of a mode class (small ranks; see ttc_pass_class_range)
__device__ __forceinline__ void class_range(const DevProb& P, int mc, int& c0, int& c1) {
  if (mc == PC_FIRST) {
    c0 = 0;
    c1 = P.chunk_base[1];
  } else if (mc == PC_LAST) {
    c0 = P.chunk_base[P.m - 1];
    c1 = P.chunk_base[P.m];
  } else {
    c0 = P.chunk_base[1];
    c1 = P.chunk_base[P.m - 1];
  }
}

// MC: a mode class.  The first and last modes (and every mode at small
// ranks) reduce one chunk per warp; the interior modes at large ranks
// (R >= 16) one chunk per block.
template <typename T, int R, int RC, int MC>
__device__ __forceinline__ void sample_project(const DevProb& P, const int blk) {
  if constexpr (MC == PC_MIDDLE && R >= 16) {
    sample_project_interior<T, R, RC>(P, P.chunk_base[1] + blk);
  } else {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5;
    int c0, c1;
    class_range(P, MC, c0, c1);
    const int call = c0 + blk * kWarps + warp;
    if (call >= c1) return;
    sample_project_warp<T, R, RC, MC>(P, call, reinterpret_cast<T*>(smraw) + warp * R * R);
  }
}

// resident blocks per SM the register budget is sized for: FP32 first/last
// modes (one gather per entry, r accumulators) keep four 256-thread blocks,
// small FP32 interior ranks two (16 warps, two gathers in flight each), and
// so do FP32 interior ranks up to 24 (the block-per-chunk form: 128
// registers instead of the 160 it takes unbounded, which left one block of
// 8 warps per SM to hide the row gathers)
template <typename T, int RC, int MC>
constexpr int min_blocks() {
  return sizeof(T) != 4 ? 1
         : RC > 8 ? (RC <= 24 ? 2 : 1)
         : (MC == PC_FIRST || MC == PC_LAST) ? (RC <= 6 ? 4 : 3)
         : (MC == PC_MIDDLE && RC <= 5) ? 2 : 1;
}

template <typename T, int R, int RC, int MC>
__global__ void __launch_bounds__(TTC_NT, (min_blocks<T, RC, MC>())) k_sample_project(const DevProb P) {
  sample_project<T, R, RC, MC>(P, blockIdx.x);
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

// copies a problem descriptor into shared memory (8-byte words)
__device__ __forceinline__ void stage_desc(const DevProb* __restrict__ src, DevProb* dst) {
  static_assert(sizeof(DevProb) % 8 == 0, "descriptor size");
  const uint2* s = reinterpret_cast<const uint2*>(src);
  uint2* d = reinterpret_cast<uint2*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(DevProb) / 8); i += blockDim.x) d[i] = __ldg(s + i);
  __syncthreads();
}

template <typename T, int R, int RC, int MC>
__global__ void __launch_bounds__(TTC_NT, (min_blocks<T, RC, MC>())) k_sample_project_batch(
    const DevProb* __restrict__ probs, const int* __restrict__ base, int nprob) {
  __shared__ __align__(16) DevProb Ps;
  const int p = find_problem(base, nprob, blockIdx.x);
  stage_desc(probs + p, &Ps);
  sample_project<T, R, RC, MC>(Ps, blockIdx.x - __ldg(base + p));
}

// per mode class: a slice per warp, or (interior modes, R >= 16) the slice
// and the staged rows of the block
template <typename T, int R, int RC>
inline size_t pass_smem_class(int mc) {
  if (R >= 16 && mc == PC_MIDDLE) return sizeof(T) * (size_t)(R * R + 2 * TTC_NT * ((RC + 3) & ~3));
  return sizeof(T) * (size_t)(kWarps * R * R);
}

// the pass of a single problem (g == nullptr) or a batch group: small ranks
// as one launch per mode class (first, interior, last), large ranks as one
// launch over all chunks
template <typename T, int R, int RC>
int launch(const PassLaunch& L) {
  const size_t sm0 = pass_smem_class<T, R, RC>(PC_FIRST), sm1 = pass_smem_class<T, R, RC>(PC_MIDDLE),
               sm2 = pass_smem_class<T, R, RC>(PC_LAST);
  {
    // the interior class on the issuing stream, the first and last classes
    // on the fork's streams (when given), joined back before returning
    cudaStream_t sf = L.st, sl = L.st;
    if (L.fork) {
      TTC_CUDA(cudaEventRecord(L.fork->fork, L.st));
      TTC_CUDA(cudaStreamWaitEvent(L.fork->aux[0], L.fork->fork, 0));
      TTC_CUDA(cudaStreamWaitEvent(L.fork->aux[1], L.fork->fork, 0));
      sf = L.fork->aux[0];
      sl = L.fork->aux[1];
    }
    if (L.g) {
      if (L.g->pass_blocks_c[PC_FIRST] > 0)
        k_sample_project_batch<T, R, RC, PC_FIRST><<<L.g->pass_blocks_c[PC_FIRST], TTC_NT, sm0, sf>>>(
            L.g->probs, L.g->pass_base_c[PC_FIRST], L.g->nprob);
      if (L.g->pass_blocks_c[PC_MIDDLE] > 0)
        k_sample_project_batch<T, R, RC, PC_MIDDLE><<<L.g->pass_blocks_c[PC_MIDDLE], TTC_NT, sm1, L.st>>>(
            L.g->probs, L.g->pass_base_c[PC_MIDDLE], L.g->nprob);
      if (L.g->pass_blocks_c[PC_LAST] > 0)
        k_sample_project_batch<T, R, RC, PC_LAST><<<L.g->pass_blocks_c[PC_LAST], TTC_NT, sm2, sl>>>(
            L.g->probs, L.g->pass_base_c[PC_LAST], L.g->nprob);
    } else {
      const int b0 = ttc_pass_class_blocks(*L.P, PC_FIRST), b1 = ttc_pass_class_blocks(*L.P, PC_MIDDLE),
                b2 = ttc_pass_class_blocks(*L.P, PC_LAST);
      if (b0 > 0) k_sample_project<T, R, RC, PC_FIRST><<<b0, TTC_NT, sm0, sf>>>(*L.P);
      if (b1 > 0) k_sample_project<T, R, RC, PC_MIDDLE><<<b1, TTC_NT, sm1, L.st>>>(*L.P);
      if (b2 > 0) k_sample_project<T, R, RC, PC_LAST><<<b2, TTC_NT, sm2, sl>>>(*L.P);
    }
    TTC_CUDA(cudaGetLastError());
    if (L.fork) {
      TTC_CUDA(cudaEventRecord(L.fork->join[0], sf));
      TTC_CUDA(cudaEventRecord(L.fork->join[1], sl));
      TTC_CUDA(cudaStreamWaitEvent(L.st, L.fork->join[0], 0));
      TTC_CUDA(cudaStreamWaitEvent(L.st, L.fork->join[1], 0));
    }
  }
  return TTC_OK;
}

template <typename T, int R, int RC, int MC>
int opt_in_class(size_t smem) {
  if (smem > 48 * 1024) {
    TTC_CUDA(cudaFuncSetAttribute(k_sample_project<T, R, RC, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    TTC_CUDA(cudaFuncSetAttribute(k_sample_project_batch<T, R, RC, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  }
  return TTC_OK;
}
template <typename T, int R, int RC>
int opt_in() {
  TTC_TRY((opt_in_class<T, R, RC, PC_FIRST>(pass_smem_class<T, R, RC>(PC_FIRST))));
  TTC_TRY((opt_in_class<T, R, RC, PC_MIDDLE>(pass_smem_class<T, R, RC>(PC_MIDDLE))));
  TTC_TRY((opt_in_class<T, R, RC, PC_LAST>(pass_smem_class<T, R, RC>(PC_LAST))));
  return TTC_OK;
}

}  // namespace ttc_pass
