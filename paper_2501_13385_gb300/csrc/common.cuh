// Shared definitions of the ttc CUDA library: limits, the device-side problem
// descriptor, error plumbing and block-level small dense linear algebra used
// by the FP64 stages (Grams, SPD inverses, symmetric eigendecomposition).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ttc.h"

#define TTC_MAXM 16      // maximum tensor order
#define TTC_MAXR 32      // maximum TT-rank
#define TTC_MAXQ 64      // maximum rank of the rank-2r TT of the retraction
#define TTC_CHUNK 1024   // Omega entries per block of the sampled pass
#define TTC_NT 256       // threads per block of the sampled pass

// ---------------------------------------------------------------------------
// Device descriptor of one completion problem.  Everything the kernels touch
// is reachable from here; the host fills it once per layout.
// Core k (0-based) is stored slice-major: T_k(x) is an r[k] x r[k+1]
// row-major block at offset x * r[k] * r[k+1].
// ---------------------------------------------------------------------------
struct DevProb {
  int m;
  int N;
  int W;                       // 32-bit code words per entry (1, 2 or 4)
  int n[TTC_MAXM];
  int r[TTC_MAXM + 1];
  int cword[TTC_MAXM];         // code word holding mode k
  int cshift[TTC_MAXM];        // bit offset of mode k in that word
  int cbits[TTC_MAXM];         // bits of mode k
  double p;                    // N / d*
  double inv_min_n;            // 1 / min_k n_k
  double inv_2m;               // 1 / (2m)
  int keep_residual;           // write g[] in input order during the pass
  int steepest;                // step size by exact line search (Eq. (PRGD stepsize))
  int uniform;                 // G_{l,i} = I (RGD)
  int weighted_retraction;     // Remark 3.6: W^{-1/2} SVD^tt_r W^{1/2}
  int step_fp64;               // an FP64 step: FP64 pass and FP64 refinement of the retraction's SVDs
  int dense_ff;                // the block-per-slice dense stages' slice products in float-float (ff.cuh)

  // current iterate
  double* core64[TTC_MAXM];    // FP64 master, slice-major, unpadded
  // padded mirrors read by the sampled pass: slice x of core k starts at
  // x * R * R (16-byte aligned); row a of the slice starts at a * R, except for
  // cores with r_{k+1} = 1 whose slice is one contiguous vector
  int R;                       // rank bucket (4, 8, 16 or 32) = row stride
  float* core32p[TTC_MAXM];
  double* core64p[TTC_MAXM];
  double* prev64[TTC_MAXM];    // copy of T_l for the step-change metric

  // interface tables: prefix L_j(x_0..x_{j-1}) = T_0(x_0)...T_{j-1}(x_{j-1})
  // (a row of length r_j) and suffix R_j(x_j..x_{d-1}) = T_j(x_j)...T_{d-1}(x_{d-1})
  // (a column of length r_j), for all index combinations.  A table covers
  // modes whose code fields share one 32-bit word; its row index is those
  // fields as they sit in the word (the lowest mode in the lowest bits), so
  // rows of coordinates >= n_j exist but are never read.  Row g at g * R.
  int ntab;
  int tab_side[2 * TTC_MAXM];     // 0 prefix, 1 suffix
  int tab_j[2 * TTC_MAXM];
  long long tab_rows[2 * TTC_MAXM];
  long long tab_row0[2 * TTC_MAXM];
  long long tab_total;
  int tab_word[2 * TTC_MAXM];     // table row = (code word tab_word >> tab_shift) & (2^tab_bits - 1):
  int tab_shift[2 * TTC_MAXM];    // the bit-concatenated coordinates of the table's modes
  int tab_bits[2 * TTC_MAXM];
  int pre_tab[TTC_MAXM];          // mode k: table giving the prefix over modes < k (-1: none)
  int suf_tab[TTC_MAXM];          // mode k: table giving the suffix over modes > k (-1: none)
  float* tab32;
  double* tab64;

  // Omega layout, per mode, in mode-k order
  const uint32_t* code[TTC_MAXM];
  const float* y32[TTC_MAXM];
  const double* y64[TTC_MAXM];
  const int* perm[TTC_MAXM];
  const int* seg[TTC_MAXM];      // n_k + 1 offsets
  const int* cfirst[TTC_MAXM];   // n_k + 1: chunks of slice x are [cfirst[x], cfirst[x+1])
  const int* cseg[TTC_MAXM];     // slice of each chunk
  int nchunk[TTC_MAXM];
  int chunk_base[TTC_MAXM + 1];  // prefix of nchunk over modes
  void* part;                    // chunk partials: [chunk][1 + r_k r_{k+1}] (float or double)
  int part_stride;               // elements per chunk partial (max over modes)

  // outputs of the Omega pass
  double* s[TTC_MAXM];           // slice energies, n_k
  double* wt[TTC_MAXM];          // this step's slice weights, n_k x 2: G_k(x)^{+1/(2m)}, G_k(x)^{-1/(2m)}
  double* E[TTC_MAXM];           // n_k x r_k x r_{k+1}
  double* B1[TTC_MAXM];          // steepest step: update cores at unit step, n_k x r_k x r_{k+1}
  float* B1_32p[TTC_MAXM];       // the same in FP32, padded like core32p (FP32 steps evaluate with it)
  double* B1_64p[TTC_MAXM];      // the same in FP64, padded like core64p (FP64 steps)
  float* ztab32;                 // steepest step: the tangent part of the prefix tables' rows (tab32 layout)
  double* ztab64;                // the same for FP64 steps (tab64 layout)
  double* zw;                    // steepest step: per slice G^{1/(2m)} <Lam B1 Gam, B1> (all modes)
  double* tpart;                 // steepest step: block partials of ||P_Omega Z||^2
  double* g;                     // residual in input order (when keep_residual)

  // dense-stage buffers
  double* C[TTC_MAXM];           // rank-2r cores, n_k x q_k x q_{k+1}
  int q[TTC_MAXM + 1];
  double* small;                 // small matrices, offsets below
  int off_lam[TTC_MAXM + 1];     // Lam[k]: r_k x r_k, left Gram of W^{1/2} T up to core k-1
  int off_gam[TTC_MAXM + 1];     // Gam[k]: r_k x r_k, right Gram of W^{1/2} T from core k
  int off_lami[TTC_MAXM + 1];    // inverse of Lam[k]
  int off_gami[TTC_MAXM + 1];    // inverse of Gam[k]
  int off_h[TTC_MAXM];           // H_k = sum_x T_k(x)^T E_k(x): r_{k+1} x r_{k+1}
  int off_qm[TTC_MAXM];          // Q_k = Lam[k+1]^{-1} H_k Gam[k+1]^{-1}
  int off_psi[TTC_MAXM + 1];     // Psi[k]: q_k x q_k right Gram of the rank-2r TT
  int off_nk[TTC_MAXM];          // N_k: q_{k+1} x q_{k+1}
  int off_pk[TTC_MAXM];          // P_k: q_{k+1} x r_{k+1}
  int off_sk[TTC_MAXM];          // S_k: r_{k+1} x q_{k+1}
  int off_mlam[3][TTC_MAXM + 1];  // metric Gram sweep: A^T A, A^T B, B^T B left Grams
  double* red;                   // partial sums of slice reductions
  long long red_metric;          // offset of the metric's partials in red
  double* red2;                  // group partials of the dense stages' two-level reductions
  long long red2_metric;         // offset of the metric's group partials in red2
  int* gctr;                     // group counters of the two-level reductions
  double* scal;                  // scalars, see SC_* below
  unsigned* flags;               // = (unsigned*)(scal + SC_FLAGS): bit 0 non-finite, bit 1 lost rank
  int* counters;                 // completion counters of the fused reductions (reset by their last block)

  // ground truth (optional)
  int has_truth;
  int rt[TTC_MAXM + 1];
  double* truth[TTC_MAXM];
  long long dstar;               // product of n_k (0 if it overflows)
};

enum {
  SC_G2 = 0,        // ||g||^2
  SC_EPS = 1,
  SC_ALPHA = 2,
  SC_ALPHA_OVR = 3, // > 0: use this step size
  SC_EPS_FIXED = 4, // > 0: use this eps
  SC_FLAGS = 5,     // bit 0: non-finite seen; bit 1: lost rank in the retraction
  SC_METRIC = 6,    // last metric (sum of squares)
  SC_NORM = 7,      // reference norm^2 of the metric
  SC_EPS_REL = 8,
  SC_ALPHA_SCALE = 9,
  SC_SUBIT = 10,    // Jacobi sweeps of the retraction's bond SVDs in the last iteration (all bonds)
  SC_COUNT = 16
};

// ---------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------
void ttc_record_cuda_error(cudaError_t e);
#define TTC_CUDA(call)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) {                             \
      ttc_record_cuda_error(_e);                         \
      return TTC_ECUDA;                                  \
    }                                                    \
  } while (0)
#define TTC_TRY(call)                                    \
  do {                                                   \
    int _s = (call);                                     \
    if (_s != TTC_OK) return _s;                         \
  } while (0)

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// offset of element (a, b) inside a padded slice of core k
__device__ __forceinline__ int pad_idx(const DevProb& P, int k, int a, int b) {
  return P.r[k + 1] == 1 ? a : a * P.R + b;
}

__device__ __forceinline__ int code_coord(const DevProb& P, const uint32_t* words, int k) {
  return (int)((words[P.cword[k]] >> P.cshift[k]) & ((1u << P.cbits[k]) - 1u));
}

// the packed code of one entry, held in registers (selected without indexing)
struct Code {
  uint32_t w0, w1, w2, w3;
  __device__ __forceinline__ uint32_t word(int i) const {
    return i == 0 ? w0 : (i == 1 ? w1 : (i == 2 ? w2 : w3));
  }
};
__device__ __forceinline__ Code load_code(const DevProb& P, int k, int e) {
  Code c;
  const uint32_t* p = P.code[k] + (long long)e * P.W;
  c.w0 = __ldg(p);
  c.w1 = P.W > 1 ? __ldg(p + 1) : 0u;
  c.w2 = P.W > 2 ? __ldg(p + 2) : 0u;
  c.w3 = P.W > 3 ? __ldg(p + 3) : 0u;
  return c;
}
__device__ __forceinline__ int code_coord(const DevProb& P, const Code& c, int k) {
  return (int)((c.word(P.cword[k]) >> P.cshift[k]) & ((1u << P.cbits[k]) - 1u));
}

// One entry of a tensor train in FP64: v <- v C_k(x_k) along the train, with
// element (i, j) of core k's slice x read through the layout functor
// (C.at(k, x, i, j), C.r(k) the ranks).  Two rank-sized arrays are live.
template <typename Cores>
__device__ __forceinline__ double tt_chain_value(const Cores& C, int d, const int* xs) {
  double v[TTC_MAXR], t[TTC_MAXR];
  v[0] = 1.0;
  for (int k = 0; k < d; ++k) {
    const int p = C.r(k), q = C.r(k + 1), x = xs[k];
    for (int j = 0; j < q; ++j) {
      double a0 = 0.0, a1 = 0.0;
      int i = 0;
      for (; i + 1 < p; i += 2) {
        a0 = fma(v[i], C.at(k, x, i, j), a0);
        a1 = fma(v[i + 1], C.at(k, x, i + 1, j), a1);
      }
      if (i < p) a0 = fma(v[i], C.at(k, x, i, j), a0);
      t[j] = a0 + a1;
    }
    for (int j = 0; j < q; ++j) v[j] = t[j];
  }
  return v[0];
}

// Per-block partial sums of ||A - B||^2 and ||B||^2 over the d* entries
// (linear index l, last mode fastest) of two tensor trains, every entry
// evaluated in FP64; the block's sums go to part[2 blockIdx], part[2 blockIdx + 1].
// blockDim.x must be 256.
template <typename CoresA, typename CoresB>
__device__ __forceinline__ void tt_dist_block(const CoresA& A, const CoresB& B, int d, const int* n, long long dstar,
                                              double* part) {
  __shared__ double sh1[256];
  __shared__ double sh2[256];
  double d2 = 0.0, b2 = 0.0;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < dstar;
       l += (long long)gridDim.x * blockDim.x) {
    int xs[TTC_MAXM];
    long long t = l;
    for (int k = d - 1; k >= 0; --k) {
      xs[k] = (int)(t % n[k]);
      t /= n[k];
    }
    const double va = tt_chain_value(A, d, xs);
    const double vb = tt_chain_value(B, d, xs);
    const double df = va - vb;
    d2 = fma(df, df, d2);
    b2 = fma(vb, vb, b2);
  }
  sh1[threadIdx.x] = d2;
  sh2[threadIdx.x] = b2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sh1[threadIdx.x] += sh1[threadIdx.x + s];
      sh2[threadIdx.x] += sh2[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sh1[0];
    part[2 * blockIdx.x + 1] = sh2[0];
  }
}

// C (M x N, ldc) = alpha * op(A) * op(B) (+ beta * C when accumulate), on data
// visible to the whole block; threads stride over the M*N outputs.  The caller
// synchronises.  op(A) is M x K: A[i*lda + k] or, transposed, A[k*lda + i].
// The inner sum runs as four independent FMA chains (k mod 4), added at the
// end: in a block of 8 warps a dependent FP64 FMA advances every ~150
// cycles on GB300 (~1.7 FP64 FMAs per clock per SM), so one chain per
// output would leave the pipe idle.
template <typename T>
__device__ void blk_gemm(int M, int N, int K, const T* A, int lda, bool ta, const T* B, int ldb,
                         bool tb, T* C, int ldc, T alpha, bool accumulate) {
  const int sa = ta ? lda : 1, sb = tb ? 1 : ldb;
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    int i = idx / N, j = idx - (idx / N) * N;
    const T* a = ta ? A + i : A + i * lda;
    const T* b = tb ? B + j * ldb : B + j;
    T c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    int k = 0;
    for (; k + 3 < K; k += 4) {
      c0 = fma(a[k * sa], b[k * sb], c0);
      c1 = fma(a[(k + 1) * sa], b[(k + 1) * sb], c1);
      c2 = fma(a[(k + 2) * sa], b[(k + 2) * sb], c2);
      c3 = fma(a[(k + 3) * sa], b[(k + 3) * sb], c3);
    }
    for (; k < K; ++k) c0 = fma(a[k * sa], b[k * sb], c0);
    const T acc = (c0 + c1) + (c2 + c3);
    C[i * ldc + j] = accumulate ? fma(alpha, acc, C[i * ldc + j]) : alpha * acc;
  }
}

// Block-level small dense linear algebra lives in linalg.cuh.
