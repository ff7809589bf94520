// Block-level small dense linear algebra in FP64 on shared-memory matrices:
// deterministic block sums, SPD inverse by Cholesky, and the symmetric
// eigendecomposition (cyclic Jacobi, round-robin parallel ordering) that the
// retraction's truncated SVDs are built from.  Every routine must be called
// by all threads of the block; matrices are row-major n x n with n <= 64.
#pragma once
#include "common.cuh"

// Deterministic block-wide sum (fixed tree order); blockDim.x a power of two.
// max that propagates NaN (fmax drops it): accuracy checks must fail on NaN
__device__ __forceinline__ double nanmax(double a, double b) { return (a != a || b != b) ? (a + b) : fmax(a, b); }

static __device__ double blk_sum(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double out = sh[0];
  __syncthreads();
  return out;
}

// In-place inverse of an SPD matrix: A = L L^T (right-looking Cholesky in
// `work`), L^{-1} by forward substitution column by column, A^{-1} = L^{-T} L^{-1}.
// `work` holds n*n doubles, `flag` one int in shared memory.  A pivot that
// is not positive is replaced by a tiny positive value and reported (returns 1).
static __device__ int blk_spd_inverse(double* A, int n, double* work, int* flag) {
  const int tid = threadIdx.x, bd = blockDim.x;
  if (tid == 0) *flag = 0;
  for (int i = tid; i < n * n; i += bd) work[i] = A[i];
  __syncthreads();
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(work[i * n + i]));
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      double d = work[j * n + j];
      if (!(d > 1e-300 * (scale > 0 ? scale : 1.0))) {
        d = 1e-300 * (scale > 0 ? scale : 1.0) + 1e-300;
        *flag = 1;
      }
      work[j * n + j] = sqrt(d);
    }
    __syncthreads();
    double piv = work[j * n + j];
    for (int i = j + 1 + tid; i < n; i += bd) work[i * n + j] /= piv;
    __syncthreads();
    int t = n - j - 1;
    for (int idx = tid; idx < t * t; idx += bd) {
      int i = j + 1 + idx / t, k = j + 1 + idx % t;
      if (k <= i) work[i * n + k] -= work[i * n + j] * work[k * n + j];
    }
    __syncthreads();
  }
  // columns of L^{-1} (lower triangular) into A
  for (int c = tid; c < n; c += bd) {
    for (int i = 0; i < n; ++i) A[i * n + c] = 0.0;
    A[c * n + c] = 1.0 / work[c * n + c];
    for (int i = c + 1; i < n; ++i) {
      double acc = 0.0;
      for (int k = c; k < i; ++k) acc = fma(work[i * n + k], A[k * n + c], acc);
      A[i * n + c] = -acc / work[i * n + i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += bd) {
    int i = idx / n, j = idx % n;
    int k0 = i > j ? i : j;
    double acc = 0.0;
    for (int k = k0; k < n; ++k) acc = fma(A[k * n + i], A[k * n + j], acc);
    work[idx] = acc;
  }
  __syncthreads();
  for (int i = tid; i < n * n; i += bd) A[i] = work[i];
  __syncthreads();
  return *flag;
}

// A = V diag(w) V^T for symmetric A (destroyed).  Cyclic Jacobi: each sweep
// runs n'-1 rounds (n' = n rounded up to even) of n'/2 disjoint rotations in
// the round-robin (circle) order, every rotation zeroing its a_pq with
// tan(phi) = sgn(theta) / (|theta| + sqrt(theta^2 + 1)),
// theta = (a_qq - a_pp) / (2 a_pq).  Sweeps stop when the off-diagonal mass
// is below 1e-30 of the total.  Eigenvalues sorted descending.
// work: n*n + 4*TTC_MAXQ + blockDim.x doubles.
static __device__ void blk_sym_eig(double* A, int n, double* V, double* w, double* work) {
  const int tid = threadIdx.x, bd = blockDim.x;
  const int n2 = n + (n & 1);
  const int np = n2 / 2;
  double* cs_c = work + n * n;
  double* cs_s = cs_c + TTC_MAXQ;
  int* pp = (int*)(cs_s + TTC_MAXQ);
  int* qq = pp + TTC_MAXQ;
  double* red = (double*)(qq + TTC_MAXQ);
  for (int i = tid; i < n * n; i += bd) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = tid; i < n * n; i += bd) {
      double a = A[i];
      if (i / n != i % n) off += a * a;
      tot += a * a;
    }
    off = blk_sum(off, red);
    tot = blk_sum(tot, red);
    if (off <= 1e-30 * tot || tot == 0.0) break;
    for (int t = 0; t < n2 - 1; ++t) {
      for (int i = tid; i < np; i += bd) {
        int pa = (i == 0) ? 0 : ((i - 1 + t) % (n2 - 1)) + 1;
        int posb = n2 - 1 - i;
        int pb = ((posb - 1 + t) % (n2 - 1)) + 1;
        int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = A[p * n + q];
          if (apq != 0.0) {
            double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            double tt = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
            if (theta < 0) tt = -tt;
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
          }
        }
        cs_c[i] = c;
        cs_s[i] = s;
        pp[i] = p;
        qq[i] = q;
      }
      __syncthreads();
      for (int idx = tid; idx < np * n; idx += bd) {   // rows p, q
        int i = idx / n, j = idx % n;
        int p = pp[i], q = qq[i];
        if (q < n) {
          double c = cs_c[i], s = cs_s[i];
          double apj = A[p * n + j], aqj = A[q * n + j];
          A[p * n + j] = c * apj - s * aqj;
          A[q * n + j] = s * apj + c * aqj;
        }
      }
      __syncthreads();
      for (int idx = tid; idx < np * n; idx += bd) {   // columns p, q of A and V
        int i = idx / n, j = idx % n;
        int p = pp[i], q = qq[i];
        if (q < n) {
          double c = cs_c[i], s = cs_s[i];
          double ajp = A[j * n + p], ajq = A[j * n + q];
          A[j * n + p] = c * ajp - s * ajq;
          A[j * n + q] = s * ajp + c * ajq;
          double vjp = V[j * n + p], vjq = V[j * n + q];
          V[j * n + p] = c * vjp - s * vjq;
          V[j * n + q] = s * vjp + c * vjq;
        }
      }
      __syncthreads();
    }
  }
  // sort descending: order into pp (as ints), then permute V's columns
  if (tid == 0) {
    for (int i = 0; i < n; ++i) pp[i] = i;
    for (int i = 0; i < n; ++i) {
      int best = i;
      for (int j = i + 1; j < n; ++j)
        if (A[pp[j] * n + pp[j]] > A[pp[best] * n + pp[best]]) best = j;
      int tmp = pp[i]; pp[i] = pp[best]; pp[best] = tmp;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += bd) w[i] = A[pp[i] * n + pp[i]];
  for (int idx = tid; idx < n * n; idx += bd) work[idx] = V[idx];
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += bd) {
    int j = idx / n, c = idx % n;
    V[idx] = work[j * n + pp[c]];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Warp-level helpers for the small factorizations.  GB300's FP64 pipe has a
// 64-cycle dependent-FMA latency, so factorizations with long sequential
// chains (Cholesky pivots, Jacobi rotations) run in FP32 and are brought to
// FP64 accuracy by refinement steps that are matrix products only.
// ---------------------------------------------------------------------------

// One warp: lower Cholesky factor L of the SPD matrix A (FP64 input, n <= 32)
// in FP32, and Li = L^{-1} (lower) in FP32.  L, Li: n*n floats (row-major).
// Returns 1 if a pivot was not positive (it is then replaced by a tiny value).
static __device__ int warp_chol_inv32(const double* A, int lda, int n, float* L, float* Li, int* pow2 = nullptr) {
  const int lane = threadIdx.x & 31;
  // factor A 2^{-2k} (exact scaling, largest diagonal in [1/4, 4)) so FP32
  // neither overflows nor underflows; with pow2 the caller gets k and the
  // factors of A are L 2^k and Li 2^{-k}
  int k2 = 0;
  if (pow2) {
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) dmax = fmax(dmax, fabs(A[i * lda + i]));
    if (dmax > 0.0 && dmax <= 1.7e308) {
      int e;
      frexp(dmax, &e);
      k2 = e / 2;
    }
    *pow2 = k2;
  }
  const double sc = ldexp(1.0, -2 * k2);   // exact power of two
  for (int idx = lane; idx < n * n; idx += 32) {
    int i = idx / n, k = idx - (idx / n) * n;
    L[idx] = (k <= i) ? (float)(A[i * lda + k] * sc) : 0.f;
  }
  __syncwarp();
  float scale = 0.f;
  for (int i = 0; i < n; ++i) scale = fmaxf(scale, fabsf(L[i * n + i]));
  int bad = 0;
  for (int j = 0; j < n; ++j) {
    float d = L[j * n + j];
    if (!(d > 1e-30f * scale + 1e-38f)) {
      d = 1e-30f * scale + 1e-38f;
      bad = 1;
    }
    float ljj = sqrtf(d), inv = 1.f / ljj;
    __syncwarp();
    for (int i = j + lane; i < n; i += 32) L[i * n + j] = (i == j) ? ljj : L[i * n + j] * inv;
    __syncwarp();
    for (int i = j + 1 + lane; i < n; i += 32) {
      float lij = L[i * n + j];
      for (int k = j + 1; k <= i; ++k) L[i * n + k] = fmaf(-lij, L[k * n + j], L[i * n + k]);
    }
    __syncwarp();
  }
  for (int c = lane; c < n; c += 32) {
    for (int i = 0; i < c; ++i) Li[i * n + c] = 0.f;
    Li[c * n + c] = 1.f / L[c * n + c];
    for (int i = c + 1; i < n; ++i) {
      float acc = 0.f;
      for (int k = c; k < i; ++k) acc = fmaf(L[i * n + k], Li[k * n + c], acc);
      Li[i * n + c] = -acc / L[i * n + i];
    }
  }
  __syncwarp();
  return bad;
}

// C (M x N, ldc) = alpha op(A) op(B) (+ C when accumulate) by one warp.
template <typename T>
__device__ void warp_gemm(int M, int N, int K, const T* A, int lda, bool ta, const T* B, int ldb, bool tb, T* C,
                          int ldc, T alpha, bool accumulate) {
  const int lane = threadIdx.x & 31;
  for (int idx = lane; idx < M * N; idx += 32) {
    int i = idx / N, j = idx - (idx / N) * N;
    T acc = 0;
    for (int k = 0; k < K; ++k) {
      T a = ta ? A[k * lda + i] : A[i * lda + k];
      T b = tb ? B[j * ldb + k] : B[k * ldb + j];
      acc = fma(a, b, acc);
    }
    C[i * ldc + j] = accumulate ? fma(alpha, acc, C[i * ldc + j]) : alpha * acc;
  }
  __syncwarp();
}

// One warp: X = A^{-1} for SPD A (n <= 32), FP64 result.  X0 = L^{-T} L^{-1}
// from the FP32 Cholesky, then Newton-Schulz steps X <- X + X (I - A X) in
// FP64 (each squares the relative error).  Returns max |I - A X| after the
// last step, or a huge value if the pivots failed, so the caller can fall
// back to the FP64 factorization.  Scratch: L, Li (n*n floats), T (2 n*n doubles).
static __device__ double warp_spd_inverse(const double* A, int lda, int n, double* X, int ldx, float* L, float* Li,
                                          double* T) {
  const int lane = threadIdx.x & 31;
  int k2 = 0;
  int bad = warp_chol_inv32(A, lda, n, L, Li, &k2);
  const double sc = ldexp(1.0, -2 * k2);
  for (int idx = lane; idx < n * n; idx += 32) {
    int i = idx / n, j = idx - (idx / n) * n;
    int k0 = i > j ? i : j;
    double acc = 0.0;
    for (int k = k0; k < n; ++k) acc = fma((double)Li[k * n + i], (double)Li[k * n + j], acc);
    X[i * ldx + j] = acc * sc;   // A^{-1} = 2^{-2k} (A 2^{-2k})^{-1}
  }
  __syncwarp();
  double* T1 = T;
  double* T2 = T + n * n;
  double res = 0.0;
  for (int it = 0; it < 4; ++it) {
    warp_gemm<double>(n, n, n, A, lda, false, X, ldx, false, T1, n, -1.0, false);   // T1 = -A X
    for (int i = lane; i < n; i += 32) T1[i * n + i] += 1.0;                          // T1 = I - A X
    __syncwarp();
    res = 0.0;
    for (int idx = lane; idx < n * n; idx += 32) res = nanmax(res, fabs(T1[idx]));
    for (int o = 16; o > 0; o >>= 1) res = nanmax(res, __shfl_xor_sync(0xffffffffu, res, o));
    if (!(res < 1.0)) break;                   // no contraction: leave it to the FP64 path
    if (it >= 2 && res < 1e-13) break;         // converged
    warp_gemm<double>(n, n, n, X, ldx, false, T1, n, false, T2, n, 1.0, false);      // T2 = X T1
    for (int idx = lane; idx < n * n; idx += 32) {
      int i = idx / n, j = idx - (idx / n) * n;
      X[i * ldx + j] += T2[idx];
    }
    __syncwarp();
  }
  return (bad || !(res < 1.0)) ? 1e300 : res;
}

// Deterministic block-wide maximum of one double per thread.
static __device__ double blk_max(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = nanmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  double out = sh[0];
  __syncthreads();
  return out;
}

// FP64 lower Cholesky factor of SPD G (n x n, ldg) and Li = L^{-1} (n x n,
// row-major), block-parallel (the slow but robust path, for matrices whose
// conditioning defeats the FP32 factorization).  `work` holds n*n doubles.
// A pivot that is not positive is replaced by a tiny value (flag set).
static __device__ void blk_chol_linv64(const double* G, int ldg, int n, double* Li, double* work, int* flag) {
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int i = tid; i < n * n; i += bd) work[i] = G[(i / n) * ldg + (i % n)];
  __syncthreads();
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(work[i * n + i]));
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      double d = work[j * n + j];
      double floor_ = 1e-300 * (scale > 0 ? scale : 1.0) + 1e-300;
      if (!(d > floor_)) {
        d = floor_;
        *flag = 1;
      }
      work[j * n + j] = sqrt(d);
    }
    __syncthreads();
    const double piv = work[j * n + j];
    for (int i = j + 1 + tid; i < n; i += bd) work[i * n + j] /= piv;
    __syncthreads();
    const int t = n - j - 1;
    for (int idx = tid; idx < t * t; idx += bd) {
      int i = j + 1 + idx / t, k = j + 1 + idx % t;
      if (k <= i) work[i * n + k] -= work[i * n + j] * work[k * n + j];
    }
    __syncthreads();
  }
  for (int c = tid; c < n; c += bd) {
    for (int i = 0; i < c; ++i) Li[i * n + c] = 0.0;
    Li[c * n + c] = 1.0 / work[c * n + c];
    for (int i = c + 1; i < n; ++i) {
      double acc = 0.0;
      for (int k = c; k < i; ++k) acc = fma(work[i * n + k], Li[k * n + c], acc);
      Li[i * n + c] = -acc / work[i * n + i];
    }
  }
  __syncthreads();
}
