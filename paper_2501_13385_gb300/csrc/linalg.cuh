// Block-level small dense linear algebra on shared-memory matrices:
// deterministic block sums, SPD inverse by Cholesky, semidefinite Cholesky
// factors and the one-sided Jacobi SVD that the retraction's truncated SVDs
// are built from.  Every routine must be called
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

// ---------------------------------------------------------------------------
// Warp-level helpers for the small factorizations.  GB300's FP64 pipe issues
// ~1.7 FMAs per clock per SM (a block's 8 warps each advance a dependent
// FP64 chain every ~150 cycles), so factorizations with long sequential
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

// C (M x N, ldc) = alpha op(A) op(B) (+ C when accumulate) by one warp.  Four
// independent FMA chains per output (k mod 4): FP64 chains advance slowly
// on this GPU (~1.7 FP64 FMAs per clock per SM).
template <typename T>
__device__ void warp_gemm(int M, int N, int K, const T* A, int lda, bool ta, const T* B, int ldb, bool tb, T* C,
                          int ldc, T alpha, bool accumulate) {
  const int lane = threadIdx.x & 31;
  const int sa = ta ? lda : 1, sb = tb ? 1 : ldb;
  for (int idx = lane; idx < M * N; idx += 32) {
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

// ---------------------------------------------------------------------------
// Factors and SVDs for the retraction's bonds.
// ---------------------------------------------------------------------------

// Upper Cholesky factors of two symmetric positive semidefinite n x n
// matrices (row-major, n <= 64) at once, in place: A = R_A^T R_A and
// B = R_B^T R_B.  Right-looking, one barrier per pivot: the Schur
// complement is updated whole (both triangles), so the update of pivot j
// reads column j below the diagonal while row j is scaled into the factor.
// Each thread keeps fixed (row, column) offsets, so no integer division runs
// inside the pivot loop.  A pivot at or below 1e-14 of the largest diagonal
// entry is rounding noise of a numerically singular Gram (its square root
// would turn noise of 1e-16 into rows of size 1e-8): it gives a zero row,
// which keeps R^T R equal to the matrix on its numerical range.  The strict
// lower triangles are zeroed.  diag: 2n doubles.
static __device__ void blk_chol2_upper_psd(double* A, double* B, int n, double* diag) {
  const int tid = threadIdx.x, bd = blockDim.x;
  __syncthreads();
  double ma = 0.0, mb = 0.0;
  for (int i = 0; i < n; ++i) {
    ma = fmax(ma, A[i * n + i]);
    mb = fmax(mb, B[i * n + i]);
  }
  const double ta = 1e-14 * ma, tb = 1e-14 * mb;
  // half the threads per matrix; within a half, thread h owns columns
  // c = h mod 64 + 64 w and rows i = h div 64 + rs v of the trailing block
  const int half = bd / 2, second = tid >= half, h = second ? tid - half : tid;
  double* M = second ? B : A;
  const double tm = second ? tb : ta;
  const int c0 = h & 63, i0 = h >> 6, rs = max(1, half >> 6);
  for (int j = 0; j < n; ++j) {
    const double d = M[j * n + j];
    const double rr = (d > tm) ? rsqrt(d) : 0.0;
    const double r2 = rr * rr;
    for (int c = j + 1 + c0; c < n; c += 64) {
      const double mcj = M[c * n + j] * r2;
      for (int i = j + 1 + i0; i < n; i += rs) M[i * n + c] = fma(-M[i * n + j], mcj, M[i * n + c]);
    }
    if (h == 0) diag[(second ? n : 0) + j] = d * rr;   // sqrt(d), or 0
    for (int c = j + 1 + h; c < n; c += half) M[j * n + c] *= rr;
    __syncthreads();
  }
  for (int idx = tid; idx < 2 * n * n; idx += bd) {
    const bool sb = idx >= n * n;
    const int e = sb ? idx - n * n : idx;
    const int i = e / n, c = e - (e / n) * n;
    double* X = sb ? B : A;
    if (c < i) X[e] = 0.0;
    else if (c == i) X[e] = diag[(sb ? n : 0) + i];
  }
  __syncthreads();
}

// One-sided (Hestenes) Jacobi: plane rotations of the columns of G (n x n,
// n <= 64, column-major: column j at G + j*ld, the same for V) until they are mutually
// orthogonal, so that G V = U diag(sigma), with the rotations accumulated in
// V (column-major, enter with the starting basis).  A sweep is the
// round-robin ordering: n' - 1 rounds (n' = n rounded up to even) of n'/2
// disjoint pairs; each pair is handled by a group of lp lanes (4 for n <= 16,
// else 8; a lane owns every lp-th row), so a block of 256 threads treats all
// pairs of a round at once.  Pair (p, q) is rotated when
// |g_p . g_q| > tol ||g_p|| ||g_q||, by the angle that zeroes the
// off-diagonal of its 2 x 2 Gram [[a, c], [c, b]]:
//   t = sgn(z) / (|z| + sqrt(1 + z^2)),  z = (b - a) / (2c),
//   g_p <- cs g_p - sn g_q,  g_q <- sn g_p + cs g_q,  cs = 1/sqrt(1 + t^2), sn = t cs.
// The sums of a pair are butterfly reductions over its lanes, identical on
// every lane, so the lanes agree on the rotation.  Columns whose squared
// norm is at or below `floor` are zero to the working precision and are not
// rotated (their directions are noise and never settle).  Stops after a
// sweep without rotations or after max_sweeps; returns the sweeps run.  The
// rotations act on the factor, not on its Gram, so singular values of very
// different sizes keep their relative accuracy.
template <typename T>
static __device__ int blk_hestenes(T* G, T* V, int n, int ld, T tol, T floor, int max_sweeps) {
  const int lp = n <= 16 ? 4 : 8;
  const int lane = threadIdx.x & 31;
  const int slot = (threadIdx.x >> 5) * (32 / lp) + lane / lp;
  const int nslots = (blockDim.x >> 5) * (32 / lp);
  const int sub = lane & (lp - 1);
  const int n2 = n + (n & 1), np = n2 / 2;
  const int passes = (np + nslots - 1) / nslots;
  // the round-robin pairs (p < q) of every round, once: integer division is
  // slow, and the rounds are latency-bound
  __shared__ unsigned char pairs[2 * 63 * 32];
  __syncthreads();
  for (int idx = threadIdx.x; idx < (n2 - 1) * np; idx += blockDim.x) {
    const int t = idx / np, i = idx - t * np;
    const int pa = (i == 0) ? 0 : ((i - 1 + t) % (n2 - 1)) + 1;
    const int pb = ((n2 - 2 - i + t) % (n2 - 1)) + 1;
    pairs[2 * idx] = (unsigned char)min(pa, pb);
    pairs[2 * idx + 1] = (unsigned char)max(pa, pb);
  }
  int sweep = 0;
  while (sweep < max_sweeps) {
    int mine = 0;   // this thread rotated in this sweep
    __syncthreads();
    for (int t = 0; t < n2 - 1; ++t) {
      for (int pass = 0; pass < passes; ++pass) {
        const int i = slot + pass * nslots;
        int p = 0, q = 0;
        bool act = false;
        if (i < np) {
          p = pairs[2 * (t * np + i)];
          q = pairs[2 * (t * np + i) + 1];
          act = q < n;   // not the dummy column of an odd n
        }
        constexpr int MR = 8;   // rows per lane: n <= 16 with lp = 4, n <= 64 with lp = 8
        T ca[MR], cb[MR];
        T al = T(0), be = T(0), ga = T(0);
#pragma unroll
        for (int h = 0; h < MR; ++h) {
          const int row = sub + h * lp;
          ca[h] = (act && row < n) ? G[p * ld + row] : T(0);
          cb[h] = (act && row < n) ? G[q * ld + row] : T(0);
          al = fma(ca[h], ca[h], al);
          be = fma(cb[h], cb[h], be);
          ga = fma(ca[h], cb[h], ga);
        }
        for (int o = lp / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        // a column below the floor is zero to the working precision: its
        // direction is noise and never settles, so it is not rotated
        if (act && fmin(al, be) > floor && ga * ga > tol * tol * (al * be)) {
          T tt, cs;
          // the angle needs no correct rounding: a rotation by a slightly
          // different angle is still orthogonal, and the next sweep removes
          // what it leaves; so it is found in FP32 with fast reciprocals
          // (FP64 from FP64 sums: b - a in FP64 first; a chain of FP64
          // divisions and square roots is slow on this GPU)
          float zn, zd;
          if constexpr (sizeof(T) == 4) {
            zn = be - al;
            zd = 2.f * ga;
          } else {
            // scaled by a power of two (exact) that brings |ga| into [1, 2):
            // sums of tiny columns would underflow FP32
            const int eg = (__double2hiint(ga) >> 20) & 0x7ff;
            const double sc = __hiloint2double((2046 - eg) << 20, 0);
            zn = (float)fmin(fmax((be - al) * sc, -1e30), 1e30);
            zd = 2.f * (float)(ga * sc);
          }
          const float z = __fdividef(zn, zd);
          const float az = fabsf(z);
          const float tf = az > 1e15f ? __fdividef(0.5f, z) : copysignf(__frcp_rn(az + sqrtf(fmaf(z, z, 1.f))), z);
          if constexpr (sizeof(T) == 4) {
            tt = tf;
            cs = rsqrtf(fmaf(tt, tt, 1.f));
          } else {
            // cs = 1 / sqrt(1 + t^2) to FP64 accuracy for the t used, so that
            // cs^2 + sn^2 = 1 and the rotation stays orthogonal: Newton's
            // iteration for the inverse square root, y <- y (3 - x y^2) / 2,
            // from the FP32 value (relative error ~2^-22 -> ~1e-13 -> FP64)
            tt = (double)tf;
            const double x = fma(tt, tt, 1.0);
            double y = (double)rsqrtf((float)x);
            for (int it = 0; it < 2; ++it) y = fma(y, fma(-0.5 * x, y * y, 0.5), y);
            cs = y;
          }
          const T sn = cs * tt;
#pragma unroll
          for (int h = 0; h < MR; ++h) {
            const int row = sub + h * lp;
            if (row < n) {
              G[p * ld + row] = fma(cs, ca[h], -sn * cb[h]);
              G[q * ld + row] = fma(sn, ca[h], cs * cb[h]);
              const T x = V[p * ld + row], y = V[q * ld + row];
              V[p * ld + row] = fma(cs, x, -sn * y);
              V[q * ld + row] = fma(sn, x, cs * y);
            }
          }
          mine = 1;
        }
      }
      __syncthreads();
    }
    ++sweep;
    if (!__syncthreads_or(mine)) break;
  }
  return sweep;
}

// One-sided Jacobi in FP32 by a single warp (the other warps of the block wait
// at the closing barrier): column-major G and V with an odd leading dimension
// ld >= n, so that the columns the lanes of a round read at the same row sit
// in different banks.  The n'/2 pairs of a round (n' = n rounded up to even)
// are spread over the 32 lanes, lp lanes per pair (8, 4, 2 or 1 as n'/2 is
// at most 4, 8, 16 or 32), each lane owning every lp-th row; rounds are
// separated by __syncwarp only, so a round costs the dependent arithmetic of
// one pair (the block-wide form pays a block barrier and idle warps per
// round).  Pair (p, q) is rotated as in blk_hestenes; columns at or below
// `floor` are not rotated.  Returns the sweeps run.
static __device__ int warp_hestenes32(float* G, float* V, int n, int ld, float tol, float floor, int max_sweeps) {
  __shared__ unsigned char wpairs[2 * 63 * 32];
  __shared__ int wsweeps;
  const int n2 = n + (n & 1), np = n2 / 2;
  __syncthreads();
  for (int idx = threadIdx.x; idx < (n2 - 1) * np; idx += blockDim.x) {
    const int t = idx / np, i = idx - t * np;
    const int pa = (i == 0) ? 0 : ((i - 1 + t) % (n2 - 1)) + 1;
    const int pb = ((n2 - 2 - i + t) % (n2 - 1)) + 1;
    wpairs[2 * idx] = (unsigned char)min(pa, pb);
    wpairs[2 * idx + 1] = (unsigned char)max(pa, pb);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lp = np <= 4 ? 8 : np <= 8 ? 4 : np <= 16 ? 2 : 1;
    const int lane = threadIdx.x, slot = lane / lp, sub = lane - slot * lp;
    int sweep = 0;
    while (sweep < max_sweeps) {
      int mine = 0;
      for (int t = 0; t < n2 - 1; ++t) {
        int p = 0, q = 0;
        bool act = false;
        if (slot < np) {
          p = wpairs[2 * (t * np + slot)];
          q = wpairs[2 * (t * np + slot) + 1];
          act = q < n;   // not the dummy column of an odd n
        }
        const float* gp = G + p * ld;
        const float* gq = G + q * ld;
        float al0 = 0.f, be0 = 0.f, ga0 = 0.f, al1 = 0.f, be1 = 0.f, ga1 = 0.f;
        if (act) {
          int row = sub;
          for (; row + lp < n; row += 2 * lp) {
            const float a0 = gp[row], b0 = gq[row], a1 = gp[row + lp], b1 = gq[row + lp];
            al0 = fmaf(a0, a0, al0);
            be0 = fmaf(b0, b0, be0);
            ga0 = fmaf(a0, b0, ga0);
            al1 = fmaf(a1, a1, al1);
            be1 = fmaf(b1, b1, be1);
            ga1 = fmaf(a1, b1, ga1);
          }
          if (row < n) {
            const float a0 = gp[row], b0 = gq[row];
            al0 = fmaf(a0, a0, al0);
            be0 = fmaf(b0, b0, be0);
            ga0 = fmaf(a0, b0, ga0);
          }
        }
        float al = al0 + al1, be = be0 + be1, ga = ga0 + ga1;
        for (int o = lp / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (act && fminf(al, be) > floor && ga * ga > tol * tol * (al * be)) {
          // the angle needs no correct rounding: fast reciprocals
          const float z = __fdividef(be - al, 2.f * ga);
          const float az = fabsf(z);
          const float tt = az > 1e15f ? __fdividef(0.5f, z) : copysignf(__frcp_rn(az + sqrtf(fmaf(z, z, 1.f))), z);
          const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = cs * tt;
          float* wp = G + p * ld;
          float* wq = G + q * ld;
          float* vp = V + p * ld;
          float* vq = V + q * ld;
          for (int row = sub; row < n; row += lp) {
            const float a = wp[row], b = wq[row];
            wp[row] = fmaf(cs, a, -sn * b);
            wq[row] = fmaf(sn, a, cs * b);
            const float x = vp[row], y = vq[row];
            vp[row] = fmaf(cs, x, -sn * y);
            vq[row] = fmaf(sn, x, cs * y);
          }
          mine = 1;
        }
        __syncwarp();
      }
      ++sweep;
      if (!__any_sync(0xffffffffu, mine)) break;
    }
    if (lane == 0) wsweeps = sweep;
  }
  __syncthreads();
  return wsweeps;
}
