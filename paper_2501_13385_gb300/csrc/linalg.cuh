// Block-level small dense linear algebra in FP64 on shared-memory matrices:
// deterministic block sums, SPD inverse by Cholesky, and the symmetric
// eigendecomposition (cyclic Jacobi, round-robin parallel ordering) that the
// retraction's truncated SVDs are built from.  Every routine must be called
// by all threads of the block; matrices are row-major n x n with n <= 64.
#pragma once
#include "common.cuh"

// Deterministic block-wide sum (fixed tree order); blockDim.x a power of two.
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
