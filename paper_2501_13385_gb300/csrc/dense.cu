// Dense stage of one PRGD iteration, all in FP64 on the device:
//
//  (1) eps_l, alpha_l from ||G_l||^2 (step-size form of Theorem 4.1);
//      G_k(x) = eps + s_k(x) is the diagonal of G_{l,k} (Section 3.2).
//  (2) Grams of T^ = W^{1/2} T (Proposition 3.1: T^_k(x) = G_k(x)^{1/(4m)} T_k(x)):
//        Lam[k+1] = sum_x G_k(x)^{1/(2m)} T_k(x)^T Lam[k] T_k(x)      (left)
//        Gam[k]   = sum_x G_k(x)^{1/(2m)} T_k(x) Gam[k+1] T_k(x)^T    (right)
//      and H_k = sum_x T_k(x)^T E_k(x).
//  (3) The weighted tangent projection of Lemma 3.5 (Eq. (tsp in nm)),
//      taken at the left-orthogonal decomposition U of T^ with T^<=k = U^<=k R_k,
//      R_k^T R_k = Lam[k], written back in the gauge of the iterate's own
//      cores.  With the sparse factor E_k from the sampled pass, the update
//      core of W_l = T_l - alpha tilde P_T W^{-1} G_l for mode k becomes
//        B_k(x) = -alpha [ G_k(x)^{-1/(2m)} Lam[k]^{-1} E_k(x) Gam[k+1]^{-1}
//                          - T_k(x) Lam[k+1]^{-1} H_k Gam[k+1]^{-1} ]    (k < d-1)
//        B_{d-1}(x) = -alpha G_{d-1}(x)^{-1/(2m)} Lam[d-1]^{-1} E_{d-1}(x),
//      which is R_{k-1}^{-1} (-alpha G_k^{-1/(4m)} A^_k) R_k with A^_k the
//      Lemma 3.5 component: the weights and R factors of the projection cancel
//      into r x r Gram inverses.
//  (4) W_l in rank-2r TT form (rank bound of Section 3.1):
//        C_0 = [B_0  T_0],  C_k = [[T_k, 0], [B_k, T_k]],  C_{d-1} = [[T_{d-1}], [T_{d-1} + B_{d-1}]].
//  (5) T_{l+1} = SVD^tt_r(W_l), Algorithm 1 evaluated on the rank-2r TT:
//      right Grams Psi[k] = sum_x C_k(x) Psi[k+1] C_k(x)^T; then for each bond
//      k, with C'_k = S_{k-1} C_k:  N_k = sum_x C'_k(x)^T C'_k(x),
//      Psi[k+1] = K K^T (eigendecomposition), K^T N_k K = V Sigma^2 V^T,
//      P_k = K V_{:,1:r} Sigma^{-1},  new core T_k(x) = C'_k(x) P_k (left-
//      orthogonal), S_k = P_k^T N_k.  The last core is S_{d-2} C_{d-1}(x).
//      The top-r left singular vectors of (T^{<=k-1} (x) I)^T W^{<k>} are
//      exactly those of L(C'_k) K, so this is Algorithm 1, not an approximation
//      of it.
// Every reduction over slices is split over blocks and summed in a fixed
// order, so results are reproducible bit for bit.
#include <algorithm>
#include <vector>

#include "ctx.h"
#include "linalg.cuh"

namespace {

enum Op { OP_LAM = 0, OP_GAM = 1, OP_H = 2, OP_PSI = 3, OP_N = 4 };

struct Job {
  int op, k;
  int nb;          // blocks
  int dim;         // output is dim x dim
  long long red;   // offset in P.red of the partials
  int dst;         // offset in P.small of the result (-1: none)
};

struct JobList {
  int njob;
  Job job[TTC_MAXM + 4];
};

constexpr int kDenseThreads = 256;

__device__ __forceinline__ double wpow(const DevProb& P, int k, int x, double e) {
  return pow(P.scal[SC_EPS] + P.s[k][x], e);
}

// one block: accumulates the contributions of slices blk, blk+nb, ... of one job
__global__ void __launch_bounds__(kDenseThreads) k_reduce(const DevProb P, const JobList L) {
  extern __shared__ __align__(16) double sm[];
  int b = blockIdx.x, j = 0;
  while (b >= L.job[j].nb) {
    b -= L.job[j].nb;
    ++j;
  }
  const Job J = L.job[j];
  const int k = J.k, m = P.m;
  const int dim = J.dim;
  double* acc = sm;                 // dim x dim
  double* Y = sm + dim * dim;       // up to 64 x 64
  for (int i = threadIdx.x; i < dim * dim; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const int nk = P.n[k];
  const int ra = P.r[k], rb = P.r[k + 1];
  const double invm2 = 1.0 / (2.0 * m);
  for (int x = b; x < nk; x += J.nb) {
    const double* T = P.core64[k] + (long long)x * ra * rb;
    if (J.op == OP_LAM) {   // acc += w2 T^T (Lam T)
      const double* Lam = P.small + P.off_lam[k];
      blk_gemm<double>(ra, rb, ra, Lam, ra, false, T, rb, false, Y, rb, 1.0, false);
      __syncthreads();
      blk_gemm<double>(rb, rb, ra, T, rb, true, Y, rb, false, acc, rb, wpow(P, k, x, invm2), true);
    } else if (J.op == OP_GAM) {   // acc += w2 (T Gam) T^T
      const double* Gam = P.small + P.off_gam[k + 1];
      blk_gemm<double>(ra, rb, rb, T, rb, false, Gam, rb, false, Y, rb, 1.0, false);
      __syncthreads();
      blk_gemm<double>(ra, ra, rb, Y, rb, false, T, rb, true, acc, ra, wpow(P, k, x, invm2), true);
    } else if (J.op == OP_H) {     // acc += T^T E
      const double* E = P.E[k] + (long long)x * ra * rb;
      blk_gemm<double>(rb, rb, ra, T, rb, true, E, rb, false, acc, rb, 1.0, true);
    } else if (J.op == OP_PSI) {   // acc += (C Psi) C^T
      const int qa = P.q[k], qb = P.q[k + 1];
      const double* C = P.C[k] + (long long)x * qa * qb;
      const double* Psi = P.small + P.off_psi[k + 1];
      blk_gemm<double>(qa, qb, qb, C, qb, false, Psi, qb, false, Y, qb, 1.0, false);
      __syncthreads();
      blk_gemm<double>(qa, qa, qb, Y, qb, false, C, qb, true, acc, qa, 1.0, true);
    } else {                       // OP_N: C' = S_{k-1} C ; acc += C'^T C'
      const int qa = P.q[k], qb = P.q[k + 1];
      const double* C = P.C[k] + (long long)x * qa * qb;
      if (k == 0) {
        blk_gemm<double>(qb, qb, qa, C, qb, true, C, qb, false, acc, qb, 1.0, true);
      } else {
        const double* S = P.small + P.off_sk[k - 1];   // r_k x q_k
        blk_gemm<double>(ra, qb, qa, S, qa, false, C, qb, false, Y, qb, 1.0, false);
        __syncthreads();
        blk_gemm<double>(qb, qb, ra, Y, qb, true, Y, qb, false, acc, qb, 1.0, true);
      }
    }
    __syncthreads();
  }
  double* out = P.red + J.red + (long long)b * dim * dim;
  for (int i = threadIdx.x; i < dim * dim; i += blockDim.x) out[i] = acc[i];
}

// sums the partials of every job in block order and stores the result
__global__ void k_reduce_finish(const DevProb P, const JobList L) {
  const Job J = L.job[blockIdx.x];
  if (J.dst < 0) return;
  const int dd = J.dim * J.dim;
  for (int i = threadIdx.x; i < dd; i += blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < J.nb; ++b) a += P.red[J.red + (long long)b * dd + i];
    P.small[J.dst + i] = a;
  }
}

__global__ void k_eps_alpha(const DevProb P) {
  __shared__ double sh[kDenseThreads];
  double v = 0.0;
  for (int x = threadIdx.x; x < P.n[0]; x += blockDim.x) v += P.s[0][x];
  double g2 = blk_sum(v, sh);
  if (threadIdx.x == 0) {
    double eps = P.scal[SC_EPS_FIXED] > 0.0 ? P.scal[SC_EPS_FIXED]
                                            : fmax(P.scal[SC_EPS_REL] * g2 * P.inv_min_n, 1e-300);
    double alpha = P.scal[SC_ALPHA_OVR] > 0.0 ? P.scal[SC_ALPHA_OVR] : P.scal[SC_ALPHA_SCALE] * sqrt(eps) / P.p;
    P.scal[SC_G2] = g2;
    P.scal[SC_EPS] = eps;
    P.scal[SC_ALPHA] = alpha;
    if (!isfinite(g2)) P.scal[SC_FLAGS] = (double)(((int)P.scal[SC_FLAGS]) | 1);
  }
}

// Lam[k]^{-1}, Gam[k]^{-1} and Q_k = Lam[k+1]^{-1} H_k Gam[k+1]^{-1}
__global__ void __launch_bounds__(kDenseThreads) k_small_proj(const DevProb P) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int flag;
  const int m = P.m;
  double* A = sm;                       // 32 x 32
  double* work = sm + TTC_MAXR * TTC_MAXR;
  double* t1 = work + TTC_MAXR * TTC_MAXR;
  int bad = 0;
  for (int k = 1; k < m; ++k) {       // Lam[k], k = 1..m-1 (Lam[0] = 1)
    const int r = P.r[k];
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) A[i] = P.small[P.off_lam[k] + i];
    __syncthreads();
    bad |= blk_spd_inverse(A, r, work, &flag);
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) P.small[P.off_lami[k] + i] = A[i];
    __syncthreads();
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) A[i] = P.small[P.off_gam[k] + i];
    __syncthreads();
    bad |= blk_spd_inverse(A, r, work, &flag);
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) P.small[P.off_gami[k] + i] = A[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.small[P.off_lami[0]] = 1.0 / P.small[P.off_lam[0]];
    P.small[P.off_gami[m]] = 1.0 / P.small[P.off_gam[m]];
  }
  __syncthreads();
  for (int k = 0; k + 1 < m; ++k) {
    const int r = P.r[k + 1];
    blk_gemm<double>(r, r, r, P.small + P.off_lami[k + 1], r, false, P.small + P.off_h[k], r, false, t1, r, 1.0, false);
    __syncthreads();
    blk_gemm<double>(r, r, r, t1, r, false, P.small + P.off_gami[k + 1], r, false, P.small + P.off_qm[k], r, 1.0,
                     false);
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) P.scal[SC_FLAGS] = (double)(((int)P.scal[SC_FLAGS]) | 2);
}

// one block per slice (k, x): B_k(x) and the block core C_k(x)
__global__ void __launch_bounds__(128) k_build_C(const DevProb P) {
  __shared__ double t1[TTC_MAXR * TTC_MAXR];
  __shared__ double B[TTC_MAXR * TTC_MAXR];
  int blk = blockIdx.x, k = 0;
  while (k < P.m - 1 && blk >= P.n[k]) {
    blk -= P.n[k];
    ++k;
  }
  const int x = blk, m = P.m;
  const int ra = P.r[k], rb = P.r[k + 1];
  const double alpha = P.scal[SC_ALPHA];
  const double wi = wpow(P, k, x, -1.0 / (2.0 * m));
  const double* T = P.core64[k] + (long long)x * ra * rb;
  const double* E = P.E[k] + (long long)x * ra * rb;
  // t1 = Lam[k]^{-1} E
  blk_gemm<double>(ra, rb, ra, P.small + P.off_lami[k], ra, false, E, rb, false, t1, rb, 1.0, false);
  __syncthreads();
  // B = -alpha wi t1 Gam[k+1]^{-1}
  blk_gemm<double>(ra, rb, rb, t1, rb, false, P.small + P.off_gami[k + 1], rb, false, B, rb, -alpha * wi, false);
  __syncthreads();
  if (k + 1 < m) {   // B += alpha T Q_k
    blk_gemm<double>(ra, rb, rb, T, rb, false, P.small + P.off_qm[k], rb, false, B, rb, alpha, true);
    __syncthreads();
  }
  const int qa = P.q[k], qb = P.q[k + 1];
  double* C = P.C[k] + (long long)x * qa * qb;
  for (int i = threadIdx.x; i < qa * qb; i += blockDim.x) {
    int a = i / qb, b = i % qb;
    double v;
    if (k == 0) {            // [B T]
      v = (b < rb) ? B[a * rb + b] : T[a * rb + (b - rb)];
    } else if (k == m - 1) { // [[T], [T + B]]
      v = (a < ra) ? T[a * rb + b] : T[(a - ra) * rb + b] + B[(a - ra) * rb + b];
    } else {                 // [[T, 0], [B, T]]
      if (a < ra)
        v = (b < rb) ? T[a * rb + b] : 0.0;
      else
        v = (b < rb) ? B[(a - ra) * rb + b] : T[(a - ra) * rb + (b - rb)];
    }
    C[i] = v;
  }
}

// Truncated-SVD factor of bond k: N_k from partials, K from Psi[k+1],
// eigen of K^T N_k K, P_k and S_k.
__global__ void __launch_bounds__(kDenseThreads) k_sweep_factor(const DevProb P, int k, long long red, int nb) {
  extern __shared__ __align__(16) double sm[];
  const int q = P.q[k + 1], r = P.r[k + 1];
  const int qq = q * q;
  double* Nk = sm;
  double* A = Nk + qq;
  double* V = A + qq;
  double* K = V + qq;
  double* T1 = K + qq;
  double* w = T1 + qq;
  double* work = w + TTC_MAXQ;
  for (int i = threadIdx.x; i < qq; i += blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += P.red[red + (long long)b * qq + i];
    Nk[i] = a;
    A[i] = P.small[P.off_psi[k + 1] + i];
  }
  __syncthreads();
  blk_sym_eig(A, q, V, w, work);
  for (int i = threadIdx.x; i < qq; i += blockDim.x) {
    int c = i % q;
    K[i] = V[i] * sqrt(fmax(w[c], 0.0));
  }
  __syncthreads();
  blk_gemm<double>(q, q, q, Nk, q, false, K, q, false, T1, q, 1.0, false);   // N K
  __syncthreads();
  blk_gemm<double>(q, q, q, K, q, true, T1, q, false, A, q, 1.0, false);    // K^T N K
  __syncthreads();
  blk_sym_eig(A, q, V, w, work);
  // P = K V[:, :r] diag(1/sigma)
  __shared__ int lost;
  if (threadIdx.x == 0) lost = 0;
  __syncthreads();
  double* Pk = P.small + P.off_pk[k];
  double smax = sqrt(fmax(w[0], 0.0));
  for (int i = threadIdx.x; i < q * r; i += blockDim.x) {
    int a = i / r, c = i % r;
    double sig = sqrt(fmax(w[c], 0.0));
    double acc = 0.0;
    for (int t = 0; t < q; ++t) acc = fma(K[a * q + t], V[t * q + c], acc);
    if (sig > 1e-300 && sig > 1e-14 * smax) {
      T1[i] = acc / sig;
    } else {
      T1[i] = 0.0;
      lost = 1;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < q * r; i += blockDim.x) Pk[i] = T1[i];
  // S = P^T N  (r x q)
  blk_gemm<double>(r, q, q, T1, r, true, Nk, q, false, P.small + P.off_sk[k], q, 1.0, false);
  if (threadIdx.x == 0 && lost) P.scal[SC_FLAGS] = (double)(((int)P.scal[SC_FLAGS]) | 2);
}

// new core k: T_k(x) = S_{k-1} C_k(x) P_k  (P_k omitted for the last core)
__global__ void __launch_bounds__(128) k_sweep_map(const DevProb P, int k) {
  __shared__ double Y[TTC_MAXR * TTC_MAXQ];
  const int x = blockIdx.x, m = P.m;
  const int qa = P.q[k], qb = P.q[k + 1];
  const int ra = P.r[k], rb = P.r[k + 1];
  const double* C = P.C[k] + (long long)x * qa * qb;
  double* T = P.core64[k] + (long long)x * ra * rb;
  float* T32 = P.core32[k] + (long long)x * ra * rb;
  const double* Cp = C;
  if (k > 0) {
    blk_gemm<double>(ra, qb, qa, P.small + P.off_sk[k - 1], qa, false, C, qb, false, Y, qb, 1.0, false);
    __syncthreads();
    Cp = Y;
  }
  if (k < m - 1) {
    const double* Pk = P.small + P.off_pk[k];
    for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
      int a = i / rb, b = i % rb;
      double acc = 0.0;
      for (int t = 0; t < qb; ++t) acc = fma(Cp[a * qb + t], Pk[t * rb + b], acc);
      T[i] = acc;
      T32[i] = (float)acc;
    }
  } else {
    for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
      T[i] = Cp[i];
      T32[i] = (float)Cp[i];
    }
  }
}

__global__ void k_copy_cores(const DevProb P, int to_prev) {
  // grid-stride over all cores
  long long tot = 0;
  for (int k = 0; k < P.m; ++k) tot += (long long)P.n[k] * P.r[k] * P.r[k + 1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    long long o = i;
    int k = 0;
    while (o >= (long long)P.n[k] * P.r[k] * P.r[k + 1]) {
      o -= (long long)P.n[k] * P.r[k] * P.r[k + 1];
      ++k;
    }
    if (to_prev)
      P.prev64[k][o] = P.core64[k][o];
    else
      P.core32[k][o] = (float)P.core64[k][o];
  }
}

// ---- metrics: squared Frobenius distance between the iterate and another TT
// Dense form (small d*): every entry is evaluated, in FP64.
__global__ void k_dense_diff(const DevProb P, int which, long long dstar, double* part) {
  __shared__ double sh1[256];
  __shared__ double sh2[256];
  double d2 = 0.0, b2 = 0.0;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < dstar; l += (long long)gridDim.x * blockDim.x) {
    int xs[TTC_MAXM];
    long long t = l;
    for (int k = P.m - 1; k >= 0; --k) {
      xs[k] = (int)(t % P.n[k]);
      t /= P.n[k];
    }
    double va[TTC_MAXQ], vb[TTC_MAXQ], tmp[TTC_MAXQ];
    va[0] = 1.0;
    vb[0] = 1.0;
    for (int k = 0; k < P.m; ++k) {
      int ra = P.r[k], rb = P.r[k + 1];
      const double* M = P.core64[k] + (long long)xs[k] * ra * rb;
      for (int b = 0; b < rb; ++b) {
        double acc = 0.0;
        for (int a = 0; a < ra; ++a) acc = fma(va[a], M[a * rb + b], acc);
        tmp[b] = acc;
      }
      for (int b = 0; b < rb; ++b) va[b] = tmp[b];
      int sa = which == 0 ? P.rt[k] : P.r[k], sb = which == 0 ? P.rt[k + 1] : P.r[k + 1];
      const double* Mb = (which == 0 ? P.truth[k] : P.prev64[k]) + (long long)xs[k] * sa * sb;
      for (int b = 0; b < sb; ++b) {
        double acc = 0.0;
        for (int a = 0; a < sa; ++a) acc = fma(vb[a], Mb[a * sb + b], acc);
        tmp[b] = acc;
      }
      for (int b = 0; b < sb; ++b) vb[b] = tmp[b];
    }
    double d = va[0] - vb[0];
    d2 = fma(d, d, d2);
    b2 = fma(vb[0], vb[0], b2);
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

__global__ void k_dense_diff_finish(const DevProb P, const double* part, int nb) {
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
      a += part[2 * i];
      b += part[2 * i + 1];
    }
    P.scal[SC_METRIC] = a;
    P.scal[SC_NORM] = b;
  }
}

// Gram-sweep form (any d*): Lam_XY <- sum_x X_k(x)^T Lam_XY Y_k(x) for the pairs
// (A,A), (A,B), (B,B); one block walks all slices of one core in order.
__global__ void __launch_bounds__(kDenseThreads) k_gram_diff_step(const DevProb P, int which, int k, double* lam) {
  extern __shared__ __align__(16) double sm[];
  const int ra = P.r[k], rb = P.r[k + 1];
  const int sa = which == 0 ? P.rt[k] : P.r[k], sb = which == 0 ? P.rt[k + 1] : P.r[k + 1];
  const double* Bc = which == 0 ? P.truth[k] : P.prev64[k];
  // lam layout: [AA: 64x64][AB: 64x64][BB: 64x64] (leading dim = current dims)
  double* LAA = lam;
  double* LAB = lam + TTC_MAXQ * TTC_MAXQ;
  double* LBB = LAB + TTC_MAXQ * TTC_MAXQ;
  double* nAA = sm;
  double* nAB = nAA + TTC_MAXQ * TTC_MAXQ;
  double* nBB = nAB + TTC_MAXQ * TTC_MAXQ;
  double* Y = nBB + TTC_MAXQ * TTC_MAXQ;
  for (int i = threadIdx.x; i < 3 * TTC_MAXQ * TTC_MAXQ; i += blockDim.x) sm[i] = 0.0;
  __syncthreads();
  for (int x = 0; x < P.n[k]; ++x) {
    const double* A = P.core64[k] + (long long)x * ra * rb;
    const double* B = Bc + (long long)x * sa * sb;
    blk_gemm<double>(ra, rb, ra, LAA, ra, false, A, rb, false, Y, rb, 1.0, false);
    __syncthreads();
    blk_gemm<double>(rb, rb, ra, A, rb, true, Y, rb, false, nAA, rb, 1.0, true);
    __syncthreads();
    blk_gemm<double>(ra, sb, sa, LAB, sa, false, B, sb, false, Y, sb, 1.0, false);
    __syncthreads();
    blk_gemm<double>(rb, sb, ra, A, rb, true, Y, sb, false, nAB, sb, 1.0, true);
    __syncthreads();
    blk_gemm<double>(sa, sb, sa, LBB, sa, false, B, sb, false, Y, sb, 1.0, false);
    __syncthreads();
    blk_gemm<double>(sb, sb, sa, B, sb, true, Y, sb, false, nBB, sb, 1.0, true);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 3 * TTC_MAXQ * TTC_MAXQ; i += blockDim.x) lam[i] = sm[i];
  __syncthreads();
  if (k == P.m - 1 && threadIdx.x == 0) {
    P.scal[SC_METRIC] = LAA[0] - 2.0 * LAB[0] + LBB[0];
    P.scal[SC_NORM] = LBB[0];
  }
}

__global__ void k_gram_diff_init(double* lam) {
  for (int i = threadIdx.x; i < 3 * TTC_MAXQ * TTC_MAXQ; i += blockDim.x) lam[i] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    lam[0] = 1.0;
    lam[TTC_MAXQ * TTC_MAXQ] = 1.0;
    lam[2 * TTC_MAXQ * TTC_MAXQ] = 1.0;
  }
}

// ---- host-side plan -------------------------------------------------------
struct Plan {
  std::vector<JobList> gram_steps;   // step j: Lam[j+1], Gam[m-1-j] (+ all H jobs at j = 0)
  std::vector<JobList> psi_steps;    // k = m-1 .. 1
  std::vector<JobList> n_steps;      // k = 0 .. m-2
  long long red_total = 0;
  double* metric_part = nullptr;
  double* gram_lam = nullptr;
};

inline int nblocks_for(int nk) { return std::max(1, std::min(nk, 1024)); }

}  // namespace

// reduction plans, one per context
#include <map>
#include <mutex>
static std::map<const ttc_ctx*, Plan> g_plan_of;
static std::mutex g_plan_mu;
static Plan& plan_of(const ttc_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  return g_plan_of[c];
}

int ttc_alloc_dense(ttc_ctx* c) {
  DevProb& P = c->hp;
  const int m = c->m;
  P.q[0] = 1;
  P.q[m] = 1;
  for (int k = 1; k < m; ++k) P.q[k] = 2 * c->r[k];
  // small matrices
  int off = 0;
  auto take = [&](int count) {
    int o = off;
    off += (count + 7) & ~7;
    return o;
  };
  for (int k = 0; k <= m; ++k) {
    int r = c->r[k];
    P.off_lam[k] = take(r * r);
    P.off_gam[k] = take(r * r);
    P.off_lami[k] = take(r * r);
    P.off_gami[k] = take(r * r);
    P.off_psi[k] = take(P.q[k] * P.q[k]);
  }
  for (int k = 0; k < m; ++k) {
    int r = c->r[k + 1], q = P.q[k + 1];
    P.off_h[k] = take(r * r);
    P.off_qm[k] = take(r * r);
    P.off_nk[k] = take(q * q);
    P.off_pk[k] = take(q * r);
    P.off_sk[k] = take(r * q);
  }
  double* small = nullptr;
  TTC_TRY(ttc_alloc(c, (void**)&small, sizeof(double) * (size_t)off, false));
  TTC_CUDA(cudaMemset(small, 0, sizeof(double) * (size_t)off));
  P.small = small;
  // Lam[0] = Gam[m] = Psi[m] = [1]
  double one = 1.0;
  TTC_CUDA(cudaMemcpy(small + P.off_lam[0], &one, sizeof(double), cudaMemcpyHostToDevice));
  TTC_CUDA(cudaMemcpy(small + P.off_gam[m], &one, sizeof(double), cudaMemcpyHostToDevice));
  TTC_CUDA(cudaMemcpy(small + P.off_psi[m], &one, sizeof(double), cudaMemcpyHostToDevice));
  for (int k = 0; k < m; ++k) {
    double* Ck = nullptr;
    TTC_TRY(ttc_alloc(c, (void**)&Ck, sizeof(double) * (size_t)c->n[k] * P.q[k] * P.q[k + 1], false));
    P.C[k] = Ck;
    double* pv = nullptr;
    TTC_TRY(ttc_alloc(c, (void**)&pv, sizeof(double) * (size_t)c->n[k] * c->r[k] * c->r[k + 1], false));
    P.prev64[k] = pv;
  }
  double* scal = nullptr;
  TTC_TRY(ttc_alloc(c, (void**)&scal, sizeof(double) * SC_COUNT, false));
  TTC_CUDA(cudaMemset(scal, 0, sizeof(double) * SC_COUNT));
  P.scal = scal;

  // reduction plan
  Plan pl;
  long long red = 0;
  auto mk = [&](int op, int k, int dim, int dst) {
    Job J;
    J.op = op;
    J.k = k;
    J.nb = nblocks_for((int)c->n[k]);
    J.dim = dim;
    J.red = red;
    J.dst = dst;
    red += (long long)J.nb * dim * dim;
    return J;
  };
  for (int j = 0; j + 1 < m; ++j) {
    JobList L;
    L.njob = 0;
    L.job[L.njob++] = mk(OP_LAM, j, c->r[j + 1], P.off_lam[j + 1]);
    int kg = m - 1 - j;
    L.job[L.njob++] = mk(OP_GAM, kg, c->r[kg], P.off_gam[kg]);
    if (j == 0)
      for (int k = 0; k + 1 < m; ++k) L.job[L.njob++] = mk(OP_H, k, c->r[k + 1], P.off_h[k]);
    pl.gram_steps.push_back(L);
  }
  for (int k = m - 1; k >= 1; --k) {
    JobList L;
    L.njob = 1;
    L.job[0] = mk(OP_PSI, k, P.q[k], P.off_psi[k]);
    pl.psi_steps.push_back(L);
  }
  for (int k = 0; k + 1 < m; ++k) {
    JobList L;
    L.njob = 1;
    L.job[0] = mk(OP_N, k, P.q[k + 1], -1);
    pl.n_steps.push_back(L);
  }
  pl.red_total = red;
  double* redp = nullptr;
  TTC_TRY(ttc_alloc(c, (void**)&redp, sizeof(double) * (size_t)std::max(red, 1LL), false));
  P.red = redp;
  TTC_TRY(ttc_alloc(c, (void**)&pl.metric_part, sizeof(double) * 2 * 1024, false));
  TTC_TRY(ttc_alloc(c, (void**)&pl.gram_lam, sizeof(double) * 3 * TTC_MAXQ * TTC_MAXQ, false));
  plan_of(c) = pl;

  // shared-memory opt-ins
  int qmax = 1;
  for (int k = 0; k <= m; ++k) qmax = std::max(qmax, P.q[k]);
  size_t red_smem = sizeof(double) * 2 * TTC_MAXQ * TTC_MAXQ;
  TTC_CUDA(cudaFuncSetAttribute(k_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red_smem));
  size_t fac_smem = sizeof(double) * (5 * TTC_MAXQ * TTC_MAXQ + TTC_MAXQ + TTC_MAXQ * TTC_MAXQ + 4 * TTC_MAXQ + kDenseThreads);
  TTC_CUDA(cudaFuncSetAttribute(k_sweep_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fac_smem));
  size_t gd_smem = sizeof(double) * 4 * TTC_MAXQ * TTC_MAXQ;
  TTC_CUDA(cudaFuncSetAttribute(k_gram_diff_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gd_smem));
  return TTC_OK;
}

static int launch_jobs(ttc_ctx* c, const JobList& L) {
  int nb = 0;
  for (int j = 0; j < L.njob; ++j) nb += L.job[j].nb;
  size_t smem = sizeof(double) * 2 * TTC_MAXQ * TTC_MAXQ;
  k_reduce<<<nb, kDenseThreads, smem, c->stream>>>(c->hp, L);
  TTC_CUDA(cudaGetLastError());
  k_reduce_finish<<<L.njob, 256, 0, c->stream>>>(c->hp, L);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 2;
  return TTC_OK;
}

int ttc_launch_dense(ttc_ctx* c) {
  const DevProb& P = c->hp;
  const int m = c->m;
  Plan& pl = plan_of(c);
  cudaStream_t st = c->stream;
  k_eps_alpha<<<1, kDenseThreads, 0, st>>>(P);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  for (auto& L : pl.gram_steps) TTC_TRY(launch_jobs(c, L));
  size_t sp_smem = sizeof(double) * 3 * TTC_MAXR * TTC_MAXR;
  k_small_proj<<<1, kDenseThreads, sp_smem, st>>>(P);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  int nslices = 0;
  for (int k = 0; k < m; ++k) nslices += (int)c->n[k];
  k_build_C<<<nslices, 128, 0, st>>>(P);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  for (auto& L : pl.psi_steps) TTC_TRY(launch_jobs(c, L));
  size_t fac_smem = sizeof(double) * (5 * TTC_MAXQ * TTC_MAXQ + TTC_MAXQ + TTC_MAXQ * TTC_MAXQ + 4 * TTC_MAXQ + kDenseThreads);
  for (int k = 0; k + 1 < m; ++k) {
    const JobList& L = pl.n_steps[k];
    size_t smem = sizeof(double) * 2 * TTC_MAXQ * TTC_MAXQ;
    k_reduce<<<L.job[0].nb, kDenseThreads, smem, st>>>(P, L);
    TTC_CUDA(cudaGetLastError());
    k_sweep_factor<<<1, kDenseThreads, fac_smem, st>>>(P, k, L.job[0].red, L.job[0].nb);
    TTC_CUDA(cudaGetLastError());
    k_sweep_map<<<(int)c->n[k], 128, 0, st>>>(P, k);
    TTC_CUDA(cudaGetLastError());
    c->nlaunch += 3;
  }
  k_sweep_map<<<(int)c->n[m - 1], 128, 0, st>>>(P, m - 1);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  return TTC_OK;
}

int ttc_launch_save_prev(ttc_ctx* c) {
  k_copy_cores<<<264, 256, 0, c->stream>>>(c->hp, 1);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  return TTC_OK;
}

int ttc_launch_mirror32(ttc_ctx* c) {
  k_copy_cores<<<264, 256, 0, c->stream>>>(c->hp, 0);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  return TTC_OK;
}

int ttc_launch_metric(ttc_ctx* c, int which) {
  const DevProb& P = c->hp;
  Plan& pl = plan_of(c);
  if (which == 0 && !P.has_truth) return TTC_EINVAL;
  if (P.dstar > 0 && P.dstar <= (1LL << 20)) {
    int nb = (int)std::min<long long>(1024, (P.dstar + 255) / 256);
    k_dense_diff<<<nb, 256, 0, c->stream>>>(P, which, P.dstar, pl.metric_part);
    TTC_CUDA(cudaGetLastError());
    k_dense_diff_finish<<<1, 32, 0, c->stream>>>(P, pl.metric_part, nb);
    TTC_CUDA(cudaGetLastError());
    c->nlaunch += 2;
    return TTC_OK;
  }
  k_gram_diff_init<<<1, 256, 0, c->stream>>>(pl.gram_lam);
  size_t smem = sizeof(double) * 4 * TTC_MAXQ * TTC_MAXQ;
  for (int k = 0; k < P.m; ++k) {
    k_gram_diff_step<<<1, kDenseThreads, smem, c->stream>>>(P, which, k, pl.gram_lam);
    TTC_CUDA(cudaGetLastError());
  }
  c->nlaunch += 1 + P.m;
  return TTC_OK;
}

void ttc_free_plan(const ttc_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plan_of.erase(c);
}
