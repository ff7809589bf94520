// Dense stage of one PRGD iteration on the device (FP64 results):
//
//  (1) eps_l, alpha_l from ||G_l||^2 (step-size form of Theorem 4.1); done by
//      the last block of the slice reduction of the sampled pass.
//      G_k(x) = eps + s_k(x) is the diagonal of G_{l,k} (Section 3.2).
//  (2) Grams of T^ = W^{1/2} T (Proposition 3.1: T^_k(x) = G_k(x)^{1/(4m)} T_k(x)):
//        Lam[k+1] = sum_x G_k(x)^{1/(2m)} T_k(x)^T Lam[k] T_k(x)      (left)
//        Gam[k]   = sum_x G_k(x)^{1/(2m)} T_k(x) Gam[k+1] T_k(x)^T    (right)
//      and H_k = sum_x T_k(x)^T E_k(x).
//  (3) The weighted tangent projection of Lemma 3.5 (Eq. (tsp in nm)), taken
//      at the left-orthogonal decomposition U of T^ with T^<=k = U^<=k R_k,
//      R_k^T R_k = Lam[k], written back in the gauge of the iterate's own
//      cores.  With the sparse factor E_k of the sampled pass, the update core
//      of W_l = T_l - alpha tilde P_T W^{-1} G_l for mode k is
//        B_k(x) = -alpha [ G_k(x)^{-1/(2m)} Lam[k]^{-1} E_k(x) Gam[k+1]^{-1}
//                          - T_k(x) Lam[k+1]^{-1} H_k Gam[k+1]^{-1} ]    (k < d-1)
//        B_{d-1}(x) = -alpha G_{d-1}(x)^{-1/(2m)} Lam[d-1]^{-1} E_{d-1}(x),
//      i.e. R_{k-1}^{-1} (-alpha G_k^{-1/(4m)} A^_k) R_k with A^_k the Lemma 3.5
//      component: weights and R factors cancel into r x r Gram inverses.
//  (4) W_l in rank-2r TT form (rank bound of Section 3.1):
//        C_0 = [B_0  T_0],  C_k = [[T_k, 0], [B_k, T_k]],  C_{d-1} = [[T_{d-1}], [T_{d-1} + B_{d-1}]].
//  (5) T_{l+1} = SVD^tt_r(W_l), Algorithm 1 evaluated on the rank-2r TT:
//      right Grams Psi[k] = sum_x C_k(x) Psi[k+1] C_k(x)^T; then bond by bond,
//      with C'_k = S_{k-1} C_k and N_k = sum_x C'_k(x)^T C'_k(x), the top-r
//      left singular vectors of (T^{<=k-1} (x) I)^T W^{<k>} = L(C'_k) C^{>=k+1}
//      are L(C'_k) u for the dominant r-dimensional invariant subspace u of
//      Psi[k+1] N_k (since M M^T L(C') u = L(C') Psi N u).  That subspace is
//      u = R_P^T w, w the top-r right singular vectors of G = R_N R_P^T
//      (upper Cholesky factors N_k = R_N^T R_N, Psi[k+1] = R_P^T R_P), from a
//      one-sided Jacobi SVD of G (FP32 sweeps, FP64 sweeps in FP64 steps); the
//      new core is T_k(x) = C'_k(x) P_k with P_k = U R^{-1}, R^T R = U^T N_k U,
//      so it is left-orthogonal; S_k = P_k^T N_k; the last core is S_{d-2} C_{d-1}.
//      This is Algorithm 1 itself, not an approximation of it.
//
// FP64 on GB300 issues ~1.7 FMAs per clock per SM (a dependent FMA of each of
// a block's 8 warps every ~150 cycles), so every factorization
// with a long sequential chain runs in FP32 (Cholesky) and is lifted to FP64
// accuracy by matrix products only (Newton-Schulz for inverses, a second-order
// correction for the final normalisation).
//
// Reductions over slices are split over blocks; the last block to finish sums
// the block partials in block order (deterministic) and runs the small
// factorization that follows, so each stage is one launch.  The powers
// G_k(x)^{+-1/(2m)} are computed once per step into a per-slice table by the
// kernel that saves the previous cores, which runs after the slice reduction
// (when eps is final) and before the first stage.  In a batch, members on the
// warp-per-slice path run each stage as one launch over a chunk of members
// (blocks mapped to members by prefix arrays).
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <mutex>
#include <vector>

#include "ctx.h"
#include "ff.cuh"
#include "linalg.cuh"

namespace {

enum Op { OP_LAM = 0, OP_GAM = 1, OP_H = 2, OP_PSI = 3, OP_N = 4, OP_DAA = 5, OP_DAB = 6, OP_DBB = 7 };
enum Post { POST_NONE = 0, POST_SMALL_PROJ = 1, POST_BOND = 2, POST_METRIC = 3 };

struct Job {
  int op, k;
  int nb;            // reduction blocks
  int rows, cols;    // output is rows x cols
  long long red;     // offset in P.red of the block partials
  long long red2;    // offset in P.red2 of the group partials (groups of kGroup blocks)
  int dst;           // offset in P.small of the result
};

struct Stage {
  int njob;
  int post, post_k;
  int counter;       // index into P.counters
  int which;         // metric stages: 0 truth, 1 previous iterate
  int nmap;          // slice maps run by the first blocks
  int map_k[2];
  int map_nb[2];     // blocks of each map on the block-per-slice path (slices strided over them)
  Job job[TTC_MAXM + 4];
};

// Outputs a warp-per-slice job computes: the Grams Lam, Gam, Psi and N are
// symmetric, so only their upper triangles (row <= column, packed row by
// row) are accumulated and mirrored; T^T E (OP_H) is computed whole.
__host__ __device__ inline bool warp_job_sym(const Job& J) { return J.op != OP_H; }
__host__ __device__ inline int warp_job_outputs(const Job& J) {
  return warp_job_sym(J) ? J.rows * (J.rows + 1) / 2 : J.rows * J.cols;
}

constexpr int kThreads = 256;
constexpr int kWarpJacobiMax = 16;   // widest bond whose FP32 Jacobi sweeps run on one warp

// y = v^{-1/(2m)} by Newton's iteration for inverse roots,
// y <- y (1 + (1 - v y^{2m}) / (2m)), started from the FP32 power (relative
// error ~1e-7); each step squares the error, two steps reach FP64 rounding.
// (No FP64 pow or division: long FP64 chains are slow on this GPU, ~1.7 FP64
// FMAs per clock per SM.)
__device__ __forceinline__ double ipow_2m(double y, int two_m) {
  double acc = 1.0, base = y;
  for (int e = two_m; e > 0; e >>= 1) {
    if (e & 1) acc *= base;
    base *= base;
  }
  return acc;
}
// c = 1/(2m) in FP64 (from the descriptor)
__device__ __forceinline__ double inv_root(double v, int m, double c) {
  const int two_m = 2 * m;
  // seed: v^{-1/(2m)} = 2^{-(e + log2 f)/(2m)} with v = f 2^e and
  // e = 2m q + rr (0 <= rr < 2m, integer division): 2^{-q}, built exactly
  // from its exponent bits (|q| <= 512 for normal v), times the FP32 power
  // 2^{-(rr + log2 f)/(2m)} of an argument in (-1, 1/(2m)]; relative error
  // ~1e-7, FP64 rounding after the two Newton steps
  int e;
  const double f = frexp(v, &e);
  int q = e / two_m, rr = e - q * two_m;
  if (rr < 0) {
    rr += two_m;
    q -= 1;
  }
  const float tf = -((float)rr + log2f((float)f)) * (float)c;
  double y = (double)exp2f(tf) * __longlong_as_double((long long)(1023 - q) << 52);
  for (int it = 0; it < 2; ++it) y = y * fma(c, fma(-v, ipow_2m(y, two_m), 1.0), 1.0);
  return y;
}
// the slice weights of this step, G_k(x) = eps + s_k(x) (Eq. 3.2's diagonal
// preconditioner): wt[k][2x] = G^{+1/(2m)}, wt[k][2x+1] = G^{-1/(2m)}, one
// thread per slice, written once per step after the slice energies and eps
// are final and read by every dense stage
__device__ __forceinline__ void slice_weights(const DevProb& P, long long t, long long nt) {
  if (P.uniform) return;
  const double eps = P.scal[SC_EPS];
  for (int k = 0; k < P.m; ++k) {
    for (long long x = t; x < P.n[k]; x += nt) {
      const double v = eps + P.s[k][x];
      const double y = inv_root(v, P.m, P.inv_2m);                        // v^{-1/(2m)}
      P.wt[k][2 * x] = v * ipow_2m(y, 2 * P.m - 1);                       // v^{1/(2m)} = v * y^{2m-1}
      P.wt[k][2 * x + 1] = y;
    }
  }
}
// G_k(x)^{+1/(2m)} (sign > 0) or G_k(x)^{-1/(2m)} (sign < 0); 1 with the
// uniform metric (RGD)
__device__ __forceinline__ double gpow(const DevProb& P, int k, int x, int sign) {
  if (P.uniform) return 1.0;
  return P.wt[k][2 * x + (sign < 0 ? 1 : 0)];
}

// ---- per-slice contributions ------------------------------------------------
__device__ void slice_contrib(const DevProb& P, const Stage& S, const Job& J, int x, double* acc, double* Y) {
  const int k = J.k;
  const int ra = P.r[k], rb = P.r[k + 1];
  const double* T = P.core64[k] + (long long)x * ra * rb;
  switch (J.op) {
    case OP_LAM: {   // acc += w2 T^T (Lam T)
      blk_gemm<double>(ra, rb, ra, P.small + P.off_lam[k], ra, false, T, rb, false, Y, rb, 1.0, false);
      __syncthreads();
      blk_gemm<double>(rb, rb, ra, T, rb, true, Y, rb, false, acc, rb, gpow(P, k, x, +1), true);
      break;
    }
    case OP_GAM: {   // acc += w2 (T Gam) T^T
      blk_gemm<double>(ra, rb, rb, T, rb, false, P.small + P.off_gam[k + 1], rb, false, Y, rb, 1.0, false);
      __syncthreads();
      blk_gemm<double>(ra, ra, rb, Y, rb, false, T, rb, true, acc, ra, gpow(P, k, x, +1), true);
      break;
    }
    case OP_H: {     // acc += T^T E
      const double* E = P.E[k] + (long long)x * ra * rb;
      blk_gemm<double>(rb, rb, ra, T, rb, true, E, rb, false, acc, rb, 1.0, true);
      break;
    }
    case OP_PSI: {   // acc += (C Psi) C^T
      const int qa = P.q[k], qb = P.q[k + 1];
      const double* C = P.C[k] + (long long)x * qa * qb;
      blk_gemm<double>(qa, qb, qb, C, qb, false, P.small + P.off_psi[k + 1], qb, false, Y, qb, 1.0, false);
      __syncthreads();
      blk_gemm<double>(qa, qa, qb, Y, qb, false, C, qb, true, acc, qa, 1.0, true);
      break;
    }
    case OP_N: {     // C' = S_{k-1} C ; acc += C'^T C'
      const int qa = P.q[k], qb = P.q[k + 1];
      const double* C = P.C[k] + (long long)x * qa * qb;
      if (k == 0) {
        blk_gemm<double>(qb, qb, qa, C, qb, true, C, qb, false, acc, qb, 1.0, true);
      } else {
        blk_gemm<double>(ra, qb, qa, P.small + P.off_sk[k - 1], qa, false, C, qb, false, Y, qb, 1.0, false);
        __syncthreads();
        blk_gemm<double>(qb, qb, ra, Y, qb, true, Y, qb, false, acc, qb, 1.0, true);
      }
      break;
    }
    default: {       // Gram sweep of the iterate A and another TT B
      const int sa = S.which == 0 ? P.rt[k] : P.r[k], sb = S.which == 0 ? P.rt[k + 1] : P.r[k + 1];
      const double* B = (S.which == 0 ? P.truth[k] : P.prev64[k]) + (long long)x * sa * sb;
      if (J.op == OP_DAA) {
        blk_gemm<double>(ra, rb, ra, P.small + P.off_mlam[0][k], ra, false, T, rb, false, Y, rb, 1.0, false);
        __syncthreads();
        blk_gemm<double>(rb, rb, ra, T, rb, true, Y, rb, false, acc, rb, 1.0, true);
      } else if (J.op == OP_DAB) {
        blk_gemm<double>(ra, sb, sa, P.small + P.off_mlam[1][k], sa, false, B, sb, false, Y, sb, 1.0, false);
        __syncthreads();
        blk_gemm<double>(rb, sb, ra, T, rb, true, Y, sb, false, acc, sb, 1.0, true);
      } else {
        blk_gemm<double>(sa, sb, sa, P.small + P.off_mlam[2][k], sa, false, B, sb, false, Y, sb, 1.0, false);
        __syncthreads();
        blk_gemm<double>(sb, sb, sa, B, sb, true, Y, sb, false, acc, sb, 1.0, true);
      }
      break;
    }
  }
  __syncthreads();
}

// ---- small factorizations run by the last block ----------------------------

// Lam[k]^{-1}, Gam[k]^{-1} (k = 1..d-1), then Q_k = Lam[k+1]^{-1} H_k Gam[k+1]^{-1};
// one warp per matrix (FP32 Cholesky + FP64 Newton-Schulz); matrices whose
// residual stays above 1e-12 are redone by the block in FP64.
__device__ void post_small_proj(const DevProb& P, double* sm) {
  const int m = P.m, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  __shared__ int redo[2 * TTC_MAXM];
  __shared__ int flag;
  int rmax = 1;
  for (int k = 0; k <= m; ++k) rmax = max(rmax, P.r[k]);
  const int nn = rmax * rmax;
  // per warp: T (2 nn doubles), then L, Li (nn floats each)
  double* T = sm + warp * 2 * nn;
  float* Lf = reinterpret_cast<float*>(sm + nw * 2 * nn) + warp * 2 * nn;
  float* Lif = Lf + nn;
  if (threadIdx.x == 0) flag = 0;
  for (int j = warp; j < 2 * (m - 1); j += nw) {
    const int k = 1 + (j >> 1);
    const int r = P.r[k];
    const double* A = P.small + ((j & 1) ? P.off_gam[k] : P.off_lam[k]);
    double* X = P.small + ((j & 1) ? P.off_gami[k] : P.off_lami[k]);
    double res = warp_spd_inverse(A, r, r, X, r, Lf, Lif, T);
    if (lane == 0) redo[j] = !(res < 1e-12);
  }
  if (threadIdx.x == 0) {
    P.small[P.off_lami[0]] = 1.0 / P.small[P.off_lam[0]];
    P.small[P.off_gami[m]] = 1.0 / P.small[P.off_gam[m]];
  }
  __threadfence_block();
  __syncthreads();
  for (int j = 0; j < 2 * (m - 1); ++j) {          // FP64 fallback, whole block
    if (!redo[j]) continue;
    const int k = 1 + (j >> 1);
    const int r = P.r[k];
    const double* A = P.small + ((j & 1) ? P.off_gam[k] : P.off_lam[k]);
    double* X = P.small + ((j & 1) ? P.off_gami[k] : P.off_lami[k]);
    double* Ac = sm;
    double* work = sm + r * r;
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) Ac[i] = A[i];
    __syncthreads();
    blk_spd_inverse(Ac, r, work, &flag);
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) X[i] = Ac[i];
    __threadfence_block();
    __syncthreads();
  }
  for (int k = warp; k + 1 < m; k += nw) {
    const int r = P.r[k + 1];
    warp_gemm<double>(r, r, r, P.small + P.off_lami[k + 1], r, false, P.small + P.off_h[k], r, false, T, r, 1.0,
                      false);
    warp_gemm<double>(r, r, r, T, r, false, P.small + P.off_gami[k + 1], r, false, P.small + P.off_qm[k], r, 1.0,
                      false);
  }
  __syncthreads();
  if (threadIdx.x == 0 && flag) atomicOr(P.flags, 2u);
}

// sum_{t0 <= t < t1} x[t * sx] y[t * sy] with four independent FP64 chains
// (in a block of 8 warps a dependent FP64 FMA advances every ~150 cycles here)
__device__ __forceinline__ double dot4(const double* x, int sx, const double* y, int sy, int t0, int t1) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int t = t0;
  for (; t + 3 < t1; t += 4) {
    a0 = fma(x[t * sx], y[t * sy], a0);
    a1 = fma(x[(t + 1) * sx], y[(t + 1) * sy], a1);
    a2 = fma(x[(t + 2) * sx], y[(t + 2) * sy], a2);
    a3 = fma(x[(t + 3) * sx], y[(t + 3) * sy], a3);
  }
  for (; t < t1; ++t) a0 = fma(x[t * sx], y[t * sy], a0);
  return (a0 + a1) + (a2 + a3);
}

// Bond k of the retraction: from N_k (in P.small) and Psi[k+1], P_k and S_k.
// The top-r left singular vectors of (T^{<=k-1} (x) I)^T W^{<k>} =
// L(C'_k) C^{>=k+1} are L(C'_k) u, u spanning the dominant r-dimensional
// invariant subspace of Psi[k+1] N_k (M M^T L(C') u = L(C') Psi N u).  With
// the upper Cholesky factors N_k = R_N^T R_N and Psi[k+1] = R_P^T R_P, the
// matrix G = R_N R_P^T has G^T G = R_P N_k R_P^T, so u = R_P^T w for the
// top-r right singular vectors w of G.  Those come from one-sided Jacobi on
// G's columns: FP32 sweeps from the identity, then, when the step needs FP64
// accuracy, FP64 sweeps on G V32 from the FP32 basis (quadratic convergence:
// one or two sweeps).  Jacobi computes the whole SVD, so a small gap between
// the r-th and (r+1)-th singular values costs no extra iterations.
__device__ void post_bond(const DevProb& P, int k, double* sm) {
  const int q = P.q[k + 1], r = P.r[k + 1];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int qq = q * q;
  const int ld = q | 1;            // odd leading dimension of the FP32 Jacobi's columns
  const int qs = q * (q + 1);      // doubles per region
  double* N = sm;                  // q x q, unscaled (the normalisation below)
  double* RP = N + qs;             // Psi (scaled) -> R_P
  double* RN = RP + qs;            // N (scaled) -> R_N -> E -> G V (column-major)
  double* GG = RN + qs;            // G (column-major) -> U, W
  float* G32 = reinterpret_cast<float*>(GG + qs);   // q x ld floats each, column-major (later an FP64 q x q)
  float* V32 = G32 + q * ld;
  double* VD = GG + 2 * qs;        // the FP64 basis V (column-major, leading dimension q)
  double* red = VD + qs;           // blockDim doubles
  double* dg = red + bd;           // 2q doubles
  __shared__ int bad;
  __shared__ int order[TTC_MAXQ];
  __shared__ double scl[2];   // powers of two that scale Psi and N to unit size
  for (int i = tid; i < qq; i += bd) N[i] = P.small[P.off_nk[k] + i];
  if (tid == 0) bad = 0;
  __syncthreads();
  const double* Psi = P.small + P.off_psi[k + 1];
  if (tid < 32) {
    // both are PSD Grams: the largest entry is on the diagonal
    double mp = 0.0, mn = 0.0;
    for (int i = tid; i < q; i += 32) {
      mp = nanmax(mp, fabs(Psi[i * q + i]));
      mn = nanmax(mn, fabs(N[i * q + i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
      mp = nanmax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
      mn = nanmax(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if (tid == 0) {
      int ep = 0, en = 0;
      if (mp > 0.0 && mp <= 1.7e308) frexp(mp, &ep);
      if (mn > 0.0 && mn <= 1.7e308) frexp(mn, &en);
      scl[0] = ldexp(1.0, -ep);
      scl[1] = ldexp(1.0, -en);
    }
  }
  __syncthreads();
  for (int i = tid; i < qq; i += bd) {
    RP[i] = Psi[i] * scl[0];
    RN[i] = N[i] * scl[1];
  }
  blk_chol2_upper_psd(RN, RP, q, dg);
  // R_N transposed (into GG for now), so that lanes with consecutive rows
  // of G read consecutive words below
  for (int idx = tid; idx < qq; idx += bd) {
    const int t = idx / q, i = idx - t * q;
    GG[idx] = RN[i * q + t];
  }
  __syncthreads();
  for (int idx = tid; idx < qq; idx += bd) RN[idx] = GG[idx];
  __syncthreads();
  // G = R_N R_P^T, column-major: G[i][j] = sum_{t >= max(i, j)} R_N[i][t] R_P[j][t]
  double fro = 0.0;
  for (int idx = tid; idx < qq; idx += bd) {
    const int j = idx / q, i = idx - j * q;
    const double acc = dot4(RN + i, q, RP + j * q, 1, max(i, j), q);
    GG[idx] = acc;
    G32[j * ld + i] = (float)acc;
    V32[j * ld + i] = (i == j) ? 1.f : 0.f;
    fro = fma(acc, acc, fro);
  }
  fro = blk_sum(fro, red);   // ||G||_F^2: columns below 1e-14 of it (FP32) are zero
  // FP32 sweeps to 1e-5: the subspace error left (~1e-5 sigma_r sigma_{r+1} /
  // (sigma_r^2 - sigma_{r+1}^2)) moves the iterate by less than the FP32 pass
  // does; FP64 steps refine below
  // up to 16 columns (8 pairs a round, 4 lanes each) one warp runs the
  // rounds without block barriers; wider bonds need the whole block's lanes
  int sweeps = q <= kWarpJacobiMax ? warp_hestenes32(G32, V32, q, ld, 1e-5f, (float)(1e-14 * fro), 24)
                                   : blk_hestenes<float>(G32, V32, q, ld, 1e-5f, (float)(1e-14 * fro), 24);
  const bool fp64 = P.step_fp64 != 0;
  // the basis in FP64 (converted once: conversions are FP64-pipe work)
  for (int idx = tid; idx < qq; idx += bd) {
    const int j = idx / q, i = idx - j * q;
    VD[idx] = (double)V32[j * ld + i];
  }
  if (fp64) {
    // V made orthonormal in FP64, V (I - E/2 + 3 E^2 / 8) with
    // E = V^T V - I (error O(|E|^3)); then FP64 sweeps on G V
    __syncthreads();
    for (int idx = tid; idx < qq; idx += bd) {     // E (R_N is not needed any more)
      const int j = idx / q, i = idx - j * q;
      RN[idx] = dot4(VD + i * q, 1, VD + j * q, 1, 0, q) - ((i == j) ? 1.0 : 0.0);
    }
    __syncthreads();
    double* F = reinterpret_cast<double*>(G32);     // G32 and V32 are not needed any more
    for (int idx = tid; idx < qq; idx += bd) {     // F = I - E/2 + 3/8 E^2
      const int j = idx / q, i = idx - j * q;
      const double acc = dot4(RN + i, q, RN + j * q, 1, 0, q);
      F[idx] = fma(0.375, acc, ((i == j) ? 1.0 : 0.0) - 0.5 * RN[idx]);
    }
    __syncthreads();
    for (int idx = tid; idx < qq; idx += bd) {     // V F (into RN: E is not needed any more)
      const int j = idx / q, i = idx - j * q;
      RN[idx] = dot4(VD + i, q, F + j * q, 1, 0, q);
    }
    __syncthreads();
    for (int idx = tid; idx < qq; idx += bd) VD[idx] = RN[idx];   // V
    __syncthreads();
    for (int idx = tid; idx < qq; idx += bd) {     // G V (G is not needed afterwards)
      const int j = idx / q, i = idx - j * q;
      RN[idx] = dot4(GG + i, q, VD + j * q, 1, 0, q);
    }
    sweeps += blk_hestenes<double>(RN, VD, q, q, 1e-14, 1e-30 * fro, 8);
  }
  __syncthreads();
  // squared singular values (column norms), NaN ordered last
  for (int j = tid; j < q; j += bd) {
    double s2 = 0.0;
    if (fp64) {
      s2 = dot4(RN + j * q, 1, RN + j * q, 1, 0, q);
    } else {
      float f = 0.f;
      for (int i = 0; i < q; ++i) f = fmaf(G32[j * ld + i], G32[j * ld + i], f);
      s2 = f;
    }
    dg[j] = (s2 == s2) ? s2 : -1.0;
  }
  __syncthreads();
  // descending order, ties by column index (a permutation for any input)
  for (int j = tid; j < q; j += bd) {
    int rk = 0;
    for (int i = 0; i < q; ++i) rk += (dg[i] > dg[j]) || (dg[i] == dg[j] && i < j);
    order[rk] = j;
  }
  __syncthreads();
  // U = R_P^T w, w the top-r columns of V (q x r, row-major)
  double* U = GG;
  double* W = GG + q * r;
  for (int idx = tid; idx < q * r; idx += bd) {   // lanes along a: R_P rows read as consecutive words
    const int c = idx / q, a = idx - (idx / q) * q;
    const int col = order[c];
    U[a * r + c] = dot4(RP + a, q, VD + col * q, 1, 0, a + 1);
  }
  __syncthreads();
  double* Bm = GG + qs;            // r x r (over G32, V32 and VD, which are not needed any more)
  double* scr = Bm + r * r;        // 5 r*r
  float* Lf = reinterpret_cast<float*>(scr + 5 * r * r);
  float* Lif = Lf + r * r;
  // normalisation: T_k = C' U R^{-1} with R^T R = G = U^T N U; R^{-1} from the
  // FP32 Cholesky of G checked by E = R^{-T} G R^{-1} - I (FP64 Cholesky when
  // ||E|| >= 1e-4), then polished: R^{-1} (I - E/2 + 3E^2/8)
  double* G = scr;
  double* Li = scr + r * r;
  double* work = Li + r * r;
  double* E = work + r * r;
  double* F = E + r * r;
  blk_gemm<double>(q, r, q, N, q, false, U, r, false, W, r, 1.0, false);         // W = N U
  __syncthreads();
  blk_gemm<double>(r, r, q, U, r, true, W, r, false, G, r, 1.0, false);          // G = U^T N U
  __syncthreads();
  __shared__ int pow2n[1];
  if (tid < 32) warp_chol_inv32(G, r, r, Lf, Lif, &pow2n[0]);
  __syncthreads();
  double* Rinv = Bm;
  const double scn = ldexp(1.0, -pow2n[0]);
  for (int i = tid; i < r * r; i += blockDim.x) {                                 // Rinv = L^{-T}
    int a = i / r, c = i - (i / r) * r;
    Rinv[i] = (double)Lif[c * r + a] * scn;
  }
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    blk_gemm<double>(r, r, r, G, r, false, Rinv, r, false, F, r, 1.0, false);    // F = G Rinv
    __syncthreads();
    blk_gemm<double>(r, r, r, Rinv, r, true, F, r, false, E, r, 1.0, false);     // E = Rinv^T G Rinv
    __syncthreads();
    double em = 0.0;
    for (int i = tid; i < r * r; i += blockDim.x) {
      double v = E[i] - (((i / r) == (i % r)) ? 1.0 : 0.0);
      E[i] = v;
      em = nanmax(em, fabs(v));
    }
    em = blk_max(em, red);
    if (em < 1e-4) break;
    // FP64 Cholesky instead
    blk_chol_linv64(G, r, r, Li, work, &bad);
    for (int i = tid; i < r * r; i += blockDim.x) {
      int a = i / r, c = i - (i / r) * r;
      Rinv[i] = Li[c * r + a];
    }
    __syncthreads();
  }
  blk_gemm<double>(r, r, r, E, r, false, E, r, false, F, r, 0.375, false);       // F = 3/8 E^2
  __syncthreads();
  for (int i = tid; i < r * r; i += blockDim.x) F[i] += (((i / r) == (i % r)) ? 1.0 : 0.0) - 0.5 * E[i];
  __syncthreads();
  blk_gemm<double>(r, r, r, Rinv, r, false, F, r, false, work, r, 1.0, false);   // Rinv F
  __syncthreads();
  double* Pk = P.small + P.off_pk[k];
  blk_gemm<double>(q, r, r, U, r, false, work, r, false, Pk, r, 1.0, false);     // P = U R^{-1}
  __threadfence_block();
  __syncthreads();
  blk_gemm<double>(r, q, q, Pk, r, true, N, q, false, P.small + P.off_sk[k], q, 1.0, false);   // S = P^T N
  if (tid == 0 && bad) atomicOr(P.flags, 2u);
  if (tid == 0) P.scal[SC_SUBIT] = (k == 0 ? 0.0 : P.scal[SC_SUBIT]) + (double)sweeps;
}

// new core k: T_k(x) = S_{k-1} C_k(x) P_k  (no P for the last core)
__device__ void slice_map(const DevProb& P, int k, int x, double* Y) {
  const int m = P.m;
  const int qa = P.q[k], qb = P.q[k + 1];
  const int ra = P.r[k], rb = P.r[k + 1];
  const double* C = P.C[k] + (long long)x * qa * qb;
  double* T = P.core64[k] + (long long)x * ra * rb;
  float* T32 = P.core32p[k] + (long long)x * P.R * P.R;
  double* T64 = P.core64p[k] + (long long)x * P.R * P.R;
  const double* Cp = C;
  if (k > 0) {
    blk_gemm<double>(ra, qb, qa, P.small + P.off_sk[k - 1], qa, false, C, qb, false, Y, qb, 1.0, false);
    __syncthreads();
    Cp = Y;
  }
  // Remark 3.6: the rounding ran on W^{1/2} W_l; undo the weight
  const double wu = P.weighted_retraction ? sqrt(gpow(P, k, x, -1)) : 1.0;
  if (k < m - 1) {
    const double* Pk = P.small + P.off_pk[k];
    for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
      int a = i / rb, b = i - (i / rb) * rb;
      double acc = 0.0;
      for (int t = 0; t < qb; ++t) acc = fma(Cp[a * qb + t], Pk[t * rb + b], acc);
      acc *= wu;
      T[i] = acc;
      T32[pad_idx(P, k, a, b)] = (float)acc;
      T64[pad_idx(P, k, a, b)] = acc;
    }
  } else {
    for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
      int a = i / rb, b = i - (i / rb) * rb;
      const double v = Cp[i] * wu;
      T[i] = v;
      T32[pad_idx(P, k, a, b)] = (float)v;
      T64[pad_idx(P, k, a, b)] = v;
    }
  }
}

// ---- float-float slice products of FP32 steps (block-per-slice path) --------
// The same sums as slice_contrib and slice_map, on the FP32 pipe (ff.cuh):
// operands are split into float-float pairs as they are staged in shared
// memory, transposed where needed so that every product is rows against
// rows (out(i, j) = sum_t A(i, t) B(j, t)), with odd leading dimensions so
// that the rows the lanes of a warp read fall in different banks.  The
// symmetric Grams (Lam, Gam, Psi, N) are accumulated on their upper triangle
// only and mirrored when the block writes its partial.

constexpr int kFFMaxOut = 9;   // outputs per thread: a 64 x 64 triangle (2080) over 256 threads

__device__ __forceinline__ int ff_ld(int cols) { return cols | 1; }

// dst (rows x cols, leading dimension ld) = split(src), src row-major with
// leading dimension lds; with `trans` dst is cols x rows: dst[j][i] = src[i][j]
__device__ void ff_stage(float2* dst, int ld, const double* src, int rows, int cols, int lds, bool trans) {
  for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
    const int i = idx / cols, j = idx - (idx / cols) * cols;
    const float2 v = ffa::split(src[i * lds + j]);
    if (trans)
      dst[j * ld + i] = v;
    else
      dst[i * ld + j] = v;
  }
}

// out (M x N, leading dimension ldo) = A (M x K) B^T with B given as N x K
// rows; results renormalised float-float pairs
__device__ void ff_mm_rows(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, float2* out,
                           int ldo) {
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - (idx / N) * N;
    float s, c;
    ffa::dot(A + i * lda, B + j * ldb, K, s, c);
    out[i * ldo + j] = ffa::renorm(s, c);
  }
}

// this thread's u-th output as i * 65536 + j, or -1: the packed upper
// triangle (row by row, j >= i) of a rows x rows result when `sym`, else
// row-major rows x cols
__device__ __forceinline__ int ff_output(int u, bool sym, int rows, int cols) {
  const int p = threadIdx.x + u * blockDim.x;
  if (sym) {
    if (p >= rows * (rows + 1) / 2) return -1;
    // row r starts at r n - r (r - 1) / 2: invert the quadratic in FP32
    // (exact integers below 2^24), then correct a rounding off by one
    const float b = 2.f * rows + 1.f;
    int r = (int)floorf(0.5f * (b - sqrtf(b * b - 8.f * (float)p)));
    r = max(0, min(r, rows - 1));
    if (r * rows - r * (r - 1) / 2 > p) --r;
    else if ((r + 1) * rows - (r + 1) * r / 2 <= p) ++r;
    const int start = r * rows - r * (r - 1) / 2;
    return (r << 16) | (r + p - start);
  }
  if (p >= rows * cols) return -1;
  return ((p / cols) << 16) | (p - (p / cols) * cols);
}

// One reduction block of a slice job of an FP32 step: its slices' sum of the
// job's products, written to the block's partial (rows x cols, mirrored
// when symmetric) in FP64.
__device__ void stage_job_ff(const DevProb& P, const Job& J, int b, double* smd) {
  float2* sm = reinterpret_cast<float2*>(smd);
  const int k = J.k;
  const int ra = P.r[k], rb = P.r[k + 1], qa = P.q[k], qb = P.q[k + 1];
  int qm = 1;
  for (int t = 0; t <= P.m; ++t) qm = max(qm, P.q[t]);
  const int reg = qm * (qm + 1);           // float2 per region
  float2* F = sm;                          // the fixed matrix of the job
  float2* X = F + reg;                     // the slice's operand
  float2* Y = X + reg;                     // the first product
  float2* X2 = Y + reg;                    // a second slice operand (E of OP_H)
  const bool sym = J.op != OP_H;
  float as[kFFMaxOut], ac[kFFMaxOut];
  int oij[kFFMaxOut];
#pragma unroll
  for (int u = 0; u < kFFMaxOut; ++u) {
    as[u] = ac[u] = 0.f;
    oij[u] = ff_output(u, sym, J.rows, J.cols);
  }
  // the fixed matrix (the same for every slice)
  int ldF = 1;
  switch (J.op) {
    case OP_LAM: ldF = ff_ld(ra); ff_stage(F, ldF, P.small + P.off_lam[k], ra, ra, ra, false); break;
    case OP_GAM: ldF = ff_ld(rb); ff_stage(F, ldF, P.small + P.off_gam[k + 1], rb, rb, rb, false); break;
    case OP_PSI: ldF = ff_ld(qb); ff_stage(F, ldF, P.small + P.off_psi[k + 1], qb, qb, qb, false); break;
    case OP_N:
      if (k > 0) {
        ldF = ff_ld(qa);
        ff_stage(F, ldF, P.small + P.off_sk[k - 1], ra, qa, qa, false);
      }
      break;
    default: break;
  }
  for (int x = b; x < P.n[k]; x += J.nb) {
    __syncthreads();   // the previous slice's reads are done (and F is staged)
    const double* T = P.core64[k] + (long long)x * ra * rb;
    const double* C = P.C[k] + (long long)x * qa * qb;
    const float2 *L = nullptr, *R = nullptr;   // the second product: out(i, j) = sum_t L(i, t) R(j, t)
    int ldL = 1, ldR = 1, K = 0;
    float2 w = make_float2(1.f, 0.f);
    switch (J.op) {
      case OP_LAM: {   // acc += w T^T (Lam T): Y^T = T^T Lam (Lam symmetric), out = w T^T Y
        const int ldX = ff_ld(ra);
        ff_stage(X, ldX, T, ra, rb, rb, true);                 // T^T: rb x ra
        __syncthreads();
        ff_mm_rows(rb, ra, ra, X, ldX, F, ldF, Y, ldX);         // Y^T: rb x ra
        L = X; ldL = ldX; R = Y; ldR = ldX; K = ra;
        w = ffa::split(gpow(P, k, x, +1));
        break;
      }
      case OP_GAM: {   // acc += w (T Gam) T^T: Y = T Gam, out = w Y T^T
        const int ldX = ff_ld(rb);
        ff_stage(X, ldX, T, ra, rb, rb, false);                // T: ra x rb
        __syncthreads();
        ff_mm_rows(ra, rb, rb, X, ldX, F, ldF, Y, ldX);         // Y: ra x rb
        L = Y; ldL = ldX; R = X; ldR = ldX; K = rb;
        w = ffa::split(gpow(P, k, x, +1));
        break;
      }
      case OP_H: {     // acc += T^T E
        const int ldX = ff_ld(ra);
        ff_stage(X, ldX, T, ra, rb, rb, true);                 // T^T: rb x ra
        ff_stage(X2, ldX, P.E[k] + (long long)x * ra * rb, ra, rb, rb, true);
        L = X; ldL = ldX; R = X2; ldR = ldX; K = ra;
        break;
      }
      case OP_PSI: {   // acc += (C Psi) C^T: Y = C Psi (Psi symmetric), out = Y C^T
        const int ldX = ff_ld(qb);
        ff_stage(X, ldX, C, qa, qb, qb, false);                // C: qa x qb
        __syncthreads();
        ff_mm_rows(qa, qb, qb, X, ldX, F, ldF, Y, ldX);         // Y: qa x qb
        L = Y; ldL = ldX; R = X; ldR = ldX; K = qb;
        break;
      }
      default: {       // OP_N: C' = S_{k-1} C, acc += C'^T C'
        const int ldX = ff_ld(qa);
        ff_stage(X, ldX, C, qa, qb, qb, true);                 // C^T: qb x qa
        if (k == 0) {
          L = X; ldL = ldX; R = X; ldR = ldX; K = qa;
        } else {
          __syncthreads();
          const int ldY = ff_ld(ra);
          ff_mm_rows(qb, ra, qa, X, ldX, F, ldF, Y, ldY);       // C'^T: qb x ra
          L = Y; ldL = ldY; R = Y; ldR = ldY; K = ra;
        }
        break;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kFFMaxOut; ++u) {
      if (oij[u] >= 0) {
        const int i = oij[u] >> 16, j = oij[u] & 0xffff;
        float s, c;
        ffa::dot(L + i * ldL, R + j * ldR, K, s, c);
        ffa::acc_scaled(as[u], ac[u], w, s, c);
      }
    }
  }
  const int dd = J.rows * J.cols;
  double* out = P.red + J.red + (long long)b * dd;
#pragma unroll
  for (int u = 0; u < kFFMaxOut; ++u) {
    if (oij[u] >= 0) {
      const int i = oij[u] >> 16, j = oij[u] & 0xffff;
      const double v = ffa::join(as[u], ac[u]);
      out[i * J.cols + j] = v;
      if (sym) out[j * J.cols + i] = v;
    }
  }
}

// new core k at slices b, b + nb, ... (the sums of slice_map in float-float)
__device__ void slice_map_ff(const DevProb& P, int k, int b, int nb, double* smd) {
  float2* sm = reinterpret_cast<float2*>(smd);
  const int m = P.m;
  const int qa = P.q[k], qb = P.q[k + 1];
  const int ra = P.r[k], rb = P.r[k + 1];
  int qm = 1;
  for (int t = 0; t <= m; ++t) qm = max(qm, P.q[t]);
  const int reg = qm * (qm + 1);
  float2* Sf = sm;                 // S_{k-1}: ra x qa
  float2* Ct = Sf + reg;           // C^T: qb x qa
  float2* Cp = Ct + reg;           // C' = S_{k-1} C: ra x qb
  float2* Pt = Cp + reg;           // P_k^T: rb x qb
  const int ldC = ff_ld(qb), ldS = ff_ld(qa);
  // the fixed factors once per block: S_{k-1} and P_k^T
  if (k > 0) ff_stage(Sf, ldS, P.small + P.off_sk[k - 1], ra, qa, qa, false);
  if (k < m - 1) ff_stage(Pt, ldC, P.small + P.off_pk[k], qb, rb, rb, true);
  for (int x = b; x < P.n[k]; x += nb) {
    __syncthreads();   // the fixed factors are staged, the previous slice's reads are done
    const double* C = P.C[k] + (long long)x * qa * qb;
    if (k > 0) {
      ff_stage(Ct, ldS, C, qa, qb, qb, true);
      __syncthreads();
      ff_mm_rows(ra, qb, qa, Sf, ldS, Ct, ldS, Cp, ldC);
    } else {
      ff_stage(Cp, ldC, C, qa, qb, qb, false);   // C' = C (qa = ra = 1)
    }
    __syncthreads();
    // Remark 3.6: the rounding ran on W^{1/2} W_l; undo the weight
    const double wu = P.weighted_retraction ? sqrt(gpow(P, k, x, -1)) : 1.0;
    double* T = P.core64[k] + (long long)x * ra * rb;
    float* T32 = P.core32p[k] + (long long)x * P.R * P.R;
    double* T64 = P.core64p[k] + (long long)x * P.R * P.R;
    for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
      const int a = i / rb, bcol = i - (i / rb) * rb;
      double v;
      if (k < m - 1) {
        float s, c;
        ffa::dot(Cp + a * ldC, Pt + bcol * ldC, qb, s, c);
        v = ffa::join(s, c);
      } else {
        const float2 e = Cp[a * ldC + bcol];
        v = ffa::join(e.x, e.y);
      }
      if (P.weighted_retraction) v *= wu;
      T[i] = v;
      T32[pad_idx(P, k, a, bcol)] = (float)v;
      T64[pad_idx(P, k, a, bcol)] = v;
    }
  }
}

// Sums n partial rows of d values (src + row * d) into dst[0..d) in a fixed
// order: G = blockDim / d thread groups split the rows, each thread keeps
// four independent register accumulators (loads pipeline, FP64 adds
// overlap), and the groups are combined in group order through shared
// memory.  With `check`, a non-finite total flags the step.
__device__ void sum_rows(const DevProb& P, const double* src, int n, int d, double* dst, double* sm, bool check) {
  const int groups = max(1, min((int)blockDim.x / max(d, 1), 32));
  if (groups == 1) {
    // wide rows: each thread sums whole columns, two at a time with eight
    // rows of each in flight (the partials come from L2, whose latency
    // sets the time of this serial tail of a stage), in a fixed order
    const int bd = blockDim.x;
    for (int i0 = threadIdx.x; i0 < d; i0 += 2 * bd) {
      const int i1 = i0 + bd;
      const bool two = i1 < d;
      double a[8], c[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = c[u] = 0.0;
      for (int bb = 0; bb < n; bb += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (bb + u < n) {
            a[u] += __ldcg(src + (long long)(bb + u) * d + i0);
            if (two) c[u] += __ldcg(src + (long long)(bb + u) * d + i1);
          }
        }
      }
      const double t0 = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
      dst[i0] = t0;
      if (check && !isfinite(t0)) atomicOr(P.flags, 1u);
      if (two) {
        const double t1 = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
        dst[i1] = t1;
        if (check && !isfinite(t1)) atomicOr(P.flags, 1u);
      }
    }
    __syncthreads();
    return;
  }
  for (int base = 0; base < d; base += blockDim.x / groups) {
    const int per = blockDim.x / groups;
    const int g = threadIdx.x / per, i = base + (threadIdx.x - g * per);
    double v = 0.0;
    if (g < groups && i < d) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int bb = g;
      for (; bb + 3 * groups < n; bb += 4 * groups) {
        a0 += __ldcg(src + (long long)bb * d + i);
        a1 += __ldcg(src + (long long)(bb + groups) * d + i);
        a2 += __ldcg(src + (long long)(bb + 2 * groups) * d + i);
        a3 += __ldcg(src + (long long)(bb + 3 * groups) * d + i);
      }
      for (; bb < n; bb += groups) a0 += __ldcg(src + (long long)bb * d + i);
      v = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    if (g < groups) sm[threadIdx.x] = v;
    __syncthreads();
    if (g == 0 && i < d) {
      double tot = 0.0;
      for (int gg = 0; gg < groups; ++gg) tot += sm[gg * per + threadIdx.x];
      dst[i] = tot;
      if (check && !isfinite(tot)) atomicOr(P.flags, 1u);   // an overflowed iterate ends the step as non-finite
    }
    __syncthreads();
  }
}

// Reduction blocks per group of the stage reduction's first level, and the
// group counters a stage may use (jobs of at most 1024 blocks each).
constexpr int kGroup = 16;
constexpr int kGroupCounters = (TTC_MAXM + 4) * (1024 / kGroup);
__host__ __device__ inline int job_groups(int nb) { return (nb + kGroup - 1) / kGroup; }

// The reduction of a stage after reduction block b of job j has written its
// partial: the last block of each group of kGroup consecutive blocks sums
// the group's partials in block order into a group partial, and the last
// group of the stage sums every job's group partials in group order into
// P.small (a fixed tree, so results are reproducible), resets the counters
// and returns true; every other block returns false.  Spreading the sums
// over the group finishers keeps the stage's last block from adding all
// block partials alone on one SM.
__device__ bool stage_reduce(const DevProb& P, const Stage& S, int j, int b, double* sm) {
  __shared__ int last;
  const Job& J = S.job[j];
  const int dd = J.rows * J.cols;
  const int g = b / kGroup, g0 = g * kGroup, gn = min(kGroup, J.nb - g0);
  int gidx = g, total = 0;
  for (int t = 0; t < S.njob; ++t) {
    if (t < j) gidx += job_groups(S.job[t].nb);
    total += job_groups(S.job[t].nb);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(P.gctr + gidx, 1) == gn - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  sum_rows(P, P.red + J.red + (long long)g0 * dd, gn, dd, P.red2 + J.red2 + (long long)g * dd, sm, false);
  if (threadIdx.x == 0) P.gctr[gidx] = 0;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(P.counters + S.counter, 1) == total - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int t = 0; t < S.njob; ++t) {
    const Job& Jt = S.job[t];
    sum_rows(P, P.red2 + Jt.red2, job_groups(Jt.nb), Jt.rows * Jt.cols, P.small + Jt.dst, sm, true);
  }
  if (threadIdx.x == 0) P.counters[S.counter] = 0;
  __threadfence_block();
  __syncthreads();
  return true;
}

// ---- the stage kernel --------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 3) k_stage(const DevProb P, const Stage S) {
  extern __shared__ __align__(16) double sm[];
  int b = blockIdx.x;
  for (int i = 0; i < S.nmap; ++i) {     // slice maps first
    const int k = S.map_k[i];
    if (b < S.map_nb[i]) {
      if (P.dense_ff) {
        slice_map_ff(P, k, b, S.map_nb[i], sm);
      } else {
        for (int x = b; x < P.n[k]; x += S.map_nb[i]) {
          __syncthreads();   // the previous slice's scratch reads are done
          slice_map(P, k, x, sm);
        }
      }
      return;
    }
    b -= S.map_nb[i];
  }
  int j = 0;
  while (b >= S.job[j].nb) {
    b -= S.job[j].nb;
    ++j;
  }
  const Job J = S.job[j];
  if (P.dense_ff && J.op <= OP_N) {
    stage_job_ff(P, J, b, sm);           // the slice products in float-float
  } else {
    const int dd = J.rows * J.cols;
    double* acc = sm;
    double* Y = sm + dd;
    for (int i = threadIdx.x; i < dd; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    for (int x = b; x < P.n[J.k]; x += J.nb) slice_contrib(P, S, J, x, acc, Y);
    double* out = P.red + J.red + (long long)b * dd;
    for (int i = threadIdx.x; i < dd; i += blockDim.x) out[i] = acc[i];
  }
  if (!stage_reduce(P, S, j, b, sm)) return;   // the stage's last group finisher continues
  // (the small projection and the bond run in k_post, a one-block launch
  // after this one: their shared memory would otherwise be reserved by every
  // block of the stage and halve the blocks an SM holds)
  if (S.post == POST_METRIC && S.post_k == P.m - 1 && threadIdx.x == 0) {
    double aa = P.small[P.off_mlam[0][P.m]], ab = P.small[P.off_mlam[1][P.m]], bbv = P.small[P.off_mlam[2][P.m]];
    P.scal[SC_METRIC] = aa - 2.0 * ab + bbv;
    P.scal[SC_NORM] = bbv;
  }
}

// the factorizations that follow a block-per-slice stage, on one block: the
// Gram inverses and Q_k (POST_SMALL_PROJ) or a bond of the rounding (POST_BOND)
__global__ void __launch_bounds__(kThreads) k_post(const DevProb P, const Stage S) {
  extern __shared__ __align__(16) double sm[];
  if (S.post == POST_SMALL_PROJ)
    post_small_proj(P, sm);
  else if (S.post == POST_BOND)
    post_bond(P, S.post_k, sm);
}

// ---- warp-per-slice forms (ranks <= 8, so q <= 16) --------------------------
// One warp handles one slice at a time: the slice is staged in the warp's
// shared scratch, intermediate products are spread over the lanes, and every
// lane owns NO outputs of the r x r (or q x q) result, accumulated in
// registers over the warp's slices with NO independent FMA chains (FP64 has a
// long dependent latency here).  The eight warps of a block are then summed in
// warp order, so results stay reproducible.

constexpr int kWarpsW = kThreads / 32;

// a warp's scratch: three q_max x q_max matrices of the problem (so blocks of
// small problems take little shared memory and more of them stay resident)
__device__ __forceinline__ int wscr_mat(const DevProb& P) {
  int q = 1;
  for (int k = 0; k <= P.m; ++k) q = max(q, P.q[k]);
  return q * q;
}
inline int wscr_mat_host(const DevProb& P) {
  int q = 1;
  for (int k = 0; k <= P.m; ++k) q = std::max(q, P.q[k]);
  return q * q;
}

// Y (M x N, ld N) = alpha X (M x K, ld ldx) Z (K x N, ld ldz), spread over
// the lanes; the unscaled form spends no FP64 multiply on alpha = 1 (the FP64
// pipe is the bound of the batched dense stages on this GPU)
template <bool kScale>
__device__ __forceinline__ void warp_mm_t(double* Y, const double* X, int ldx, const double* Z, int ldz, int M, int N,
                                          int K, double alpha) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < M * N; e += 32) {
    const int i = e / N, j = e - (e / N) * N;
    double a0 = 0.0, a1 = 0.0;   // two chains: FP64 chains advance slowly here
    int t = 0;
    for (; t + 1 < K; t += 2) {
      a0 = fma(X[i * ldx + t], Z[t * ldz + j], a0);
      a1 = fma(X[i * ldx + t + 1], Z[(t + 1) * ldz + j], a1);
    }
    if (t < K) a0 = fma(X[i * ldx + t], Z[t * ldz + j], a0);
    const double acc = a0 + a1;
    Y[e] = kScale ? alpha * acc : acc;
  }
  __syncwarp();
}
__device__ __forceinline__ void warp_mm(double* Y, const double* X, int ldx, const double* Z, int ldz, int M, int N,
                                        int K) {
  warp_mm_t<false>(Y, X, ldx, Z, ldz, M, N, K, 1.0);
}
__device__ __forceinline__ void warp_mm_scaled(double* Y, const double* X, int ldx, const double* Z, int ldz, int M,
                                               int N, int K, double alpha) {
  warp_mm_t<true>(Y, X, ldx, Z, ldz, M, N, K, alpha);
}

// warp copy of n contiguous doubles
__device__ __forceinline__ void warp_load(double* dst, const double* src, int n) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < n; i += 32) dst[i] = src[i];
  __syncwarp();
}

// acc[t] += w sum_i L[i*ldl + ia[t]] R[i*ldr + ib[t]]   (columns against columns)
template <int NO>
__device__ __forceinline__ void acc_cols(double (&acc)[NO], const int (&ia)[NO], const int (&ib)[NO], const double* L,
                                         int ldl, const double* R, int ldr, int K, double w) {
  double t[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) t[u] = 0.0;
  for (int i = 0; i < K; ++i) {
#pragma unroll
    for (int u = 0; u < NO; ++u) t[u] = fma(L[i * ldl + ia[u]], R[i * ldr + ib[u]], t[u]);
  }
#pragma unroll
  for (int u = 0; u < NO; ++u) acc[u] = fma(w, t[u], acc[u]);
}
// acc[t] += w sum_i L[ia[t]*ldl + i] R[ib[t]*ldr + i]   (rows against rows)
template <int NO>
__device__ __forceinline__ void acc_rows(double (&acc)[NO], const int (&ia)[NO], const int (&ib)[NO], const double* L,
                                         int ldl, const double* R, int ldr, int K, double w) {
  double t[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) t[u] = 0.0;
  for (int i = 0; i < K; ++i) {
#pragma unroll
    for (int u = 0; u < NO; ++u) t[u] = fma(L[ia[u] * ldl + i], R[ib[u] * ldr + i], t[u]);
  }
#pragma unroll
  for (int u = 0; u < NO; ++u) acc[u] = fma(w, t[u], acc[u]);
}

// the contribution of slice x to job J (same sums as slice_contrib)
template <int NO>
__device__ void warp_contrib(const DevProb& P, const Job& J, int x, double (&acc)[NO], const int (&ia)[NO],
                             const int (&ib)[NO], double* scr) {
  const int k = J.k;
  const int ra = P.r[k], rb = P.r[k + 1];
  double* A = scr;
  double* Y = scr + wscr_mat(P);
  switch (J.op) {
    case OP_LAM: {   // acc += w2 T^T (Lam T)
      warp_load(A, P.core64[k] + (long long)x * ra * rb, ra * rb);
      warp_mm(Y, P.small + P.off_lam[k], ra, A, rb, ra, rb, ra);
      acc_cols<NO>(acc, ia, ib, A, rb, Y, rb, ra, gpow(P, k, x, +1));
      break;
    }
    case OP_GAM: {   // acc += w2 (T Gam) T^T
      warp_load(A, P.core64[k] + (long long)x * ra * rb, ra * rb);
      warp_mm(Y, A, rb, P.small + P.off_gam[k + 1], rb, ra, rb, rb);
      acc_rows<NO>(acc, ia, ib, Y, rb, A, rb, rb, gpow(P, k, x, +1));
      break;
    }
    case OP_H: {     // acc += T^T E
      warp_load(A, P.core64[k] + (long long)x * ra * rb, ra * rb);
      warp_load(Y, P.E[k] + (long long)x * ra * rb, ra * rb);
      acc_cols<NO>(acc, ia, ib, A, rb, Y, rb, ra, 1.0);
      break;
    }
    case OP_PSI: {   // acc += (C Psi) C^T
      const int qa = P.q[k], qb = P.q[k + 1];
      warp_load(A, P.C[k] + (long long)x * qa * qb, qa * qb);
      warp_mm(Y, A, qb, P.small + P.off_psi[k + 1], qb, qa, qb, qb);
      acc_rows<NO>(acc, ia, ib, Y, qb, A, qb, qb, 1.0);
      break;
    }
    default: {       // OP_N: C' = S_{k-1} C ; acc += C'^T C'
      const int qa = P.q[k], qb = P.q[k + 1];
      warp_load(A, P.C[k] + (long long)x * qa * qb, qa * qb);
      if (k == 0) {
        acc_cols<NO>(acc, ia, ib, A, qb, A, qb, qa, 1.0);
      } else {
        warp_mm(Y, P.small + P.off_sk[k - 1], qa, A, qb, ra, qb, qa);
        acc_cols<NO>(acc, ia, ib, Y, qb, Y, qb, ra, 1.0);
      }
      break;
    }
  }
  __syncwarp();
}

// new core k at slice x from C'_k = S_{k-1} C_k (same as slice_map)
__device__ void warp_slice_map(const DevProb& P, int k, int x, double* scr) {
  const int lane = threadIdx.x & 31;
  const int m = P.m;
  const int qa = P.q[k], qb = P.q[k + 1];
  const int ra = P.r[k], rb = P.r[k + 1];
  double* A = scr;
  double* Y = scr + wscr_mat(P);
  double* Z = scr + 2 * wscr_mat(P);
  warp_load(A, P.C[k] + (long long)x * qa * qb, qa * qb);
  const double* Cp = A;
  if (k > 0) {
    warp_mm(Y, P.small + P.off_sk[k - 1], qa, A, qb, ra, qb, qa);
    Cp = Y;
  }
  const double* Tn = Cp;
  if (k < m - 1) {
    warp_mm(Z, Cp, qb, P.small + P.off_pk[k], rb, ra, rb, qb);
    Tn = Z;
  }
  double* T = P.core64[k] + (long long)x * ra * rb;
  float* T32 = P.core32p[k] + (long long)x * P.R * P.R;
  double* T64 = P.core64p[k] + (long long)x * P.R * P.R;
  const double wu = P.weighted_retraction ? sqrt(gpow(P, k, x, -1)) : 1.0;   // Remark 3.6
  for (int i = lane; i < ra * rb; i += 32) {
    const int a = i / rb, b = i - (i / rb) * rb;
    const double v = Tn[i] * wu;
    T[i] = v;
    T32[pad_idx(P, k, a, b)] = (float)v;
    T64[pad_idx(P, k, a, b)] = v;
  }
  __syncwarp();
}

template <int NO>
__device__ __forceinline__ void stage_w_body(const DevProb& P, const Stage& S, int b) {
  extern __shared__ __align__(16) double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* scr = sm + warp * 3 * wscr_mat(P);
  for (int i = 0; i < S.nmap; ++i) {     // slice maps first, one slice per warp
    const int k = S.map_k[i];
    const int nbm = (P.n[k] + kWarpsW - 1) / kWarpsW;
    if (b < nbm) {
      const int x = b * kWarpsW + warp;
      if (x < P.n[k]) warp_slice_map(P, k, x, scr);
      return;
    }
    b -= nbm;
  }
  int j = 0;
  while (b >= S.job[j].nb) {
    b -= S.job[j].nb;
    ++j;
  }
  const Job J = S.job[j];
  const int dd = J.rows * J.cols;
  const bool sym = warp_job_sym(J);
  const int nout = warp_job_outputs(J);
  double acc[NO];
  int ia[NO], ib[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    acc[u] = 0.0;
    int o = min(lane + 32 * u, nout - 1);
    if (sym) {             // packed upper triangle: row i holds rows - i entries
      int i = 0;
      while (o >= J.rows - i) {
        o -= J.rows - i;
        ++i;
      }
      ia[u] = i;
      ib[u] = i + o;
    } else {
      ia[u] = o / J.cols;
      ib[u] = o - ia[u] * J.cols;
    }
  }
  const int stride = J.nb * kWarpsW;
  for (int x = b * kWarpsW + warp; x < P.n[J.k]; x += stride) warp_contrib<NO>(P, J, x, acc, ia, ib, scr);
  __syncthreads();                       // the scratch becomes the warp-sum area
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    if (lane + 32 * u < nout) {
      sm[warp * dd + ia[u] * J.cols + ib[u]] = acc[u];
      if (sym) sm[warp * dd + ib[u] * J.cols + ia[u]] = acc[u];
    }
  }
  __syncthreads();
  double* out = P.red + J.red + (long long)b * dd;
  for (int o = threadIdx.x; o < dd; o += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kWarpsW; ++w) t += sm[w * dd + o];
    out[o] = t;
  }
  if (!stage_reduce(P, S, j, b, sm)) return;   // the stage's last group finisher continues
  if (S.post == POST_SMALL_PROJ) {
    post_small_proj(P, sm);
  } else if (S.post == POST_BOND) {
    post_bond(P, S.post_k, sm);
  }
}

template <int NO>
__global__ void __launch_bounds__(kThreads) k_stage_w(const DevProb P, const Stage S) {
  stage_w_body<NO>(P, S, blockIdx.x);
}

// B_k(x) and the block core C_k(x), one slice per warp (same as k_build_C)
__device__ __forceinline__ void build_C_w_body(const DevProb& P, int blk, int nslices) {
  extern __shared__ __align__(16) double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* scr = sm + warp * 3 * wscr_mat(P);
  int g = blk * kWarpsW + warp;
  if (g >= nslices) return;
  int k = 0;
  while (k < P.m - 1 && g >= P.n[k]) {
    g -= P.n[k];
    ++k;
  }
  const int x = g, m = P.m;
  const int ra = P.r[k], rb = P.r[k + 1];
  const double alpha = P.scal[SC_ALPHA];
  const double wi = gpow(P, k, x, -1);
  double* Tt = scr;
  double* t1 = scr + wscr_mat(P);
  double* B = scr + 2 * wscr_mat(P);
  warp_load(Tt, P.core64[k] + (long long)x * ra * rb, ra * rb);
  if (P.steepest) {
    // the steepest step formed B1 = B / alpha already (k_build_B1)
    const double* B1 = P.B1[k] + (long long)x * ra * rb;
    for (int e = lane; e < ra * rb; e += 32) B[e] = alpha * B1[e];
    __syncwarp();
  } else {
    warp_mm(t1, P.small + P.off_lami[k], ra, P.E[k] + (long long)x * ra * rb, rb, ra, rb, ra);
    warp_mm_scaled(B, t1, rb, P.small + P.off_gami[k + 1], rb, ra, rb, rb, -alpha * wi);
  }
  if (k + 1 < m && !P.steepest) {
    const double* Q = P.small + P.off_qm[k];
    for (int e = lane; e < ra * rb; e += 32) {
      const int i = e / rb, j = e - (e / rb) * rb;
      double acc = 0.0;
      for (int t = 0; t < rb; ++t) acc = fma(Tt[i * rb + t], Q[t * rb + j], acc);
      B[e] = fma(alpha, acc, B[e]);
    }
    __syncwarp();
  }
  const int qa = P.q[k], qb = P.q[k + 1];
  double* C = P.C[k] + (long long)x * qa * qb;
  const double ws = P.weighted_retraction ? sqrt(gpow(P, k, x, +1)) : 1.0;   // Remark 3.6: W^{1/2} W_l
  for (int i = lane; i < qa * qb; i += 32) {
    int a = i / qb, b = i - (i / qb) * qb;
    double v;
    if (k == 0) {
      v = (b < rb) ? B[a * rb + b] : Tt[a * rb + (b - rb)];
    } else if (k == m - 1) {
      v = (a < ra) ? Tt[a * rb + b] : Tt[(a - ra) * rb + b] + B[(a - ra) * rb + b];
    } else {
      if (a < ra)
        v = (b < rb) ? Tt[a * rb + b] : 0.0;
      else
        v = (b < rb) ? B[(a - ra) * rb + b] : Tt[(a - ra) * rb + (b - rb)];
    }
    C[i] = P.weighted_retraction ? v * ws : v;
  }
}

__global__ void __launch_bounds__(kThreads) k_build_C_w(const DevProb P, int nslices) {
  build_C_w_body(P, blockIdx.x, nslices);
}

// ---- batched dense stages ----------------------------------------------------
// Members of a batch whose dense stage takes the warp-per-slice path and the
// same stage sequence (same order m) run every stage as one launch: blocks
// [base[p], base[p+1]) execute member p's stage with its own descriptor,
// plan, counters and partials, so each member computes exactly what it
// computes alone.  (With a launch per member and stage, the GPU's kernel
// launch rate, not the work, limited a batched step.)

__device__ __forceinline__ int find_member(const int* __restrict__ base, int nprob, int blk) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename X>
__device__ __forceinline__ void stage_copy(const X* __restrict__ src, X* dst) {
  static_assert(sizeof(X) % 8 == 0, "8-byte words");
  const uint2* sp = reinterpret_cast<const uint2*>(src);
  uint2* dp = reinterpret_cast<uint2*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(X) / 8); i += blockDim.x) dp[i] = __ldg(sp + i);
}

template <int NO>
__global__ void __launch_bounds__(kThreads) k_stage_w_batch(const DevProb* __restrict__ probs,
                                                            const Stage* __restrict__ stages,
                                                            const int* __restrict__ base, int nprob) {
  __shared__ __align__(16) DevProb Ps;
  __shared__ __align__(16) Stage Ss;
  const int p = find_member(base, nprob, blockIdx.x);
  stage_copy(probs + p, &Ps);
  stage_copy(stages + p, &Ss);
  __syncthreads();
  stage_w_body<NO>(Ps, Ss, blockIdx.x - __ldg(base + p));
}

__global__ void __launch_bounds__(kThreads) k_build_C_w_batch(const DevProb* __restrict__ probs,
                                                              const int* __restrict__ base, int nprob) {
  __shared__ __align__(16) DevProb Ps;
  const int p = find_member(base, nprob, blockIdx.x);
  stage_copy(probs + p, &Ps);
  __syncthreads();
  int nslices = 0;
  for (int k = 0; k < Ps.m; ++k) nslices += Ps.n[k];
  build_C_w_body(Ps, blockIdx.x - __ldg(base + p), nslices);
}

// the copy of the cores into prev64 (the step-change metric), kCopyBlocks
// blocks per member
constexpr int kCopyBlocks = 16;
__global__ void __launch_bounds__(256) k_save_prev_batch(const DevProb* __restrict__ probs, int nprob) {
  const int p = blockIdx.x / kCopyBlocks, lb = blockIdx.x - p * kCopyBlocks;
  if (p >= nprob) return;
  const DevProb& P = probs[p];
  slice_weights(P, lb * (long long)blockDim.x + threadIdx.x, (long long)kCopyBlocks * blockDim.x);
  const int m = P.m;
  for (int k = 0; k < m; ++k) {
    const long long cnt = (long long)P.n[k] * P.r[k] * P.r[k + 1];
    const double* src = P.core64[k];
    double* dst = P.prev64[k];
    for (long long i = lb * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)kCopyBlocks * blockDim.x)
      dst[i] = src[i];
  }
}

// ---- steepest step, Eq. (PRGD stepsize) ------------------------------------
// One block per slice (k, x): the update core at unit step
//   B1_k(x) = -[G_k(x)^{-1/(2m)} Lam_k^{-1} E_k(x) Gam_{k+1}^{-1} - T_k(x) Q_k]
// (W_l = T_l + sum_k [T..alpha B1_k..T], so Z = tilde P_T W^{-1} G_l =
// -sum_k [T..B1_k..T]) and G_k(x)^{1/(2m)} <Lam_k B1_k(x) Gam_{k+1}, B1_k(x)>:
// summed over all slices this is ||Z||_W^2, because the components of Z are
// W-orthogonal (Lemma 3.4) and Lam, Gam are the Grams of W^{1/2} T.
// The same sums in float-float (FP32 steps, ff.cuh): operands staged as
// float pairs in `sm` (seven regions of rmax (rmax + 1) pairs), every
// product rows against rows.
__device__ void build_B1_ff(const DevProb& P, int k, int x, int slice, float2* sm, double* red) {
  const int m = P.m, ra = P.r[k], rb = P.r[k + 1];
  int rm = 1;
  for (int t = 0; t <= m; ++t) rm = max(rm, P.r[t]);
  const int reg = rm * (rm + 1);
  float2* Li = sm;                 // Lam_k^{-1}: ra x ra      -> Lam_k
  float2* Et = Li + reg;           // E^T: rb x ra             -> Y^T = (Lam B1)^T: rb x ra
  float2* Gt = Et + reg;           // (Gam_{k+1}^{-1})^T: rb x rb -> Gam_{k+1}
  float2* Tm = Gt + reg;           // T: ra x rb
  float2* Qt = Tm + reg;           // Q_k^T: rb x rb
  float2* t1 = Qt + reg;           // Lam^{-1} E: ra x rb
  float2* Bt = t1 + reg;           // B1^T: rb x ra
  const int la = ff_ld(ra), lb = ff_ld(rb);
  ff_stage(Li, la, P.small + P.off_lami[k], ra, ra, ra, false);
  ff_stage(Et, la, P.E[k] + (long long)x * ra * rb, ra, rb, rb, true);
  ff_stage(Gt, lb, P.small + P.off_gami[k + 1], rb, rb, rb, true);
  if (k + 1 < m) {
    ff_stage(Tm, lb, P.core64[k] + (long long)x * ra * rb, ra, rb, rb, false);
    ff_stage(Qt, lb, P.small + P.off_qm[k], rb, rb, rb, true);
  }
  __syncthreads();
  ff_mm_rows(ra, rb, ra, Li, la, Et, la, t1, lb);                 // t1 = Lam^{-1} E
  __syncthreads();
  const float2 wneg = ffa::split(-gpow(P, k, x, -1));
  double* out = P.B1[k] + (long long)x * ra * rb;
  float* out32 = P.B1_32p[k] + (long long)x * P.R * P.R;
  double* out64 = P.B1_64p[k] + (long long)x * P.R * P.R;
  for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
    const int a = i / rb, b = i - (i / rb) * rb;
    float s, c, as = 0.f, ac = 0.f;
    ffa::dot(t1 + a * lb, Gt + b * lb, rb, s, c);
    ffa::acc_scaled(as, ac, wneg, s, c);                          // -w t1 Gam^{-1}
    if (k + 1 < m) {
      ffa::dot(Tm + a * lb, Qt + b * lb, rb, s, c);
      ffa::acc_scaled(as, ac, make_float2(1.f, 0.f), s, c);       // + T Q
    }
    const double v = ffa::join(as, ac);
    out[i] = v;
    const int pi = pad_idx(P, k, a, b);
    out32[pi] = (float)v;
    out64[pi] = v;
    Bt[b * la + a] = ffa::renorm(as, ac);
  }
  __syncthreads();
  // ||Z||_W^2 term: G^{1/(2m)} <Lam B1 Gam, B1>
  ff_stage(Li, la, P.small + P.off_lam[k], ra, ra, ra, false);
  ff_stage(Gt, lb, P.small + P.off_gam[k + 1], rb, rb, rb, false);
  __syncthreads();
  ff_mm_rows(rb, ra, ra, Bt, la, Li, la, Et, la);                  // (Lam B1)^T = B1^T Lam (Lam symmetric)
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
    const int a = i / rb, b = i - (i / rb) * rb;
    // (Lam B1 Gam)(a, b) = sum_c (Lam B1)(a, c) Gam(c, b): column a of (Lam B1)^T
    float s = 0.f, c = 0.f;
    for (int t = 0; t < rb; ++t) ffa::dot_step(s, c, Et[t * la + a], Gt[b * lb + t]);
    const float2 bv = Bt[b * la + a];
    acc += ffa::join(s, c) * ffa::join(bv.x, bv.y);
  }
  const double tot = blk_sum(acc, red);
  if (threadIdx.x == 0) P.zw[slice] = gpow(P, k, x, +1) * tot;
}

__global__ void __launch_bounds__(128) k_build_B1(const DevProb P) {
  __shared__ double t1[TTC_MAXR * TTC_MAXR];
  __shared__ double B[TTC_MAXR * TTC_MAXR];
  __shared__ double red[128];
  const int slice = blockIdx.x;
  int blk = slice, k = 0;
  while (k < P.m - 1 && blk >= P.n[k]) {
    blk -= P.n[k];
    ++k;
  }
  const int x = blk, m = P.m;
  if (P.dense_ff) {
    extern __shared__ __align__(16) float2 ffsm[];
    build_B1_ff(P, k, x, slice, ffsm, red);
    return;
  }
  const int ra = P.r[k], rb = P.r[k + 1];
  const double wi = gpow(P, k, x, -1);
  const double* T = P.core64[k] + (long long)x * ra * rb;
  const double* E = P.E[k] + (long long)x * ra * rb;
  blk_gemm<double>(ra, rb, ra, P.small + P.off_lami[k], ra, false, E, rb, false, t1, rb, 1.0, false);
  __syncthreads();
  blk_gemm<double>(ra, rb, rb, t1, rb, false, P.small + P.off_gami[k + 1], rb, false, B, rb, -wi, false);
  __syncthreads();
  if (k + 1 < m) {
    blk_gemm<double>(ra, rb, rb, T, rb, false, P.small + P.off_qm[k], rb, false, B, rb, 1.0, true);
    __syncthreads();
  }
  double* out = P.B1[k] + (long long)x * ra * rb;
  float* out32 = P.B1_32p[k] + (long long)x * P.R * P.R;
  double* out64 = P.B1_64p[k] + (long long)x * P.R * P.R;
  for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
    out[i] = B[i];
    const int pi = pad_idx(P, k, i / rb, i - (i / rb) * rb);
    out32[pi] = (float)B[i];
    out64[pi] = B[i];
  }
  blk_gemm<double>(ra, rb, ra, P.small + P.off_lam[k], ra, false, B, rb, false, t1, rb, 1.0, false);   // Lam B1
  __syncthreads();
  const double* Gm = P.small + P.off_gam[k + 1];
  double acc = 0.0;
  for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) {
    const int a = i / rb, b = i - (i / rb) * rb;
    double v = 0.0;
    for (int t = 0; t < rb; ++t) v = fma(t1[a * rb + t], Gm[t * rb + b], v);
    acc = fma(v, B[i], acc);
  }
  const double tot = blk_sum(acc, red);
  if (threadIdx.x == 0) P.zw[slice] = gpow(P, k, x, +1) * tot;
}

// ||P_Omega Z||^2 = sum over Omega of (sum_k l_{k-1} B1_k(x_k) r_{k+1})^2: the
// tangent TT [[T, 0], [B1, T]] evaluated entry by entry along the chain
//   (l_T, l_Z) <- (l_T T_k(x_k), l_Z T_k(x_k) + l_T B1_k(x_k)),
// in the precision of the step (FP32 steps: FP32 on the padded FP32 mirrors,
// squares summed in FP64; the step size only scales the step, so FP32's
// relative error in alpha moves the iterate by that fraction of one step, as
// the FP32 sampled pass does).  Where a prefix table covers the first modes,
// the chain starts from its row (l_T) and the row of its tangent companion
// table (l_Z), built by k_build_ztables.  Block partials; the last block forms
// alpha_l = ||Z||_W^2 / ||P_Omega Z||^2 (an explicit step size is kept).
constexpr int kTanThreads = 256;
constexpr int kTanCounter = 127;

template <typename T>
__device__ __forceinline__ const T* pcore(const DevProb& P, int k);
template <>
__device__ __forceinline__ const float* pcore<float>(const DevProb& P, int k) { return P.core32p[k]; }
template <>
__device__ __forceinline__ const double* pcore<double>(const DevProb& P, int k) { return P.core64p[k]; }
template <typename T>
__device__ __forceinline__ const T* pb1(const DevProb& P, int k);
template <>
__device__ __forceinline__ const float* pb1<float>(const DevProb& P, int k) { return P.B1_32p[k]; }
template <>
__device__ __forceinline__ const double* pb1<double>(const DevProb& P, int k) { return P.B1_64p[k]; }
template <typename T>
__device__ __forceinline__ T* ptab(const DevProb& P, bool z);
template <>
__device__ __forceinline__ float* ptab<float>(const DevProb& P, bool z) { return z ? P.ztab32 : P.tab32; }
template <>
__device__ __forceinline__ double* ptab<double>(const DevProb& P, bool z) { return z ? P.ztab64 : P.tab64; }

// 16-byte loads of a padded row (4 floats or 2 doubles at a time)
template <int RC>
__device__ __forceinline__ void ld_row16(const float* p, int len, float (&v)[RC]) {
#pragma unroll
  for (int b = 0; b < RC; b += 4) {
    if (b >= len) break;
    const float4 t = __ldg(reinterpret_cast<const float4*>(p + b));
    v[b] = t.x;
    if (b + 1 < RC) v[b + 1] = t.y;
    if (b + 2 < RC) v[b + 2] = t.z;
    if (b + 3 < RC) v[b + 3] = t.w;
  }
}
template <int RC>
__device__ __forceinline__ void ld_row16(const double* p, int len, double (&v)[RC]) {
#pragma unroll
  for (int b = 0; b < RC; b += 2) {
    if (b >= len) break;
    const double2 t = __ldg(reinterpret_cast<const double2*>(p + b));
    v[b] = t.x;
    if (b + 1 < RC) v[b + 1] = t.y;
  }
}

// (l_T, l_Z) <- (l_T T_j(x), l_Z T_j(x) + l_T B1_j(x)) on the padded mirrors
// (row stride R), register arrays of RC >= every rank
template <typename T, int R, int RC>
__device__ __forceinline__ void tangent_times(const DevProb& P, int j, int x, T (&lT)[RC], T (&lZ)[RC]) {
  constexpr int V = 16 / sizeof(T);   // values per 16-byte load
  const int ra = P.r[j], rb = P.r[j + 1];
  const T* S = pcore<T>(P, j) + (long long)x * R * R;
  const T* Bk = pb1<T>(P, j) + (long long)x * R * R;
  T nT[RC], nZ[RC];
#pragma unroll
  for (int b = 0; b < RC; ++b) {
    nT[b] = 0;
    nZ[b] = 0;
  }
  if (rb == 1) {   // the slice is one contiguous column
#pragma unroll
    for (int a0 = 0; a0 < RC; a0 += V) {
      if (a0 >= ra) break;
      T sv[V], bv[V];
      ld_row16<V>(S + a0, V, sv);
      ld_row16<V>(Bk + a0, V, bv);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        if (a0 + i < RC) {
          nT[0] = fma(lT[a0 + i], sv[i], nT[0]);
          nZ[0] = fma(lZ[a0 + i], sv[i], fma(lT[a0 + i], bv[i], nZ[0]));
        }
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < RC; ++a) {
      if (a >= ra) break;
      const T la = lT[a], za = lZ[a];
#pragma unroll
      for (int b0 = 0; b0 < RC; b0 += V) {
        if (b0 >= rb) break;
        T sv[V], bv[V];
        ld_row16<V>(S + a * R + b0, V, sv);
        ld_row16<V>(Bk + a * R + b0, V, bv);
#pragma unroll
        for (int i = 0; i < V; ++i) {
          if (b0 + i < RC) {
            nZ[b0 + i] = fma(za, sv[i], fma(la, bv[i], nZ[b0 + i]));
            nT[b0 + i] = fma(la, sv[i], nT[b0 + i]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < RC; ++b) {
    lT[b] = nT[b];
    lZ[b] = nZ[b];
  }
}

// row g of the tangent companion of table t (a prefix table over modes
// 0..jt-1), from scratch by its own chain
template <typename T, int R, int RC>
__device__ __forceinline__ void ztable_row_chain(const DevProb& P, int t, long long g) {
  const unsigned row = (unsigned)(g - P.tab_row0[t]);
  const int jt = P.tab_j[t];
  T lT[RC], lZ[RC];
#pragma unroll
  for (int a = 0; a < RC; ++a) {
    lT[a] = 0;
    lZ[a] = 0;
  }
  lT[0] = 1;
  bool valid = true;
  for (int j = 0; j < jt; ++j) {
    const int x = (int)((row >> (P.cshift[j] - P.tab_shift[t])) & ((1u << P.cbits[j]) - 1u));
    valid = valid && x < P.n[j];
    if (valid) tangent_times<T, R, RC>(P, j, x, lT, lZ);
  }
  if (!valid) return;   // a row that stands for no entry: zeroed at allocation
  T* dst = ptab<T>(P, true) + g * R;
#pragma unroll
  for (int a = 0; a < R; ++a) dst[a] = (a < RC && a < P.r[jt]) ? lZ[a < RC ? a : 0] : T(0);
}

// The tangent companion of the prefix tables: row i of ztab holds l_Z over
// the table's modes (the prefix table itself holds l_T).  A block takes 128
// consecutive rows; when they all belong to one two-mode prefix table and
// share the coordinate of its second mode (its bits lie above the first
// mode's), that mode's slices T_1(x_1), B1_1(x_1) are staged in shared memory
// once and every row is l_Z = B1_0(x_0) T_1(x_1) + T_0(x_0) B1_1(x_1) from
// the first mode's rows; otherwise each thread runs its row's chain.
template <typename T, int R, int RC>
__global__ void __launch_bounds__(128) k_build_ztables(const DevProb P) {
  __shared__ __align__(16) T sS[R * R];
  __shared__ __align__(16) T sB[R * R];
  __shared__ long long key0;
  for (long long g0 = (long long)blockIdx.x * blockDim.x; g0 < P.tab_total; g0 += (long long)gridDim.x * blockDim.x) {
    const long long g = g0 + threadIdx.x;
    const bool inr = g < P.tab_total;
    int t = 0;
    if (inr)
      while (t + 1 < P.ntab && g >= P.tab_row0[t + 1]) ++t;
    const bool pre = inr && P.tab_side[t] == 0;
    const unsigned row = inr ? (unsigned)(g - P.tab_row0[t]) : 0u;
    int x0 = 0, x1 = 0;
    long long key = -1;
    if (pre && P.tab_j[t] == 2) {
      x0 = (int)((row >> (P.cshift[0] - P.tab_shift[t])) & ((1u << P.cbits[0]) - 1u));
      x1 = (int)((row >> (P.cshift[1] - P.tab_shift[t])) & ((1u << P.cbits[1]) - 1u));
      if (x1 < P.n[1]) key = (long long)t * (1LL << 32) + x1;
    }
    __syncthreads();   // the previous rows' reads of sS, sB are done
    if (threadIdx.x == 0) key0 = key;
    __syncthreads();
    if (__syncthreads_and(key >= 0 && key == key0)) {
      const int r1 = P.r[1], r2 = P.r[2];
      const T* S1 = pcore<T>(P, 1) + (long long)x1 * R * R;
      const T* B11 = pb1<T>(P, 1) + (long long)x1 * R * R;
      for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
        sS[i] = S1[i];
        sB[i] = B11[i];
      }
      __syncthreads();
      const bool valid = x0 < P.n[0];   // rows that stand for no entry stay as zeroed at allocation
      T lT[RC], lZ[RC];
      const T* S0 = pcore<T>(P, 0) + (long long)(valid ? x0 : 0) * R * R;
      const T* B10 = pb1<T>(P, 0) + (long long)(valid ? x0 : 0) * R * R;
#pragma unroll
      for (int a = 0; a < RC; ++a) {
        lT[a] = (valid && a < r1) ? S0[a] : T(0);    // row 0 of a 1 x r_1 slice
        lZ[a] = (valid && a < r1) ? B10[a] : T(0);
      }
      T* dst = ptab<T>(P, true) + g * R;
      for (int b = 0; b < R && valid; ++b) {
        T z = T(0);
        if (b < r2) {
#pragma unroll
          for (int a = 0; a < RC; ++a) {
            if (a < r1) {
              const int ix = r2 == 1 ? a : a * R + b;   // padded mirrors: a column when r_2 = 1
              z = fma(lZ[a], sS[ix], fma(lT[a], sB[ix], z));
            }
          }
        }
        dst[b] = z;
      }
    } else if (pre) {
      ztable_row_chain<T, R, RC>(P, t, g);
    }
  }
}

template <typename T, int R, int RC>
__global__ void __launch_bounds__(kTanThreads) k_tangent_sq(const DevProb P, int nslices) {
  __shared__ double red[kTanThreads];
  __shared__ int am_last;
  // the longest prefix table: rows of l_T and l_Z over modes < j0
  const int tp = P.m >= 2 ? P.pre_tab[P.m - 1] : -1;
  const int j0 = tp >= 0 ? P.tab_j[tp] : 0;
  // entries in the layout order of mode j0 - 1, lexicographic in
  // (x_{j0-1}, ..., x_0): the lanes of a warp mostly share their table rows
  const int ord = tp >= 0 ? j0 - 1 : P.m - 1;
  double acc = 0.0;
  for (int e = blockIdx.x * kTanThreads + threadIdx.x; e < P.N; e += gridDim.x * kTanThreads) {
    const Code w = load_code(P, ord, e);
    T lT[RC], lZ[RC];
#pragma unroll
    for (int a = 0; a < RC; ++a) {
      lT[a] = 0;
      lZ[a] = 0;
    }
    if (tp >= 0) {
      const long long row =
          P.tab_row0[tp] + (long long)((w.word(P.tab_word[tp]) >> P.tab_shift[tp]) & ((1u << P.tab_bits[tp]) - 1u));
      ld_row16<RC>(ptab<T>(P, false) + row * R, RC, lT);
      ld_row16<RC>(ptab<T>(P, true) + row * R, RC, lZ);
    } else {
      lT[0] = 1;
    }
    for (int k = j0; k < P.m; ++k) tangent_times<T, R, RC>(P, k, code_coord(P, w, k), lT, lZ);
    acc = fma((double)lZ[0], (double)lZ[0], acc);
  }
  const double tot = blk_sum(acc, red);
  if (threadIdx.x == 0) P.tpart[blockIdx.x] = tot;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(P.counters + kTanCounter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double den = 0.0, num = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kTanThreads) den += __ldcg(P.tpart + i);
  den = blk_sum(den, red);
  for (int i = threadIdx.x; i < nslices; i += kTanThreads) num += __ldcg(P.zw + i);
  num = blk_sum(num, red);
  if (threadIdx.x == 0) {
    if (!(P.scal[SC_ALPHA_OVR] > 0.0)) P.scal[SC_ALPHA] = den > 0.0 ? num / den : 0.0;
    P.counters[kTanCounter] = 0;
  }
}

inline int tangent_blocks(const DevProb& P) { return std::max(1, std::min((P.N + kTanThreads - 1) / kTanThreads, 2 * 152)); }

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
  const double wi = gpow(P, k, x, -1);
  const double* T = P.core64[k] + (long long)x * ra * rb;
  const double* E = P.E[k] + (long long)x * ra * rb;
  if (P.steepest) {
    // the steepest step formed B1 = B / alpha already (k_build_B1)
    const double* B1 = P.B1[k] + (long long)x * ra * rb;
    for (int i = threadIdx.x; i < ra * rb; i += blockDim.x) B[i] = alpha * B1[i];
    __syncthreads();
  } else {
    blk_gemm<double>(ra, rb, ra, P.small + P.off_lami[k], ra, false, E, rb, false, t1, rb, 1.0, false);
    __syncthreads();
    blk_gemm<double>(ra, rb, rb, t1, rb, false, P.small + P.off_gami[k + 1], rb, false, B, rb, -alpha * wi, false);
    __syncthreads();
    if (k + 1 < m) {
      blk_gemm<double>(ra, rb, rb, T, rb, false, P.small + P.off_qm[k], rb, false, B, rb, alpha, true);
      __syncthreads();
    }
  }
  const int qa = P.q[k], qb = P.q[k + 1];
  double* C = P.C[k] + (long long)x * qa * qb;
  const double ws = P.weighted_retraction ? sqrt(gpow(P, k, x, +1)) : 1.0;   // Remark 3.6: W^{1/2} W_l
  for (int i = threadIdx.x; i < qa * qb; i += blockDim.x) {
    int a = i / qb, b = i - (i / qb) * qb;
    double v;
    if (k == 0) {
      v = (b < rb) ? B[a * rb + b] : T[a * rb + (b - rb)];
    } else if (k == m - 1) {
      v = (a < ra) ? T[a * rb + b] : T[(a - ra) * rb + b] + B[(a - ra) * rb + b];
    } else {
      if (a < ra)
        v = (b < rb) ? T[a * rb + b] : 0.0;
      else
        v = (b < rb) ? B[(a - ra) * rb + b] : T[(a - ra) * rb + (b - rb)];
    }
    C[i] = v * ws;
  }
}

__global__ void k_copy_cores(const DevProb P, int to_prev) {
  if (to_prev) slice_weights(P, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
  long long tot = 0;
  for (int k = 0; k < P.m; ++k) tot += (long long)P.n[k] * P.r[k] * P.r[k + 1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    long long o = i;
    int k = 0;
    while (o >= (long long)P.n[k] * P.r[k] * P.r[k + 1]) {
      o -= (long long)P.n[k] * P.r[k] * P.r[k + 1];
      ++k;
    }
    if (to_prev) {
      P.prev64[k][o] = P.core64[k][o];
    } else {   // padded mirrors
      const int ra = P.r[k], rb = P.r[k + 1];
      const long long x = o / (ra * rb);
      const int e = (int)(o - x * ra * rb), a = e / rb, b = e - (e / rb) * rb;
      const long long d = x * P.R * P.R + pad_idx(P, k, a, b);
      P.core32p[k][d] = (float)P.core64[k][o];
      P.core64p[k][d] = P.core64[k][o];
    }
  }
}

// ---- metrics: dense form for small d* (every entry, FP64) -------------------
// cores in the library's slice-major layout: T_k(x) an r_k x r_{k+1} block
struct SliceMajorCores {
  const double* const* core;
  const int* rk;
  __device__ __forceinline__ int r(int k) const { return rk[k]; }
  __device__ __forceinline__ double at(int k, int x, int i, int j) const {
    return core[k][((long long)x * rk[k] + i) * rk[k + 1] + j];
  }
};

__global__ void __launch_bounds__(256) k_dense_diff(const DevProb P, int which, long long dstar, double* part) {
  const SliceMajorCores A{P.core64, P.r};
  const SliceMajorCores B{which == 0 ? P.truth : P.prev64, which == 0 ? P.rt : P.r};
  tt_dist_block(A, B, P.m, P.n, dstar, part);
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

// ---- host-side plan ----------------------------------------------------------
struct Plan {
  std::vector<Stage> gram;       // Lam/Gam chains (+ H jobs in the first); the last runs small_proj
  std::vector<Stage> psi;        // k = d-1 .. 1
  std::vector<Stage> sweep;      // bond k (+ map of core k-1), then the final maps
  std::vector<Stage> metric[2];  // Gram sweep of ||A - B||^2, which = 0 truth, 1 previous
  size_t smem_stage = 0;       // block-per-slice stages (slice jobs, maps, reductions)
  size_t smem_post = 0;        // k_post: the small projection or a bond
  size_t smem_b1 = 0;         // float-float k_build_B1: seven regions of rmax (rmax + 1) float pairs
  bool warp = false;          // warp-per-slice kernels (ranks <= 8)
  size_t smem_warp = 0;
  double* metric_part = nullptr;
};

std::map<const ttc_ctx*, Plan> g_plan_of;
std::mutex g_plan_mu;

Plan& plan_of(const ttc_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  return g_plan_of[c];
}

inline int nblocks_for(int nk) { return std::max(1, std::min(nk, 1024)); }

// Blocks of a block-per-slice job: slices are strided over the blocks, each
// block taking enough slices for about kBlockWork FMAs (at most
// kMaxSlicesPerBlock: a slice costs a block a few dependent global-memory
// round trips however small it is), so that a block's fixed costs (its
// partial, the reduction protocol) are amortised and the reduction has fewer
// partials.  `work` is one slice's FMAs.
constexpr double kBlockWork = 131072.0;
constexpr int kMaxSlicesPerBlock = 8;
inline int nblocks_work(long long nk, double work) {
  const double per = std::min((double)kMaxSlicesPerBlock, std::max(1.0, std::floor(kBlockWork / std::max(work, 1.0))));
  return (int)std::max(1LL, std::min<long long>(1024, (long long)std::ceil((double)nk / per)));
}
// one slice's FMAs of each job (upper triangles of the symmetric Grams), and of a slice map
inline double slice_work(int op, int ra, int rb, int qa, int qb, int k) {
  switch (op) {
    case OP_LAM: return (double)ra * ra * rb + 0.5 * rb * (rb + 1) * ra;
    case OP_GAM: return (double)ra * rb * rb + 0.5 * ra * (ra + 1) * rb;
    case OP_H: return (double)rb * rb * ra;
    case OP_PSI: return (double)qa * qb * qb + 0.5 * qa * (qa + 1) * qb;
    default: return k == 0 ? 0.5 * qb * (qb + 1) * qa : (double)qb * ra * qa + 0.5 * qb * (qb + 1) * ra;   // OP_N
  }
}
inline double map_work(int ra, int rb, int qa, int qb) { return (double)ra * qb * qa + (double)ra * rb * qb; }
inline int nblocks_warp(int nk) { return std::max(1, std::min((nk + kWarpsW - 1) / kWarpsW, 256)); }

int launch_stage(ttc_ctx* c, const Stage& S, size_t smem, size_t smem_post) {
  int nb = 0;
  for (int i = 0; i < S.nmap; ++i) nb += S.map_nb[i];
  for (int j = 0; j < S.njob; ++j) nb += S.job[j].nb;
  k_stage<<<nb, kThreads, smem, c->stream>>>(c->hp, S);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  if (S.post == POST_SMALL_PROJ || S.post == POST_BOND) {
    k_post<<<1, kThreads, smem_post, c->stream>>>(c->hp, S);
    TTC_CUDA(cudaGetLastError());
    c->nlaunch += 1;
  }
  return TTC_OK;
}

// warp-per-slice stage: NO outputs per lane for the largest job of the stage
int launch_stage_w(ttc_ctx* c, const Stage& S, size_t smem) {
  int nb = 0, dd = 1;
  for (int i = 0; i < S.nmap; ++i) nb += (int)((c->n[S.map_k[i]] + kWarpsW - 1) / kWarpsW);
  for (int j = 0; j < S.njob; ++j) {
    nb += S.job[j].nb;
    dd = std::max(dd, warp_job_outputs(S.job[j]));
  }
  const int no = (dd + 31) / 32;
  if (no <= 1)
    k_stage_w<1><<<nb, kThreads, smem, c->stream>>>(c->hp, S);
  else if (no <= 2)
    k_stage_w<2><<<nb, kThreads, smem, c->stream>>>(c->hp, S);
  else if (no <= 4)
    k_stage_w<4><<<nb, kThreads, smem, c->stream>>>(c->hp, S);
  else if (no <= 8)
    k_stage_w<8><<<nb, kThreads, smem, c->stream>>>(c->hp, S);
  else
    return TTC_EUNSUPPORTED;
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  return TTC_OK;
}

int run_stage(ttc_ctx* c, const Plan& pl, const Stage& S) {
  return pl.warp ? launch_stage_w(c, S, pl.smem_warp) : launch_stage(c, S, pl.smem_stage, pl.smem_post);
}

}  // namespace

int ttc_alloc_dense(ttc_ctx* c) {
  DevProb& P = c->hp;
  const int m = c->m;
  P.q[0] = 1;
  P.q[m] = 1;
  for (int k = 1; k < m; ++k) P.q[k] = 2 * c->r[k];
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
    for (int t = 0; t < 3; ++t) P.off_mlam[t][k] = take(TTC_MAXR * TTC_MAXR);
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
  TTC_CUDA(cudaMemsetAsync(small, 0, sizeof(double) * (size_t)off, c->stream));
  P.small = small;
  double one = 1.0;
  TTC_CUDA(cudaMemcpyAsync(small + P.off_lam[0], &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TTC_CUDA(cudaMemcpyAsync(small + P.off_gam[m], &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TTC_CUDA(cudaMemcpyAsync(small + P.off_psi[m], &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  for (int t = 0; t < 3; ++t)
    TTC_CUDA(cudaMemcpyAsync(small + P.off_mlam[t][0], &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TTC_CUDA(cudaStreamSynchronize(c->stream));   // `one` lives on this stack frame
  for (int k = 0; k < m; ++k) {
    double* Ck = nullptr;
    TTC_TRY(ttc_alloc(c, (void**)&Ck, sizeof(double) * (size_t)c->n[k] * P.q[k] * P.q[k + 1], false));
    P.C[k] = Ck;
    double* pv = nullptr;
    TTC_TRY(ttc_alloc(c, (void**)&pv, sizeof(double) * (size_t)c->n[k] * c->r[k] * c->r[k + 1], false));
    P.prev64[k] = pv;
  }
  {   // the steepest step's buffers (also for the constant step, which may fall back to it)
    long long nsl = 0;
    for (int k = 0; k < m; ++k) {
      double* b1 = nullptr;
      TTC_TRY(ttc_alloc(c, (void**)&b1, sizeof(double) * (size_t)c->n[k] * c->r[k] * c->r[k + 1], false));
      P.B1[k] = b1;
      float* b32 = nullptr;
      double* b64 = nullptr;
      const size_t padcnt = (size_t)c->n[k] * c->rank_bucket * c->rank_bucket;
      TTC_TRY(ttc_alloc(c, (void**)&b32, sizeof(float) * padcnt, false));
      TTC_TRY(ttc_alloc(c, (void**)&b64, sizeof(double) * padcnt, false));
      TTC_CUDA(cudaMemsetAsync(b32, 0, sizeof(float) * padcnt, c->stream));   // the padding stays zero
      TTC_CUDA(cudaMemsetAsync(b64, 0, sizeof(double) * padcnt, c->stream));
      P.B1_32p[k] = b32;
      P.B1_64p[k] = b64;
      nsl += c->n[k];
    }
    TTC_TRY(ttc_alloc(c, (void**)&P.zw, sizeof(double) * (size_t)nsl, false));
    TTC_TRY(ttc_alloc(c, (void**)&P.tpart, sizeof(double) * 2 * 152, false));
  }
  double* scal = nullptr;
  TTC_TRY(ttc_alloc(c, (void**)&scal, sizeof(double) * SC_COUNT, false));
  TTC_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * SC_COUNT, c->stream));
  P.scal = scal;
  P.flags = reinterpret_cast<unsigned*>(scal + SC_FLAGS);
  int* counters = nullptr;
  TTC_TRY(ttc_alloc(c, (void**)&counters, sizeof(int) * 128, false));
  TTC_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * 128, c->stream));
  P.counters = counters;

  Plan pl;
  {
    int qm = 1;
    for (int k = 0; k <= m; ++k) qm = std::max(qm, P.q[k]);
    pl.warp = qm <= 16;
  }
  long long red = 0, red2 = 0;
  int ctr = 1;   // counter 0 belongs to the slice reduction of the sampled pass
  bool warp_jobs = pl.warp;   // the metric stages below always use the block kernel
  auto mk = [&](int op, int k, int rows, int cols, int dst) {
    Job J;
    J.op = op;
    J.k = k;
    J.nb = warp_jobs  ? nblocks_warp((int)c->n[k])
           : op <= OP_N ? nblocks_work(c->n[k], slice_work(op, c->r[k], c->r[k + 1], P.q[k], P.q[k + 1], k))
                        : nblocks_for((int)c->n[k]);
    J.rows = rows;
    J.cols = cols;
    J.red = red;
    J.red2 = red2;
    J.dst = dst;
    red += (long long)J.nb * rows * cols;
    red2 += (long long)job_groups(J.nb) * rows * cols;
    return J;
  };
  auto blank = [&]() {
    Stage S;
    memset(&S, 0, sizeof(S));
    S.counter = ctr++;
    return S;
  };
  for (int j = 0; j + 1 < m; ++j) {
    Stage S = blank();
    S.job[S.njob++] = mk(OP_LAM, j, c->r[j + 1], c->r[j + 1], P.off_lam[j + 1]);
    int kg = m - 1 - j;
    S.job[S.njob++] = mk(OP_GAM, kg, c->r[kg], c->r[kg], P.off_gam[kg]);
    if (j == 0)
      for (int k = 0; k + 1 < m; ++k) S.job[S.njob++] = mk(OP_H, k, c->r[k + 1], c->r[k + 1], P.off_h[k]);
    if (j + 2 == m) S.post = POST_SMALL_PROJ;
    pl.gram.push_back(S);
  }
  for (int k = m - 1; k >= 1; --k) {
    Stage S = blank();
    S.job[S.njob++] = mk(OP_PSI, k, P.q[k], P.q[k], P.off_psi[k]);
    pl.psi.push_back(S);
  }
  auto map_nb = [&](int k) { return nblocks_work(c->n[k], map_work(c->r[k], c->r[k + 1], P.q[k], P.q[k + 1])); };
  for (int k = 0; k + 1 < m; ++k) {
    Stage S = blank();
    if (k > 0) {
      S.nmap = 1;
      S.map_k[0] = k - 1;
      S.map_nb[0] = map_nb(k - 1);
    }
    S.job[S.njob++] = mk(OP_N, k, P.q[k + 1], P.q[k + 1], P.off_nk[k]);
    S.post = POST_BOND;
    S.post_k = k;
    pl.sweep.push_back(S);
  }
  {
    Stage S = blank();
    S.nmap = 0;
    S.map_nb[S.nmap] = map_nb(m - 2);
    S.map_k[S.nmap++] = m - 2;
    S.map_nb[S.nmap] = map_nb(m - 1);
    S.map_k[S.nmap++] = m - 1;
    pl.sweep.push_back(S);
  }
  warp_jobs = false;
  for (int which = 0; which < 2; ++which) {
    for (int k = 0; k < m; ++k) {
      Stage S = blank();
      S.which = which;
      int ra = c->r[k + 1];
      S.job[S.njob++] = mk(OP_DAA, k, ra, ra, P.off_mlam[0][k + 1]);
      S.post = POST_METRIC;
      S.post_k = k;
      pl.metric[which].push_back(S);   // AB and BB jobs are added at launch (B's ranks)
    }
  }
  if (ctr > kTanCounter) return TTC_EUNSUPPORTED;
  long long metric_extra = 0;
  for (int k = 0; k < m; ++k) metric_extra += 2LL * nblocks_for((int)c->n[k]) * TTC_MAXR * TTC_MAXR;
  double* redp = nullptr;
  TTC_TRY(ttc_alloc(c, (void**)&redp, sizeof(double) * (size_t)std::max(red + metric_extra, 1LL), false));
  P.red = redp;
  P.red_metric = red;
  // group partials: the plan's jobs, then the metric stages' extra jobs
  long long metric_extra2 = 0;
  for (int k = 0; k < m; ++k) metric_extra2 += 2LL * job_groups(nblocks_for((int)c->n[k])) * TTC_MAXR * TTC_MAXR;
  double* red2p = nullptr;
  TTC_TRY(ttc_alloc(c, (void**)&red2p, sizeof(double) * (size_t)std::max(red2 + metric_extra2, 1LL), false));
  P.red2 = red2p;
  P.red2_metric = red2;
  int* gctr = nullptr;   // group counters, reused by every stage (a stage resets the ones it used)
  TTC_TRY(ttc_alloc(c, (void**)&gctr, sizeof(int) * kGroupCounters, false));
  TTC_CUDA(cudaMemsetAsync(gctr, 0, sizeof(int) * kGroupCounters, c->stream));
  P.gctr = gctr;
  TTC_TRY(ttc_alloc(c, (void**)&pl.metric_part, sizeof(double) * 2 * 1024, false));

  int qmax = 1, rmax = 1;
  for (int k = 0; k <= m; ++k) {
    qmax = std::max(qmax, P.q[k]);
    rmax = std::max(rmax, c->r[k]);
  }
  size_t red_need = sizeof(double) * (size_t)(2 * qmax * qmax);
  red_need = std::max(red_need, sizeof(double) * (size_t)(2 * TTC_MAXR * TTC_MAXR));
  size_t proj_need = sizeof(double) * (size_t)(8 * 2 * rmax * rmax) + sizeof(float) * (size_t)(8 * 2 * rmax * rmax);
  // the bond: N, the two factors, G, the FP32 pair G32 / V32, the FP64 basis (6 regions of
  // q (q + 1) doubles), the block's reduction slots and the factor diagonals
  size_t bond_need = sizeof(double) * (size_t)(6 * qmax * (qmax + 1) + kThreads + 2 * qmax);
  // float-float slice jobs and maps of FP32 steps: four regions of q (q + 1) float pairs
  size_t ff_need = sizeof(float2) * (size_t)(4 * qmax * (qmax + 1));
  pl.smem_stage = std::max(red_need, ff_need) + 64;
  pl.smem_post = std::max(proj_need, bond_need) + 64;
  // the warp-per-slice kernels run the posts in their last block
  pl.smem_warp = pl.warp ? std::max(std::max(pl.smem_stage, pl.smem_post),
                                    sizeof(double) * (size_t)kWarpsW * 3 * wscr_mat_host(P))
                         : pl.smem_stage;
  pl.smem_b1 = sizeof(float2) * (size_t)(7 * rmax * (rmax + 1));
  {
    // the attribute is per device and shared by every context: only raise it,
    // so that contexts needing more than this one keep launching
    static std::mutex mu;
    static std::map<int, size_t> granted;
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0;
    TTC_CUDA(cudaGetDevice(&dev));
    static std::map<int, bool> b1_granted;
    if (!b1_granted[dev]) {   // the largest float-float k_build_B1 (rank 32)
      TTC_CUDA(cudaFuncSetAttribute(k_build_B1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(float2) * 7 * TTC_MAXR * (TTC_MAXR + 1))));
      b1_granted[dev] = true;
    }
    if (granted[dev] < std::max(pl.smem_warp, pl.smem_post)) {
      const int sz = (int)std::max(pl.smem_warp, pl.smem_post);   // >= smem_stage
      TTC_CUDA(cudaFuncSetAttribute(k_post, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_build_C_w, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w_batch<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_stage_w_batch<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      TTC_CUDA(cudaFuncSetAttribute(k_build_C_w_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
      granted[dev] = std::max(pl.smem_warp, pl.smem_post);
    }
  }
  plan_of(c) = pl;
  return TTC_OK;
}

// the steepest step's ||P_Omega Z||^2: the tangent companion tables (when
// prefix tables exist), then the evaluation over Omega
template <typename T>
int launch_tangent(ttc_ctx* c, int tb, int nslices, cudaStream_t st) {
  const DevProb& P = c->hp;
  const int R = c->rank_bucket;
  const bool r24 = c->rank_max <= 24;   // register arrays of 24 suffice for ranks <= 24 in bucket 32
  if (P.ntab > 0 && P.m >= 2 && P.pre_tab[P.m - 1] >= 0) {
    const int zb = (int)std::min<long long>((P.tab_total + 127) / 128, 4 * 152);
    switch (R) {
      case 4: k_build_ztables<T, 4, 4><<<zb, 128, 0, st>>>(P); break;
      case 8: k_build_ztables<T, 8, 8><<<zb, 128, 0, st>>>(P); break;
      case 16: k_build_ztables<T, 16, 16><<<zb, 128, 0, st>>>(P); break;
      default:
        if (r24) k_build_ztables<T, 32, 24><<<zb, 128, 0, st>>>(P);
        else k_build_ztables<T, 32, 32><<<zb, 128, 0, st>>>(P);
        break;
    }
    TTC_CUDA(cudaGetLastError());
    c->nlaunch += 1;
  }
  switch (R) {
    case 4: k_tangent_sq<T, 4, 4><<<tb, kTanThreads, 0, st>>>(P, nslices); break;
    case 8: k_tangent_sq<T, 8, 8><<<tb, kTanThreads, 0, st>>>(P, nslices); break;
    case 16: k_tangent_sq<T, 16, 16><<<tb, kTanThreads, 0, st>>>(P, nslices); break;
    default:
      if (r24) k_tangent_sq<T, 32, 24><<<tb, kTanThreads, 0, st>>>(P, nslices);
      else k_tangent_sq<T, 32, 32><<<tb, kTanThreads, 0, st>>>(P, nslices);
      break;
  }
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 2;   // with k_build_B1
  return TTC_OK;
}

int ttc_launch_dense(ttc_ctx* c) {
  const DevProb& P = c->hp;
  const int m = c->m;
  Plan& pl = plan_of(c);
  cudaStream_t st = c->stream;
  for (auto& S : pl.gram) TTC_TRY(run_stage(c, pl, S));
  int nslices = 0;
  for (int k = 0; k < m; ++k) nslices += (int)c->n[k];
  if (P.steepest) {   // alpha_l by exact line search before the rank-2r cores are formed
    k_build_B1<<<nslices, 128, P.dense_ff ? pl.smem_b1 : 0, st>>>(P);
    TTC_CUDA(cudaGetLastError());
    const int tb = tangent_blocks(P);
    if (P.step_fp64) {   // an FP64 step: ||P_Omega Z||^2 in FP64
      TTC_TRY(launch_tangent<double>(c, tb, nslices, st));
    } else {
      TTC_TRY(launch_tangent<float>(c, tb, nslices, st));
    }
  }
  if (pl.warp)
    k_build_C_w<<<(nslices + kWarpsW - 1) / kWarpsW, kThreads, sizeof(double) * kWarpsW * 3 * wscr_mat_host(P), st>>>(
        P, nslices);
  else
    k_build_C<<<nslices, 128, 0, st>>>(P);
  TTC_CUDA(cudaGetLastError());
  c->nlaunch += 1;
  for (auto& S : pl.psi) TTC_TRY(run_stage(c, pl, S));
  for (auto& S : pl.sweep) TTC_TRY(run_stage(c, pl, S));
  return TTC_OK;
}

// ---- batched dense stages (host) ----------------------------------------------
struct DenseGroup {
  int nprob = 0, m = 0;
  DevProb* probs = nullptr;
  std::vector<Stage*> stages;   // per stage of the sequence (gram, psi, sweep): one Stage per member
  std::vector<int*> base;       // per stage: block prefix over the members
  std::vector<int> blocks, no;
  int* base_c = nullptr;        // rank-2r assembly
  int blocks_c = 0;
  size_t smem = 0, smem_c = 0;
};

bool ttc_dense_batchable(const ttc_ctx* c) { return plan_of(c).warp && !c->hp.steepest; }

void ttc_dense_group_destroy(DenseGroup* g) {
  if (!g) return;
  cudaFree(g->probs);
  for (auto* p : g->stages) cudaFree(p);
  for (auto* p : g->base) cudaFree(p);
  cudaFree(g->base_c);
  delete g;
}

int ttc_dense_group_create(ttc_ctx* const* members, int count, DenseGroup** out) {
  *out = nullptr;
  if (count < 1) return TTC_EINVAL;
  DenseGroup* g = new (std::nothrow) DenseGroup();
  if (!g) return TTC_ENOMEM;
  g->nprob = count;
  g->m = members[0]->m;
  std::vector<DevProb> descs;
  std::vector<const Plan*> plans;
  for (int i = 0; i < count; ++i) {
    if (members[i]->m != g->m || !ttc_dense_batchable(members[i])) {
      ttc_dense_group_destroy(g);
      return TTC_EINVAL;
    }
    descs.push_back(members[i]->hp);
    plans.push_back(&plan_of(members[i]));
    g->smem = std::max(g->smem, plans.back()->smem_warp);
  }
  auto upload = [&](void** dst, const void* src, size_t bytes) {
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) ttc_record_cuda_error(e);
    return e;
  };
  cudaError_t e = upload((void**)&g->probs, descs.data(), sizeof(DevProb) * count);
  // the stage sequence: Gram chains (m-1), right Grams of the rank-2r TT (m-1), bonds and maps (m)
  const int nst = 3 * g->m - 2;
  for (int si = 0; si < nst && e == cudaSuccess; ++si) {
    std::vector<Stage> st(count);
    std::vector<int> base(1, 0);
    int dd = 1;
    for (int i = 0; i < count; ++i) {
      const Plan& pl = *plans[i];
      const Stage& S = si < g->m - 1 ? pl.gram[si] : si < 2 * g->m - 2 ? pl.psi[si - (g->m - 1)]
                                                                    : pl.sweep[si - (2 * g->m - 2)];
      st[i] = S;
      int nb = 0;
      for (int j = 0; j < S.nmap; ++j) nb += (int)((members[i]->n[S.map_k[j]] + kWarpsW - 1) / kWarpsW);
      for (int j = 0; j < S.njob; ++j) {
        nb += S.job[j].nb;
        dd = std::max(dd, warp_job_outputs(S.job[j]));
      }
      base.push_back(base.back() + nb);
    }
    Stage* sd = nullptr;
    int* bd = nullptr;
    e = upload((void**)&sd, st.data(), sizeof(Stage) * count);
    g->stages.push_back(sd);
    if (e == cudaSuccess) e = upload((void**)&bd, base.data(), sizeof(int) * base.size());
    g->base.push_back(bd);
    g->blocks.push_back(base.back());
    g->no.push_back((dd + 31) / 32);
  }
  if (e == cudaSuccess) {
    std::vector<int> base(1, 0);
    for (int i = 0; i < count; ++i) {
      int nsl = 0;
      for (int k = 0; k < g->m; ++k) nsl += (int)members[i]->n[k];
      base.push_back(base.back() + (nsl + kWarpsW - 1) / kWarpsW);
      g->smem_c = std::max(g->smem_c, sizeof(double) * (size_t)kWarpsW * 3 * wscr_mat_host(members[i]->hp));
    }
    e = upload((void**)&g->base_c, base.data(), sizeof(int) * base.size());
    g->blocks_c = base.back();
  }
  if (e != cudaSuccess) {
    ttc_dense_group_destroy(g);
    return e == cudaErrorMemoryAllocation ? TTC_ENOMEM : TTC_ECUDA;
  }
  *out = g;
  return TTC_OK;
}

// save-previous copy, Gram stages, rank-2r assembly, right Grams, bonds: one
// launch each for all members of the group
int ttc_dense_group_launch(const DenseGroup* g, cudaStream_t st, long long* kernels) {
  long long n = 0;
  k_save_prev_batch<<<g->nprob * kCopyBlocks, 256, 0, st>>>(g->probs, g->nprob);
  TTC_CUDA(cudaGetLastError());
  ++n;
  auto stage = [&](int si) -> int {
    const int no = g->no[si];
    if (no <= 1)
      k_stage_w_batch<1><<<g->blocks[si], kThreads, g->smem, st>>>(g->probs, g->stages[si], g->base[si], g->nprob);
    else if (no <= 2)
      k_stage_w_batch<2><<<g->blocks[si], kThreads, g->smem, st>>>(g->probs, g->stages[si], g->base[si], g->nprob);
    else if (no <= 4)
      k_stage_w_batch<4><<<g->blocks[si], kThreads, g->smem, st>>>(g->probs, g->stages[si], g->base[si], g->nprob);
    else if (no <= 8)
      k_stage_w_batch<8><<<g->blocks[si], kThreads, g->smem, st>>>(g->probs, g->stages[si], g->base[si], g->nprob);
    else
      return TTC_EUNSUPPORTED;
    TTC_CUDA(cudaGetLastError());
    ++n;
    return TTC_OK;
  };
  const int m = g->m;
  for (int si = 0; si < m - 1; ++si) TTC_TRY(stage(si));
  k_build_C_w_batch<<<g->blocks_c, kThreads, g->smem_c, st>>>(g->probs, g->base_c, g->nprob);
  TTC_CUDA(cudaGetLastError());
  ++n;
  for (int si = m - 1; si < 3 * m - 2; ++si) TTC_TRY(stage(si));
  if (kernels) *kernels += n;
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
  // Gram sweep: one stage per core with the AA, AB and BB jobs
  const int m = P.m;
  for (int k = 0; k < m; ++k) {
    Stage S = pl.metric[which][k];
    long long red = P.red_metric, red2 = P.red2_metric;
    const int ra = P.r[k + 1];
    const int sb = which == 0 ? P.rt[k + 1] : P.r[k + 1];
    Job J = S.job[0];
    J.op = OP_DAB;
    J.rows = ra;
    J.cols = sb;
    J.red = red;
    J.red2 = red2;
    J.dst = P.off_mlam[1][k + 1];
    red += (long long)J.nb * ra * sb;
    red2 += (long long)job_groups(J.nb) * ra * sb;
    S.job[S.njob++] = J;
    J.op = OP_DBB;
    J.rows = sb;
    J.cols = sb;
    J.red = red;
    J.red2 = red2;
    J.dst = P.off_mlam[2][k + 1];
    S.job[S.njob++] = J;
    TTC_TRY(launch_stage(c, S, pl.smem_stage, 0));
  }
  return TTC_OK;
}

void ttc_free_plan(const ttc_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plan_of.erase(c);
}
