// Omega layout builder (once per problem): validates the observed index set,
// packs coordinates into 32-bit code words, and for every mode k builds the
// stable order of the entries by x_k with the CSR offsets of the mode-k
// slices and the chunk lists the sampled pass walks.  Mode k's order is the
// stable sort by x_k of mode k-1's (mode 0's of the input order), so it is
// lexicographic in (x_k, x_{k-1}, ..., x_0): inside a mode-k slice, entries
// that share the prefix (x_0 .. x_{k-1}) are adjacent, and the prefix-table
// rows the passes read for them are read by neighbouring lanes.
// Duplicate indices are found by a lexicographic order built from the same
// stable per-mode sort (LSD over modes d..1).  Problem statement: Omega is a
// set of observed indices and P_Omega samples T on it (Eq. (model: Low TT)).
#include <algorithm>
#include <vector>

#include "ctx.h"

namespace {

constexpr int kTile = 256;   // entries per block in the radix passes

__global__ void k_validate_pack(const int32_t* __restrict__ idx, const double* __restrict__ y, int N,
                                DevProb P, uint32_t* __restrict__ code, int* __restrict__ flags) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  int bad = 0;
  for (int k = 0; k < P.m; ++k) {
    int x = idx[(long long)e * P.m + k];
    if (x < 0 || x >= P.n[k]) {
      bad |= 1;
      x = 0;
    }
    w[P.cword[k]] |= ((uint32_t)x) << P.cshift[k];
  }
  double v = y[e];
  if (!isfinite(v)) bad |= 4;
  for (int i = 0; i < P.W; ++i) code[(long long)e * P.W + i] = w[i];
  if (bad) atomicOr(flags, bad);
}

__device__ __forceinline__ int digit_of(const uint32_t* code, int W, int e, int word, int shift, int dbits) {
  return (int)((code[(long long)e * W + word] >> shift) & ((1u << dbits) - 1u));
}

// per-tile histogram of one radix digit; counts are digit-major [digit][tile]
__global__ void k_digit_hist(const int* __restrict__ perm_in, const uint32_t* __restrict__ code, int W, int N,
                             int word, int shift, int dbits, int ntiles, int* __restrict__ counts) {
  __shared__ int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int j = blockIdx.x * kTile + threadIdx.x;
  if (j < N) atomicAdd(&h[digit_of(code, W, perm_in[j], word, shift, dbits)], 1);
  __syncthreads();
  int nd = 1 << dbits;
  for (int d = threadIdx.x; d < nd; d += blockDim.x) counts[(long long)d * ntiles + blockIdx.x] = h[d];
}

// stable scatter: warps of the tile are taken in order, and inside a warp the
// entries with equal digit are ranked by lane
__global__ void k_digit_scatter(const int* __restrict__ perm_in, int* __restrict__ perm_out,
                                const uint32_t* __restrict__ code, int W, int N, int word, int shift, int dbits,
                                int ntiles, const int* __restrict__ offsets) {
  __shared__ int base[256];
  int nd = 1 << dbits;
  for (int d = threadIdx.x; d < nd; d += blockDim.x) base[d] = offsets[(long long)d * ntiles + blockIdx.x];
  __syncthreads();
  int j = blockIdx.x * kTile + threadIdx.x;
  int valid = j < N;
  int e = valid ? perm_in[j] : 0;
  int d = valid ? digit_of(code, W, e, word, shift, dbits) : 256;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) {
    if (warp == wv) {
      unsigned mask = __match_any_sync(0xffffffffu, d);
      int rank = __popc(mask & ((1u << lane) - 1u));
      int pos = valid ? base[d] + rank : 0;
      __syncwarp();
      if (valid) {
        perm_out[pos] = e;
        if (rank == 0) base[d] += __popc(mask);
      }
    }
    __syncthreads();
  }
}

// single-block exclusive scan of n ints (in place), writes the total to *total
__global__ void k_scan(int* __restrict__ a, long long n, int* __restrict__ total) {
  __shared__ long long part[1024];
  long long per = (n + blockDim.x - 1) / blockDim.x;
  long long b = threadIdx.x * per, e = min(n, b + per);
  long long s = 0;
  for (long long i = b; i < e; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      long long v = part[t];
      part[t] = run;
      run += v;
    }
    if (total) *total = (int)run;
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (long long i = b; i < e; ++i) {
    int v = a[i];
    a[i] = (int)run;
    run += v;
  }
}

// Multi-block exclusive scan for long count arrays (the digit-major radix
// counts hold 256 per tile): block sums of consecutive segments, a scan of
// the block sums, then each block scans its segment from its offset.  Same
// integers as k_scan; the single-block k_scan took ~0.1 ms per radix pass.
constexpr int kScanThreads = 256;
__global__ void __launch_bounds__(kScanThreads) k_scan_blocksum(const int* __restrict__ a, long long n, long long L,
                                                                long long* __restrict__ bsum) {
  __shared__ long long sh[kScanThreads];
  const long long b0 = blockIdx.x * L, e0 = min(n, b0 + L);
  long long s = 0;
  for (long long i = b0 + threadIdx.x; i < e0; i += kScanThreads) s += a[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kScanThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

// exclusive scan of nb <= 1024 block sums in place (one block of 1024)
__global__ void __launch_bounds__(1024) k_scan_top(long long* __restrict__ bsum, int nb, int* __restrict__ total) {
  __shared__ long long sh[1024];
  const int t = threadIdx.x;
  const long long v = t < nb ? bsum[t] : 0;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long w = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += w;
    __syncthreads();
  }
  if (t < nb) bsum[t] = sh[t] - v;
  if (t == 1023 && total) *total = (int)sh[t];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int* __restrict__ a, long long n, long long L,
                                                             const long long* __restrict__ bsum) {
  __shared__ long long sh[kScanThreads];
  __shared__ long long base;
  const int t = threadIdx.x;
  if (t == 0) base = bsum[blockIdx.x];
  const long long b0 = blockIdx.x * L, e0 = min(n, b0 + L);
  for (long long c0 = b0; c0 < e0; c0 += kScanThreads) {
    const long long i = c0 + t;
    const int v = i < e0 ? a[i] : 0;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
      const long long w = t >= o ? sh[t - o] : 0;
      __syncthreads();
      sh[t] += w;
      __syncthreads();
    }
    const long long incl = sh[t], bb = base;
    __syncthreads();
    if (i < e0) a[i] = (int)(bb + incl - v);
    if (t == kScanThreads - 1) base = bb + incl;
    __syncthreads();
  }
}

// exclusive scan of a[0..n) in place; total (if given) receives the sum;
// bsum: 1024 long longs of scratch
void scan_ints(int* a, long long n, int* total, long long* bsum, cudaStream_t st) {
  if (n <= 16384) {
    k_scan<<<1, 1024, 0, st>>>(a, n, total);
    return;
  }
  long long L = std::max(4096LL, (n + 1023) / 1024);
  L = (L + kScanThreads - 1) / kScanThreads * kScanThreads;
  const int nb = (int)((n + L - 1) / L);   // <= 1024
  k_scan_blocksum<<<nb, kScanThreads, 0, st>>>(a, n, L, bsum);
  k_scan_top<<<1, 1024, 0, st>>>(bsum, nb, total);
  k_scan_apply<<<nb, kScanThreads, 0, st>>>(a, n, L, bsum);
}

__global__ void k_iota(int* __restrict__ p, int N) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) p[j] = j;
}

__global__ void k_dup_check(const int* __restrict__ perm, const uint32_t* __restrict__ code, int W, int N,
                            int* __restrict__ flags) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j <= 0 || j >= N) return;
  int a = perm[j], b = perm[j - 1];
  bool same = true;
  for (int w = 0; w < W; ++w) same = same && (code[(long long)a * W + w] == code[(long long)b * W + w]);
  if (same) atomicOr(flags, 2);
}

__global__ void k_gather_mode(const int* __restrict__ perm, const uint32_t* __restrict__ code_in,
                              const double* __restrict__ y, int W, int N, uint32_t* __restrict__ code_out,
                              float* __restrict__ y32, double* __restrict__ y64) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  int e = perm[j];
  for (int w = 0; w < W; ++w) code_out[(long long)j * W + w] = code_in[(long long)e * W + w];
  double v = y[e];
  y64[j] = v;
  y32[j] = (float)v;
}

// seg[x] = first position whose coordinate is >= x (x = 0..n), from sorted order
__global__ void k_seg_bounds(const int* __restrict__ perm, const uint32_t* __restrict__ code, int W, int N,
                             int word, int shift, int bits, int nk, int* __restrict__ seg) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  uint32_t mask = (bits >= 32) ? 0xffffffffu : ((1u << bits) - 1u);
  int key = (int)((code[(long long)perm[j] * W + word] >> shift) & mask);
  int prev = (j == 0) ? -1 : (int)((code[(long long)perm[j - 1] * W + word] >> shift) & mask);
  for (int x = prev + 1; x <= key; ++x) seg[x] = j;
  if (j == N - 1)
    for (int x = key + 1; x <= nk; ++x) seg[x] = N;
}

__global__ void k_chunk_counts(const int* __restrict__ seg, int nk, int chunk, int* __restrict__ cnt) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < nk) cnt[x] = (seg[x + 1] - seg[x] + chunk - 1) / chunk;
  if (x == nk) cnt[x] = 0;
}

__global__ void k_chunk_fill(const int* __restrict__ cfirst, int nk, int* __restrict__ cseg) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nk) return;
  for (int c = cfirst[x]; c < cfirst[x + 1]; ++c) cseg[c] = x;
}

inline int nblk(long long n, int bs) { return (int)((n + bs - 1) / bs); }

// stable LSD radix sort of perm_in by the coordinate of mode k (8-bit digits)
int sort_by_mode(ttc_ctx* c, const uint32_t* code, const int* perm_in, int* perm_out, int* tmp_perm, int k,
                 int* counts, long long* bsum) {
  const DevProb& P = c->hp;
  int N = P.N;
  int ntiles = nblk(N, kTile);
  int bits = P.cbits[k];
  cudaStream_t st = c->stream;
  if (bits == 0) {
    TTC_CUDA(cudaMemcpyAsync(perm_out, perm_in, sizeof(int) * N, cudaMemcpyDeviceToDevice, st));
    return TTC_OK;
  }
  int passes = (bits + 7) / 8;
  const int* src = perm_in;
  for (int ps = 0; ps < passes; ++ps) {
    int dbits = std::min(8, bits - 8 * ps);
    // ping-pong so that the last pass lands in perm_out
    int* dst = ((passes - 1 - ps) % 2 == 0) ? perm_out : tmp_perm;
    int shift = P.cshift[k] + 8 * ps;
    long long ncount = (long long)(1 << dbits) * ntiles;
    k_digit_hist<<<ntiles, kTile, 0, st>>>(src, code, P.W, N, P.cword[k], shift, dbits, ntiles, counts);
    scan_ints(counts, ncount, nullptr, bsum, st);
    k_digit_scatter<<<ntiles, kTile, 0, st>>>(src, dst, code, P.W, N, P.cword[k], shift, dbits, ntiles, counts);
    TTC_CUDA(cudaGetLastError());
    src = dst;
  }
  return TTC_OK;
}

}  // namespace

int ttc_build_layout(ttc_ctx* c, const int32_t* idx_host, const double* y_host) {
  DevProb& P = c->hp;
  const int m = c->m, N = c->N;
  cudaStream_t st = c->stream;

  // code word packing: fields never straddle a 32-bit word
  int word = 0, shift = 0;
  for (int k = 0; k < m; ++k) {
    int bits = 0;
    while ((1LL << bits) < c->n[k]) ++bits;
    if (shift + bits > 32) {
      ++word;
      shift = 0;
    }
    P.cword[k] = word;
    P.cshift[k] = shift;
    P.cbits[k] = bits;
    shift += bits;
  }
  int W = word + 1;
  if (W == 3) W = 4;
  if (W > 4) return TTC_EUNSUPPORTED;
  P.W = W;
  P.N = N;

  // temporaries
  int32_t* idx_d = nullptr;
  double* y_d = nullptr;
  uint32_t* code_in = nullptr;
  int *pa = nullptr, *pb = nullptr, *pt = nullptr, *counts = nullptr, *flags = nullptr, *scr = nullptr;
  long long* bsum = nullptr;
  int ntiles = nblk(N, kTile);
  long long ncount_max = 256LL * ntiles;
  long long maxn = 0;
  for (int k = 0; k < m; ++k) maxn = std::max(maxn, c->n[k]);
  auto cleanup = [&]() {
    for (void* q : {(void*)idx_d, (void*)y_d, (void*)code_in, (void*)pa, (void*)pb, (void*)pt, (void*)counts,
                    (void*)flags, (void*)scr, (void*)bsum})
      ttc_pool_free(q, st);
  };
#define LTRY(call)                        \
  do {                                    \
    cudaError_t _e = (call);              \
    if (_e != cudaSuccess) {              \
      ttc_record_cuda_error(_e);          \
      cleanup();                          \
      return _e == cudaErrorMemoryAllocation ? TTC_ENOMEM : TTC_ECUDA; \
    }                                     \
  } while (0)
  LTRY(ttc_pool_alloc((void**)&idx_d, sizeof(int32_t) * (size_t)N * m, st));
  LTRY(ttc_pool_alloc((void**)&y_d, sizeof(double) * (size_t)N, st));
  LTRY(ttc_pool_alloc((void**)&code_in, sizeof(uint32_t) * (size_t)N * W, st));
  LTRY(ttc_pool_alloc((void**)&pa, sizeof(int) * (size_t)N, st));
  LTRY(ttc_pool_alloc((void**)&pb, sizeof(int) * (size_t)N, st));
  LTRY(ttc_pool_alloc((void**)&pt, sizeof(int) * (size_t)N, st));
  LTRY(ttc_pool_alloc((void**)&counts, sizeof(int) * (size_t)std::max(ncount_max, maxn + 2), st));
  LTRY(ttc_pool_alloc((void**)&flags, sizeof(int) * (4 + TTC_MAXM), st));   // flags, then per-mode chunk totals
  LTRY(ttc_pool_alloc((void**)&bsum, sizeof(long long) * 1024, st));
  LTRY(ttc_pool_alloc((void**)&scr, sizeof(int) * (size_t)(maxn + 2), st));
  LTRY(cudaMemcpyAsync(idx_d, idx_host, sizeof(int32_t) * (size_t)N * m, cudaMemcpyHostToDevice, st));
  LTRY(cudaMemcpyAsync(y_d, y_host, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, st));
  LTRY(cudaMemsetAsync(flags, 0, sizeof(int) * 4, st));
  k_validate_pack<<<nblk(N, 256), 256, 0, st>>>(idx_d, y_d, N, P, code_in, flags);
  LTRY(cudaGetLastError());
  int hflags = 0;
  LTRY(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  LTRY(cudaStreamSynchronize(st));
  if (hflags & 1) { cleanup(); return TTC_ERANGE; }
  if (hflags & 4) { cleanup(); return TTC_ENONFINITE; }

  // duplicates: lexicographic order by stable passes over modes m-1 .. 0
  k_iota<<<nblk(N, 256), 256, 0, st>>>(pa, N);
  for (int k = m - 1; k >= 0; --k) {
    int s = sort_by_mode(c, code_in, pa, pb, pt, k, counts, bsum);
    if (s != TTC_OK) { cleanup(); return s; }
    std::swap(pa, pb);
  }
  k_dup_check<<<nblk(N, 256), 256, 0, st>>>(pa, code_in, W, N, flags);
  LTRY(cudaGetLastError());
  LTRY(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  LTRY(cudaStreamSynchronize(st));
  if (hflags & 2) { cleanup(); return TTC_EDUP; }

  // per-mode layouts; each mode's chunk list is allocated for its bound
  // sum_x ceil(n_x / chunk) <= N / chunk + n_k, and the totals are read back
  // once after all modes
  int maxstride = 1;
  int* totals = flags + 4;
  for (int k = 0; k < m; ++k) {
    int nk = (int)c->n[k];
    uint32_t* code_k = nullptr;
    float* y32 = nullptr;
    double* y64 = nullptr;
    int *perm = nullptr, *seg = nullptr, *cfirst = nullptr, *cseg = nullptr;
    int s = TTC_OK;
    if ((s = ttc_alloc(c, (void**)&code_k, sizeof(uint32_t) * (size_t)N * W, true)) ||
        (s = ttc_alloc(c, (void**)&y32, sizeof(float) * (size_t)N, true)) ||
        (s = ttc_alloc(c, (void**)&y64, sizeof(double) * (size_t)N, true)) ||
        (s = ttc_alloc(c, (void**)&perm, sizeof(int) * (size_t)N, true)) ||
        (s = ttc_alloc(c, (void**)&seg, sizeof(int) * (size_t)(nk + 1), true)) ||
        (s = ttc_alloc(c, (void**)&cfirst, sizeof(int) * (size_t)(nk + 1), true))) {
      cleanup();
      return s;
    }
    const int* from = pa;
    if (k == 0)
      k_iota<<<nblk(N, 256), 256, 0, st>>>(pa, N);
    else
      from = P.perm[k - 1];   // chained: lexicographic in (x_k, ..., x_0)
    if ((s = sort_by_mode(c, code_in, from, perm, pt, k, counts, bsum)) != TTC_OK) { cleanup(); return s; }
    k_gather_mode<<<nblk(N, 256), 256, 0, st>>>(perm, code_in, y_d, W, N, code_k, y32, y64);
    k_seg_bounds<<<nblk(N, 256), 256, 0, st>>>(perm, code_in, W, N, P.cword[k], P.cshift[k], P.cbits[k], nk, seg);
    k_chunk_counts<<<nblk(nk + 1, 256), 256, 0, st>>>(seg, nk, TTC_CHUNK, cfirst);
    scan_ints(cfirst, nk + 1, totals + k, bsum, st);
    LTRY(cudaGetLastError());
    const long long bound = (long long)N / TTC_CHUNK + nk + 1;
    if ((s = ttc_alloc(c, (void**)&cseg, sizeof(int) * (size_t)bound, true)) != TTC_OK) {
      cleanup();
      return s;
    }
    k_chunk_fill<<<nblk(nk, 256), 256, 0, st>>>(cfirst, nk, cseg);
    LTRY(cudaGetLastError());
    P.code[k] = code_k;
    P.y32[k] = y32;
    P.y64[k] = y64;
    P.perm[k] = perm;
    P.seg[k] = seg;
    P.cfirst[k] = cfirst;
    P.cseg[k] = cseg;
    maxstride = std::max(maxstride, 1 + c->r[k] * c->r[k + 1]);
  }
  int htot[TTC_MAXM] = {0};
  LTRY(cudaMemcpyAsync(htot, totals, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
  LTRY(cudaStreamSynchronize(st));
  int base = 0;
  for (int k = 0; k < m; ++k) {
    P.nchunk[k] = htot[k];
    P.chunk_base[k] = base;
    base += htot[k];
  }
  P.chunk_base[m] = base;
  P.part_stride = maxstride;
  void* part = nullptr;
  int s = ttc_alloc(c, &part, sizeof(double) * (size_t)std::max(base, 1) * maxstride, true);
  if (s != TTC_OK) { cleanup(); return s; }
  P.part = part;
  double* g = nullptr;
  if ((s = ttc_alloc(c, (void**)&g, sizeof(double) * (size_t)N, true)) != TTC_OK) { cleanup(); return s; }
  P.g = g;
  LTRY(cudaStreamSynchronize(st));
  cleanup();
#undef LTRY
  return TTC_OK;
}
