// An allocation-free entry point: the squared Frobenius distance between two
// tensor trains held in caller-provided device memory, with the per-block
// partial sums kept in a file-scope device array instead of memory obtained
// from cudaMalloc.
//
// Who needs this: callers that may not allocate device memory at all, e.g. a
// real-time or embedded loop with a fixed memory budget decided up front, or
// code running inside another framework that owns every device allocation
// (its own pool allocator) and forbids raw cudaMalloc/cudaFree.  They pass
// inputs and outputs; the library brings only this fixed scratch array.
//
// The paper has no counterpart of this call; it evaluates the same quantity
// as the stopping rule's distance (relative error of an iterate).
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kStaticBlocks = 1024;      // maximum number of blocks (partials) per call
constexpr int kStaticThreads = 256;
constexpr long long kMaxEntries = 1LL << 32;   // largest d* accepted (every entry is evaluated)
constexpr double kMaxWork = 17179869184.0;      // largest FP64 FMA count accepted, 2^34 (d* times the
                                                // chain products of one entry of A and of B)

// Scratch: two doubles (sum of squared differences, sum of squares of B) per
// block.  Every GPU that loads the library holds these 16 KiB until exit.
static __device__ __align__(256) double g_dist_scratch[2 * kStaticBlocks];

struct TTPair {
  int d;
  int n[TTC_MAXM];
  int ra[TTC_MAXM + 1];
  int rb[TTC_MAXM + 1];
  const double* a[TTC_MAXM];   // core k: ra[k] x n[k] x ra[k+1], row-major
  const double* b[TTC_MAXM];
};

// cores in the layout of the C ABI: core k is ra[k] x n[k] x ra[k+1], row-major
struct HostLayoutCores {
  const double* const* core;
  const int* rk;
  const int* nk;
  __device__ __forceinline__ int r(int k) const { return rk[k]; }
  __device__ __forceinline__ double at(int k, int x, int i, int j) const {
    return core[k][((long long)i * nk[k] + x) * rk[k + 1] + j];
  }
};

__global__ void __launch_bounds__(kStaticThreads) k_dist_partial(const TTPair T, long long dstar, double* scratch) {
  const HostLayoutCores A{T.a, T.ra, T.n};
  const HostLayoutCores B{T.b, T.rb, T.n};
  tt_dist_block(A, B, T.d, T.n, dstar, scratch);
}

// sums the partials of this call in block order (every slot < nb was written
// by this call's first kernel, so nothing needs clearing)
__global__ void k_dist_finish(const double* scratch, int nb, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
      a += scratch[2 * i];
      b += scratch[2 * i + 1];
    }
    out[0] = a;
    out[1] = b;
  }
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in).
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    return TTC_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TTC_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dist_scratch);
    if (e != cudaSuccess) {
      ttc_record_cuda_error(e);
      return TTC_ECUDA;
    }
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return TTC_OK;
}

}  // namespace

extern "C" int ttc_tt_dist2_static(int d, const int64_t* n, const int32_t* ra, const double* const* a_dev,
                                   const int32_t* rb, const double* const* b_dev, double* out_dev,
                                   void* cuda_stream) {
  if (!n || !ra || !rb || !a_dev || !b_dev || !out_dev) return TTC_EINVAL;
  if (d < 1) return TTC_EINVAL;
  if (d > TTC_MAXM) return TTC_EUNSUPPORTED;
  if (ra[0] != 1 || ra[d] != 1 || rb[0] != 1 || rb[d] != 1) return TTC_EINVAL;
  TTPair T;
  T.d = d;
  long long dstar = 1;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1 || !a_dev[k] || !b_dev[k]) return TTC_EINVAL;
    if (n[k] > (1LL << 30) || dstar > kMaxEntries / n[k]) return TTC_EUNSUPPORTED;
    dstar *= n[k];
    T.n[k] = (int)n[k];
    T.a[k] = a_dev[k];
    T.b[k] = b_dev[k];
  }
  for (int k = 0; k <= d; ++k) {
    if (ra[k] < 1 || rb[k] < 1) return TTC_EINVAL;
    if (ra[k] > TTC_MAXR || rb[k] > TTC_MAXR) return TTC_EUNSUPPORTED;
    T.ra[k] = ra[k];
    T.rb[k] = rb[k];
  }
  // bound the work, not only d*: a rank-32 train of many small modes would
  // otherwise keep the GPU busy for minutes
  double per_entry = 0.0;
  for (int k = 0; k < d; ++k) per_entry += (double)ra[k] * ra[k + 1] + (double)rb[k] * rb[k + 1];
  if ((double)dstar * per_entry > kMaxWork) return TTC_EUNSUPPORTED;
  double* scratch = nullptr;
  int s = scratch_for_current_device(&scratch);
  if (s != TTC_OK) return s;
  long long want = (dstar + kStaticThreads - 1) / kStaticThreads;
  int nb = (int)(want < kStaticBlocks ? want : kStaticBlocks);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_dist_partial<<<nb, kStaticThreads, 0, st>>>(T, dstar, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_dist_finish<<<1, 32, 0, st>>>(scratch, nb, out_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    ttc_record_cuda_error(e);
    return TTC_ECUDA;
  }
  return TTC_OK;
}
