// Allocation-free weighted integral: sum_i w_i u_i with the same Neumaier
// compensation as fr_mass_integral but its own fixed summation order
// (contiguous 2048-value blocks, then the block partials in order), for
// callers that cannot call cudaMalloc (see include/fr_pcpf.h,
// fr_mass_integral_noalloc).
//
// Its scratch (per-block partial sums, the last-block counter and the result)
// is one file-scope __device__ array.  Host code cannot use the array's name
// as a device address, so the address is fetched with cudaGetSymbolAddress
// once per device (on that device's first call) and passed to the kernel.
#include <cuda_runtime.h>

#include "../../include/fr_pcpf.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 8;
constexpr int64_t kMaxPartials = FR_NOALLOC_MAX_BLOCKS;
constexpr int kMaxDevices = 64;

// [0, 2*kMaxPartials): (sum, compensation) per block; then the result; then
// the last-block counter (an unsigned long long stored in a double slot).
static __device__ __align__(256) double g_integral_scratch[2 * kMaxPartials + 2];

double* g_scratch_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ void neu_add(double& s, double& c, double x) {
  const double t = s + x;
  c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

__global__ void k_weighted_sum(const double* __restrict__ u, const double* __restrict__ w, int64_t n,
                               double* scratch) {
  __shared__ double ss[kThreads], sc[kThreads];
  __shared__ bool last;
  double s = 0.0, c = 0.0;
  const int64_t base = (int64_t)blockIdx.x * kThreads * kItemsPerThread;
  for (int k = 0; k < kItemsPerThread; ++k) {
    const int64_t g = base + (int64_t)k * kThreads + threadIdx.x;
    if (g < n) neu_add(s, c, w[g] * u[g]);
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch + 2 * kMaxPartials + 1);
  if (threadIdx.x == 0) {
    double bs = 0.0, bc = 0.0;
    for (int t = 0; t < kThreads; ++t) {
      neu_add(bs, bc, ss[t]);
      bc += sc[t];
    }
    scratch[2 * blockIdx.x] = bs;
    scratch[2 * blockIdx.x + 1] = bc;
    __threadfence();
    last = atomicAdd(counter, 1ull) == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double ts = 0.0, tc = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      neu_add(ts, tc, ((volatile double*)scratch)[2 * b]);
      tc += ((volatile double*)scratch)[2 * b + 1];
    }
    scratch[2 * kMaxPartials] = ts + tc;
    *counter = 0ull;
  }
}

}  // namespace

extern "C" int fr_mass_integral_noalloc(const double* dev_u, const double* dev_w, int64_t n, double* out_host,
                                        void* stream) {
  if (!dev_u || !dev_w || !out_host || n < 0) return FR_EINVAL;
  if (n > FR_NOALLOC_MAX_VALUES) return FR_EINVAL;  // beyond the static scratch capacity
  if (n == 0) {
    *out_host = 0.0;
    return FR_OK;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FR_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return FR_EUNSUPPORTED;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_integral_scratch) != cudaSuccess) return FR_ECUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  double* scratch = g_scratch_ptr[dev];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the counter must start at zero even if an earlier launch was abandoned
  if (cudaMemsetAsync(scratch + 2 * kMaxPartials + 1, 0, sizeof(double), s) != cudaSuccess) return FR_ECUDA;
  const int64_t per_block = (int64_t)kThreads * kItemsPerThread;
  const int64_t grid = (n + per_block - 1) / per_block;
  k_weighted_sum<<<(unsigned)grid, kThreads, 0, s>>>(dev_u, dev_w, n, scratch);
  if (cudaGetLastError() != cudaSuccess) return FR_ECUDA;
  if (cudaMemcpyAsync(out_host, scratch + 2 * kMaxPartials, sizeof(double), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return FR_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FR_ECUDA;
  return FR_OK;
}
