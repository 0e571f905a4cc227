// Kernel tables per element type, order and precision (see k_*.cu).
#pragma once
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace frp {

typedef void (*LaunchFn)(const KArgs&, cudaStream_t);

struct KernelSet {
  LaunchFn kb[2] = {nullptr, nullptr};  // [mode]: 0 physical, 1 preconditioning
  LaunchFn ka[2] = {nullptr, nullptr};
  int max_blocks = 0;                   // upper bound on blocks of any launch (per element count)
  LaunchFn vcache = nullptr;            // fills the spatial velocity cache (nullptr: not supported)
  LaunchFn mconst = nullptr;            // fills the per-element metric records (tensor elements)
  bool prepared = false;                // shared-memory limits set for every kernel of the set
};

// Return false if the (order, precision) pair is not built.
bool kernels_quad(int order, int precision, int64_t E, int variant, KernelSet* ks);
bool kernels_hex(int order, int precision, int64_t E, int variant, KernelSet* ks);
bool kernels_tri(int order, int precision, int64_t E, int variant, KernelSet* ks);

template <typename K>
inline void launch_kernel(K kern, size_t smem, int et, const KArgs& A, cudaStream_t s, int threads = kThreads) {
  const int64_t grid = (A.E + et - 1) / et;
  kern<<<(unsigned)grid, threads, smem, s>>>(A);
}

}  // namespace frp
