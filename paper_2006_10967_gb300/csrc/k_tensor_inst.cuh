// Instantiation helpers for the tensor kernels (included by k_quad.cu, k_hex.cu).
#pragma once
#include "kdispatch.hpp"
#include "ktensor.cuh"

namespace frp {

template <int DIM, int N, typename T, int MODE>
void launch_kb_tensor(const KArgs& A, cudaStream_t s) {
  using LY = KBLayout<DIM, N, T, MODE>;
  launch_kernel(kb_tensor<DIM, N, T, MODE>, LY::SMEM, LY::ET, A, s, LY::THREADS);
}

template <int DIM, int N, typename T, int MODE>
void launch_ka_tensor(const KArgs& A, cudaStream_t s) {
  using LY = KALayout<DIM, N, T, MODE>;
  launch_kernel(ka_tensor<DIM, N, T, MODE>, LY::SMEM, LY::ET, A, s, LY::THREADS);
}

template <int DIM, int N, typename T>
void launch_mconst(const KArgs& A, cudaStream_t s) {
  const int64_t g = (A.E + kThreads - 1) / kThreads;
  k_metric_const<DIM, T><<<(unsigned)(g < 152 * 8 ? g : 152 * 8), kThreads, 0, s>>>(A, TS<DIM, N>::NG, TS<DIM, N>::NU);
}

template <int DIM, int N, typename T>
void launch_vcache(const KArgs& A, cudaStream_t s) {
  k_vel_cache<DIM, N, T><<<152 * 8, kThreads, 0, s>>>(A);
}

// Shared-memory opt-in of one (kb, ka) pair; done when the kernel table is
// filled, so that no launch (and no graph capture) has to do it.
template <int DIM, int N, typename T, int MODE>
bool prepare_tensor() {
  return cudaFuncSetAttribute(kb_tensor<DIM, N, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KBLayout<DIM, N, T, MODE>::SMEM) == cudaSuccess &&
         cudaFuncSetAttribute(ka_tensor<DIM, N, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KALayout<DIM, N, T, MODE>::SMEM) == cudaSuccess;
}

template <int DIM, int N, typename T>
void fill_tensor(int64_t E, KernelSet* ks) {
  ks->prepared = prepare_tensor<DIM, N, T, 0>() && prepare_tensor<DIM, N, T, 1>();
  ks->vcache = launch_vcache<DIM, N, T>;
  ks->mconst = launch_mconst<DIM, N, T>;
  ks->kb[0] = launch_kb_tensor<DIM, N, T, 0>;
  ks->kb[1] = launch_kb_tensor<DIM, N, T, 1>;
  ks->ka[0] = launch_ka_tensor<DIM, N, T, 0>;
  ks->ka[1] = launch_ka_tensor<DIM, N, T, 1>;
  const int et_min = KBLayout<DIM, N, T, 0>::ET < KALayout<DIM, N, T, 0>::ET ? KBLayout<DIM, N, T, 0>::ET
                                                                              : KALayout<DIM, N, T, 0>::ET;
  const int et_min1 = KBLayout<DIM, N, T, 1>::ET < KALayout<DIM, N, T, 1>::ET ? KBLayout<DIM, N, T, 1>::ET
                                                                               : KALayout<DIM, N, T, 1>::ET;
  const int et = et_min < et_min1 ? et_min : et_min1;
  ks->max_blocks = (int)((E + et - 1) / et);
}

}  // namespace frp
