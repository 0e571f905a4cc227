// Instantiation helpers for the tensor kernels (included by k_quad.cu, k_hex.cu).
#pragma once
#include "kdispatch.hpp"
#include "ktensor.cuh"

namespace frp {

template <int DIM, int N, typename T, int MODE, int TD = 1>
void launch_kb_tensor(const KArgs& A, cudaStream_t s) {
  using LY = KBLayout<DIM, N, T, MODE, TD>;
  launch_kernel(kb_tensor<DIM, N, T, MODE, TD>, LY::SMEM, LY::ET, A, s, LY::THREADS);
}

template <int DIM, int N, typename T, int MODE, int TD = 1>
void launch_ka_tensor(const KArgs& A, cudaStream_t s) {
  using LY = KALayout<DIM, N, T, MODE, TD>;
  if constexpr (StageKA<DIM, T, MODE>::v) {
    switch (A.stage) {
      case 1: launch_kernel(ka_tensor<DIM, N, T, MODE, TD, 1>, LY::SMEM, LY::ET, A, s, LY::THREADS); return;
      case 2: launch_kernel(ka_tensor<DIM, N, T, MODE, TD, 2>, LY::SMEM, LY::ET, A, s, LY::THREADS); return;
      case 3: launch_kernel(ka_tensor<DIM, N, T, MODE, TD, 3>, LY::SMEM, LY::ET, A, s, LY::THREADS); return;
      case 4: launch_kernel(ka_tensor<DIM, N, T, MODE, TD, 4>, LY::SMEM, LY::ET, A, s, LY::THREADS); return;
      default: break;
    }
  }
  launch_kernel(ka_tensor<DIM, N, T, MODE, TD>, LY::SMEM, LY::ET, A, s, LY::THREADS);
}

template <int DIM, int N, typename T, int MODE, int TD, int SF>
bool prepare_ka() {
  return cudaFuncSetAttribute(ka_tensor<DIM, N, T, MODE, TD, SF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KALayout<DIM, N, T, MODE, TD>::SMEM) == cudaSuccess;
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
template <int DIM, int N, typename T, int MODE, int TD = 1>
bool prepare_tensor() {
  bool ok = cudaFuncSetAttribute(kb_tensor<DIM, N, T, MODE, TD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)KBLayout<DIM, N, T, MODE, TD>::SMEM) == cudaSuccess &&
            prepare_ka<DIM, N, T, MODE, TD, -2>();
  if constexpr (StageKA<DIM, T, MODE>::v)
    ok = ok && prepare_ka<DIM, N, T, MODE, TD, 1>() && prepare_ka<DIM, N, T, MODE, TD, 2>() &&
         prepare_ka<DIM, N, T, MODE, TD, 3>() && prepare_ka<DIM, N, T, MODE, TD, 4>();
  return ok;
}

// TB, TA: the tile divisors of the physical-step residual and update
// kernels (the kernel variant; the preconditioning kernels keep the default
// tiles)
template <int DIM, int N, typename T, int TB = 1, int TA = 1>
void fill_tensor(int64_t E, KernelSet* ks) {
  ks->prepared = prepare_tensor<DIM, N, T, 0, TB>() && prepare_tensor<DIM, N, T, 0, TA>() &&
                 prepare_tensor<DIM, N, T, 1>();
  ks->vcache = launch_vcache<DIM, N, T>;
  ks->mconst = launch_mconst<DIM, N, T>;
  ks->kb[0] = launch_kb_tensor<DIM, N, T, 0, TB>;
  ks->kb[1] = launch_kb_tensor<DIM, N, T, 1>;
  ks->ka[0] = launch_ka_tensor<DIM, N, T, 0, TA>;
  ks->ka[1] = launch_ka_tensor<DIM, N, T, 1>;
  const int et_min = KBLayout<DIM, N, T, 0, TB>::ET < KALayout<DIM, N, T, 0, TA>::ET ? KBLayout<DIM, N, T, 0, TB>::ET
                                                                                      : KALayout<DIM, N, T, 0, TA>::ET;
  const int et_min1 = KBLayout<DIM, N, T, 1>::ET < KALayout<DIM, N, T, 1>::ET ? KBLayout<DIM, N, T, 1>::ET
                                                                               : KALayout<DIM, N, T, 1>::ET;
  const int et = et_min < et_min1 ? et_min : et_min1;
  ks->max_blocks = (int)((E + et - 1) / et);
}

}  // namespace frp
