// Triangle kernel instantiations (p = 1..5, fp64 and mixed).
#include "kdispatch.hpp"
#include "ktri.cuh"

namespace frp {

template <int P, typename T, int MODE>
void launch_kb_tri(const KArgs& A, cudaStream_t s) {
  using LY = KBTriLayout<P, T, MODE>;
  launch_kernel(kb_tri<P, T, MODE>, LY::SMEM, LY::ET, A, s);
}

template <int P, typename T, int MODE>
void launch_ka_tri(const KArgs& A, cudaStream_t s) {
  using LY = KATriLayout<P, T, MODE>;
  launch_kernel(ka_tri<P, T, MODE>, LY::SMEM, LY::ET, A, s);
}

template <int P, typename T, int MODE>
bool prepare_tri() {
  return cudaFuncSetAttribute(kb_tri<P, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KBTriLayout<P, T, MODE>::SMEM) == cudaSuccess &&
         cudaFuncSetAttribute(ka_tri<P, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KATriLayout<P, T, MODE>::SMEM) == cudaSuccess;
}

template <int P, typename T>
void fill_tri(int64_t E, KernelSet* ks) {
  ks->prepared = prepare_tri<P, T, 0>() && prepare_tri<P, T, 1>();
  ks->kb[0] = launch_kb_tri<P, T, 0>;
  ks->kb[1] = launch_kb_tri<P, T, 1>;
  ks->ka[0] = launch_ka_tri<P, T, 0>;
  ks->ka[1] = launch_ka_tri<P, T, 1>;
  int et = KBTriLayout<P, T, 0>::ET;
  if (KATriLayout<P, T, 0>::ET < et) et = KATriLayout<P, T, 0>::ET;
  if (KBTriLayout<P, T, 1>::ET < et) et = KBTriLayout<P, T, 1>::ET;
  if (KATriLayout<P, T, 1>::ET < et) et = KATriLayout<P, T, 1>::ET;
  ks->max_blocks = (int)((E + et - 1) / et);
}

bool kernels_tri(int order, int precision, int64_t E, KernelSet* ks) {
#define FRP_T(P)                                        \
  case P:                                               \
    if (precision == 0) fill_tri<P, double>(E, ks);     \
    else fill_tri<P, float>(E, ks);                     \
    return true;
  switch (order) {
    FRP_T(1) FRP_T(2) FRP_T(3) FRP_T(4) FRP_T(5)
    default: return false;
  }
#undef FRP_T
}

}  // namespace frp
