// Triangle kernel instantiations (p = 1..5, fp64 and mixed).
#include "kdispatch.hpp"
#include "ktri.cuh"

namespace frp {

template <int P, typename T, int MODE, bool TC>
void launch_kb_tri(const KArgs& A, cudaStream_t s) {
  using LY = KBTriLayout<P, T, MODE, TC>;
  launch_kernel(kb_tri<P, T, MODE, TC>, LY::SMEM, LY::ET, A, s);
}

template <int P, typename T, int MODE, bool TC>
void launch_ka_tri(const KArgs& A, cudaStream_t s) {
  using LY = KATriLayout<P, T, MODE, TC>;
  launch_kernel(ka_tri<P, T, MODE, TC>, LY::SMEM, LY::ET, A, s);
}

template <int P, typename T, int MODE, bool TC>
bool prepare_tri() {
  return cudaFuncSetAttribute(kb_tri<P, T, MODE, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KBTriLayout<P, T, MODE, TC>::SMEM) == cudaSuccess &&
         cudaFuncSetAttribute(ka_tri<P, T, MODE, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KATriLayout<P, T, MODE, TC>::SMEM) == cudaSuccess;
}

template <int P, typename T>
void launch_vcache_tri(const KArgs& A, cudaStream_t s) {
  k_vel_cache_tri<P, T><<<152 * 8, kThreads, 0, s>>>(A);
}

template <int P, typename T, bool TC>
void fill_tri(int64_t E, KernelSet* ks) {
  ks->prepared = prepare_tri<P, T, 0, TC>() && prepare_tri<P, T, 1, TC>();
  ks->vcache = launch_vcache_tri<P, T>;
  ks->kb[0] = launch_kb_tri<P, T, 0, TC>;
  ks->kb[1] = launch_kb_tri<P, T, 1, TC>;
  ks->ka[0] = launch_ka_tri<P, T, 0, TC>;
  ks->ka[1] = launch_ka_tri<P, T, 1, TC>;
  int et = KBTriLayout<P, T, 0, TC>::ET;
  if (KATriLayout<P, T, 0, TC>::ET < et) et = KATriLayout<P, T, 0, TC>::ET;
  if (KBTriLayout<P, T, 1, TC>::ET < et) et = KBTriLayout<P, T, 1, TC>::ET;
  if (KATriLayout<P, T, 1, TC>::ET < et) et = KATriLayout<P, T, 1, TC>::ET;
  ks->max_blocks = (int)((E + et - 1) / et);
}

// variant 0: scalar dot products; variant 1 (float path only): the operator
// applies on tensor cores
bool kernels_tri(int order, int precision, int64_t E, int variant, KernelSet* ks) {
  if (variant < 0 || variant > 1 || (variant == 1 && precision == 0)) return false;
#define FRP_T(P)                                                      \
  case P:                                                             \
    if (precision == 0) fill_tri<P, double, false>(E, ks);            \
    else if (variant == 0) fill_tri<P, float, false>(E, ks);          \
    else fill_tri<P, float, true>(E, ks);                             \
    return true;
  switch (order) {
    FRP_T(1) FRP_T(2) FRP_T(3) FRP_T(4) FRP_T(5)
    default: return false;
  }
#undef FRP_T
}

}  // namespace frp
