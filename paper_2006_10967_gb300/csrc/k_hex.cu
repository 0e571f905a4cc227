// Hexahedron kernel instantiations (p = 1..5, fp64 and mixed).
#include "k_tensor_inst.cuh"

namespace frp {
// Variants (mixed precision; FP64 has variant 0 only): the tiles of the
// physical-step residual and update kernels, 0 (default, default),
// 1 (half, half), 2 (default, half), 3 (half, default)
bool kernels_hex(int order, int precision, int64_t E, int variant, KernelSet* ks) {
  if (variant < 0 || variant > 3 || (variant > 0 && precision == 0)) return false;
#define FRP_H(P)                                                          \
  case P:                                                                 \
    if (precision == 0) fill_tensor<3, P + 1, double>(E, ks);             \
    else if (variant == 0) fill_tensor<3, P + 1, float>(E, ks);           \
    else if (variant == 1) fill_tensor<3, P + 1, float, 2, 2>(E, ks);     \
    else if (variant == 2) fill_tensor<3, P + 1, float, 1, 2>(E, ks);     \
    else fill_tensor<3, P + 1, float, 2, 1>(E, ks);                       \
    return true;
  switch (order) {
    FRP_H(1) FRP_H(2) FRP_H(3) FRP_H(4) FRP_H(5)
    default: return false;
  }
#undef FRP_H
}
}  // namespace frp
