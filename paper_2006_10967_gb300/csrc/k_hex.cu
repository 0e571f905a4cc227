// Hexahedron kernel instantiations (p = 1..5, fp64 and mixed).
#include "k_tensor_inst.cuh"

namespace frp {
// variant 0: the default tiles; variant 1 (mixed precision only): the
// physical-step kernels with half tiles
bool kernels_hex(int order, int precision, int64_t E, int variant, KernelSet* ks) {
  if (variant < 0 || variant > 1 || (variant == 1 && precision == 0)) return false;
#define FRP_H(P)                                                        \
  case P:                                                               \
    if (precision == 0) fill_tensor<3, P + 1, double>(E, ks);           \
    else if (variant == 0) fill_tensor<3, P + 1, float>(E, ks);         \
    else fill_tensor<3, P + 1, float, 2>(E, ks);                        \
    return true;
  switch (order) {
    FRP_H(1) FRP_H(2) FRP_H(3) FRP_H(4) FRP_H(5)
    default: return false;
  }
#undef FRP_H
}
}  // namespace frp
