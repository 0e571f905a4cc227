// Quadrilateral kernel instantiations (p = 1..6, fp64 and mixed).
#include "k_tensor_inst.cuh"

namespace frp {
// Variants (mixed precision; FP64 has variant 0 only): the tiles of the
// physical-step residual and update kernels, 0 (default, default),
// 1 (half, half), 2 (default, half), 3 (half, default)
bool kernels_quad(int order, int precision, int64_t E, int variant, KernelSet* ks) {
  if (variant < 0 || variant > 3 || (variant > 0 && precision == 0)) return false;
#define FRP_Q(P)                                                          \
  case P:                                                                 \
    if (precision == 0) fill_tensor<2, P + 1, double>(E, ks);             \
    else if (variant == 0) fill_tensor<2, P + 1, float>(E, ks);           \
    else if (variant == 1) fill_tensor<2, P + 1, float, 2, 2>(E, ks);     \
    else if (variant == 2) fill_tensor<2, P + 1, float, 1, 2>(E, ks);     \
    else fill_tensor<2, P + 1, float, 2, 1>(E, ks);                       \
    return true;
  switch (order) {
    FRP_Q(1) FRP_Q(2) FRP_Q(3) FRP_Q(4) FRP_Q(5) FRP_Q(6)
    default: return false;
  }
#undef FRP_Q
}
}  // namespace frp
