// Quadrilateral kernel instantiations (p = 1..6, fp64 and mixed).
#include "k_tensor_inst.cuh"

namespace frp {
// variant 0: the default tiles; variant 1 (mixed precision only): the
// physical-step kernels with half tiles
bool kernels_quad(int order, int precision, int64_t E, int variant, KernelSet* ks) {
  if (variant < 0 || variant > 1 || (variant == 1 && precision == 0)) return false;
#define FRP_Q(P)                                                        \
  case P:                                                               \
    if (precision == 0) fill_tensor<2, P + 1, double>(E, ks);           \
    else if (variant == 0) fill_tensor<2, P + 1, float>(E, ks);         \
    else fill_tensor<2, P + 1, float, 2>(E, ks);                        \
    return true;
  switch (order) {
    FRP_Q(1) FRP_Q(2) FRP_Q(3) FRP_Q(4) FRP_Q(5) FRP_Q(6)
    default: return false;
  }
#undef FRP_Q
}
}  // namespace frp
