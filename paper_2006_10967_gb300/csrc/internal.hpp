// Internal host-side types of libfrpcpf (not part of the C ABI).
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/fr_pcpf.h"
#include "refel.hpp"

struct fr_mesh {
  int dim = 0, etype = 0, order = 0;
  int n = 0;        // p + 1
  int nu = 0, nf = 0, nfaces = 0, nfp = 0, nverts = 0, ncoef = 0;
  int64_t E = 0;
  std::vector<double> geo;     // E * dim * ncoef map coefficients
  std::vector<int32_t> fnbr;   // E * nf: (partner global flux point << 1) | isL
  std::vector<double> xu;      // E * nu * dim physical solution points
  std::vector<double> wdet;    // E * nu: w_i det J_ei
  frp::Tensor1D t1;            // quad/hex operators
  frp::TriRef tri;             // tri operators
  double h = 0.0, volume = 0.0;
  int64_t n_boundary = 0;
};
