// Element mapping x = M(xi) and its Jacobian (Section 3.1, Eqs. maintranseq,
// maintranseq2), shared by the host mesh builder and the device kernels.
//
// Straight-sided elements; per element and physical component the map is a
// polynomial in the reference coordinates with coefficients c_k:
//   quad (bilinear):  1, xi, eta, xi*eta
//   tri  (affine):    1, xi, eta
//   hex  (trilinear): 1, xi, eta, zeta, xi*eta, xi*zeta, eta*zeta, xi*eta*zeta
// stored element-major as geo[e][comp][k].
#pragma once

#ifdef __CUDACC__
#define FRP_HD __host__ __device__ __forceinline__
#else
#define FRP_HD inline
#endif

namespace frp {

enum { ET_QUAD = 0, ET_TRI = 1, ET_HEX = 2 };

template <int ET> struct Geo;
template <> struct Geo<ET_QUAD> { static constexpr int DIM = 2, NC = 4, NV = 4; };
template <> struct Geo<ET_TRI> { static constexpr int DIM = 2, NC = 3, NV = 3; };
template <> struct Geo<ET_HEX> { static constexpr int DIM = 3, NC = 8, NV = 8; };

template <int ET, typename R>
FRP_HD void map_point(const R* g, const R* xi, R* x) {
  constexpr int NC = Geo<ET>::NC, DIM = Geo<ET>::DIM;
  for (int c = 0; c < DIM; ++c) {
    const R* k = g + c * NC;
    if (ET == ET_QUAD) x[c] = k[0] + k[1] * xi[0] + k[2] * xi[1] + k[3] * xi[0] * xi[1];
    else if (ET == ET_TRI) x[c] = k[0] + k[1] * xi[0] + k[2] * xi[1];
    else
      x[c] = k[0] + k[1] * xi[0] + k[2] * xi[1] + k[3] * xi[2] + k[4] * xi[0] * xi[1] +
             k[5] * xi[0] * xi[2] + k[6] * xi[1] * xi[2] + k[7] * xi[0] * xi[1] * xi[2];
  }
}

// J[i][a] = d x_i / d xi_a
template <int ET, typename R>
FRP_HD void jacobian(const R* g, const R* xi, R J[3][3]) {
  constexpr int NC = Geo<ET>::NC, DIM = Geo<ET>::DIM;
  for (int c = 0; c < DIM; ++c) {
    const R* k = g + c * NC;
    if (ET == ET_QUAD) {
      J[c][0] = k[1] + k[3] * xi[1];
      J[c][1] = k[2] + k[3] * xi[0];
    } else if (ET == ET_TRI) {
      J[c][0] = k[1];
      J[c][1] = k[2];
    } else {
      J[c][0] = k[1] + k[4] * xi[1] + k[5] * xi[2] + k[7] * xi[1] * xi[2];
      J[c][1] = k[2] + k[4] * xi[0] + k[6] * xi[2] + k[7] * xi[0] * xi[2];
      J[c][2] = k[3] + k[5] * xi[0] + k[6] * xi[1] + k[7] * xi[0] * xi[1];
    }
  }
}

// S = det J * J^{-1} (the adjugate), S[a][i] = det J * d xi_a / d x_i; returns det J.
template <int DIM, typename R>
FRP_HD R adjugate(const R J[3][3], R S[3][3]) {
  if (DIM == 2) {
    S[0][0] = J[1][1];
    S[0][1] = -J[0][1];
    S[1][0] = -J[1][0];
    S[1][1] = J[0][0];
    return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
    S[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    S[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    S[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    S[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    S[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    S[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    S[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    S[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    S[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * S[0][0] + J[0][1] * S[1][0] + J[0][2] * S[2][0];
  }
}

}  // namespace frp
