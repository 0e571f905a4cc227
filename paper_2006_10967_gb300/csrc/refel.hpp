// Reference-element data for the FR operators (host side, double precision).
//
// Section 3.1: Gauss-Legendre solution points on tensor elements, flux points
// coinciding with solution-point lines, the nodal basis l_i built from an
// orthonormal modal basis through the Vandermonde matrix, and the
// DG-recovering correction functions (Huynh's Radau g_L, g_R on lines; the
// DG lift on triangles).  Section 3.2: the orthonormal modal coefficients
// chi = V^{-1} u used by the resolution indicator.
#pragma once
#include <cstdint>
#include <vector>

namespace frp {

constexpr int kMaxN = 7;  // p <= 6

struct Tensor1D {
  int n = 0;                 // points per line (p + 1)
  double x[kMaxN], w[kMaxN]; // Gauss-Legendre points and weights
  double lend[2][kMaxN];     // l_j(-1), l_j(+1)
  double D[kMaxN][kMaxN];    // D[i][j] = l_j'(x_i)
  double gLd[kMaxN];         // g_L'(x_i), left Radau correction derivative
  double gRd[kMaxN];         // g_R'(x_i) = -g_L'(-x_i)
  double Vinv[kMaxN][kMaxN]; // chi_m = sum_j Vinv[m][j] u_j (orthonormal Legendre)
};

// Triangle with reference vertices (-1,-1), (1,-1), (-1,1); edge e runs from
// vertex e to vertex (e+1)%3 with n Gauss-Legendre flux points.
struct TriRef {
  int p = 0, nu = 0, nf = 0;
  std::vector<double> xu;    // nu x 2
  std::vector<double> xf;    // nf x 2
  std::vector<double> nref;  // nf x 2 unit outward normals
  std::vector<double> L;     // nf x nu:  l_i(x^f_k)
  std::vector<double> Dr, Ds;// nu x nu: d l_j/d r (x_i), d l_j/d s (x_i)
  std::vector<double> LIFT;  // nu x nf: (div g_k)(x_i)
  std::vector<double> Vinv;  // nu x nu
  std::vector<uint8_t> high; // nu: mode has total degree p
  std::vector<double> wq;    // nu: int l_i
};

void build_tensor1d(int p, Tensor1D& t);
void build_tri(int p, TriRef& t);

// Small dense helpers
bool invert(int n, const double* A, double* Ainv);

}  // namespace frp
