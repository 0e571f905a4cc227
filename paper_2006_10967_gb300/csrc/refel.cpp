// Reference-element construction (see refel.hpp).
#include "refel.hpp"

#include <cmath>
#include <cstring>

namespace frp {

// Legendre P_k(x) and P_k'(x) for k = 0..n by the Bonnet recurrence and
// P'_{k+1} = P'_{k-1} + (2k+1) P_k.
static void legendre_all(int n, double x, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n == 0) return;
  P[1] = x;
  dP[1] = 1.0;
  for (int k = 1; k < n; ++k) {
    P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
    dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
  }
}

// Gauss-Legendre nodes by Newton iteration from Chebyshev-like guesses.
static void gauss_legendre(int n, double* x, double* w) {
  double P[kMaxN + 2], dP[kMaxN + 2];
  for (int i = 0; i < n; ++i) {
    double r = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      legendre_all(n, r, P, dP);
      double dr = P[n] / dP[n];
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    legendre_all(n, r, P, dP);
    x[i] = r;
    w[i] = 2.0 / ((1.0 - r * r) * dP[n] * dP[n]);
  }
  // exact symmetry
  for (int i = 0; i < n / 2; ++i) {
    double a = 0.5 * (x[n - 1 - i] - x[i]);
    x[i] = -a;
    x[n - 1 - i] = a;
    double b = 0.5 * (w[i] + w[n - 1 - i]);
    w[i] = w[n - 1 - i] = b;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

static double lagrange(int n, const double* x, int j, double t) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) v *= (t - x[m]) / (x[j] - x[m]);
  return v;
}

bool invert(int n, const double* A, double* Ainv) {
  std::vector<double> M(n * 2 * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      M[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r * 2 * n + c]) > std::fabs(M[piv * 2 * n + c])) piv = r;
    if (std::fabs(M[piv * 2 * n + c]) < 1e-300) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(M[c * 2 * n + j], M[piv * 2 * n + j]);
    double d = M[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * 2 * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
  return true;
}

void build_tensor1d(int p, Tensor1D& t) {
  const int n = p + 1;
  t.n = n;
  gauss_legendre(n, t.x, t.w);
  for (int j = 0; j < n; ++j) {
    t.lend[0][j] = lagrange(n, t.x, j, -1.0);
    t.lend[1][j] = lagrange(n, t.x, j, 1.0);
  }
  // barycentric differentiation matrix
  double b[kMaxN];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) prod *= (t.x[j] - t.x[m]);
    b[j] = 1.0 / prod;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      t.D[i][j] = (b[j] / b[i]) / (t.x[i] - t.x[j]);
      diag -= t.D[i][j];
    }
    t.D[i][i] = diag;
  }
  // g_L = (-1)^{p+1}/2 (P_{p+1} - P_p): g_L(-1) = 1, g_L(1) = 0
  double P[kMaxN + 2], dP[kMaxN + 2];
  const double sgn = (p + 1) % 2 == 0 ? 1.0 : -1.0;
  for (int i = 0; i < n; ++i) {
    legendre_all(p + 1, t.x[i], P, dP);
    t.gLd[i] = sgn * 0.5 * (dP[p + 1] - dP[p]);
  }
  for (int i = 0; i < n; ++i) t.gRd[i] = -t.gLd[n - 1 - i];
  // orthonormal Legendre Vandermonde V[j][m] = sqrt((2m+1)/2) P_m(x_j)
  double V[kMaxN * kMaxN], Vi[kMaxN * kMaxN];
  for (int j = 0; j < n; ++j) {
    legendre_all(p, t.x[j], P, dP);
    for (int m = 0; m < n; ++m) V[j * n + m] = std::sqrt((2.0 * m + 1.0) / 2.0) * P[m];
  }
  invert(n, V, Vi);
  for (int m = 0; m < n; ++m)
    for (int j = 0; j < n; ++j) t.Vinv[m][j] = Vi[m * n + j];
}

// ---------------------------------------------------------------------------
// Triangle: orthonormal Dubiner basis psi_ij(r,s) = sqrt(2) Q_i(a) R_ij(b) (1-b)^i
// with a = 2(1+r)/(1-s) - 1, b = s, Q_i the normalised Legendre and R_ij the
// normalised Jacobi P_j^{(2i+1,0)}.

static double jacobi(int n, double al, double be, double x, double* deriv) {
  // value and derivative by recurrence on (P_{k-1}, P_k) and dP = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}
  auto val = [](int n, double al, double be, double x) {
    double p0 = 1.0;
    if (n == 0) return p0;
    double p1 = 0.5 * (al - be + (al + be + 2.0) * x);
    for (int k = 2; k <= n; ++k) {
      double c1 = 2.0 * k * (k + al + be) * (2.0 * k + al + be - 2.0);
      double c2 = (2.0 * k + al + be - 1.0) * (al * al - be * be);
      double c3 = (2.0 * k + al + be - 2.0) * (2.0 * k + al + be - 1.0) * (2.0 * k + al + be);
      double c4 = 2.0 * (k + al - 1.0) * (k + be - 1.0) * (2.0 * k + al + be);
      double p2 = ((c2 + c3 * x) * p1 - c4 * p0) / c1;
      p0 = p1;
      p1 = p2;
    }
    return p1;
  };
  if (deriv) *deriv = n == 0 ? 0.0 : 0.5 * (n + al + be + 1.0) * val(n - 1, al + 1.0, be + 1.0, x);
  return val(n, al, be, x);
}

static double jacobi_norm(int n, double al, double be) {
  return std::pow(2.0, al + be + 1.0) / (2.0 * n + al + be + 1.0) *
         std::tgamma(n + al + 1.0) * std::tgamma(n + be + 1.0) /
         (std::tgamma(n + al + be + 1.0) * std::tgamma(n + 1.0));
}

// values (and gradients) of all nm = (p+1)(p+2)/2 modes at (r, s), s < 1
static void dubiner(int p, double r, double s, double* P, double* Gr, double* Gs) {
  const double a = 2.0 * (1.0 + r) / (1.0 - s) - 1.0, b = s, om = 1.0 - b;
  int m = 0;
  for (int i = 0; i <= p; ++i) {
    for (int j = 0; j <= p - i; ++j, ++m) {
      double dA, dB;
      const double ni = std::sqrt(jacobi_norm(i, 0.0, 0.0));
      const double nj = std::sqrt(jacobi_norm(j, 2.0 * i + 1.0, 0.0));
      double A = jacobi(i, 0.0, 0.0, a, &dA) / ni;
      dA /= ni;
      double B = jacobi(j, 2.0 * i + 1.0, 0.0, b, &dB) / nj;
      dB /= nj;
      const double omi = std::pow(om, i);
      const double omi1 = i > 0 ? std::pow(om, i - 1) : 0.0;
      P[m] = std::sqrt(2.0) * A * B * omi;
      if (Gr) {
        Gr[m] = i > 0 ? std::sqrt(2.0) * 2.0 * dA * B * omi1 : 0.0;
        double t1 = i > 0 ? dA * (1.0 + a) * B * omi1 : 0.0;
        double t3 = i > 0 ? -i * A * B * omi1 : 0.0;
        Gs[m] = std::sqrt(2.0) * (t1 + A * dB * omi + t3);
      }
    }
  }
}

void build_tri(int p, TriRef& t) {
  const int n = p + 1;
  const int nu = n * (n + 1) / 2, nf = 3 * n;
  t.p = p;
  t.nu = nu;
  t.nf = nf;
  double g[kMaxN], w[kMaxN];
  gauss_legendre(n, g, w);
  // Solution points: the Blyth-Pozrikidis map of 1D nodes v on [0, 1]:
  // lattice index (i, j, k), i + j + k = p, goes to the barycentric point
  // l_a = (1 + 2 v_a - v_b - v_c)/3 (symmetric, interior, positive
  // interpolatory weights).  The nodes are the Gauss-Legendre points for
  // p <= 4 and the Chebyshev points of the second kind for p = 5,
  // cos(m pi / (p + 2)), m = p + 1, ..., 1, whose advection operator has no
  // growing mode where the Gauss-Legendre one does.
  double v1[kMaxN];
  for (int m = 0; m < n; ++m)
    v1[m] = p == 5 ? 0.5 * (std::cos((double)(n - m) * M_PI / (double)(n + 1)) + 1.0) : 0.5 * (g[m] + 1.0);
  t.xu.resize(nu * 2);
  int c = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i <= p - j; ++i, ++c) {
      const int k = p - i - j;
      const double vi = v1[i], vj = v1[j], vk = v1[k];
      const double l1 = (1.0 + 2.0 * vi - vj - vk) / 3.0;
      const double l2 = (1.0 + 2.0 * vj - vi - vk) / 3.0;
      const double l0 = 1.0 - l1 - l2;
      t.xu[2 * c] = l1 - l0 - l2;  // vertices (-1,-1), (1,-1), (-1,1)
      t.xu[2 * c + 1] = l2 - l0 - l1;
    }
  const double V[3][2] = {{-1, -1}, {1, -1}, {-1, 1}};
  const double s2 = std::sqrt(2.0);
  const double nrm[3][2] = {{0, -1}, {1 / s2, 1 / s2}, {-1, 0}};
  const double len[3] = {2.0, 2.0 * s2, 2.0};
  t.xf.resize(nf * 2);
  t.nref.resize(nf * 2);
  std::vector<double> wf(nf);
  for (int e = 0; e < 3; ++e)
    for (int k = 0; k < n; ++k) {
      const int f = e * n + k;
      const double lam = 0.5 * (1.0 + g[k]);
      const int e1 = (e + 1) % 3;
      t.xf[2 * f] = (1.0 - lam) * V[e][0] + lam * V[e1][0];
      t.xf[2 * f + 1] = (1.0 - lam) * V[e][1] + lam * V[e1][1];
      t.nref[2 * f] = nrm[e][0];
      t.nref[2 * f + 1] = nrm[e][1];
      wf[f] = w[k] * 0.5 * len[e];
    }
  std::vector<double> Vm(nu * nu), Vinv(nu * nu), Gr(nu * nu), Gs(nu * nu), Pf(nf * nu);
  for (int i = 0; i < nu; ++i)
    dubiner(p, t.xu[2 * i], t.xu[2 * i + 1], &Vm[i * nu], &Gr[i * nu], &Gs[i * nu]);
  for (int k = 0; k < nf; ++k) dubiner(p, t.xf[2 * k], t.xf[2 * k + 1], &Pf[k * nu], nullptr, nullptr);
  invert(nu, Vm.data(), Vinv.data());
  t.Vinv = Vinv;
  t.L.assign(nf * nu, 0.0);
  for (int k = 0; k < nf; ++k)
    for (int i = 0; i < nu; ++i) {
      double acc = 0.0;
      for (int m = 0; m < nu; ++m) acc += Pf[k * nu + m] * Vinv[m * nu + i];
      t.L[k * nu + i] = acc;
    }
  t.Dr.assign(nu * nu, 0.0);
  t.Ds.assign(nu * nu, 0.0);
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j) {
      double ar = 0.0, as = 0.0;
      for (int m = 0; m < nu; ++m) {
        ar += Gr[i * nu + m] * Vinv[m * nu + j];
        as += Gs[i * nu + m] * Vinv[m * nu + j];
      }
      t.Dr[i * nu + j] = ar;
      t.Ds[i * nu + j] = as;
    }
  // LIFT = (V V^T) E, E[i][k] = wf[k] l_i(x^f_k)
  std::vector<double> VVt(nu * nu, 0.0);
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j) {
      double acc = 0.0;
      for (int m = 0; m < nu; ++m) acc += Vm[i * nu + m] * Vm[j * nu + m];
      VVt[i * nu + j] = acc;
    }
  t.LIFT.assign(nu * nf, 0.0);
  for (int i = 0; i < nu; ++i)
    for (int k = 0; k < nf; ++k) {
      double acc = 0.0;
      for (int j = 0; j < nu; ++j) acc += VVt[i * nu + j] * wf[k] * t.L[k * nu + j];
      t.LIFT[i * nf + k] = acc;
    }
  t.high.assign(nu, 0);
  int m = 0;
  for (int i = 0; i <= p; ++i)
    for (int j = 0; j <= p - i; ++j, ++m) t.high[m] = (i + j == p) ? 1 : 0;
  // int psi_0 = sqrt(2) (psi_0 = 1/sqrt(2) on an area-2 triangle)
  t.wq.resize(nu);
  for (int i = 0; i < nu; ++i) t.wq[i] = Vinv[0 * nu + i] * std::sqrt(2.0);
}

}  // namespace frp
