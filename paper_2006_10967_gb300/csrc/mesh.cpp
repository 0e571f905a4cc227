// Host mesh builder of libfrpcpf: reference operators, element geometry and
// face pairing.  Section 3.1: the element mapping and its Jacobian; flux
// points that coincide physically with the neighbour's flux points.
// Section 3.3: unmatched faces are walls with copy ghost states.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>

#include "geom.cuh"
#include "internal.hpp"

using namespace frp;

namespace {

const double kQuadV[4][3] = {{-1, -1, 0}, {1, -1, 0}, {1, 1, 0}, {-1, 1, 0}};
const double kHexV[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                            {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
const double kTriV[3][3] = {{-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

const double* ref_vertex(int etype, int v) {
  return etype == FR_QUAD ? kQuadV[v] : etype == FR_HEX ? kHexV[v] : kTriV[v];
}

// reference coordinates of solution point i / flux point k
void upt_ref(const fr_mesh& m, int i, double* xi) {
  if (m.etype == FR_TRI) {
    xi[0] = m.tri.xu[2 * i];
    xi[1] = m.tri.xu[2 * i + 1];
    return;
  }
  int r = i;
  for (int a = 0; a < m.dim; ++a) {
    xi[a] = m.t1.x[r % m.n];
    r /= m.n;
  }
}

void fpt_ref(const fr_mesh& m, int k, double* xi) {
  if (m.etype == FR_TRI) {
    xi[0] = m.tri.xf[2 * k];
    xi[1] = m.tri.xf[2 * k + 1];
    return;
  }
  const int f = k / m.nfp, a = f / 2, s = f % 2;
  int r = k % m.nfp;
  for (int b = 0; b < m.dim; ++b) {
    if (b == a) {
      xi[b] = s ? 1.0 : -1.0;
    } else {
      xi[b] = m.t1.x[r % m.n];
      r /= m.n;
    }
  }
}

// reference normal of flux point k
void fpt_normal(const fr_mesh& m, int k, double* nr) {
  if (m.etype == FR_TRI) {
    nr[0] = m.tri.nref[2 * k];
    nr[1] = m.tri.nref[2 * k + 1];
    return;
  }
  const int f = k / m.nfp, a = f / 2, s = f % 2;
  for (int b = 0; b < m.dim; ++b) nr[b] = b == a ? (s ? 1.0 : -1.0) : 0.0;
}

void face_vertices(const fr_mesh& m, int f, std::vector<int>& out) {
  out.clear();
  if (m.etype == FR_TRI) {
    out.push_back(f);
    out.push_back((f + 1) % 3);
    return;
  }
  const int a = f / 2;
  const double v = (f % 2) ? 1.0 : -1.0;
  for (int q = 0; q < m.nverts; ++q)
    if (ref_vertex(m.etype, q)[a] == v) out.push_back(q);
}

template <int ET>
void geo_coeffs(const double* X /*nv x dim*/, int dim, double* c /*dim x NC*/) {
  constexpr int NC = Geo<ET>::NC;
  if (ET == ET_TRI) {
    for (int d = 0; d < dim; ++d) {
      const double c1 = 0.5 * (X[1 * dim + d] - X[0 * dim + d]);
      const double c2 = 0.5 * (X[2 * dim + d] - X[0 * dim + d]);
      c[d * NC + 0] = X[0 * dim + d] + c1 + c2;
      c[d * NC + 1] = c1;
      c[d * NC + 2] = c2;
    }
    return;
  }
  const int nv = Geo<ET>::NV;
  for (int d = 0; d < dim; ++d)
    for (int k = 0; k < NC; ++k) c[d * NC + k] = 0.0;
  for (int v = 0; v < nv; ++v) {
    const double* r = ref_vertex(ET == ET_QUAD ? FR_QUAD : FR_HEX, v);
    double B[8];
    if (ET == ET_QUAD) {
      B[0] = 1; B[1] = r[0]; B[2] = r[1]; B[3] = r[0] * r[1];
    } else {
      B[0] = 1; B[1] = r[0]; B[2] = r[1]; B[3] = r[2];
      B[4] = r[0] * r[1]; B[5] = r[0] * r[2]; B[6] = r[1] * r[2]; B[7] = r[0] * r[1] * r[2];
    }
    for (int d = 0; d < dim; ++d)
      for (int k = 0; k < NC; ++k) c[d * NC + k] += B[k] * X[v * dim + d] / nv;
  }
  // Round-off of the sums above leaves ~1e-17 h in coefficients that are
  // zero for the element's shape (the cross terms of a parallelogram or
  // parallelepiped, the off-diagonal terms of an axis-aligned box) when the
  // node coordinates are not dyadic; set coefficients below 1e-13 of the
  // element's largest linear coefficient to zero, so that such elements are
  // recognised as affine (one metric per element) and axis-aligned.
  double scale = 0.0;
  for (int d = 0; d < dim; ++d)
    for (int k = 1; k <= dim; ++k) scale = std::max(scale, std::fabs(c[d * NC + k]));
  for (int d = 0; d < dim; ++d)
    for (int k = 1; k < NC; ++k)
      if (std::fabs(c[d * NC + k]) < 1e-13 * scale) c[d * NC + k] = 0.0;
}

void point_and_jac(const fr_mesh& m, int64_t e, const double* xi, double* x, double J[3][3]) {
  const double* g = &m.geo[e * m.dim * m.ncoef];
  if (m.etype == FR_QUAD) { map_point<ET_QUAD>(g, xi, x); jacobian<ET_QUAD>(g, xi, J); }
  else if (m.etype == FR_TRI) { map_point<ET_TRI>(g, xi, x); jacobian<ET_TRI>(g, xi, J); }
  else { map_point<ET_HEX>(g, xi, x); jacobian<ET_HEX>(g, xi, J); }
}

struct FaceKey {
  std::array<int64_t, 15> k;  // sorted vertex keys, then the centroid key
  int64_t e;
  int f;
};

int build(const fr_mesh_desc* d, fr_mesh& m) {
  const int dim = d->dim, et = d->etype, p = d->order;
  if (!((et == FR_QUAD && dim == 2) || (et == FR_TRI && dim == 2) || (et == FR_HEX && dim == 3)))
    return FR_EINVAL;
  if (p < 1) return FR_EINVAL;
  if ((et == FR_QUAD && p > 6) || (et == FR_HEX && p > 5) || (et == FR_TRI && p > 5))
    return FR_EUNSUPPORTED;
  if (d->n_nodes <= 0 || d->n_elems <= 0 || !d->nodes || !d->conn) return FR_EINVAL;
  m.dim = dim;
  m.etype = et;
  m.order = p;
  m.n = p + 1;
  m.E = d->n_elems;
  if (et == FR_TRI) {
    build_tri(p, m.tri);
    m.nu = m.tri.nu;
    m.nf = m.tri.nf;
    m.nfaces = 3;
    m.nfp = m.n;
    m.nverts = 3;
    m.ncoef = 3;
  } else {
    build_tensor1d(p, m.t1);
    m.nu = dim == 2 ? m.n * m.n : m.n * m.n * m.n;
    m.nfp = dim == 2 ? m.n : m.n * m.n;
    m.nfaces = 2 * dim;
    m.nf = m.nfaces * m.nfp;
    m.nverts = dim == 2 ? 4 : 8;
    m.ncoef = dim == 2 ? 4 : 8;
  }
  if ((int64_t)m.E * m.nf >= (int64_t(1) << 30)) return FR_EUNSUPPORTED;
  for (int64_t i = 0; i < m.E * m.nverts; ++i)
    if (d->conn[i] < 0 || d->conn[i] >= d->n_nodes) return FR_EINVAL;
  for (int64_t i = 0; i < d->n_nodes * dim; ++i)
    if (!std::isfinite(d->nodes[i])) return FR_EINVAL;
  for (int a = 0; a < dim; ++a)
    if (d->periodic[a] && !(d->period[a] > 0.0)) return FR_EINVAL;

  // geometry coefficients
  m.geo.resize(m.E * dim * m.ncoef);
  std::vector<double> X(m.nverts * dim);
  for (int64_t e = 0; e < m.E; ++e) {
    for (int v = 0; v < m.nverts; ++v)
      for (int c = 0; c < dim; ++c) X[v * dim + c] = d->nodes[d->conn[e * m.nverts + v] * dim + c];
    double* g = &m.geo[e * dim * m.ncoef];
    if (et == FR_QUAD) geo_coeffs<ET_QUAD>(X.data(), dim, g);
    else if (et == FR_TRI) geo_coeffs<ET_TRI>(X.data(), dim, g);
    else geo_coeffs<ET_HEX>(X.data(), dim, g);
  }
  // solution points, weights, det J > 0 at solution and flux points
  std::vector<double> wref(m.nu);
  for (int i = 0; i < m.nu; ++i) {
    if (et == FR_TRI) wref[i] = m.tri.wq[i];
    else {
      double w = 1.0;
      int r = i;
      for (int a = 0; a < dim; ++a) { w *= m.t1.w[r % m.n]; r /= m.n; }
      wref[i] = w;
    }
  }
  m.xu.resize(m.E * m.nu * dim);
  m.wdet.resize(m.E * m.nu);
  double vol = 0.0;
  for (int64_t e = 0; e < m.E; ++e) {
    for (int i = 0; i < m.nu; ++i) {
      double xi[3] = {0, 0, 0}, x[3], J[3][3], S[3][3];
      upt_ref(m, i, xi);
      point_and_jac(m, e, xi, x, J);
      const double dj = dim == 2 ? adjugate<2>(J, S) : adjugate<3>(J, S);
      if (!(dj > 0.0)) return FR_EINVAL;
      for (int c = 0; c < dim; ++c) m.xu[(e * m.nu + i) * dim + c] = x[c];
      m.wdet[e * m.nu + i] = wref[i] * dj;
      vol += wref[i] * dj;
    }
    for (int k = 0; k < m.nf; ++k) {
      double xi[3] = {0, 0, 0}, x[3], J[3][3], S[3][3];
      fpt_ref(m, k, xi);
      point_and_jac(m, e, xi, x, J);
      const double dj = dim == 2 ? adjugate<2>(J, S) : adjugate<3>(J, S);
      if (!(dj > 0.0)) return FR_EINVAL;
    }
  }
  m.volume = vol;
  m.h = et == FR_TRI ? std::sqrt(2.0 * vol / m.E) : std::pow(vol / m.E, 1.0 / dim);

  // ---- faces: sorted, wrapped, quantised vertex coordinates
  // on a periodic axis the quantum is rounded to divide the period (inv[a]
  // = P[a] / period), so a vertex and its periodic image share a key
  const double quantum = 1e-7 * m.h;
  int64_t P[3] = {0, 0, 0};
  double inv[3] = {1.0 / quantum, 1.0 / quantum, 1.0 / quantum};
  for (int a = 0; a < dim; ++a)
    if (d->periodic[a]) {
      P[a] = std::llround(d->period[a] / quantum);
      inv[a] = (double)P[a] / d->period[a];
    }
  std::vector<FaceKey> keys;
  keys.reserve(m.E * m.nfaces);
  std::vector<int> fv;
  for (int64_t e = 0; e < m.E; ++e)
    for (int f = 0; f < m.nfaces; ++f) {
      face_vertices(m, f, fv);
      std::vector<std::array<int64_t, 3>> vk(fv.size());
      for (size_t q = 0; q < fv.size(); ++q) {
        const double* x = &d->nodes[d->conn[e * m.nverts + fv[q]] * dim];
        for (int a = 0; a < 3; ++a) {
          int64_t v = a < dim ? std::llround(x[a] * inv[a]) : 0;
          if (a < dim && P[a] > 0) v = ((v % P[a]) + P[a]) % P[a];
          vk[q][a] = v;
        }
      }
      std::sort(vk.begin(), vk.end());
      FaceKey fk;
      fk.k.fill(INT64_MIN);
      for (size_t q = 0; q < vk.size(); ++q)
        for (int a = 0; a < 3; ++a) fk.k[q * 3 + a] = vk[q][a];
      // the wrapped centroid separates faces whose vertices all coincide
      // modulo the period (an element that is its own periodic neighbour)
      for (int a = 0; a < dim; ++a) {
        double c = 0.0;
        for (size_t q = 0; q < fv.size(); ++q) c += d->nodes[d->conn[e * m.nverts + fv[q]] * dim + a];
        int64_t v = std::llround(c / fv.size() * inv[a]);
        if (P[a] > 0) v = ((v % P[a]) + P[a]) % P[a];
        fk.k[12 + a] = v;
      }
      fk.e = e;
      fk.f = f;
      keys.push_back(fk);
    }
  std::sort(keys.begin(), keys.end(), [](const FaceKey& a, const FaceKey& b) {
    if (a.k != b.k) return a.k < b.k;
    if (a.e != b.e) return a.e < b.e;
    return a.f < b.f;
  });

  // default: every flux point is its own partner and an L point (wall)
  m.fnbr.resize(m.E * m.nf);
  for (int64_t g = 0; g < m.E * m.nf; ++g) m.fnbr[g] = (int32_t)((g << 1) | 1);
  std::vector<char> matched(m.E * m.nfaces, 0);

  std::vector<double> x1(m.nfp * 3), x2(m.nfp * 3);
  auto face_points = [&](int64_t e, int f, std::vector<double>& out) {
    for (int q = 0; q < m.nfp; ++q) {
      double xi[3] = {0, 0, 0}, J[3][3];
      fpt_ref(m, f * m.nfp + q, xi);
      point_and_jac(m, e, xi, &out[q * 3], J);
    }
  };
  auto centroid_sum = [&](int64_t e, int f) {
    face_vertices(m, f, fv);
    double s = 0.0;
    for (int q : fv)
      for (int a = 0; a < dim; ++a) s += d->nodes[d->conn[e * m.nverts + q] * dim + a];
    return s / fv.size();
  };
  size_t i = 0;
  while (i < keys.size()) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].k == keys[i].k) ++j;
    if (j - i > 2) return FR_EINVAL;
    if (j - i == 2) {
      const int64_t e1 = keys[i].e, e2 = keys[i + 1].e;
      const int f1 = keys[i].f, f2 = keys[i + 1].f;
      face_points(e1, f1, x1);
      face_points(e2, f2, x2);
      bool first_L = e1 != e2 ? (e1 < e2) : (centroid_sum(e1, f1) > centroid_sum(e2, f2));
      for (int q = 0; q < m.nfp; ++q) {
        int best = -1;
        double bd = 1e300;
        for (int r = 0; r < m.nfp; ++r) {
          double dd = 0.0;
          for (int a = 0; a < dim; ++a) {
            double dx = x1[q * 3 + a] - x2[r * 3 + a];
            if (d->periodic[a]) dx -= d->period[a] * std::nearbyint(dx / d->period[a]);
            dd += dx * dx;
          }
          if (dd < bd) { bd = dd; best = r; }
        }
        if (std::sqrt(bd) > 1e-6 * m.h) return FR_EINVAL;
        const int64_t g1 = e1 * m.nf + f1 * m.nfp + q;
        const int64_t g2 = e2 * m.nf + f2 * m.nfp + best;
        m.fnbr[g1] = (int32_t)((g2 << 1) | (first_L ? 1 : 0));
        m.fnbr[g2] = (int32_t)((g1 << 1) | (first_L ? 0 : 1));
      }
      matched[e1 * m.nfaces + f1] = matched[e2 * m.nfaces + f2] = 1;
    }
    i = j;
  }
  m.n_boundary = 0;
  for (int64_t k = 0; k < m.E * m.nfaces; ++k)
    if (!matched[k]) m.n_boundary += m.nfp;
  return FR_OK;
}

}  // namespace

extern "C" int fr_mesh_create(const fr_mesh_desc* desc, fr_mesh** out) {
  if (!desc || !out) return FR_EINVAL;
  *out = nullptr;
  fr_mesh* m = new (std::nothrow) fr_mesh();
  if (!m) return FR_ENOMEM;
  int rc;
  try {
    rc = build(desc, *m);
  } catch (const std::bad_alloc&) {
    rc = FR_ENOMEM;
  } catch (...) {
    rc = FR_EINVAL;
  }
  if (rc != FR_OK) {
    delete m;
    return rc;
  }
  *out = m;
  return FR_OK;
}

extern "C" int fr_mesh_info_get(const fr_mesh* m, fr_mesh_info* info) {
  if (!m || !info) return FR_EINVAL;
  info->dim = m->dim;
  info->etype = m->etype;
  info->order = m->order;
  info->nu = m->nu;
  info->nf = m->nf;
  info->n_faces_per_elem = m->nfaces;
  info->n_elems = m->E;
  info->n_dof = m->E * m->nu;
  info->n_boundary_fpts = m->n_boundary;
  info->h = m->h;
  info->volume = m->volume;
  return FR_OK;
}

extern "C" int fr_mesh_solution_points(const fr_mesh* m, double* out) {
  if (!m || !out) return FR_EINVAL;
  std::memcpy(out, m->xu.data(), m->xu.size() * sizeof(double));
  return FR_OK;
}

extern "C" int fr_mesh_quadrature(const fr_mesh* m, double* out) {
  if (!m || !out) return FR_EINVAL;
  std::memcpy(out, m->wdet.data(), m->wdet.size() * sizeof(double));
  return FR_OK;
}

extern "C" int fr_mesh_concat(const fr_mesh* const* meshes, int n, fr_mesh** out) {
  if (!meshes || n < 1 || !out) return FR_EINVAL;
  *out = nullptr;
  const fr_mesh* m0 = meshes[0];
  if (!m0) return FR_EINVAL;
  int64_t E = 0;
  for (int i = 0; i < n; ++i) {
    const fr_mesh* mi = meshes[i];
    if (!mi || mi->etype != m0->etype || mi->order != m0->order || mi->dim != m0->dim) return FR_EINVAL;
    E += mi->E;
  }
  if (E * m0->nf >= (int64_t(1) << 30)) return FR_EUNSUPPORTED;
  fr_mesh* u = new (std::nothrow) fr_mesh();
  if (!u) return FR_ENOMEM;
  try {
    *u = *m0;
    u->E = E;
    u->geo.clear();
    u->fnbr.clear();
    u->xu.clear();
    u->wdet.clear();
    u->volume = 0.0;
    u->n_boundary = 0;
    double hsum = 0.0;
    int64_t off = 0;
    for (int i = 0; i < n; ++i) {
      const fr_mesh* mi = meshes[i];
      u->geo.insert(u->geo.end(), mi->geo.begin(), mi->geo.end());
      u->xu.insert(u->xu.end(), mi->xu.begin(), mi->xu.end());
      u->wdet.insert(u->wdet.end(), mi->wdet.begin(), mi->wdet.end());
      for (int32_t w : mi->fnbr) {
        const int64_t g = (int64_t)(w >> 1) + off * mi->nf;
        u->fnbr.push_back((int32_t)((g << 1) | (w & 1)));
      }
      u->volume += mi->volume;
      u->n_boundary += mi->n_boundary;
      hsum += mi->h * mi->E;
      off += mi->E;
    }
    u->h = hsum / E;
  } catch (const std::bad_alloc&) {
    delete u;
    return FR_ENOMEM;
  }
  *out = u;
  return FR_OK;
}

extern "C" void fr_mesh_destroy(fr_mesh* m) { delete m; }
