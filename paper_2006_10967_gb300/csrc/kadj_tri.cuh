// Hand-written discrete adjoint (vector-Jacobian product) of the FR residual
// of the physical system on straight-sided triangles: the transpose, step by
// step in reverse order, of kb_tri / ka_tri (Steps 1-6 of Section 3.1 with
// the dense reference operators L, D_r, D_s, LIFT and one affine metric per
// element).  The same three kernels as the tensor-element adjoint
// (kadj.cuh), with the same arguments:
//   adj_a_tri : lam_div = -lam / det J and Y = LIFT^T lam_div at every flux
//               point (the adjoint of the lifted flux jumps)
//   adj_b_tri : forward recomputation of the element (traces, gradient,
//               fluxes), the reverse of Steps 6, 4, 5, 3 and 1; the adjoint
//               of the common flux out of L takes this side's Y times its
//               face scale and the partner's Y times the partner's face scale
//               (the two sides of an edge see different reference edges)
//   adj_c_tri : gathers the partners' lamuo, adds L^T of it, and applies the
//               RK4 adjoint recurrence.
// FP64 only; the velocity is evaluated analytically, as in the forward
// triangle kernels.  adj_b_tri<P, 1> is the preconditioning system's
// (Eq. pseudotimesystem), as adj_b<.., 1> of kadj.cuh: the flux -nu_s q, the
// penalty, the source tanh(psi0 / |q|)(1 - |q|) and the element viscosity's
// dependence on psi through the resolution indicator.
#pragma once
#include "kadj.cuh"
#include "ktri.cuh"

namespace frp {

template <int P>
struct AdjTriLayout {
  using S = TriS<P>;
  // per element (doubles): U / lam_U, q, lam_f~ -> lam_q -> lam_q~, lam_div,
  // uf, uo, luf, luo, lam_qf, geometry, metric
  static constexpr int PER_EL = 2 * S::NU + 4 * S::NU + 4 * S::NU + 2 * S::NU + 8 * S::NF + 4 * S::NF + S::NG + 5;
  static constexpr int BYTES_EL = PER_EL * 8 + S::NF;
  static constexpr int ETr = 40960 / BYTES_EL;
  static constexpr int ET = ETr < 1 ? 1 : (ETr > 64 ? 64 : ETr);
  static constexpr int THREADS = 256;
  static constexpr size_t SMEM = (size_t)ET * BYTES_EL + sizeof(TriOpsS<P, double>) + 64;
};

// the transformed normal of flux point k of an element with metric m: pn =
// S^T n~, |pn|, n = pn / |pn|
__device__ __forceinline__ double tri_normal(const double* mt, const double* nref, double* nh) {
  const double p0 = mt[0] * nref[0] + mt[2] * nref[1];
  const double p1 = mt[1] * nref[0] + mt[3] * nref[1];
  const double pm = sqrt(p0 * p0 + p1 * p1);
  nh[0] = p0 / pm;
  nh[1] = p1 / pm;
  return pm;
}

template <int P>
__global__ void __launch_bounds__(256) adj_a_tri(const AdjArgs B) {
  using S = TriS<P>;
  using LY = AdjTriLayout<P>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, ET = LY::ET;
  const KArgs& A = B.K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TriOpsS<P, double>& op = *reinterpret_cast<TriOpsS<P, double>*>(smem_raw);
  double* ld = reinterpret_cast<double*>(smem_raw + ((sizeof(TriOpsS<P, double>) + 15) & ~size_t(15)));  // [ET][2][NU]
  __shared__ double djs[ET];
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const int tid = threadIdx.x;
  load_tri_ops<P, double>(A.trid, op);
  for (int el = tid; el < ne; el += blockDim.x) {
    TriMet<double> m;
    tri_metric(A.geo + (e0 + el) * NG, m);
    djs[el] = m.dj;
  }
  __syncthreads();
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x)
    ld[idx] = -B.lam_scale * B.lamk[e0 * 2 * NU + idx] / djs[idx / (2 * NU)];
  __syncthreads();
  for (int idx = tid; idx < ne * 2 * NF; idx += blockDim.x) {
    const int c = idx / NF, k = idx % NF;
    double y = 0.0;
    for (int i = 0; i < NU; ++i) y += op.LIFT[i][k] * ld[c * NU + i];
    B.Y[e0 * 2 * NF + idx] = y;
  }
}

template <int P, int MODE = 0>
__global__ void __launch_bounds__(256) adj_b_tri(const AdjArgs B) {
  using S = TriS<P>;
  using LY = AdjTriLayout<P>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, ET = LY::ET;
  const KArgs& A = B.K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TriOpsS<P, double>& op = *reinterpret_cast<TriOpsS<P, double>*>(smem_raw);
  double* us = reinterpret_cast<double*>(smem_raw + ((sizeof(TriOpsS<P, double>) + 15) & ~size_t(15)));
  double* q = us + ET * 2 * NU;        // [ET][2][2][NU] physical gradient
  double* lf = q + ET * 4 * NU;        // [ET][2][2][NU] lam_f~ -> lam_q -> lam_q~
  double* ld = lf + ET * 4 * NU;       // [ET][2][NU]
  double* uf = ld + ET * 2 * NU;       // [ET][2][NF]
  double* uo = uf + ET * 2 * NF;
  double* luf = uo + ET * 2 * NF;
  double* luo = luf + ET * 2 * NF;
  double* lqf = luo + ET * 2 * NF;     // [ET][2][2][NF]
  double* gs = lqf + ET * 4 * NF;      // [ET][NG]
  double* met = gs + ET * NG;          // [ET][5]: S00 S01 S10 S11 det J
  unsigned char* lm = reinterpret_cast<unsigned char*>(met + ET * 5);

  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const int tid = threadIdx.x;
  const double* ustg = reinterpret_cast<const double*>(A.ustg);
  const double* tr = reinterpret_cast<const double*>(A.tr);
  const BulkConst<double>& BC = A.cd;
  const PrmT<double> Pm = BC.prm;
  const double g = time_factor(A, A.t);
  const bool coef = MODE == 0 && B.want_coef && BC.vel.kind == 3;
  __shared__ double nu_e[ET], dnu_e[ET], lnu_e[ET];  // MODE 1: nu_s, d nu_s / d s, lam of nu_s
  load_tri_ops<P, double>(A.trid, op);
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) us[idx] = ustg[e0 * 2 * NU + idx];
  for (int idx = tid; idx < ne * NG; idx += blockDim.x) gs[idx] = A.geo[e0 * NG + idx];
  __syncthreads();
  for (int el = tid; el < ne; el += blockDim.x) {
    TriMet<double> m;
    tri_metric(gs + el * NG, m);
    met[el * 5 + 0] = m.S[0][0];
    met[el * 5 + 1] = m.S[0][1];
    met[el * 5 + 2] = m.S[1][0];
    met[el * 5 + 3] = m.S[1][1];
    met[el * 5 + 4] = m.dj;
  }
  // ---- forward: traces and partner traces (Steps 1-2)
  for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
    const int el = idx / NF, k = idx % NF;
    const int32_t own = (int32_t)((e0 + el) * NF + k);
    const int32_t w = A.fnbr[own];
    const int64_t pg = (int64_t)partner<NF>(A, w, own);
    lm[el * NF + k] = (unsigned char)(w & 1);
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      double acc = 0.0;
      for (int j = 0; j < NU; ++j) acc += op.L[k][j] * us[(el * 2 + fld) * NU + j];
      uf[(el * 2 + fld) * NF + k] = acc;
      uo[(el * 2 + fld) * NF + k] = (w & 1) ? tr[((pg / NF) * 2 + fld) * NF + pg % NF] : acc;
    }
  }
  __syncthreads();
  // ---- forward: corrected gradient (Step 3) and lam_div
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    const double* mt = met + el * 5;
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      double q0 = 0, q1 = 0;
      for (int j = 0; j < NU; ++j) {
        q0 += op.Dr[i][j] * us[(el * 2 + fld) * NU + j];
        q1 += op.Ds[i][j] * us[(el * 2 + fld) * NU + j];
      }
      for (int k = 0; k < NF; ++k) {
        const double jmp = lm[el * NF + k] ? uo[(el * 2 + fld) * NF + k] - uf[(el * 2 + fld) * NF + k] : 0.0;
        const double lj = op.LIFT[i][k] * jmp;
        q0 += lj * op.nref[k][0];
        q1 += lj * op.nref[k][1];
      }
      q[((el * 2 + fld) * 2 + 0) * NU + i] = (mt[0] * q0 + mt[2] * q1) / mt[4];
      q[((el * 2 + fld) * 2 + 1) * NU + i] = (mt[1] * q0 + mt[3] * q1) / mt[4];
      ld[(el * 2 + fld) * NU + i] = -B.lam_scale * B.lamk[((e0 + el) * 2 + fld) * NU + i] / mt[4];
    }
  }
  __syncthreads();
  if constexpr (MODE == 1) {
    // forward sensor (as kb_tri<.., 1>): chi = V^-1 psi, s = log10(top / all)
    for (int el = tid; el < ne; el += blockDim.x) {
      double tot = 0.0, hi = 0.0;
      for (int m = 0; m < NU; ++m) {
        double c = 0.0;
        for (int j = 0; j < NU; ++j) c += op.Vinv[m][j] * us[(el * 2 + 1) * NU + j];
        tot += c * c;
        if (op.high[m]) hi += c * c;
      }
      double nu = 0.0, dnu = 0.0;
      if (tot > 0.0 && hi > 0.0) {
        const double se = log10(hi / tot);
        const double lo = A.prm.s0 - A.prm.kappa, up = A.prm.s0 + A.prm.kappa;
        const double w = M_PI / (2.0 * A.prm.kappa);
        if (se > up) {
          nu = A.prm.nu_max;
        } else if (se >= lo) {
          nu = 0.5 * A.prm.nu_max * (1.0 + sin(w * (se - A.prm.s0)));
          dnu = 0.5 * A.prm.nu_max * w * cos(w * (se - A.prm.s0));
        }
      }
      nu_e[el] = nu;
      dnu_e[el] = dnu;
      lnu_e[el] = 0.0;
    }
    __syncthreads();
  }
  // ---- reverse of Step 6: lam_f~_a = D_a^T lam_div - L^T (n~_a Y)
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) {
    const int c = idx / NU, j = idx % NU;  // c = element-field column
    const double* Yc = B.Y + (e0 * 2 + c) * NF;
    double a0 = 0, a1 = 0;
    for (int i = 0; i < NU; ++i) {
      a0 += op.Dr[i][j] * ld[c * NU + i];
      a1 += op.Ds[i][j] * ld[c * NU + i];
    }
    for (int k = 0; k < NF; ++k) {
      const double lk = op.L[k][j] * Yc[k];
      a0 -= lk * op.nref[k][0];
      a1 -= lk * op.nref[k][1];
    }
    lf[(c * 2 + 0) * NU + j] = a0;
    lf[(c * 2 + 1) * NU + j] = a1;
  }
  __syncthreads();
  if constexpr (MODE == 1) {
    // ---- reverse of Step 4 and of the source (psi slot)
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, i = idx % NU;
      const double* mt = met + el * 5;
      double q1[2], lg[2], lnu = 0.0;
      for (int c = 0; c < 2; ++c) q1[c] = q[((el * 2 + 1) * 2 + c) * NU + i];
      // lam_g = S^T lam_g~ with g~_a = sum_c S[a][c] g_c, g = -nu q
      for (int c = 0; c < 2; ++c) {
        lg[c] = mt[0 * 2 + c] * lf[((el * 2 + 1) * 2 + 0) * NU + i] + mt[1 * 2 + c] * lf[((el * 2 + 1) * 2 + 1) * NU + i];
        lnu -= lg[c] * q1[c];
      }
      const double lsrc = B.lam_scale * B.lamk[((e0 + el) * 2 + 1) * NU + i];
      const double qm = sqrt(q1[0] * q1[0] + q1[1] * q1[1]), m = fmax(qm, Pm.delta);
      const double p0 = A.psi0[(e0 + el) * NU + i];
      const double t = tanh(p0 / m), sech2 = 1.0 - t * t;
      const double dq = qm > 0.0 ? (-t - (qm > Pm.delta ? (1.0 - qm) * sech2 * p0 / (m * m) : 0.0)) / qm : 0.0;
      const double nu = nu_e[el];
      for (int c = 0; c < 2; ++c) {
        lf[((el * 2 + 1) * 2 + c) * NU + i] = -nu * lg[c] + lsrc * dq * q1[c];
        lf[((el * 2 + 0) * 2 + c) * NU + i] = 0.0;
      }
      B.lam_psi0[(e0 + el) * NU + i] += lsrc * (1.0 - qm) * sech2 / m;
      us[(el * 2 + 0) * NU + i] = 0.0;
      us[(el * 2 + 1) * NU + i] = 0.0;
      atomicAdd(&lnu_e[el], lnu);
    }
    // ---- reverse of Step 5 at L flux points (psi slot)
    for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
      const int el = idx / NF, k = idx % NF;
      for (int fld = 0; fld < 2; ++fld) {
        for (int c = 0; c < 2; ++c) lqf[((el * 2 + fld) * 2 + c) * NF + k] = 0.0;
        luf[(el * 2 + fld) * NF + k] = 0.0;
        luo[(el * 2 + fld) * NF + k] = 0.0;
      }
      if (!lm[el * NF + k]) continue;
      const int32_t own = (int32_t)((e0 + el) * NF + k);
      const int64_t pg = (int64_t)partner<NF>(A, A.fnbr[own], own);
      const bool bnd = pg == own;
      double nh[2];
      const double pm = tri_normal(met + el * 5, op.nref[k], nh);
      double pmR = pm;
      if (!bnd) {
        TriMet<double> mp;
        tri_metric(A.geo + (pg / NF) * NG, mp);
        const double mpv[4] = {mp.S[0][0], mp.S[0][1], mp.S[1][0], mp.S[1][1]};
        double nr[2];
        pmR = tri_normal(mpv, op.nref[pg % NF], nr);
      }
      double gn = 0.0;
      for (int c = 0; c < 2; ++c) {
        double a = 0.0;
        for (int j = 0; j < NU; ++j) a += op.L[k][j] * q[((el * 2 + 1) * 2 + c) * NU + j];
        gn += nh[c] * a;
      }
      const double y = B.Y[((e0 + el) * 2 + 1) * NF + k];
      const double lF = bnd ? pm * y : pm * y - pmR * B.Y[((pg / NF) * 2 + 1) * NF + pg % NF];
      const double nu = nu_e[el];
      luf[(el * 2 + 1) * NF + k] = lF * Pm.tau_pseudo;
      luo[(el * 2 + 1) * NF + k] = -lF * Pm.tau_pseudo;
      for (int c = 0; c < 2; ++c) lqf[((el * 2 + 1) * 2 + c) * NF + k] = -lF * nu * nh[c];
      atomicAdd(&lnu_e[el], -lF * gn);
    }
  } else {
  // ---- reverse of Step 4 at solution points
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    const double* mt = met + el * 5;
    const double xi[2] = {A.trid.xu[2 * i], A.trid.xu[2 * i + 1]};
    double x[3], v[3];
    map_point<ET_TRI, double>(gs + el * NG, xi, x);
    velocity<2, double>(BC.vel, x, g, v);
    const int kn = Pm.nphi ? 0 : 1;
    double q0[2], q1[2], l0[2], l1[2];
    for (int c = 0; c < 2; ++c) {
      q0[c] = q[((el * 2 + 0) * 2 + c) * NU + i];
      q1[c] = q[((el * 2 + kn) * 2 + c) * NU + i];
    }
    // lam_f = S^T lam_f~ with f~_a = sum_c S[a][c] f_c
    for (int c = 0; c < 2; ++c) {
      l0[c] = mt[0 * 2 + c] * lf[((el * 2 + 0) * 2 + 0) * NU + i] + mt[1 * 2 + c] * lf[((el * 2 + 0) * 2 + 1) * NU + i];
      l1[c] = mt[0 * 2 + c] * lf[((el * 2 + 1) * 2 + 0) * NU + i] + mt[1 * 2 + c] * lf[((el * 2 + 1) * 2 + 1) * NU + i];
    }
    const double v2 = v[0] * v[0] + v[1] * v[1], vm = sqrt(v2), M = fmax(vm, Pm.gamma);
    const double qn = sqrt(q1[0] * q1[0] + q1[1] * q1[1]), gm = fmax(qn, Pm.delta);
    const double ph = us[(el * 2 + 0) * NU + i], ps = us[(el * 2 + 1) * NU + i];
    const double pp = ph * (1.0 - ph);
    double lv0 = 0, lv1 = 0, lq1n = 0, la = 0;
    for (int c = 0; c < 2; ++c) {
      const double av = Pm.eps * q0[c] - Pm.gamma * pp / gm * q1[c];
      lv0 += l0[c] * v[c];
      lv1 += l1[c] * v[c];
      lq1n += l0[c] * q1[c];
      la += l0[c] * av;
    }
    // f0 = phi v - M (eps q_phi - gamma phi(1-phi) q_n / gm),  f1 = psi v
    const double lphi = lv0 + M * Pm.gamma * (1.0 - 2.0 * ph) / gm * lq1n;
    const double beta = M * Pm.gamma * pp;
    double n1[2], nl = 0;
    for (int c = 0; c < 2; ++c) {
      n1[c] = qn > Pm.delta ? q1[c] / qn : 0.0;
      nl += n1[c] * l0[c];
    }
    double lqp[2], lqn[2];
    for (int c = 0; c < 2; ++c) {
      lqp[c] = -M * Pm.eps * l0[c];
      lqn[c] = qn > Pm.delta ? beta * (l0[c] - n1[c] * nl) / qn : beta * l0[c] / Pm.delta;
    }
    for (int c = 0; c < 2; ++c) {
      // the normal's field is phi itself for the unpreconditioned method
      lf[((el * 2 + 0) * 2 + c) * NU + i] = lqp[c] + (kn == 0 ? lqn[c] : 0.0);
      lf[((el * 2 + 1) * 2 + c) * NU + i] = kn == 1 ? lqn[c] : 0.0;
    }
    us[(el * 2 + 0) * NU + i] = lphi;
    us[(el * 2 + 1) * NU + i] = lv1;
    if (coef) {
      const double dM = vm > Pm.gamma ? 1.0 / vm : 0.0;
      double* o = B.lv + ((e0 + el) * (NU + NF) + i) * 2;
      for (int c = 0; c < 2; ++c) o[c] = ph * l0[c] + ps * l1[c] - la * v[c] * dM;
    }
  }
  // ---- reverse of Step 5 at L flux points
  for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
    const int el = idx / NF, k = idx % NF;
    for (int fld = 0; fld < 2; ++fld) {
      for (int c = 0; c < 2; ++c) lqf[((el * 2 + fld) * 2 + c) * NF + k] = 0.0;
      luf[(el * 2 + fld) * NF + k] = 0.0;
      luo[(el * 2 + fld) * NF + k] = 0.0;
    }
    if (coef) {
      double* o = B.lv + ((e0 + el) * (NU + NF) + NU + k) * 2;
      o[0] = o[1] = 0.0;
    }
    if (!lm[el * NF + k]) continue;
    const int32_t own = (int32_t)((e0 + el) * NF + k);
    const int64_t pg = (int64_t)partner<NF>(A, A.fnbr[own], own);
    const bool bnd = pg == own;
    const double* mt = met + el * 5;
    double nh[2];
    const double pm = tri_normal(mt, op.nref[k], nh);
    double x[3], v[3];
    map_point<ET_TRI, double>(gs + el * NG, op.xf[k], x);
    velocity<2, double>(BC.vel, x, g, v);
    const int kn = Pm.nphi ? 0 : 1;
    double qf0[2], qf1[2];
    for (int c = 0; c < 2; ++c) {
      double a0 = 0, a1 = 0;
      for (int j = 0; j < NU; ++j) {
        a0 += op.L[k][j] * q[((el * 2 + 0) * 2 + c) * NU + j];
        a1 += op.L[k][j] * q[((el * 2 + kn) * 2 + c) * NU + j];
      }
      qf0[c] = a0;
      qf1[c] = a1;
    }
    // lam of the common flux out of L: this side lifts |pn_L| F, the partner
    // -|pn_R| F at its own point
    double lF[2];
    double pmR = pm;
    if (!bnd) {
      TriMet<double> mp;
      tri_metric(A.geo + (pg / NF) * NG, mp);
      const double mpv[4] = {mp.S[0][0], mp.S[0][1], mp.S[1][0], mp.S[1][1]};
      double nr[2];
      pmR = tri_normal(mpv, op.nref[pg % NF], nr);
    }
    for (int fld = 0; fld < 2; ++fld) {
      const double y = B.Y[((e0 + el) * 2 + fld) * NF + k];
      lF[fld] = bnd ? pm * y : pm * y - pmR * B.Y[((pg / NF) * 2 + fld) * NF + pg % NF];
    }
    const double vn = v[0] * nh[0] + v[1] * nh[1];
    const double vm = sqrt(v[0] * v[0] + v[1] * v[1]), M = fmax(vm, Pm.gamma);
    const double qn = sqrt(qf1[0] * qf1[0] + qf1[1] * qf1[1]), gm = fmax(qn, Pm.delta);
    const double pL = uf[(el * 2 + 0) * NF + k], pR = uo[(el * 2 + 0) * NF + k];
    const double sL = uf[(el * 2 + 1) * NF + k], sR = uo[(el * 2 + 1) * NF + k];
    const double pp = pL * (1.0 - pL);
    double nq = nh[0] * qf1[0] + nh[1] * qf1[1], fvn = 0;
    for (int c = 0; c < 2; ++c) fvn += nh[c] * (Pm.eps * qf0[c] - Pm.gamma * pp / gm * qf1[c]);
    // Fp = 1/2 (pL + pR) vn - M fvn + tau (pL - pR);  Fs = 1/2 (sL + sR) vn + tau_psi (sL - sR)
    luf[(el * 2 + 0) * NF + k] = lF[0] * (0.5 * vn + Pm.tau + M * Pm.gamma * (1.0 - 2.0 * pL) / gm * nq);
    luo[(el * 2 + 0) * NF + k] = lF[0] * (0.5 * vn - Pm.tau);
    luf[(el * 2 + 1) * NF + k] = lF[1] * (0.5 * vn + Pm.tau_psi);
    luo[(el * 2 + 1) * NF + k] = lF[1] * (0.5 * vn - Pm.tau_psi);
    double n1[2], n1h = 0;
    for (int c = 0; c < 2; ++c) {
      n1[c] = qn > Pm.delta ? qf1[c] / qn : 0.0;
      n1h += n1[c] * nh[c];
    }
    const double beta = M * Pm.gamma * pp;
    for (int c = 0; c < 2; ++c) {
      const double lp = -lF[0] * M * Pm.eps * nh[c];
      const double ln = lF[0] * (qn > Pm.delta ? beta * (nh[c] - n1h * n1[c]) / qn : beta * nh[c] / Pm.delta);
      lqf[((el * 2 + 0) * 2 + c) * NF + k] = lp + (kn == 0 ? ln : 0.0);
      lqf[((el * 2 + 1) * 2 + c) * NF + k] = kn == 1 ? ln : 0.0;
    }
    if (coef) {
      const double dM = vm > Pm.gamma ? 1.0 / vm : 0.0;
      double* o = B.lv + ((e0 + el) * (NU + NF) + NU + k) * 2;
      for (int c = 0; c < 2; ++c)
        o[c] = lF[0] * (0.5 * (pL + pR) * nh[c] - fvn * v[c] * dM) + lF[1] * 0.5 * (sL + sR) * nh[c];
    }
  }
  }
  __syncthreads();
  // ---- lam_q += L^T lam_qf, then lam_q~_a = sum_b S[a][b] lam_q_b / det J
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, j = idx % NU;
    const double* mt = met + el * 5;
    for (int fld = 0; fld < 2; ++fld) {
      double lq[2];
      for (int c = 0; c < 2; ++c) {
        double a = lf[((el * 2 + fld) * 2 + c) * NU + j];
        for (int k = 0; k < NF; ++k) a += op.L[k][j] * lqf[((el * 2 + fld) * 2 + c) * NF + k];
        lq[c] = a;
      }
      lf[((el * 2 + fld) * 2 + 0) * NU + j] = (mt[0] * lq[0] + mt[1] * lq[1]) / mt[4];
      lf[((el * 2 + fld) * 2 + 1) * NU + j] = (mt[2] * lq[0] + mt[3] * lq[1]) / mt[4];
    }
  }
  __syncthreads();
  // ---- reverse of Step 3's lift: lam_jump = sum_c n~_c LIFT^T lam_q~_c at L points
  for (int idx = tid; idx < ne * 2 * NF; idx += blockDim.x) {
    const int c = idx / NF, k = idx % NF, el = c / 2;
    if (!lm[el * NF + k]) continue;
    double lj = 0.0;
    for (int i = 0; i < NU; ++i)
      lj += op.LIFT[i][k] * (op.nref[k][0] * lf[(c * 2 + 0) * NU + i] + op.nref[k][1] * lf[(c * 2 + 1) * NU + i]);
    luo[c * NF + k] += lj;   // jump = u_o - u^f
    luf[c * NF + k] -= lj;
  }
  __syncthreads();
  if constexpr (MODE == 1) {
    // the element viscosity's dependence on psi: lam_psi += lam_nu dnu/ds
    // ds/dchi V^-1, ds/dchi_m = 2 chi_m (top_m / hi - 1 / tot) / ln 10; chi
    // (slot 0) and the weights (slot 1) in the lam_div region, free by now
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, m = idx % NU;
      double c = 0.0;
      for (int j = 0; j < NU; ++j) c += op.Vinv[m][j] * ustg[((e0 + el) * 2 + 1) * NU + j];
      ld[(el * 2 + 0) * NU + m] = c;
    }
    __syncthreads();
    for (int el = tid; el < ne; el += blockDim.x) {
      double tot = 0.0, hi = 0.0;
      for (int m = 0; m < NU; ++m) {
        const double c = ld[(el * 2 + 0) * NU + m];
        tot += c * c;
        if (op.high[m]) hi += c * c;
      }
      const double w = lnu_e[el] * dnu_e[el];
      for (int m = 0; m < NU; ++m) {
        const double c = ld[(el * 2 + 0) * NU + m];
        ld[(el * 2 + 1) * NU + m] = w == 0.0 ? 0.0 : w * 2.0 * c * ((op.high[m] ? 1.0 / hi : 0.0) - 1.0 / tot) / M_LN10;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, j = idx % NU;
      double a = 0.0;
      for (int m = 0; m < NU; ++m) a += op.Vinv[m][j] * ld[(el * 2 + 1) * NU + m];
      us[(el * 2 + 1) * NU + j] += a;
    }
    __syncthreads();
  }
  // ---- reverse of Step 3's derivative and of Step 1: lam_U += D^T lam_q~ + L^T lam_uf
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) {
    const int c = idx / NU, j = idx % NU;
    double a = us[idx];
    for (int i = 0; i < NU; ++i) a += op.Dr[i][j] * lf[(c * 2 + 0) * NU + i] + op.Ds[i][j] * lf[(c * 2 + 1) * NU + i];
    for (int k = 0; k < NF; ++k) a += op.L[k][j] * luf[c * NF + k];
    B.lamU[e0 * 2 * NU + idx] = a;
  }
  for (int idx = tid; idx < ne * 2 * NF; idx += blockDim.x) B.lamuo[e0 * 2 * NF + idx] = luo[idx];
}

template <int P>
__global__ void __launch_bounds__(256) adj_c_tri(const AdjArgs B) {
  using S = TriS<P>;
  using LY = AdjTriLayout<P>;
  constexpr int NU = S::NU, NF = S::NF, ET = LY::ET;
  const KArgs& A = B.K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TriOpsS<P, double>& op = *reinterpret_cast<TriOpsS<P, double>*>(smem_raw);
  double* gv = reinterpret_cast<double*>(smem_raw + ((sizeof(TriOpsS<P, double>) + 15) & ~size_t(15)));  // [ET][2][NF]
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const int tid = threadIdx.x;
  load_tri_ops<P, double>(A.trid, op);
  // the partner's adjoint of the trace it read from this element's point k
  for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
    const int el = idx / NF, k = idx % NF;
    const int32_t own = (int32_t)((e0 + el) * NF + k);
    const int64_t pg = (int64_t)partner<NF>(A, A.fnbr[own], own);
    for (int fld = 0; fld < 2; ++fld) gv[(el * 2 + fld) * NF + k] = B.lamuo[((pg / NF) * 2 + fld) * NF + pg % NF];
  }
  __syncthreads();
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) {
    const int c = idx / NU, j = idx % NU;
    double a = B.lamU[e0 * 2 * NU + idx];
    for (int k = 0; k < NF; ++k) a += op.L[k][j] * gv[c * NF + k];
    const int64_t gi = e0 * 2 * NU + idx;
    const double lp = B.Lp[gi];
    B.Lu[gi] = (B.first ? lp : B.Lu[gi]) + a;
    if (B.Lk) B.Lk[gi] = B.c_lp * lp + B.c_a * a;
  }
}

// cos/sin(2 pi k_m . x) of every stream-function mode m at every solution
// and flux point of the triangles (as k_coef_table)
template <int P>
__global__ void k_coef_table_tri(const KArgs A, double* cs) {
  using S = TriS<P>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG;
  const VelDescT<double>& V = A.cd.vel;
  const int M = V.n_modes;
  const int64_t n = A.E * (NU + NF);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / (NU + NF);
    const int p = (int)(g % (NU + NF));
    const double* xr = p < NU ? A.trid.xu + 2 * p : A.trid.xf + 2 * (p - NU);
    const double xi[2] = {xr[0], xr[1]};
    double x[3];
    map_point<ET_TRI, double>(A.geo + e * NG, xi, x);
    for (int m = 0; m < M; ++m) {
      double sn, c;
      scpi(2.0 * (V.kx[m] * x[0] + V.ky[m] * x[1]), &sn, &c);
      cs[(g * M + m) * 2 + 0] = c;
      cs[(g * M + m) * 2 + 1] = sn;
    }
  }
}

}  // namespace frp
