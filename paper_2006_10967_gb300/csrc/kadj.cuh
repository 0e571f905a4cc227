// Hand-written discrete adjoint (vector-Jacobian product) of the FR residual
// of the physical system on tensor elements.  The paper has no adjoint; this
// is the transpose, step by step in reverse order, of the forward kernels of
// ktensor.cuh (Steps 1-6 of Section 3.1), for the gradient of a misfit of
// phi at the final time with respect to the initial fields and the velocity
// coefficients.
//
// For a stage input U and an adjoint weight lam of its rate R(U) (both
// fields), the three kernels compute a = (dR/dU)^T lam and accumulate
// (dR/dc)^T lam over the stream-function coefficients c:
//   adj_a : lam_div = -lam / det J; the adjoints of the lifted flux jumps at
//           every flux point -> Y (global)
//   adj_b : forward recomputation of the element (traces, gradient, fluxes)
//           and the reverse of Steps 6, 4, 5, 3 and 1 on the element; the
//           adjoint of the common flux out of L gathers Y from the partner;
//           writes the element part of a and the adjoint of the partner
//           traces (lamuo, global)
//   adj_c : gathers the partners' lamuo, adds L^T of it, and applies the
//           RK4 adjoint recurrence.
// adj_b<.., 1> is the same for the preconditioning system of psi (Eq.
// pseudotimesystem): R_p = -J^{-1} div~ g~ + S with g = -nu_s(psi) q, the
// common flux n.g_L + tau_p (psi_L - psi_R) and S = tanh(psi0 / max(|q|,
// delta)) (1 - |q|); besides the gradient path it carries the element
// viscosity's dependence on psi (through the resolution indicator, Eqs.
// resolutionIndicator and nu_s) and accumulates dR_p/dpsi0 (lam_psi0).  The
// phi slot of the stage arrays is carried with zero weight.
// For a stream-function velocity adj_b also stores, per solution and flux
// point, the adjoint of the velocity there (lv); k_coef_acc contracts it with
// the derivative of the velocity with respect to each coefficient, from a
// table of cos/sin(2 pi k_m . x) at the points made once per sweep
// (k_coef_table), into per-block partial sums.
#pragma once
#include "ktensor.cuh"

namespace frp {

struct AdjArgs {
  KArgs K;              // forward arguments: K.ustg = stage input, K.tr = its traces, K.t = stage time
  const double* lamk;   // E x 2 x NU adjoint weight of the stage rate (times lam_scale)
  double lam_scale;
  double* Y;            // E x 2 x NF
  double* lamU;         // E x 2 x NU
  double* lamuo;        // E x 2 x NF
  double* coefp;        // [blocks][2 * n_modes] coefficient gradient partials (accumulated)
  int want_coef;
  double* lv;           // stream velocity: E x (NU + NF) x 2 adjoint of the velocity at each point
  // adj_c: RK4 recurrence  Lu = (first ? Lp : Lu) + a ;  Lk = c_lp * Lp + c_a * a
  const double* Lp;
  double* Lu;
  double* Lk;
  double c_lp, c_a;
  int first;
  double* lam_psi0;     // preconditioning sweep: E x NU, += (dR_p/dpsi0)^T lam (adj_b<.., 1>)
};

template <int DIM, int N>
struct AdjLayout {
  using S = TS<DIM, N>;
  static constexpr int LN = S::NFP;
  // adj_b shared memory per element (doubles)
  static constexpr int PER_EL = 2 * S::NU            // U, later lam_U
                                + 2 * DIM * S::NU    // q
                                + 2 * DIM * S::NU    // lam_f~, later lam_q, lam_q~
                                + 2 * S::NU          // lam_div
                                + 4 * 2 * S::NF      // uf, uo, luf, luo
                                + 2 * DIM * S::NF    // lam_qf
                                + S::NG;
  static constexpr int BYTES_EL = PER_EL * 8 + S::NF;
  static constexpr int ET_T = 256 / LN < 1 ? 1 : 256 / LN;
  static constexpr int ET_S = 49152 / BYTES_EL < 1 ? 1 : 49152 / BYTES_EL;
  static constexpr int ET = ET_T < ET_S ? ET_T : ET_S;
  static constexpr int THREADS = ET * LN;
  static constexpr size_t SMEM = (size_t)ET * BYTES_EL + 64;
};

// cos/sin(2 pi k_m . x) of every stream-function mode m at every solution
// and flux point of the mesh: cs[((e (NU + NF) + p) M + m) 2 + {0, 1}].
template <int DIM, int N>
__global__ void k_coef_table(const KArgs A, double* cs) {
  using S = TS<DIM, N>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG;
  const VelDescT<double>& V = A.cd.vel;
  const int M = V.n_modes;
  const int64_t n = A.E * (NU + NF);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / (NU + NF);
    const int p = (int)(g % (NU + NF));
    double xi[3], x[3];
    if (p < NU) upt_xi<DIM, N>(p, A.cd.ops.x, xi);
    else fpt_xi<DIM, N>(p - NU, A.cd.ops.x, xi);
    map_point<S::ET_, double>(A.geo + e * NG, xi, x);
    for (int m = 0; m < M; ++m) {
      double sn, c;
      scpi(2.0 * (V.kx[m] * x[0] + V.ky[m] * x[1]), &sn, &c);
      cs[(g * M + m) * 2 + 0] = c;
      cs[(g * M + m) * 2 + 1] = sn;
    }
  }
}

// Coefficient gradient of one stage: with v = g sum_m 2 pi (A_m cos th_m -
// B_m sin th_m)(k_y, -k_x), th_m = 2 pi k_m . x, the stage adds
//   dA_m += 2 pi g sum_p w_pm cos th_pm,  dB_m -= 2 pi g sum_p w_pm sin th_pm,
//   w_pm = k_y,m lv0_p - k_x,m lv1_p,
// over the points p of block b's share, to coefp[b][.] (no atomics).
// Launch: blocks = the partial slots, 256 threads = 32 mode lanes x 8 groups.
__global__ void k_coef_acc(const double* lv, const double* cs, int64_t npts, VelDescT<double> V, double g,
                           double* coefp) {
  const int M = V.n_modes, M2 = 2 * M;
  const int m = threadIdx.x & 31, grp = threadIdx.x >> 5, ngrp = blockDim.x >> 5;
  const int64_t per = (npts + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = (int64_t)blockIdx.x * per, p1 = p0 + per < npts ? p0 + per : npts;
  double ac = 0.0, as = 0.0;
  if (m < M) {
    const double kx = V.kx[m], ky = V.ky[m];
    for (int64_t p = p0 + grp; p < p1; p += ngrp) {
      const double w = ky * lv[2 * p] - kx * lv[2 * p + 1];
      ac += w * cs[(p * M + m) * 2 + 0];
      as += w * cs[(p * M + m) * 2 + 1];
    }
  }
  __shared__ double red[2][8][32];
  red[0][grp][m] = ac;
  red[1][grp][m] = as;
  __syncthreads();
  if (grp == 0 && m < M) {
    double sc = 0.0, ss = 0.0;
    for (int q = 0; q < ngrp; ++q) {
      sc += red[0][q][m];
      ss += red[1][q][m];
    }
    const double f = 2.0 * M_PI * g;
    coefp[(int64_t)blockIdx.x * M2 + m] += f * sc;
    coefp[(int64_t)blockIdx.x * M2 + M + m] -= f * ss;
  }
}

// ---------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256) adj_a(const AdjArgs B) {
  using S = TS<DIM, N>;
  using LY = AdjLayout<DIM, N>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, NFP = S::NFP, ET = LY::ET, LN = LY::LN;
  const KArgs& A = B.K;
  __shared__ double ld[ET * 2 * NU];
  __shared__ double gs[ET * NG];
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const int tid = threadIdx.x;
  const TensorOpsT<double>& O = A.cd.ops;
  for (int idx = tid; idx < ne * NG; idx += blockDim.x) gs[idx] = A.geo[e0 * NG + idx];
  __syncthreads();
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) {
    const int el = idx / (2 * NU), i = idx % NU;
    double xi[3], Sm[3][3];
    upt_xi<DIM, N>(i, O.x, xi);
    const double dj = metric<DIM>(gs + el * NG, xi, Sm);
    ld[idx] = -B.lam_scale * B.lamk[e0 * 2 * NU + idx] / dj;
  }
  __syncthreads();
  const int lel = tid / LN, ll = tid % LN;
  if (lel >= ne) return;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const int st = ipow(N, a), base = line_base<DIM, N>(a, ll);
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      const double* l = ld + (lel * 2 + fld) * NU + base;
      double c0 = 0, c1 = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        c0 -= O.gLd[j] * l[j * st];
        c1 += O.gRd[j] * l[j * st];
      }
      double* Y = B.Y + ((e0 + lel) * 2 + fld) * NF;
      Y[(2 * a) * NFP + ll] = c0;
      Y[(2 * a + 1) * NFP + ll] = c1;
    }
  }
}

// ---------------------------------------------------------------------------
template <int DIM, int N, int MODE = 0>
__global__ void __launch_bounds__(256) adj_b(const AdjArgs B) {
  using S = TS<DIM, N>;
  using LY = AdjLayout<DIM, N>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, NFP = S::NFP, ET = LY::ET, LN = LY::LN;
  const KArgs& A = B.K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* us = reinterpret_cast<double*>(smem_raw);  // [ET][2][NU]  U, later lam_U
  double* qt = us + ET * 2 * NU;                       // [ET][2][DIM][NU] q
  double* lf = qt + ET * 2 * DIM * NU;                 // [ET][2][DIM][NU] lam_f~ -> lam_q -> lam_q~
  double* ld = lf + ET * 2 * DIM * NU;                 // [ET][2][NU] lam_div
  double* uf = ld + ET * 2 * NU;                       // [ET][2][NF]
  double* uo = uf + ET * 2 * NF;
  double* luf = uo + ET * 2 * NF;
  double* luo = luf + ET * 2 * NF;
  double* lqf = luo + ET * 2 * NF;                     // [ET][2][DIM][NF]
  double* gs = lqf + ET * 2 * DIM * NF;                // [ET][NG]
  unsigned char* lm = reinterpret_cast<unsigned char*>(gs + ET * NG);

  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const int tid = threadIdx.x;
  const double* ustg = reinterpret_cast<const double*>(A.ustg);
  const double* tr = reinterpret_cast<const double*>(A.tr);
  const BulkConst<double>& BC = A.cd;
  const TensorOpsT<double>& O = BC.ops;
  const PrmT<double> P = BC.prm;
  const double g = time_factor(A, A.t);
  const bool coef = MODE == 0 && B.want_coef && BC.vel.kind == 3 && DIM == 2;
  __shared__ double nu_e[ET], dnu_e[ET], lnu_e[ET];  // MODE 1: nu_s, d nu_s / d s, lam of nu_s
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) us[idx] = ustg[e0 * 2 * NU + idx];
  for (int idx = tid; idx < ne * NG; idx += blockDim.x) gs[idx] = A.geo[e0 * NG + idx];
  __syncthreads();
  const int lel = tid / LN, ll = tid % LN;
  const bool lact = lel < ne;

  // ---- forward: traces, partner traces, gradient (as in kb_tensor) --------
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (lact) {
      const int st = ipow(N, a), base = line_base<DIM, N>(a, ll);
      const int k0 = (2 * a) * NFP + ll, k1 = k0 + NFP;
      const int32_t w0 = A.fnbr[(e0 + lel) * NF + k0], w1 = A.fnbr[(e0 + lel) * NF + k1];
      lm[lel * NF + k0] = (unsigned char)(w0 & 1);
      lm[lel * NF + k1] = (unsigned char)(w1 & 1);
#pragma unroll
      for (int fld = 0; fld < 2; ++fld) {
        const double* ul = us + (lel * 2 + fld) * NU + base;
        double v[N], f0 = 0, f1 = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          v[j] = ul[j * st];
          f0 += O.lend[0][j] * v[j];
          f1 += O.lend[1][j] * v[j];
        }
        // partner traces: in the own slots with FaceScatter (see ka_tensor),
        // else in the partner's
        const int64_t g0 = FaceScatter<DIM>::v ? (e0 + lel) * NF + k0
                                                : (int64_t)partner<NF>(A, w0, (int32_t)((e0 + lel) * NF + k0));
        const int64_t g1 = FaceScatter<DIM>::v ? (e0 + lel) * NF + k1
                                                : (int64_t)partner<NF>(A, w1, (int32_t)((e0 + lel) * NF + k1));
        const double o0 = (w0 & 1) ? tr[((g0 / NF) * 2 + fld) * NF + g0 % NF] : f0;
        const double o1 = (w1 & 1) ? tr[((g1 / NF) * 2 + fld) * NF + g1 % NF] : f1;
        const int fo = (lel * 2 + fld) * NF;
        uf[fo + k0] = f0;
        uf[fo + k1] = f1;
        uo[fo + k0] = o0;
        uo[fo + k1] = o1;
        const double jm = o0 - f0, jp = o1 - f1;
        double* qa = qt + ((lel * 2 + fld) * DIM + a) * NU + base;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          double acc = O.gLd[j] * jm + O.gRd[j] * jp;
#pragma unroll
          for (int m = 0; m < N; ++m) acc += O.D[j][m] * v[m];
          qa[j * st] = acc;
        }
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    double xi[3], Sm[3][3];
    upt_xi<DIM, N>(i, O.x, xi);
    const double dj = metric<DIM>(gs + el * NG, xi, Sm);
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      double* q = qt + (el * 2 + fld) * DIM * NU + i;
      double qv[3];
#pragma unroll
      for (int c = 0; c < DIM; ++c) qv[c] = q[c * NU];
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        double r = 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) r += Sm[c][b] * qv[c];
        q[b * NU] = r / dj;
      }
      ld[(el * 2 + fld) * NU + i] = -B.lam_scale * B.lamk[((e0 + el) * 2 + fld) * NU + i] / dj;
    }
  }
  __syncthreads();
  if constexpr (MODE == 1) {
    // forward sensor of the element (as kb_tensor<.., 1>): modal coefficients
    // chi = V^-1 psi (tensor product), s = log10(top / all), nu_s(s)
    for (int el = tid; el < ne; el += blockDim.x) {
      const double* ps = us + (el * 2 + 1) * NU;
      double tot = 0.0, hi = 0.0;
      for (int m = 0; m < NU; ++m) {
        double c = 0.0;
        for (int i = 0; i < NU; ++i) {
          double v = 1.0;
#pragma unroll
          for (int b = 0; b < DIM; ++b) v *= O.Vinv[ucoord<N>(m, b)][ucoord<N>(i, b)];
          c += v * ps[i];
        }
        tot += c * c;
        bool top = false;
#pragma unroll
        for (int b = 0; b < DIM; ++b) top = top || (ucoord<N>(m, b) == N - 1);
        if (top) hi += c * c;
      }
      double nu = 0.0, dnu = 0.0;
      if (tot > 0.0 && hi > 0.0) {
        const double se = log10(hi / tot);
        const double lo = A.prm.s0 - A.prm.kappa, up = A.prm.s0 + A.prm.kappa;
        const double nmax = A.prm.nu_max, w = M_PI / (2.0 * A.prm.kappa);
        if (se > up) {
          nu = nmax;
        } else if (se >= lo) {
          nu = 0.5 * nmax * (1.0 + sin(w * (se - A.prm.s0)));
          dnu = 0.5 * nmax * w * cos(w * (se - A.prm.s0));
        }
      }
      nu_e[el] = nu;
      dnu_e[el] = dnu;
      lnu_e[el] = 0.0;
    }
    __syncthreads();
  }

  // ---- reverse of Step 6 by axis: lam_f~ from the derivative and the lifts
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (lact) {
      const int st = ipow(N, a), base = line_base<DIM, N>(a, ll);
#pragma unroll
      for (int fld = 0; fld < 2; ++fld) {
        const double* l = ld + (lel * 2 + fld) * NU + base;
        double lv[N], c0 = 0, c1 = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          lv[j] = l[j * st];
          c0 -= O.gLd[j] * lv[j];
          c1 += O.gRd[j] * lv[j];
        }
        double* o = lf + ((lel * 2 + fld) * DIM + a) * NU + base;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          double acc = O.lend[0][m] * c0 - O.lend[1][m] * c1;
#pragma unroll
          for (int j = 0; j < N; ++j) acc += O.D[j][m] * lv[j];
          o[m * st] = acc;
        }
      }
    }
  }
  __syncthreads();

  if constexpr (MODE == 1) {
    // ---- reverse of Step 4 and of the source at solution points (psi slot)
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, i = idx % NU;
      double xi[3], Sm[3][3];
      upt_xi<DIM, N>(i, O.x, xi);
      metric<DIM>(gs + el * NG, xi, Sm);
      double q[3], lg[3], q2 = 0.0, lnu = 0.0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        q[c] = qt[((el * 2 + 1) * DIM + c) * NU + i];
        q2 += q[c] * q[c];
      }
      // lam_g = S^T lam_g~ with g~ = S g, g = -nu q
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double sc = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) sc += Sm[a][c] * lf[((el * 2 + 1) * DIM + a) * NU + i];
        lg[c] = sc;
        lnu -= sc * q[c];
      }
      // source S = tanh(psi0 / m)(1 - |q|), m = max(|q|, delta), weight lam_src
      const double lsrc = B.lam_scale * B.lamk[((e0 + el) * 2 + 1) * NU + i];
      const double qm = sqrt(q2), m = fmax(qm, P.delta);
      const double p0 = A.psi0[(e0 + el) * NU + i];
      const double t = tanh(p0 / m), sech2 = 1.0 - t * t;
      const double dq = qm > 0.0 ? (-t - (qm > P.delta ? (1.0 - qm) * sech2 * p0 / (m * m) : 0.0)) / qm : 0.0;
      const double nu = nu_e[el];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        lf[((el * 2 + 1) * DIM + c) * NU + i] = -nu * lg[c] + lsrc * dq * q[c];
        lf[((el * 2 + 0) * DIM + c) * NU + i] = 0.0;
      }
      B.lam_psi0[(e0 + el) * NU + i] += lsrc * (1.0 - qm) * sech2 / m;
      us[(el * 2 + 0) * NU + i] = 0.0;  // lam_U (direct part): none
      us[(el * 2 + 1) * NU + i] = 0.0;
      atomicAdd(&lnu_e[el], lnu);
    }
    // ---- reverse of Step 5 at L flux points (psi slot)
    for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
      const int el = idx / NF, k = idx % NF;
#pragma unroll
      for (int fld = 0; fld < 2; ++fld) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) lqf[((el * 2 + fld) * DIM + c) * NF + k] = 0.0;
        luf[(el * 2 + fld) * NF + k] = 0.0;
        luo[(el * 2 + fld) * NF + k] = 0.0;
      }
      if (!lm[el * NF + k]) continue;
      const int64_t gk = (e0 + el) * NF + k;
      const int64_t pg = (int64_t)partner<NF>(A, A.fnbr[gk], (int32_t)gk);
      const bool bnd = pg == gk;
      int a, s, b0;
      fline<DIM, N>(k, a, s, b0);
      double xi[3], Sm[3][3];
      fpt_xi<DIM, N>(k, O.x, xi);
      metric<DIM>(gs + el * NG, xi, Sm);
      double pn[3], pm = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double sac = Sm[0][c];
#pragma unroll
        for (int b = 1; b < DIM; ++b)
          if (b == a) sac = Sm[b][c];
        pn[c] = (s ? 1.0 : -1.0) * sac;
        pm += pn[c] * pn[c];
      }
      pm = sqrt(pm);
      const int st = ipow(N, a);
      double gn = 0.0, nh[3];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        nh[c] = pn[c] / pm;
        const double* ql = qt + ((el * 2 + 1) * DIM + c) * NU + b0;
        double acc = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += (s ? O.lend[1][j] : O.lend[0][j]) * ql[j * st];
        gn += nh[c] * acc;
      }
      // F~ = pm (-nu n.q_f + tau_p (psi_L - psi_R)) enters this side's lift
      // and (negated) the partner's
      const double y = B.Y[((e0 + el) * 2 + 1) * NF + k];
      const double lF = pm * (bnd ? y : y - B.Y[((pg / NF) * 2 + 1) * NF + pg % NF]);
      const double nu = nu_e[el];
      luf[(el * 2 + 1) * NF + k] = lF * P.tau_pseudo;
      luo[(el * 2 + 1) * NF + k] = -lF * P.tau_pseudo;
#pragma unroll
      for (int c = 0; c < DIM; ++c) lqf[((el * 2 + 1) * DIM + c) * NF + k] = -lF * nu * nh[c];
      atomicAdd(&lnu_e[el], -lF * gn);
    }
  } else {
  // ---- reverse of Step 4 at solution points ---------------------------------
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    double xi[3], Sm[3][3], x[3], v[3];
    upt_xi<DIM, N>(i, O.x, xi);
    metric<DIM>(gs + el * NG, xi, Sm);
    if (A.vsu) {  // the forward kernels' velocity: g(t) times the cached v(x)
      const double* vc = reinterpret_cast<const double*>(A.vsu) + (e0 + el) * DIM * NU + i;
#pragma unroll
      for (int c = 0; c < DIM; ++c) v[c] = g * vc[c * NU];
    } else {
      map_point<S::ET_, double>(gs + el * NG, xi, x);
      velocity<DIM, double>(BC.vel, x, g, v);
    }
    double q0[3], q1[3], l0[3], l1[3], v2 = 0, g2 = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      q0[c] = qt[((el * 2 + 0) * DIM + c) * NU + i];
      q1[c] = qt[((el * 2 + 1) * DIM + c) * NU + i];
      v2 += v[c] * v[c];
      g2 += q1[c] * q1[c];
    }
    // lam_f = S^T lam_f~
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double s0 = 0, s1 = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        s0 += Sm[a][c] * lf[((el * 2 + 0) * DIM + a) * NU + i];
        s1 += Sm[a][c] * lf[((el * 2 + 1) * DIM + a) * NU + i];
      }
      l0[c] = s0;
      l1[c] = s1;
    }
    const double vm = sqrt(v2), M = fmax(vm, P.gamma);
    const double qn = sqrt(g2), gm = fmax(qn, P.delta);
    const double ph = us[(el * 2 + 0) * NU + i], ps = us[(el * 2 + 1) * NU + i];
    const double pp = ph * (1.0 - ph);
    double lv0 = 0, lv1 = 0, lq1n = 0, la = 0;
    double av[3];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      av[c] = P.eps * q0[c] - P.gamma * pp / gm * q1[c];
      lv0 += l0[c] * v[c];
      lv1 += l1[c] * v[c];
      lq1n += l0[c] * q1[c];
      la += l0[c] * av[c];
    }
    // f0 = phi v - M (eps q0 - gamma phi(1-phi) q1 / gm),  f1 = psi v
    const double lphi = lv0 + M * P.gamma * (1.0 - 2.0 * ph) / gm * lq1n;
    const double lpsi = lv1;
    const double beta = M * P.gamma * pp;
    double* lq = lf;  // lam_q overwrites lam_f~ (this point only)
    double n1[3];
#pragma unroll
    for (int c = 0; c < DIM; ++c) n1[c] = qn > P.delta ? q1[c] / qn : 0.0;
    double nl = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) nl += n1[c] * l0[c];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      lq[((el * 2 + 0) * DIM + c) * NU + i] = -M * P.eps * l0[c];
      lq[((el * 2 + 1) * DIM + c) * NU + i] = qn > P.delta ? beta * (l0[c] - n1[c] * nl) / qn : beta * l0[c] / P.delta;
    }
    us[(el * 2 + 0) * NU + i] = lphi;  // lam_U (direct part) overwrites U
    us[(el * 2 + 1) * NU + i] = lpsi;
    if (coef) {
      double lvv[3];
      const double dM = vm > P.gamma ? 1.0 / vm : 0.0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) lvv[c] = ph * l0[c] + ps * l1[c] - la * v[c] * dM;
      double* o = B.lv + ((e0 + el) * (NU + NF) + i) * 2;
      o[0] = lvv[0];
      o[1] = lvv[1];
    }
  }
  // ---- reverse of Step 5 at L flux points ------------------------------------
  for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
    const int el = idx / NF, k = idx % NF;
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) lqf[((el * 2 + fld) * DIM + c) * NF + k] = 0.0;
      luf[(el * 2 + fld) * NF + k] = 0.0;
      luo[(el * 2 + fld) * NF + k] = 0.0;
    }
    if (coef) {
      double* o = B.lv + ((e0 + el) * (NU + NF) + NU + k) * 2;  // R points: no contribution
      o[0] = 0.0;
      o[1] = 0.0;
    }
    if (!lm[el * NF + k]) continue;
    const int64_t gk = (e0 + el) * NF + k;
    const int32_t w = A.fnbr[gk];
    const int64_t pg = (int64_t)partner<NF>(A, w, (int32_t)gk);
    const bool bnd = pg == gk;
    int a, s, b0;
    fline<DIM, N>(k, a, s, b0);
    double xi[3], Sm[3][3], x[3], v[3];
    fpt_xi<DIM, N>(k, O.x, xi);
    metric<DIM>(gs + el * NG, xi, Sm);
    double pn[3], pm = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double sac = Sm[0][c];
#pragma unroll
      for (int b = 1; b < DIM; ++b)
        if (b == a) sac = Sm[b][c];
      pn[c] = (s ? 1.0 : -1.0) * sac;
      pm += pn[c] * pn[c];
    }
    pm = sqrt(pm);
    double nh[3];
#pragma unroll
    for (int c = 0; c < DIM; ++c) nh[c] = pn[c] / pm;
    if (A.vsf) {  // the forward kernels' velocity: g(t) times the cached v(x)
      const double* vc = reinterpret_cast<const double*>(A.vsf) + (e0 + el) * DIM * NF + k;
#pragma unroll
      for (int c = 0; c < DIM; ++c) v[c] = g * vc[c * NF];
    } else {
      map_point<S::ET_, double>(gs + el * NG, xi, x);
      velocity<DIM, double>(BC.vel, x, g, v);
    }
    const int st = ipow(N, a);
    double qf0[3], qf1[3];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const double* q0l = qt + ((el * 2 + 0) * DIM + c) * NU + b0;
      const double* q1l = qt + ((el * 2 + 1) * DIM + c) * NU + b0;
      double a0 = 0, a1 = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const double lw = s ? O.lend[1][j] : O.lend[0][j];
        a0 += lw * q0l[j * st];
        a1 += lw * q1l[j * st];
      }
      qf0[c] = a0;
      qf1[c] = a1;
    }
    // lam of the physical common flux out of L: the transformed flux pm F
    // enters this side's lift and (negated) the partner's
    double lF[2];
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      const double y = B.Y[((e0 + el) * 2 + fld) * NF + k];
      lF[fld] = pm * (bnd ? y : y - B.Y[((pg / NF) * 2 + fld) * NF + pg % NF]);
    }
    double vn = 0, v2 = 0, g2 = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      vn += v[c] * nh[c];
      v2 += v[c] * v[c];
      g2 += qf1[c] * qf1[c];
    }
    const double vm = sqrt(v2), M = fmax(vm, P.gamma);
    const double qn = sqrt(g2), gm = fmax(qn, P.delta);
    const double pL = uf[(el * 2 + 0) * NF + k], pR = uo[(el * 2 + 0) * NF + k];
    const double sL = uf[(el * 2 + 1) * NF + k], sR = uo[(el * 2 + 1) * NF + k];
    double nq = 0, fvn = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) nq += nh[c] * qf1[c];
    const double pp = pL * (1.0 - pL);
#pragma unroll
    for (int c = 0; c < DIM; ++c) fvn += nh[c] * (P.eps * qf0[c] - P.gamma * pp / gm * qf1[c]);
    // Fp = 1/2 (pL + pR) vn - M fvn + tau (pL - pR);  Fs = 1/2 (sL + sR) vn + tau_psi (sL - sR)
    luf[(el * 2 + 0) * NF + k] = lF[0] * (0.5 * vn + P.tau + M * P.gamma * (1.0 - 2.0 * pL) / gm * nq);
    luo[(el * 2 + 0) * NF + k] = lF[0] * (0.5 * vn - P.tau);
    luf[(el * 2 + 1) * NF + k] = lF[1] * (0.5 * vn + P.tau_psi);
    luo[(el * 2 + 1) * NF + k] = lF[1] * (0.5 * vn - P.tau_psi);
    double n1[3], n1h = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      n1[c] = qn > P.delta ? qf1[c] / qn : 0.0;
      n1h += n1[c] * nh[c];
    }
    const double beta = M * P.gamma * pp;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      lqf[((el * 2 + 0) * DIM + c) * NF + k] = -lF[0] * M * P.eps * nh[c];
      lqf[((el * 2 + 1) * DIM + c) * NF + k] =
          lF[0] * (qn > P.delta ? beta * (nh[c] - n1h * n1[c]) / qn : beta * nh[c] / P.delta);
    }
    if (coef) {
      const double dM = vm > P.gamma ? 1.0 / vm : 0.0;
      double lvv[3];
#pragma unroll
      for (int c = 0; c < DIM; ++c)
        lvv[c] = lF[0] * (0.5 * (pL + pR) * nh[c] - fvn * v[c] * dM) + lF[1] * 0.5 * (sL + sR) * nh[c];
      double* o = B.lv + ((e0 + el) * (NU + NF) + NU + k) * 2;
      o[0] = lvv[0];
      o[1] = lvv[1];
    }
  }
  }
  __syncthreads();

  // ---- lam_q += L^T lam_qf, one pass per axis ------------------------------
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (lact) {
      const int st = ipow(N, a), base = line_base<DIM, N>(a, ll);
      const int k0 = (2 * a) * NFP + ll, k1 = k0 + NFP;
#pragma unroll
      for (int fld = 0; fld < 2; ++fld)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const double g0 = lqf[((lel * 2 + fld) * DIM + c) * NF + k0];
          const double g1 = lqf[((lel * 2 + fld) * DIM + c) * NF + k1];
          double* o = lf + ((lel * 2 + fld) * DIM + c) * NU + base;
#pragma unroll
          for (int j = 0; j < N; ++j) o[j * st] += O.lend[0][j] * g0 + O.lend[1][j] * g1;
        }
    }
    __syncthreads();
  }
  // ---- lam_q~ = J^{-1} lam_q -------------------------------------------------
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    double xi[3], Sm[3][3];
    upt_xi<DIM, N>(i, O.x, xi);
    const double dj = metric<DIM>(gs + el * NG, xi, Sm);
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      double* l = lf + (el * 2 + fld) * DIM * NU + i;
      double lv[3];
#pragma unroll
      for (int b = 0; b < DIM; ++b) lv[b] = l[b * NU];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        double r = 0;
#pragma unroll
        for (int b = 0; b < DIM; ++b) r += Sm[a][b] * lv[b];
        l[a * NU] = r / dj;
      }
    }
  }
  __syncthreads();
  // ---- reverse of Step 3 and Step 1 by axis: D^T, the jump adjoints, L^T ---
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (lact) {
      const int st = ipow(N, a), base = line_base<DIM, N>(a, ll);
      const int k0 = (2 * a) * NFP + ll, k1 = k0 + NFP;
      const bool L0 = lm[lel * NF + k0], L1 = lm[lel * NF + k1];
#pragma unroll
      for (int fld = 0; fld < 2; ++fld) {
        const double* lq = lf + ((lel * 2 + fld) * DIM + a) * NU + base;
        double lv[N], jm = 0, jp = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          lv[j] = lq[j * st];
          jm += O.gLd[j] * lv[j];
          jp += O.gRd[j] * lv[j];
        }
        const int fo = (lel * 2 + fld) * NF;
        // jump = isL ? uo - uf : 0
        double u0 = luf[fo + k0], u1 = luf[fo + k1];
        if (L0) {
          luo[fo + k0] += jm;
          u0 -= jm;
        }
        if (L1) {
          luo[fo + k1] += jp;
          u1 -= jp;
        }
        double* o = us + (lel * 2 + fld) * NU + base;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          double acc = O.lend[0][m] * u0 + O.lend[1][m] * u1;
#pragma unroll
          for (int j = 0; j < N; ++j) acc += O.D[j][m] * lv[j];
          o[m * st] += acc;
        }
      }
    }
    __syncthreads();
  }
  if constexpr (MODE == 1) {
    // the element viscosity's dependence on psi: lam_psi += lam_nu dnu/ds
    // ds/dchi V^-1, with ds/dchi_m = 2 chi_m (top_m / hi - 1 / tot) / ln 10;
    // chi (slot 0) and ds/dchi (slot 1) in the lam_div region, free by now
    const double* psg = reinterpret_cast<const double*>(A.ustg);
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, m = idx % NU;
      double c = 0.0;
      for (int j = 0; j < NU; ++j) {
        double v = 1.0;
#pragma unroll
        for (int b = 0; b < DIM; ++b) v *= O.Vinv[ucoord<N>(m, b)][ucoord<N>(j, b)];
        c += v * psg[((e0 + el) * 2 + 1) * NU + j];
      }
      ld[(el * 2 + 0) * NU + m] = c;
    }
    __syncthreads();
    for (int el = tid; el < ne; el += blockDim.x) {
      double tot = 0.0, hi = 0.0;
      for (int m = 0; m < NU; ++m) {
        const double c = ld[(el * 2 + 0) * NU + m];
        bool top = false;
#pragma unroll
        for (int b = 0; b < DIM; ++b) top = top || (ucoord<N>(m, b) == N - 1);
        tot += c * c;
        if (top) hi += c * c;
      }
      const double w = lnu_e[el] * dnu_e[el];
      for (int m = 0; m < NU; ++m) {
        bool top = false;
#pragma unroll
        for (int b = 0; b < DIM; ++b) top = top || (ucoord<N>(m, b) == N - 1);
        const double c = ld[(el * 2 + 0) * NU + m];
        ld[(el * 2 + 1) * NU + m] = w == 0.0 ? 0.0 : w * 2.0 * c * ((top ? 1.0 / hi : 0.0) - 1.0 / tot) / M_LN10;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, i = idx % NU;
      double acc = 0.0;
      for (int m = 0; m < NU; ++m) {
        double v = 1.0;
#pragma unroll
        for (int b = 0; b < DIM; ++b) v *= O.Vinv[ucoord<N>(m, b)][ucoord<N>(i, b)];
        acc += ld[(el * 2 + 1) * NU + m] * v;
      }
      us[(el * 2 + 1) * NU + i] += acc;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) B.lamU[e0 * 2 * NU + idx] = us[idx];
  for (int idx = tid; idx < ne * 2 * NF; idx += blockDim.x) B.lamuo[e0 * 2 * NF + idx] = luo[idx];
}

// ---------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256) adj_c(const AdjArgs B) {
  using S = TS<DIM, N>;
  using LY = AdjLayout<DIM, N>;
  constexpr int NU = S::NU, NF = S::NF, NFP = S::NFP, ET = LY::ET, LN = LY::LN;
  const KArgs& A = B.K;
  __shared__ double la[ET * 2 * NU];
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const int tid = threadIdx.x;
  const TensorOpsT<double>& O = A.cd.ops;
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) la[idx] = B.lamU[e0 * 2 * NU + idx];
  __syncthreads();
  const int lel = tid / LN, ll = tid % LN;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (lel < ne) {
      const int st = ipow(N, a), base = line_base<DIM, N>(a, ll);
      double gv[2][2];
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int32_t own = (int32_t)((e0 + lel) * NF + (2 * a + sd) * NFP + ll);
        const int64_t pg = (int64_t)partner<NF>(A, A.fnbr[own], own);
#pragma unroll
        for (int fld = 0; fld < 2; ++fld) gv[sd][fld] = B.lamuo[((pg / NF) * 2 + fld) * NF + pg % NF];
      }
#pragma unroll
      for (int fld = 0; fld < 2; ++fld) {
        double* o = la + (lel * 2 + fld) * NU + base;
#pragma unroll
        for (int j = 0; j < N; ++j) o[j * st] += O.lend[0][j] * gv[0][fld] + O.lend[1][j] * gv[1][fld];
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ne * 2 * NU; idx += blockDim.x) {
    const int64_t gi = e0 * 2 * NU + idx;
    const double a = la[idx];
    const double lp = B.Lp[gi];
    B.Lu[gi] = (B.first ? lp : B.Lu[gi]) + a;
    if (B.Lk) B.Lk[gi] = B.c_lp * lp + B.c_a * a;
  }
}

}  // namespace frp
