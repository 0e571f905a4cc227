// FR kernels for tensor-product elements (quadrilaterals, hexahedra) with
// Gauss-Legendre solution points and flux points on the solution-point lines.
//
// Every operator of Section 3.1 is applied by sum factorisation along lines:
//   Step 1  u^f   = sum_j l_j(+-1) u(line)                 (Eq. extrapolateSoln)
//   Step 2  C(u)  = u_R on both sides of a face (beta = +1/2 w.r.t. L)
//   Step 3  q~_a  = sum_j D_ij u(line_a) + g_L'(xi_i)(C-u^f)_{a,-} + g_R'(xi_i)(C-u^f)_{a,+}
//           q     = J^{-T} q~, q^f by line interpolation     (Eqs. continuousGrad, extrapolateGrad)
//   Step 4  f~    = det J J^{-1} f(u, q), f~perp = n~ . f~(x^f) (Eq. normalTransFlux)
//   Step 5  common normal flux on the L side of every face   (Eqs. commonFlux, inviscidFlux, viscousFlux)
//   Step 6  div~ f~ = sum_a D f~_a + sum_faces (div g)(F~ - f~perp)  (Eq. continuousDivFlux)
//
// Two kernels per RK stage:
//   kb_tensor : Steps 1-6 for one tile of elements.  It writes the common
//               normal flux at its L flux points (fc) and the divergence with
//               the R-side common fluxes still missing (rp).
//   ka_tensor : adds the lift of the R-side common fluxes (minus the L side's
//               flux, scaled by this side's face metric), forms
//               du/dt = -div~ f~ / det J (Step 6), applies the RK4 register
//               update and writes the flux-point traces of the next stage.
// MODE 0 is the physical system u = [phi, psi]; MODE 1 the preconditioning
// system for psi alone (Eq. pseudotimesystem) with element viscosity nu_s
// from the resolution indicator (Eqs. resolutionIndicator, nu_s).
#pragma once
#include "kcommon.cuh"

namespace frp {

template <int DIM, int N>
struct TS {
  static constexpr int NU = DIM == 2 ? N * N : N * N * N;
  static constexpr int NFP = DIM == 2 ? N : N * N;
  static constexpr int NF = 2 * DIM * NFP;
  static constexpr int NC = DIM == 2 ? 4 : 8;
  static constexpr int NG = DIM * NC;
  static constexpr int ET_ = DIM == 2 ? ET_QUAD : ET_HEX;
};

__host__ __device__ constexpr int ipow(int n, int a) { return a == 0 ? 1 : (a == 1 ? n : n * n); }

template <int N>
__device__ __forceinline__ int ucoord(int i, int a) { return (i / ipow(N, a)) % N; }

template <int DIM, int N>
__device__ __forceinline__ void fline(int k, int& a, int& s, int& base) {
  constexpr int NFP = TS<DIM, N>::NFP;
  const int f = k / NFP;
  int r = k % NFP;
  a = f >> 1;
  s = f & 1;
  base = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (b == a) continue;
    base += (r % N) * ipow(N, b);
    r /= N;
  }
}

template <int DIM, int N>
__device__ __forceinline__ int fpt_of(int i, int a, int s) {
  int m = 0, mul = 1;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (b == a) continue;
    m += ucoord<N>(i, b) * mul;
    mul *= N;
  }
  return (2 * a + s) * TS<DIM, N>::NFP + m;
}

template <int DIM, int N, typename T>
__device__ __forceinline__ void upt_xi(int i, const T* x1, T* xi) {
#pragma unroll
  for (int b = 0; b < DIM; ++b) xi[b] = x1[ucoord<N>(i, b)];
}

template <int DIM, int N, typename T>
__device__ __forceinline__ void fpt_xi(int k, const T* x1, T* xi) {
  constexpr int NFP = TS<DIM, N>::NFP;
  const int f = k / NFP, a = f >> 1, s = f & 1;
  int r = k % NFP;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (b == a) {
      xi[b] = s ? (T)1 : (T)-1;
    } else {
      xi[b] = x1[r % N];
      r /= N;
    }
  }
}

// Metric at a reference point: S = det J J^{-1}; returns det J.
template <int DIM, typename T>
__device__ __forceinline__ T metric(const T* g, const T* xi, T S[3][3]) {
  T J[3][3];
  jacobian<DIM == 2 ? ET_QUAD : ET_HEX, T>(g, xi, J);
  return adjugate<DIM, T>(J, S);
}

// Shared 1D operators in bulk precision.
template <int N, typename T>
struct SOps {
  T x[N], lend[2][N], D[N][N], gLd[N], gRd[N], Vinv[N][N];
};

template <int N, typename T>
__device__ __forceinline__ void load_ops(const TensorOps& o, SOps<N, T>& s) {
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    s.x[t] = (T)o.x[t];
    s.lend[0][t] = (T)o.lend[0][t];
    s.lend[1][t] = (T)o.lend[1][t];
    s.gLd[t] = (T)o.gLd[t];
    s.gRd[t] = (T)o.gRd[t];
  }
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    s.D[t / N][t % N] = (T)o.D[t / N][t % N];
    s.Vinv[t / N][t % N] = (T)o.Vinv[t / N][t % N];
  }
}

template <int DIM, int N, typename T, int MODE>
struct KBLayout {
  using S = TS<DIM, N>;
  static constexpr int NFLD = MODE == 0 ? 2 : 1;
  static constexpr int PER_EL_T = NFLD * S::NU        // us
                                  + 3 * NFLD * S::NF  // uf, uo, cor
                                  + NFLD * DIM * S::NU // q / f~
                                  + S::NG             // geometry
                                  + (MODE == 1 ? 2 * S::NU + 1 : 0);  // modal scratch, nu_s
  static constexpr int BYTES_EL = PER_EL_T * (int)sizeof(T) + S::NF;
  static constexpr int ETr = 40960 / BYTES_EL;
  static constexpr int ET = ETr < 1 ? 1 : (ETr > 32 ? 32 : ETr);
  static constexpr size_t SMEM = (size_t)ET * BYTES_EL + sizeof(SOps<N, T>) + 64;
};

// ============================================================================
// kb_tensor: Steps 1-6 on a tile of elements.
template <int DIM, int N, typename T, int MODE>
__global__ void __launch_bounds__(kThreads) kb_tensor(const KArgs A) {
  using S = TS<DIM, N>;
  using LY = KBLayout<DIM, N, T, MODE>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, NFLD = LY::NFLD, ET = LY::ET;
  constexpr int F0 = MODE == 0 ? 0 : 1;
  if (MODE == 1 && *(volatile int32_t*)&A.status[ST_PSEUDO_DONE]) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  SOps<N, T>& op = *reinterpret_cast<SOps<N, T>*>(smem_raw);
  T* base = reinterpret_cast<T*>(smem_raw + ((sizeof(SOps<N, T>) + 15) & ~size_t(15)));
  T* us = base;                        // [ET][NFLD][NU]
  T* uf = us + ET * NFLD * NU;         // [ET][NFLD][NF]
  T* uo = uf + ET * NFLD * NF;         // [ET][NFLD][NF]
  T* cor = uo + ET * NFLD * NF;        // [ET][NFLD][NF]
  T* q = cor + ET * NFLD * NF;         // [ET][NFLD][DIM][NU]  (later f~)
  T* gs = q + ET * NFLD * DIM * NU;    // [ET][NG]
  T* chi = gs + ET * NG;               // MODE 1: [ET][2][NU]
  T* nus = chi + (MODE == 1 ? ET * 2 * NU : 0);  // MODE 1: [ET]
  unsigned char* lm = reinterpret_cast<unsigned char*>(nus + (MODE == 1 ? ET : 0));  // [ET][NF]

  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const T* ustg = reinterpret_cast<const T*>(A.ustg);
  const T* tr = reinterpret_cast<const T*>(A.tr);
  T* fc = reinterpret_cast<T*>(A.fc);
  T* rp = reinterpret_cast<T*>(A.rp);
  const int tid = threadIdx.x;
  const double tstage = A.use_dev_time ? A.dstate[DS_TIME] + rk_c(A.stage) * A.dt : A.t;

  load_ops<N, T>(A.ops, op);
  for (int idx = tid; idx < ne * NFLD * NU; idx += blockDim.x) {
    const int el = idx / (NFLD * NU), r = idx % (NFLD * NU), fld = r / NU, i = r % NU;
    us[idx] = ustg[((e0 + el) * 2 + F0 + fld) * NU + i];
  }
  for (int idx = tid; idx < ne * NG; idx += blockDim.x) gs[idx] = (T)A.geo[e0 * NG + idx];
  __syncthreads();

  // ---- Step 1 and the partner traces (Step 2 needs them) -------------------
  for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
    const int el = idx / NF, k = idx % NF;
    int a, s, b0;
    fline<DIM, N>(k, a, s, b0);
    const int32_t w = A.fnbr[(e0 + el) * NF + k];
    const int isL = w & 1;
    const int64_t pg = (int64_t)(w >> 1);
    const int64_t pe = pg / NF, pk = pg % NF;
    lm[el * NF + k] = (unsigned char)isL;
#pragma unroll
    for (int fld = 0; fld < NFLD; ++fld) {
      const T* ul = us + (el * NFLD + fld) * NU + b0;
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += op.lend[s][j] * ul[j * ipow(N, a)];
      uf[(el * NFLD + fld) * NF + k] = acc;
      uo[(el * NFLD + fld) * NF + k] = isL ? tr[(pe * 2 + F0 + fld) * NF + pk] : acc;
    }
  }
  __syncthreads();

  // ---- Step 3: corrected gradient at solution points -----------------------
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    T xi[3], Sm[3][3];
    upt_xi<DIM, N>(i, op.x, xi);
    const T dj = metric<DIM>(gs + el * NG, xi, Sm);
    const T rdj = (T)1 / dj;
#pragma unroll
    for (int fld = 0; fld < NFLD; ++fld) {
      const T* ul = us + (el * NFLD + fld) * NU;
      const T* fo = uo + (el * NFLD + fld) * NF;
      const T* ff = uf + (el * NFLD + fld) * NF;
      const unsigned char* L = lm + el * NF;
      T qt[3];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int ia = ucoord<N>(i, a), st = ipow(N, a), lb = i - ia * st;
        T acc = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += op.D[ia][j] * ul[lb + j * st];
        const int km = fpt_of<DIM, N>(i, a, 0), kp = fpt_of<DIM, N>(i, a, 1);
        const T jm = L[km] ? fo[km] - ff[km] : (T)0;
        const T jp = L[kp] ? fo[kp] - ff[kp] : (T)0;
        qt[a] = acc + op.gLd[ia] * jm + op.gRd[ia] * jp;
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        T v = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) v += Sm[a][b] * qt[a];
        q[((el * NFLD + fld) * DIM + b) * NU + i] = v * rdj;
      }
    }
  }
  // ---- MODE 1: resolution indicator on psi and element viscosity ----------
  if (MODE == 1) {
    // chi = (Vinv x ... x Vinv) psi by DIM line passes (ping-pong in chi)
    for (int pass = 0; pass < DIM; ++pass) {
      for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
        const int el = idx / NU, i = idx % NU;
        const T* src = pass == 0 ? us + el * NU : chi + (el * 2 + ((pass - 1) & 1)) * NU;
        T* dst = chi + (el * 2 + (pass & 1)) * NU;
        const int ia = ucoord<N>(i, pass), st = ipow(N, pass), lb = i - ia * st;
        T acc = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += op.Vinv[ia][j] * src[lb + j * st];
        dst[i] = acc;
      }
      __syncthreads();
    }
    for (int el = tid; el < ne; el += blockDim.x) {
      const T* c = chi + (el * 2 + ((DIM - 1) & 1)) * NU;
      double tot = 0.0, hi = 0.0;
      for (int i = 0; i < NU; ++i) {
        const double v = (double)c[i] * (double)c[i];
        tot += v;
        bool top = false;
#pragma unroll
        for (int a = 0; a < DIM; ++a) top = top || (ucoord<N>(i, a) == N - 1);
        if (top) hi += v;
      }
      double nu = 0.0;
      if (tot > 0.0 && hi > 0.0) {
        const double se = log10(hi / tot);
        const double lo = A.prm.s0 - A.prm.kappa, up = A.prm.s0 + A.prm.kappa;
        if (se < lo) nu = 0.0;
        else if (se > up) nu = A.prm.nu_max;
        else nu = 0.5 * A.prm.nu_max * (1.0 + sin(M_PI * (se - A.prm.s0) / (2.0 * A.prm.kappa)));
      }
      nus[el] = (T)nu;
    }
  }
  __syncthreads();

  // ---- Step 5 on L flux points (needs q^f, Eq. extrapolateGrad) ------------
  for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
    const int el = idx / NF, k = idx % NF;
    if (!lm[el * NF + k]) {
#pragma unroll
      for (int fld = 0; fld < NFLD; ++fld) cor[(el * NFLD + fld) * NF + k] = 0;
      continue;
    }
    int a, s, b0;
    fline<DIM, N>(k, a, s, b0);
    T xi[3], Sm[3][3];
    fpt_xi<DIM, N>(k, op.x, xi);
    metric<DIM>(gs + el * NG, xi, Sm);
    const T sg = s ? (T)1 : (T)-1;
    T pn[3], pm = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      pn[c] = sg * Sm[a][c];
      pm += pn[c] * pn[c];
    }
    pm = sqrt_(pm);
    T nh[3];
#pragma unroll
    for (int c = 0; c < DIM; ++c) nh[c] = pn[c] / pm;
    const int st = ipow(N, a);
    if (MODE == 0) {
      T qf[2][3];
#pragma unroll
      for (int fld = 0; fld < 2; ++fld)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const T* ql = q + ((el * 2 + fld) * DIM + c) * NU + b0;
          T acc = 0;
#pragma unroll
          for (int j = 0; j < N; ++j) acc += op.lend[s][j] * ql[j * st];
          qf[fld][c] = acc;
        }
      T x[3], v[3];
      map_point<S::ET_, T>(gs + el * NG, xi, x);
      velocity<DIM, T>(A.vel, x, tstage, v);
      T vn = 0, v2 = 0, g2 = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        vn += v[c] * nh[c];
        v2 += v[c] * v[c];
        g2 += qf[1][c] * qf[1][c];
      }
      const T M = fmax(sqrt_(v2), (T)A.prm.gamma);
      const T gm = fmax(sqrt_(g2), (T)A.prm.delta);
      const T pL = uf[(el * 2 + 0) * NF + k], pR = uo[(el * 2 + 0) * NF + k];
      const T sL = uf[(el * 2 + 1) * NF + k], sR = uo[(el * 2 + 1) * NF + k];
      const T sharp = (T)A.prm.gamma * pL * ((T)1 - pL) / gm;
      T fvn = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) fvn += nh[c] * M * ((T)A.prm.eps * qf[0][c] - sharp * qf[1][c]);
      const T Fp = (T)0.5 * (pL + pR) * vn - fvn + (T)A.prm.tau * (pL - pR);
      const T Fs = (T)0.5 * (sL + sR) * vn + (T)A.prm.tau_psi * (sL - sR);
      fc[((e0 + el) * 2 + 0) * NF + k] = Fp;
      fc[((e0 + el) * 2 + 1) * NF + k] = Fs;
      cor[(el * 2 + 0) * NF + k] = pm * Fp;
      cor[(el * 2 + 1) * NF + k] = pm * Fs;
    } else {
      T gn = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const T* ql = q + (el * DIM + c) * NU + b0;
        T acc = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += op.lend[s][j] * ql[j * st];
        gn += nh[c] * acc;
      }
      const T L_ = uf[el * NF + k], R_ = uo[el * NF + k];
      const T F = -nus[el] * gn + (T)A.prm.tau_pseudo * (L_ - R_);
      fc[((e0 + el) * 2 + 1) * NF + k] = F;
      cor[el * NF + k] = pm * F;
    }
  }
  __syncthreads();

  // ---- Step 4: transformed flux at solution points (in place of q) ---------
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    T xi[3], Sm[3][3];
    upt_xi<DIM, N>(i, op.x, xi);
    const T dj = metric<DIM>(gs + el * NG, xi, Sm);
    if (MODE == 0) {
      T x[3], v[3];
      map_point<S::ET_, T>(gs + el * NG, xi, x);
      velocity<DIM, T>(A.vel, x, tstage, v);
      T qp[3], qs[3], v2 = 0, g2 = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        qp[c] = q[((el * 2 + 0) * DIM + c) * NU + i];
        qs[c] = q[((el * 2 + 1) * DIM + c) * NU + i];
        v2 += v[c] * v[c];
        g2 += qs[c] * qs[c];
      }
      const T M = fmax(sqrt_(v2), (T)A.prm.gamma);
      const T gm = fmax(sqrt_(g2), (T)A.prm.delta);
      const T ph = us[(el * 2 + 0) * NU + i], ps = us[(el * 2 + 1) * NU + i];
      const T sharp = (T)A.prm.gamma * ph * ((T)1 - ph) / gm;
      T f0[3], f1[3];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        f0[c] = ph * v[c] - M * ((T)A.prm.eps * qp[c] - sharp * qs[c]);
        f1[c] = ps * v[c];
      }
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T t0 = 0, t1 = 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          t0 += Sm[a][c] * f0[c];
          t1 += Sm[a][c] * f1[c];
        }
        q[((el * 2 + 0) * DIM + a) * NU + i] = t0;
        q[((el * 2 + 1) * DIM + a) * NU + i] = t1;
      }
    } else {
      T qs[3], g2 = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        qs[c] = q[(el * DIM + c) * NU + i];
        g2 += qs[c] * qs[c];
      }
      const T nu = nus[el];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T t0 = 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) t0 += Sm[a][c] * (-nu * qs[c]);
        q[(el * DIM + a) * NU + i] = t0;
      }
      const T qm = sqrt_(g2);
      const T p0 = (T)A.psi0[(e0 + el) * NU + i];
      const T src = tanh_(p0 / fmax(qm, (T)A.prm.delta)) * ((T)1 - qm);
      us[el * NU + i] = src * dj;  // psi itself is no longer needed
    }
  }
  __syncthreads();

  // ---- Step 4/6: discontinuous normal flux and flux jump at flux points ---
  for (int idx = tid; idx < ne * NFLD * NF; idx += blockDim.x) {
    const int el = idx / (NFLD * NF), r = idx % (NFLD * NF), fld = r / NF, k = r % NF;
    int a, s, b0;
    fline<DIM, N>(k, a, s, b0);
    const T* fl = q + ((el * NFLD + fld) * DIM + a) * NU + b0;
    const int st = ipow(N, a);
    T acc = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) acc += op.lend[s][j] * fl[j * st];
    const T fperp = s ? acc : -acc;
    cor[idx] = cor[idx] - fperp;
  }
  __syncthreads();

  // ---- Step 6: divergence with the lift of the known flux jumps ------------
  for (int idx = tid; idx < ne * NFLD * NU; idx += blockDim.x) {
    const int el = idx / (NFLD * NU), r = idx % (NFLD * NU), fld = r / NU, i = r % NU;
    const T* cr = cor + (el * NFLD + fld) * NF;
    T div = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int ia = ucoord<N>(i, a), st = ipow(N, a), lb = i - ia * st;
      const T* fl = q + ((el * NFLD + fld) * DIM + a) * NU;
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += op.D[ia][j] * fl[lb + j * st];
      div += acc - op.gLd[ia] * cr[fpt_of<DIM, N>(i, a, 0)] + op.gRd[ia] * cr[fpt_of<DIM, N>(i, a, 1)];
    }
    if (MODE == 1) div -= us[el * NU + i];
    rp[((e0 + el) * 2 + F0 + fld) * NU + i] = div;
  }
}

// ============================================================================
template <int DIM, int N, typename T, int MODE>
struct KALayout {
  using S = TS<DIM, N>;
  static constexpr int NFLD = MODE == 0 ? 2 : 1;
  static constexpr int BYTES_EL = (NFLD * S::NU + NFLD * S::NF + S::NG) * (int)sizeof(T);
  static constexpr int ETr = 24576 / BYTES_EL;
  static constexpr int ET = ETr < 1 ? 1 : (ETr > 64 ? 64 : ETr);
  static constexpr size_t SMEM = (size_t)ET * BYTES_EL + sizeof(SOps<N, T>) + 64;
};

// ka_tensor: R-side lift, du/dt, RK4 update, next-stage traces.
// stage -1 writes du/dt to A.out (fp64) and leaves the state alone;
// stage 0 only recomputes the traces of ustg.
template <int DIM, int N, typename T, int MODE>
__global__ void __launch_bounds__(kThreads) ka_tensor(const KArgs A) {
  using S = TS<DIM, N>;
  using LY = KALayout<DIM, N, T, MODE>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, NFLD = LY::NFLD, ET = LY::ET;
  constexpr int F0 = MODE == 0 ? 0 : 1;
  if (MODE == 1 && *(volatile int32_t*)&A.status[ST_PSEUDO_DONE]) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  SOps<N, T>& op = *reinterpret_cast<SOps<N, T>*>(smem_raw);
  T* base = reinterpret_cast<T*>(smem_raw + ((sizeof(SOps<N, T>) + 15) & ~size_t(15)));
  T* ys = base;                   // [ET][NFLD][NU]
  T* cr = ys + ET * NFLD * NU;    // [ET][NFLD][NF]
  T* gs = cr + ET * NFLD * NF;    // [ET][NG]

  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  T* ustg = reinterpret_cast<T*>(A.ustg);
  T* tr = reinterpret_cast<T*>(A.tr);
  const T* fc = reinterpret_cast<const T*>(A.fc);
  const T* rp = reinterpret_cast<const T*>(A.rp);
  const int tid = threadIdx.x;
  const int stage = A.stage;

  load_ops<N, T>(A.ops, op);
  for (int idx = tid; idx < ne * NG; idx += blockDim.x) gs[idx] = (T)A.geo[e0 * NG + idx];
  for (int idx = tid; idx < ne * NFLD * NU; idx += blockDim.x) {
    const int el = idx / (NFLD * NU), r = idx % (NFLD * NU), fld = r / NU, i = r % NU;
    const int64_t g = ((e0 + el) * 2 + F0 + fld) * NU + i;
    ys[idx] = stage == 0 ? ustg[g] : rp[g];
  }
  __syncthreads();

  double sq = 0.0;
  if (stage != 0) {
    // ---- common flux on R flux points: minus L's physical flux, this side's metric
    for (int idx = tid; idx < ne * NF; idx += blockDim.x) {
      const int el = idx / NF, k = idx % NF;
      const int32_t w = A.fnbr[(e0 + el) * NF + k];
      if (w & 1) {
#pragma unroll
        for (int fld = 0; fld < NFLD; ++fld) cr[(el * NFLD + fld) * NF + k] = 0;
        continue;
      }
      const int64_t pg = (int64_t)(w >> 1), pe = pg / NF, pk = pg % NF;
      T xi[3], Sm[3][3];
      fpt_xi<DIM, N>(k, op.x, xi);
      metric<DIM>(gs + el * NG, xi, Sm);
      const int a = (k / S::NFP) >> 1;
      T pm = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) pm += Sm[a][c] * Sm[a][c];
      pm = sqrt_(pm);
#pragma unroll
      for (int fld = 0; fld < NFLD; ++fld)
        cr[(el * NFLD + fld) * NF + k] = -pm * fc[(pe * 2 + F0 + fld) * NF + pk];
    }
    __syncthreads();
    // ---- du/dt and the RK4 register update
    for (int idx = tid; idx < ne * NFLD * NU; idx += blockDim.x) {
      const int el = idx / (NFLD * NU), r = idx % (NFLD * NU), fld = r / NU, i = r % NU;
      const T* c = cr + (el * NFLD + fld) * NF;
      T div = ys[idx];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int ia = ucoord<N>(i, a);
        div += -op.gLd[ia] * c[fpt_of<DIM, N>(i, a, 0)] + op.gRd[ia] * c[fpt_of<DIM, N>(i, a, 1)];
      }
      T xi[3], Sm[3][3];
      upt_xi<DIM, N>(i, op.x, xi);
      const T dj = metric<DIM>(gs + el * NG, xi, Sm);
      const double R = (double)(-div / dj);
      const int64_t g = ((e0 + el) * 2 + F0 + fld) * NU + i;
      if (stage < 0) {
        A.out[(int64_t)(F0 + fld - F0) * A.E * NU + (e0 + el) * NU + i] = R;
        continue;
      }
      double uu = A.u[g], aa = stage == 1 ? 0.0 : A.acc[g];
      const double uold = uu;
      const double y = rk_update(stage, A.dt, R, uu, aa);
      if (stage < 4) A.acc[g] = aa;
      else A.u[g] = uu;
      if (MODE == 1 && stage == 4) {
        const double d = (uu - uold) / A.dt;
        sq += d * d;
      }
      if (!isfinite(y)) atomicExch(&A.status[ST_STATUS], -4);
      const T yt = (T)y;
      ustg[g] = yt;
      ys[idx] = yt;
    }
    __syncthreads();
  }
  if (stage >= 0) {
    // ---- flux-point traces of the new stage input (Step 1 of the next stage)
    for (int idx = tid; idx < ne * NFLD * NF; idx += blockDim.x) {
      const int el = idx / (NFLD * NF), r = idx % (NFLD * NF), fld = r / NF, k = r % NF;
      int a, s, b0;
      fline<DIM, N>(k, a, s, b0);
      const T* yl = ys + (el * NFLD + fld) * NU + b0;
      const int st = ipow(N, a);
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += op.lend[s][j] * yl[j * st];
      tr[((e0 + el) * 2 + F0 + fld) * NF + k] = acc;
    }
  }
  if (MODE == 0 && stage == 4 && A.use_dev_time && blockIdx.x == 0 && tid == 0)
    A.dstate[DS_TIME] = A.dstate[DS_TIME] + A.dt;
  if (MODE == 1 && stage == 4) pseudo_rms_finish(A, block_sum(sq, red_sh), red_sh, A.E * NU);
}

}  // namespace frp
