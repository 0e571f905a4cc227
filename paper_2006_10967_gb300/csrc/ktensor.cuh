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
#include <type_traits>

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

// Affine elements (no cross terms in the map) have one metric per element;
// kernels cache it per tile: mc[el] = {S (3x3), det J}, aff[el] = 1.
template <int DIM, typename T>
__device__ __forceinline__ bool is_affine(const T* g) {
  constexpr int NC = DIM == 2 ? 4 : 8;
  bool aff = true;
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int k = DIM + 1; k < NC; ++k) aff = aff && g[c * NC + k] == (T)0;
  return aff;
}

// Metric terms at xi: from the element's precomputed record when the element
// is affine (mc: adj J row-major, det J, 1/det J, affine flag, ...; see
// k_metric_const), else from its geometry.  Returns det J; rdj, when given,
// receives 1/det J.
template <int DIM, typename T>
__device__ __forceinline__ T metric_c(const T* g, const T* xi, T S[3][3], const T* mc, T* rdj = nullptr) {
  if (mc[11] != (T)0) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) S[a][b] = mc[a * 3 + b];
    if (rdj) *rdj = mc[10];
    return mc[9];
  }
  const T dj = metric<DIM>(g, xi, S);
  if (rdj) *rdj = (T)1 / dj;
  return dj;
}

// One element's metric for the per-point loops of a line pass, where all of
// a thread's points lie in one element.  Quads hold the six bilinear Jacobian
// coefficients in registers (an affine map has a zero cross coefficient), so
// the per-point metric needs no shared-memory reads; with lanes spanning
// several elements those reads conflict (element records 8 and 16 words
// apart share banks).  Hexes, whose kernels have no registers to spare,
// read the record and geometry per point.
template <int DIM, typename T>
struct LineMetric {
  const T* g;
  const T* mc;
  __device__ __forceinline__ void load(const T* g_, const T* mc_) {
    g = g_;
    mc = mc_;
  }
  __device__ __forceinline__ T at(const T* xi, T S[3][3], T* rdj = nullptr) const {
    return metric_c<DIM>(g, xi, S, mc, rdj);
  }
};
template <typename T>
struct LineMetric<2, T> {
  T k[2][3];  // d x_c / d xi = k[c][0] + k[c][2] eta, d x_c / d eta = k[c][1] + k[c][2] xi
  __device__ __forceinline__ void load(const T* g, const T*) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      k[c][0] = g[c * 4 + 1];
      k[c][1] = g[c * 4 + 2];
      k[c][2] = g[c * 4 + 3];
    }
  }
  __device__ __forceinline__ T at(const T* xi, T S[3][3], T* rdj = nullptr) const {
    T J[3][3];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      J[c][0] = k[c][0] + k[c][2] * xi[1];
      J[c][1] = k[c][1] + k[c][2] * xi[0];
    }
    const T dj = adjugate<2, T>(J, S);
    if (rdj) *rdj = (T)1 / dj;
    return dj;
  }
};

// Per-element metric record (kMetricRec values of the bulk type), computed
// once per field from the element geometry: [0..8] the metric at the
// reference centre, [9] its determinant, [10] the reciprocal, [11] whether
// the map is affine (then [0..10] hold everywhere in the element; 2: affine
// with a diagonal Jacobian, so that separable velocity fields come from
// per-axis tables), [12..13] 1/W with W = sum_i w_i det J_i the element's
// quadrature area (FP64 value split into two bulk-type parts).  The residual
// kernel stages only the first kKbRec values.
constexpr int kKbRec = 12;  // metric-record values the residual kernel stages

template <int DIM, typename T>
__global__ void k_metric_const(const KArgs A, int NG, int NU) {
  T* mc = reinterpret_cast<T*>(A.mcg);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A.E; e += (int64_t)gridDim.x * blockDim.x) {
    const T* g = geo_of<T>(A) + e * NG;
    T xi[3] = {0, 0, 0}, S[3][3];
    const T dj = metric<DIM>(g, xi, S);
    T* o = mc + e * kMetricRec;
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) o[p * 3 + q] = (p < DIM && q < DIM) ? S[p][q] : (T)0;
    o[9] = dj;
    o[10] = (T)1 / dj;
    double W = 0.0;
    for (int i = 0; i < NU; ++i) W += A.wdet[e * NU + i];
    const double rW = 1.0 / W;
    o[12] = (T)rW;
    o[13] = (T)(rW - (double)o[12]);
    // [11]: 2 when the affine map also has a diagonal Jacobian (x_c a
    // function of xi_c alone)
    const bool aff = is_affine<DIM>(g);
    bool diag = aff;
    for (int c = 0; c < DIM; ++c)
      for (int b = 0; b < DIM; ++b)
        if (b != c) diag = diag && g[c * (DIM == 2 ? 4 : 8) + 1 + b] == (T)0;
    o[11] = diag ? (T)2 : (aff ? (T)1 : (T)0);
    o[14] = o[15] = (T)0;
  }
}

// Lines: along axis a, line l runs through the solution points whose other
// coordinates (in increasing axis order, lowest fastest) encode l; it ends
// at flux point l of faces (a, -) and (a, +).
template <int DIM, int N>
__device__ __forceinline__ int line_base(int a, int l) {
  int base = 0, r = l;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (b == a) continue;
    base += (r % N) * ipow(N, b);
    r /= N;
  }
  return base;
}

// Largest tile (elements) <= cap whose thread count ET*LN fills whole warps,
// when such a tile exists; otherwise cap.
__host__ __device__ constexpr int gcd_(int a, int b) { return b == 0 ? a : gcd_(b, a % b); }
__host__ __device__ constexpr int warp_tile(int cap, int ln) {
  return (cap / (32 / gcd_(ln, 32))) > 0 ? (cap / (32 / gcd_(ln, 32))) * (32 / gcd_(ln, 32)) : cap;
}

// Field split: on the physical step (two fields) the line passes give each
// thread one line of one field, in separate warps, so that twice the warps
// are in flight; MINB asks the compiler for registers that let MINB blocks
// share an SM.
#ifndef FRP_FIELD_SPLIT
#define FRP_FIELD_SPLIT 0
#endif
template <int THREADS, typename T>
struct MinBlocks {
  static constexpr int v = sizeof(T) == 8 ? 1 : (1280 / THREADS < 1 ? 1 : (1280 / THREADS > 8 ? 8 : 1280 / THREADS));
};

// Where a kernel finds its partner's face values.  Quads (FaceScatter):
// the producer writes each value into the slot of the element that reads it
// (ka_tensor a trace into the L-side partner's slot, kb_tensor a common flux
// into the R-side partner's slot as well as its own), so both kernels read
// their partner values from their own slots with loads that do not wait for
// the connectivity.  Hexes: each value stays in its owner's slot and the
// reader gathers it through the connectivity (the scattered stores into
// arrays larger than L2 cost more than the gathers save).
template <int DIM>
struct FaceScatter {
  static constexpr bool v = DIM == 2;
};

// Blocks of `bytes` dynamic shared memory that fit on one SM (228 KB, 1 KB
// reserved per block), at most 32.
__host__ __device__ constexpr int smem_blocks(long bytes) {
  return 233472 / (bytes + 1024) > 32 ? 32 : (int)(233472 / (bytes + 1024));
}
// Tile (elements per block, <= cap) that keeps the most active lanes resident
// on an SM under the shared-memory and thread limits, counting at most 32
// warps (beyond that the register file decides); ties go to the larger tile.
__host__ __device__ constexpr int occupancy_tile(int bytes_el, int per_block, int ln, int cap) {
  int best = 1;
  long best_lanes = -1;
  for (int et = 1; et <= cap; ++et) {
    const int threads = (et * ln + 31) / 32 * 32;
    int b = smem_blocks((long)et * bytes_el + per_block);
    if (b * threads > 2048) b = 2048 / threads;
    long lanes = (long)b * et * ln;
    if (lanes > 32 * 32) lanes = 32 * 32;
    if (lanes >= best_lanes) {
      best_lanes = lanes;
      best = et;
    }
  }
  return best;
}

// TD: tile divisor of a kernel variant (1: the default tile below; 2: half
// of it, rounded to whole warps where possible), chosen per element type,
// order and precision by the autotuner.
template <int DIM, int N, typename T, int MODE, int TD = 1>
struct KBLayout {
  using S = TS<DIM, N>;
  static constexpr int NFLD = MODE == 0 ? 2 : 1;
  static constexpr int LN = S::NFP;  // lines per axis per element
  // Quads stage the velocity cache tiles in shared memory with the state;
  // hexes read them from global memory where they are used, since the tiles
  // would take a third of the element's shared memory and cut the resident
  // warps from 28 to 16 (N = 4).
  static constexpr bool VT = MODE == 0 && DIM == 2;
  static constexpr int PER_EL_T = NFLD * S::NU          // u, later the divergence
                                  + NFLD * DIM * S::NU  // q~ -> q -> f~
                                  + 2 * NFLD * S::NF    // uo, cor
                                  + S::NG + kKbRec  // geometry, metric record (first kKbRec values)
                                  + (VT ? DIM * (S::NU + S::NF) : 0)  // velocity cache tiles
                                  + (MODE == 0 ? DIM * (N + 2) * 2 : 0)  // separable velocity tables
                                  + (MODE == 1 ? 2 * S::NU + 1 : 0);  // modal ping-pong / source, nu_s
  static constexpr int BYTES_EL = PER_EL_T * (int)sizeof(T) + 2 * S::NF;  // + L list
  static constexpr int ET_T = 256 / LN < 1 ? 1 : 256 / LN;
  static constexpr int ET_S = 57344 / BYTES_EL < 1 ? 1 : 57344 / BYTES_EL;
  static constexpr bool OCC = MODE == 0 && DIM == 3;  // tile chosen for resident warps
  static constexpr int ET0 = OCC ? occupancy_tile(BYTES_EL, 16 * 13 + 2 * (int)sizeof(T) + 64, LN, ET_T)
                                 : warp_tile(ET_T < ET_S ? ET_T : ET_S, LN);
  static constexpr int ET = TD == 1 ? ET0 : (ET0 / TD < 1 ? 1 : warp_tile(ET0 / TD, LN));
  static constexpr int FS = FRP_FIELD_SPLIT ? NFLD : 1;  // fields split across threads
  static constexpr int LINES = ET * LN;
  static constexpr int THREADS = (LINES * FS + 31) / 32 * 32;  // whole warps; idle lanes inactive
  static constexpr size_t SMEM = (size_t)ET * BYTES_EL + 16 * 13;  // + region alignment
  static_assert(ET * S::NF < 0x8000, "L-list entries keep bit 15 for the wall flag");
  static constexpr int SMB = smem_blocks((long)SMEM + ET * 2 * (int)sizeof(T) + 64);
  static constexpr int MINB = OCC && SMB < MinBlocks<THREADS, T>::v ? SMB : MinBlocks<THREADS, T>::v;
};

// ============================================================================
// kb_tensor: Steps 1-6 on a tile of ET elements.  Line passes give each
// thread one solution-point line; the 1D operators are read from the kernel
// parameters (constant bank) with compile-time indices.
template <int DIM, int N, typename T, int MODE, int TD = 1>
__device__ __forceinline__ void kb_tensor_body(const KArgs& A, const int blk) {
  using S = TS<DIM, N>;
  using LY = KBLayout<DIM, N, T, MODE, TD>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, NFP = S::NFP, NFLD = LY::NFLD, ET = LY::ET, LN = LY::LN;
  constexpr int FS = LY::FS, NQ = NFLD / FS;  // fields per thread in the line passes
  constexpr int F0 = MODE == 0 ? 0 : 1;
  constexpr bool kFuse4 = (N % 2) == 1;  // Step 4 inside the axis-0 pass of Step 6
  static_assert(FS == 1, "the line passes assume one thread per line for all fields");
  if (MODE == 1 && *(volatile int32_t*)&A.status[ST_PSEUDO_DONE]) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemCarve sc{smem_raw};
  T* us = sc.take<T>(ET * NFLD * NU);         // [ET][NFLD][NU]
  T* qt = sc.take<T>(ET * NFLD * DIM * NU);   // [ET][NFLD][DIM][NU]
  T* uo = sc.take<T>(ET * NFLD * NF);         // [ET][NFLD][NF] partner traces (own trace at R points)
  T* cor = sc.take<T>(ET * NFLD * NF);        // [ET][NFLD][NF]
  T* gs = sc.take<T>(ET * NG);                // [ET][NG]
  T* mcs = sc.take<T>(ET * kKbRec);           // [ET][kKbRec] metric records
  T* vu = sc.take<T>(LY::VT ? ET * DIM * NU : 0);  // velocity cache tiles, solution points
  T* vf = sc.take<T>(LY::VT ? ET * DIM * NF : 0);  // velocity cache tiles, flux points
  T* chi = sc.take<T>(MODE == 1 ? ET * 2 * NU : 0);   // MODE 1: [ET][2][NU]
  T* nus = sc.take<T>(MODE == 1 ? ET : 0);
  constexpr int NT = N + 2;                           // velocity table entries per axis
  T* vtab = sc.take<T>(MODE == 0 ? ET * DIM * NT * 2 : 0);  // [ET][DIM][NT][2]
  uint16_t* llist = sc.take<uint16_t>(ET * NF);       // [ET*NF] L flux points

  const int64_t e0 = (int64_t)blk * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  const T* ustg = reinterpret_cast<const T*>(A.ustg);
  const T* tr = reinterpret_cast<const T*>(A.tr);
  T* fc = reinterpret_cast<T*>(A.fc);
  T* rp = reinterpret_cast<T*>(A.rp);
  const int tid = threadIdx.x;
  const BulkConst<T>& BC = bulk<T>(A);
  const TensorOpsT<T>& O = BC.ops;
  const PrmT<T> P = BC.prm;
  __shared__ T gfac_s;
  __shared__ T gfe[ET], epe[ET];  // per-element time factor and eps (batched instances)
  __shared__ int nL;
  if (tid == 0) {
    nL = 0;
    const double tstage = A.use_dev_time ? A.dstate[DS_TIME] + rk_c(A.stage) * A.dt : A.t;
    gfac_s = time_factor_t<T>(A, tstage);
  }
  if (A.ep)
    for (int el = tid; el < ne; el += blockDim.x) {
      const ElemPar& ep = A.ep[e0 + el];
      gfe[el] = time_factor_t<T>(A, ep.t + rk_c(A.stage) * ep.dt);
      epe[el] = (T)ep.eps;
    }
  // line-pass role: line (lel, ll) of the fields fsel + q FS, q < NQ
  const int fsel = tid / LY::LINES, lin = tid % LY::LINES;
  const int lel = lin / LN, ll = lin % LN;
  const bool lact = lel < ne && fsel < FS;  // false on the idle lanes of a padded last warp
  // Prefetch this thread's line-end connectivity and partner traces for all
  // axis passes.  With FaceScatter the trace array holds the partner's trace
  // at each L flux point and both loads are independent; otherwise the
  // partner traces are gathered below, after the tile copies are issued.
  // Hexahedra read one face word per line end (face_link) instead of the
  // per-point connectivity, decoded below once the tile copies are issued;
  // wpre then holds the flags (bit 0 L side, bit 1 wall).
  int32_t wpre[DIM][2];
  T opre[DIM][2][NQ];
  [[maybe_unused]] int2 fwr[DIM][2];
  if (lact) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int k = (2 * a + sd) * NFP + ll;
        if constexpr (DIM == 3) {
          fwr[a][sd] = __ldg(A.ffw + (e0 + lel) * 6 + 2 * a + sd);
        } else {
          wpre[a][sd] = A.fnbr[(e0 + lel) * NF + k];
          if constexpr (FaceScatter<DIM>::v)
#pragma unroll
            for (int q = 0; q < NQ; ++q) opre[a][sd][q] = tr[((e0 + lel) * 2 + F0 + fsel + q * FS) * NF + k];
        }
      }
  }
  // contiguous tiles: state (both fields), geometry, velocity cache; all in
  // flight together with the connectivity loads above
  if (MODE == 0) tile_async(us, ustg + e0 * 2 * NU, ne * 2 * NU * (int)sizeof(T));
  tile_async(gs, geo_of<T>(A) + e0 * NG, ne * NG * (int)sizeof(T));
  {
    // the first kKbRec values of each record, in 16-byte granules
    constexpr int G = kKbRec * (int)sizeof(T) / 16;
    const T* src = reinterpret_cast<const T*>(A.mcg) + e0 * kMetricRec;
    for (int t = tid; t < ne * G; t += blockDim.x)
      cp_async_16(mcs + (t / G) * kKbRec + (t % G) * (16 / (int)sizeof(T)),
                  src + (t / G) * kMetricRec + (t % G) * (16 / (int)sizeof(T)));
  }
  const T* vsu = reinterpret_cast<const T*>(A.vsu);
  const T* vsf = reinterpret_cast<const T*>(A.vsf);
  if (LY::VT && A.vsu) tile_async(vu, vsu + e0 * DIM * NU, ne * DIM * NU * (int)sizeof(T));
  if (LY::VT && A.vsf) tile_async(vf, vsf + e0 * DIM * NF, ne * DIM * NF * (int)sizeof(T));
  if constexpr (DIM == 3) {
    if (lact) {
      const int fi = ll % N, fj = ll / N;
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          int32_t fl;
          const int32_t po = face_link<N, NF>(A, fwr[a][sd], e0 + lel, 2 * a + sd, fi, fj, fl);
          wpre[a][sd] = fl;
#pragma unroll
          for (int q = 0; q < NQ; ++q) opre[a][sd][q] = (fl & 1) ? tr[po + (F0 + fsel + q * FS) * NF] : (T)0;
        }
    }
  }
  if (MODE == 1)
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, i = idx % NU;
      us[idx] = ustg[((e0 + el) * 2 + F0) * NU + i];
    }
  cp_async_wait_all();
  __syncthreads();
  const T gfac = gfac_s;
  // separable velocity: per-axis tables of the elements with a diagonal map
  // (read after the first axis pass's barrier)
  const bool sepk = MODE == 0 && vel_separable(BC.vel.kind);
  if (sepk)
    for (int t = tid; t < ne * DIM * NT; t += blockDim.x) {
      const int el = t / (DIM * NT), r = t % (DIM * NT), c = r / NT, j = r % NT;
      if (mcs[el * kKbRec + 11] != (T)2) continue;
      const T* g = gs + el * NG + c * S::NC;
      const T xi = j < N ? O.x[j] : (j == N ? (T)-1 : (T)1);
      vel_tab_entry<T>(BC.vel.kind, g[0] + g[1 + c] * xi, vtab + (el * DIM * NT + r) * 2);
    }
  auto tab_of = [&](int el) -> bool { return sepk && mcs[el * kKbRec + 11] == (T)2; };

  // ---- Steps 1-3, one pass per axis: traces at the line ends, partner
  //      traces (Step 2), reference derivative plus the two end corrections;
  //      the last pass maps q~ to the physical gradient q = J^{-T} q~.
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (lact) {
      const int st = ipow(N, a);
      const int base = line_base<DIM, N>(a, ll);
      const int k0 = (2 * a) * NFP + ll, k1 = k0 + NFP;
      const int32_t w0 = wpre[a][0], w1 = wpre[a][1];
      if (fsel == 0) {
        // L points go to the compacted list of Step 5; R points get no flux here
        // entry: tile flux point, bit 15 set at walls (own partner)
        const int64_t g0 = (e0 + lel) * NF + k0, g1 = (e0 + lel) * NF + k1;
        const bool wl0 = DIM == 3 ? (w0 & 2) != 0 : (w0 >> 1) == g0;
        const bool wl1 = DIM == 3 ? (w1 & 2) != 0 : (w1 >> 1) == g1;
        if (w0 & 1) llist[atomicAdd(&nL, 1)] = (uint16_t)((lel * NF + k0) | (wl0 ? 0x8000 : 0));
        if (w1 & 1) llist[atomicAdd(&nL, 1)] = (uint16_t)((lel * NF + k1) | (wl1 ? 0x8000 : 0));
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int fld = fsel + q * FS;
        const T* ul = us + (lel * NFLD + fld) * NU + base;
        T v[N];
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = ul[j * st];
        T f0 = 0, f1 = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          f0 += O.lend[0][j] * v[j];
          f1 += O.lend[1][j] * v[j];
        }
        const T o0 = (w0 & 1) ? opre[a][0][q] : f0;
        const T o1 = (w1 & 1) ? opre[a][1][q] : f1;
        const int fo = (lel * NFLD + fld) * NF;
        uo[fo + k0] = o0;
        uo[fo + k1] = o1;
        // the own trace at L points (Step 5 reads it, then overwrites it with
        // the common flux); no correction at R points in kb
        cor[fo + k0] = (w0 & 1) ? f0 : (T)0;
        cor[fo + k1] = (w1 & 1) ? f1 : (T)0;
        const T jm = o0 - f0, jp = o1 - f1;
        T* qa = qt + ((lel * NFLD + fld) * DIM + a) * NU + base;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T acc = O.gLd[j] * jm + O.gRd[j] * jp;
#pragma unroll
          for (int m = 0; m < N; ++m) acc += O.D[j][m] * v[m];
          qa[j * st] = acc;
        }
      }
      if (MODE == 1) {
        // resolution indicator: chi = (Vinv x ... x Vinv) psi, one axis per pass
        const T* src = a == 0 ? us + lel * NU : chi + (lel * 2 + ((a - 1) & 1)) * NU;
        T* dst = chi + (lel * 2 + (a & 1)) * NU;
        T v[N];
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = src[base + j * st];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T acc = 0;
#pragma unroll
          for (int m = 0; m < N; ++m) acc += O.Vinv[j][m] * v[m];
          dst[base + j * st] = acc;
        }
      }
      if (a == DIM - 1 && DIM == 3 && mcs[lel * kKbRec + 11] == (T)2) {
        // physical gradient, diagonal metric (axis-aligned affine element):
        // q_b = S_bb q~_b / det J
        const T* mcl = mcs + lel * kKbRec;
        const T sd[3] = {mcl[0], mcl[4], mcl[8]}, rdj = mcl[10];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int i = base + j * st;
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            T* qp = qt + (lel * NFLD + fsel + q * FS) * DIM * NU + i;
#pragma unroll
            for (int b = 0; b < DIM; ++b) qp[b * NU] = (sd[b] * qp[b * NU]) * rdj;
          }
        }
      } else if (a == DIM - 1) {
        // physical gradient at this line's points (all axes are done)
        LineMetric<DIM, T> em;
        em.load(gs + lel * NG, mcs + lel * kKbRec);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int i = base + j * st;
          T xi[3], Sm[3][3];
          upt_xi<DIM, N>(i, O.x, xi);
          T rdj;
          em.at(xi, Sm, &rdj);
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            T* qp = qt + (lel * NFLD + fsel + q * FS) * DIM * NU + i;
            T qv[3];
#pragma unroll
            for (int c = 0; c < DIM; ++c) qv[c] = qp[c * NU];
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
              T r = 0;
#pragma unroll
              for (int c = 0; c < DIM; ++c) r += Sm[c][b] * qv[c];
              qp[b * NU] = r * rdj;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if (MODE == 1) {
    for (int el = tid; el < ne; el += blockDim.x) {
      const T* c = chi + (el * 2 + ((DIM - 1) & 1)) * NU;
      double tot = 0.0, hi = 0.0;
      for (int i = 0; i < NU; ++i) {
        const double v = (double)c[i] * (double)c[i];
        tot += v;
        bool top = false;
#pragma unroll
        for (int b = 0; b < DIM; ++b) top = top || (ucoord<N>(i, b) == N - 1);
        if (top) hi += v;
      }
      double nu = 0.0;
      const double nmax = A.ep ? (double)A.ep[e0 + el].nu_max : A.prm.nu_max;
      if (tot > 0.0 && hi > 0.0) {
        const double se = log10(hi / tot);
        const double lo = A.prm.s0 - A.prm.kappa, up = A.prm.s0 + A.prm.kappa;
        if (se < lo) nu = 0.0;
        else if (se > up) nu = nmax;
        else nu = 0.5 * nmax * (1.0 + sin(M_PI * (se - A.prm.s0) / (2.0 * A.prm.kappa)));
      }
      nus[el] = (T)nu;
    }
    __syncthreads();
  }

  // ---- Step 5 on L flux points (q^f by Eq. extrapolateGrad) ----------------
  const int nLpts = nL;
  for (int t = tid; t < nLpts; t += blockDim.x) {
    const int code = llist[t] & 0x7fff;
    const bool wallp = (llist[t] >> 15) != 0;  // wall point (own partner)
    const int el = code / NF, k = code % NF;
    // partner flux point: the common flux also goes to its slot on quads,
    // where the partner's ka_tensor lifts it (a wall point is its own partner)
    const int64_t og = (e0 + el) * NF + k;
    const int64_t pg = FaceScatter<DIM>::v ? (int64_t)partner<NF>(A, A.fnbr[og], (int32_t)og) : og;
    const int64_t pslot = (pg / NF) * 2 * NF + pg % NF;
    int a, s, b0;
    fline<DIM, N>(k, a, s, b0);
    T xi[3];
    fpt_xi<DIM, N>(k, O.x, xi);
    const T sg = s ? (T)1 : (T)-1;
    // transformed face normal: row a of S = det J J^{-1} (from the record on
    // affine elements)
    const T* mcl = mcs + el * kKbRec;
    const int st = ipow(N, a);
    if (MODE == 0 && DIM == 3 && mcl[11] == (T)2) {
      // diagonal metric (axis-aligned affine element): the transformed normal
      // is sg S_aa e_a, so only the normal components of the fluxes enter,
      // and the viscous flux needs q_phi along axis a and the full gradient
      // that gives the interface normal (for |q|)
      const T saa = mcl[a * 4];
      const T nha = (sg * saa > (T)0) ? (T)1 : (T)-1;
      const T pm = fabs(saa);
      const int kn = P.nphi ? 0 : 1;
      T qn[3];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const T* ql = qt + ((el * 2 + kn) * DIM + c) * NU + b0;
        T acc = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += (s ? O.lend[1][j] : O.lend[0][j]) * ql[j * st];
        qn[c] = acc;
      }
      const T qna = a == 0 ? qn[0] : (a == 1 ? qn[1] : qn[2]);
      T qpa = qna;
      if (!P.nphi) {
        const T* ql = qt + ((el * 2 + 0) * DIM + a) * NU + b0;
        T acc = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += (s ? O.lend[1][j] : O.lend[0][j]) * ql[j * st];
        qpa = acc;
      }
      T v[3];
      const T gel = A.ep ? gfe[el] : gfac;
      const T epsel = A.ep ? epe[el] : P.eps;
      if (tab_of(el)) {
        int jj[3];
#pragma unroll
        for (int b = 0; b < DIM; ++b) jj[b] = b == a ? N + s : ucoord<N>(b0, b);
        velocity_tab<DIM, NT, T>(BC.vel, vtab + el * DIM * NT * 2, jj, gel, v);
      } else if (A.vsf) {
        const T* vc = LY::VT ? vf + el * DIM * NF + k : vsf + (e0 + el) * DIM * NF + k;
#pragma unroll
        for (int c = 0; c < DIM; ++c) v[c] = gel * vc[c * NF];
      } else {
        T x[3];
        map_point<S::ET_, T>(gs + el * NG, xi, x);
        velocity<DIM, T>(BC.vel, x, gel, v);
      }
      const T va = a == 0 ? v[0] : (a == 1 ? v[1] : v[2]);
      T v2 = 0, g2 = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        v2 += v[c] * v[c];
        g2 += qn[c] * qn[c];
      }
      const T M = fmax(sqrt_(v2), P.gamma);
      const T gm = fmax(sqrt_(g2), P.delta);
      const T pL = cor[(el * 2 + 0) * NF + k], sL = cor[(el * 2 + 1) * NF + k];
      const T pR = uo[(el * 2 + 0) * NF + k], sR = uo[(el * 2 + 1) * NF + k];
      const T sharp = P.gamma * pL * ((T)1 - pL) / gm;
      const T vn = nha * va;
      const T fvn = nha * (epsel * qpa - sharp * qna);
      const bool shut = P.noflux && wallp;
      const T Fp = shut ? (T)0 : (T)0.5 * (pL + pR) * vn - M * fvn + P.tau * (pL - pR);
      const T Fs = shut ? (T)0 : (T)0.5 * (sL + sR) * vn + P.tau_psi * (sL - sR);
      const T Fp_t = pm * Fp, Fs_t = pm * Fs;
      fc[((e0 + el) * 2 + 0) * NF + k] = Fp_t;
      fc[((e0 + el) * 2 + 1) * NF + k] = Fs_t;
      if (FaceScatter<DIM>::v && !wallp) {
        fc[pslot] = Fp_t;
        fc[pslot + NF] = Fs_t;
      }
      cor[(el * 2 + 0) * NF + k] = Fp_t;
      cor[(el * 2 + 1) * NF + k] = Fs_t;
      continue;
    }
    T srow[3];
    if (mcl[11] != (T)0) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) srow[c] = mcl[a * 3 + c];
    } else {
      T Sm[3][3];
      metric<DIM>(gs + el * NG, xi, Sm);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        T sac = Sm[0][c];
#pragma unroll
        for (int b = 1; b < DIM; ++b)
          if (b == a) sac = Sm[b][c];
        srow[c] = sac;
      }
    }
    T pn[3], pm = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      pn[c] = sg * srow[c];
      pm += pn[c] * pn[c];
    }
    pm = sqrt_(pm);
    const T rpm = (T)1 / pm;
    T nh[3];
#pragma unroll
    for (int c = 0; c < DIM; ++c) nh[c] = pn[c] * rpm;
    if (MODE == 0) {
      T qf[2][3];
#pragma unroll
      for (int fld = 0; fld < 2; ++fld)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const T* ql = qt + ((el * 2 + fld) * DIM + c) * NU + b0;
          T acc = 0;
#pragma unroll
          for (int j = 0; j < N; ++j) acc += (s ? O.lend[1][j] : O.lend[0][j]) * ql[j * st];
          qf[fld][c] = acc;
        }
      T v[3];
      const T gel = A.ep ? gfe[el] : gfac;
      const T epsel = A.ep ? epe[el] : P.eps;
      if (tab_of(el)) {
        int jj[3];
#pragma unroll
        for (int b = 0; b < DIM; ++b) jj[b] = b == a ? N + s : ucoord<N>(b0, b);
        velocity_tab<DIM, NT, T>(BC.vel, vtab + el * DIM * NT * 2, jj, gel, v);
      } else if (A.vsf) {
        const T* vc = LY::VT ? vf + el * DIM * NF + k : vsf + (e0 + el) * DIM * NF + k;
#pragma unroll
        for (int c = 0; c < DIM; ++c) v[c] = gel * vc[c * NF];
      } else {
        T x[3];
        map_point<S::ET_, T>(gs + el * NG, xi, x);
        velocity<DIM, T>(BC.vel, x, gel, v);
      }
      T vn = 0, v2 = 0, g2 = 0, qn[3];  // qn: gradient giving the interface normal
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        qn[c] = P.nphi ? qf[0][c] : qf[1][c];
        vn += v[c] * nh[c];
        v2 += v[c] * v[c];
        g2 += qn[c] * qn[c];
      }
      const T M = fmax(sqrt_(v2), P.gamma);
      const T gm = fmax(sqrt_(g2), P.delta);
      const T pL = cor[(el * 2 + 0) * NF + k], sL = cor[(el * 2 + 1) * NF + k];  // own traces (Step 1)
      const T pR = uo[(el * 2 + 0) * NF + k], sR = uo[(el * 2 + 1) * NF + k];
      const T sharp = P.gamma * pL * ((T)1 - pL) / gm;
      T fvn = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) fvn += nh[c] * (epsel * qf[0][c] - sharp * qn[c]);
      const bool shut = P.noflux && wallp;  // no-flux wall point
      const T Fp = shut ? (T)0 : (T)0.5 * (pL + pR) * vn - M * fvn + P.tau * (pL - pR);
      const T Fs = shut ? (T)0 : (T)0.5 * (sL + sR) * vn + P.tau_psi * (sL - sR);
      // the transformed common flux F~ = |pn| F out of L; the R side uses -F~
      const T Fp_t = pm * Fp, Fs_t = pm * Fs;
      fc[((e0 + el) * 2 + 0) * NF + k] = Fp_t;
      fc[((e0 + el) * 2 + 1) * NF + k] = Fs_t;
      if (FaceScatter<DIM>::v && !wallp) {
        fc[pslot] = Fp_t;
        fc[pslot + NF] = Fs_t;
      }
      cor[(el * 2 + 0) * NF + k] = Fp_t;
      cor[(el * 2 + 1) * NF + k] = Fs_t;

    } else {
      T gn = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const T* ql = qt + (el * DIM + c) * NU + b0;
        T acc = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) acc += (s ? O.lend[1][j] : O.lend[0][j]) * ql[j * st];
        gn += nh[c] * acc;
      }
      const T L_ = cor[el * NF + k];  // own trace (Step 1)
      const T F = pm * (-nus[el] * gn + P.tau_pseudo * (L_ - uo[el * NF + k]));
      fc[((e0 + el) * 2 + 1) * NF + k] = F;
      if (FaceScatter<DIM>::v && !wallp) fc[pslot + NF] = F;
      cor[el * NF + k] = F;
    }
  }
  __syncthreads();

  // ---- Step 4 (even N): transformed flux at solution points (in place of q)
  if constexpr (!kFuse4) {
  for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
    const int el = idx / NU, i = idx % NU;
    T xi[3], Sm[3][3];
    upt_xi<DIM, N>(i, O.x, xi);
    // diagonal metric (axis-aligned affine hex): only S_aa enters below
    const bool dg = MODE == 0 && DIM == 3 && mcs[el * kKbRec + 11] == (T)2;
    T dj;
    if (dg) {
#pragma unroll
      for (int a = 0; a < DIM; ++a) Sm[a][a] = mcs[el * kKbRec + a * 4];
      dj = mcs[el * kKbRec + 9];
    } else {
      dj = metric_c<DIM>(gs + el * NG, xi, Sm, mcs + el * kKbRec);
    }
    if (MODE == 0) {
      T v[3];
      const T gel = A.ep ? gfe[el] : gfac;
      const T epsel = A.ep ? epe[el] : P.eps;
      if (tab_of(el)) {
        int jj[3];
#pragma unroll
        for (int b = 0; b < DIM; ++b) jj[b] = ucoord<N>(i, b);
        velocity_tab<DIM, NT, T>(BC.vel, vtab + el * DIM * NT * 2, jj, gel, v);
      } else if (A.vsu) {
        const T* vc = LY::VT ? vu + el * DIM * NU + i : vsu + (e0 + el) * DIM * NU + i;
#pragma unroll
        for (int c = 0; c < DIM; ++c) v[c] = gel * vc[c * NU];
      } else {
        T x[3];
        map_point<S::ET_, T>(gs + el * NG, xi, x);
        velocity<DIM, T>(BC.vel, x, gel, v);
      }
      T qp[3], qs[3], v2 = 0, g2 = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        qp[c] = qt[((el * 2 + 0) * DIM + c) * NU + i];
        qs[c] = qt[((el * 2 + 1) * DIM + c) * NU + i];
        v2 += v[c] * v[c];
        qs[c] = P.nphi ? qp[c] : qs[c];  // gradient giving the interface normal
        g2 += qs[c] * qs[c];
      }
      const T M = fmax(sqrt_(v2), P.gamma);
      const T gm = fmax(sqrt_(g2), P.delta);
      const T ph = us[(el * 2 + 0) * NU + i], ps = us[(el * 2 + 1) * NU + i];
      const T sharp = P.gamma * ph * ((T)1 - ph) / gm;
      T f0[3], f1[3];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        f0[c] = ph * v[c] - M * (epsel * qp[c] - sharp * qs[c]);
        f1[c] = ps * v[c];
      }
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T t0 = 0, t1 = 0;
        if (dg) {
          t0 = Sm[a][a] * f0[a];
          t1 = Sm[a][a] * f1[a];
        } else {
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            t0 += Sm[a][c] * f0[c];
            t1 += Sm[a][c] * f1[c];
          }
        }
        qt[((el * 2 + 0) * DIM + a) * NU + i] = t0;
        qt[((el * 2 + 1) * DIM + a) * NU + i] = t1;
      }
    } else {
      T qs[3], g2 = 0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        qs[c] = qt[(el * DIM + c) * NU + i];
        g2 += qs[c] * qs[c];
      }
      const T nu = nus[el];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        T t0 = 0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) t0 += Sm[a][c] * (-nu * qs[c]);
        qt[(el * DIM + a) * NU + i] = t0;
      }
      const T qm = sqrt_(g2);
      const T p0 = (T)A.psi0[(e0 + el) * NU + i];
      chi[el * 2 * NU + i] = tanh_(p0 / fmax(qm, P.delta)) * ((T)1 - qm) * dj;
    }
  }
  __syncthreads();
  }

  // ---- Steps 4 and 6 by axis.  With N odd, axis 0 first computes Step 4
  //      (the transformed flux f~ = det J J^-1 f) at its own line's points:
  //      the axis-0 component stays in registers, the others go to qt for the
  //      later axes (with N even the lanes' stride N would make that pass's
  //      shared-memory accesses conflict, so Step 4 runs above instead).  Each
  //      pass then takes the normal flux at the line ends, the flux jumps,
  //      the line derivative and the two end lifts into us.
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (lact) {
      const int st = ipow(N, a);
      const int base = line_base<DIM, N>(a, ll);
      const int k0 = (2 * a) * NFP + ll, k1 = k0 + NFP;
      T fa[NFLD][N];  // axis-a transformed flux along this line
      if (kFuse4 && a == 0) {
        const int el = lel;
        LineMetric<DIM, T> em;
        em.load(gs + el * NG, mcs + el * kKbRec);
        // diagonal metric (axis-aligned affine hex): only S_bb enters below
        const bool dg = MODE == 0 && DIM == 3 && mcs[el * kKbRec + 11] == (T)2;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int i = base + j;  // axis-0 lines are contiguous
          T xi[3], Sm[3][3];
          upt_xi<DIM, N>(i, O.x, xi);
          T dj;
          if (dg) {
#pragma unroll
            for (int b = 0; b < DIM; ++b) Sm[b][b] = mcs[el * kKbRec + b * 4];
            dj = mcs[el * kKbRec + 9];
          } else {
            dj = em.at(xi, Sm);
          }
          if (MODE == 0) {
            T v[3];
            const T gel = A.ep ? gfe[el] : gfac;
            const T epsel = A.ep ? epe[el] : P.eps;
            if (tab_of(el)) {
              int jj[3];
#pragma unroll
              for (int b = 0; b < DIM; ++b) jj[b] = ucoord<N>(i, b);
              velocity_tab<DIM, NT, T>(BC.vel, vtab + el * DIM * NT * 2, jj, gel, v);
            } else if (A.vsu) {
              const T* vc = LY::VT ? vu + el * DIM * NU + i : vsu + (e0 + el) * DIM * NU + i;
#pragma unroll
              for (int c = 0; c < DIM; ++c) v[c] = gel * vc[c * NU];
            } else {
              T x[3];
              map_point<S::ET_, T>(gs + el * NG, xi, x);
              velocity<DIM, T>(BC.vel, x, gel, v);
            }
            T qp[3], qs[3], v2 = 0, g2 = 0;
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
              qp[c] = qt[((el * 2 + 0) * DIM + c) * NU + i];
              qs[c] = qt[((el * 2 + 1) * DIM + c) * NU + i];
              v2 += v[c] * v[c];
              qs[c] = P.nphi ? qp[c] : qs[c];  // gradient giving the interface normal
              g2 += qs[c] * qs[c];
            }
            const T M = fmax(sqrt_(v2), P.gamma);
            const T gm = fmax(sqrt_(g2), P.delta);
            const T ph = us[(el * 2 + 0) * NU + i], ps = us[(el * 2 + 1) * NU + i];
            const T sharp = P.gamma * ph * ((T)1 - ph) / gm;
            T f0[3], f1[3];
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
              f0[c] = ph * v[c] - M * (epsel * qp[c] - sharp * qs[c]);
              f1[c] = ps * v[c];
            }
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
              T t0 = 0, t1 = 0;
              if (dg) {
                t0 = Sm[b][b] * f0[b];
                t1 = Sm[b][b] * f1[b];
              } else {
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                  t0 += Sm[b][c] * f0[c];
                  t1 += Sm[b][c] * f1[c];
                }
              }
              if (b == 0) {
                fa[0][j] = t0;
                fa[NFLD - 1][j] = t1;
              } else {
                qt[((el * 2 + 0) * DIM + b) * NU + i] = t0;
                qt[((el * 2 + 1) * DIM + b) * NU + i] = t1;
              }
            }
          } else {
            T qs[3], g2 = 0;
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
              qs[c] = qt[(el * DIM + c) * NU + i];
              g2 += qs[c] * qs[c];
            }
            const T nu = nus[el];
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
              T t0 = 0;
#pragma unroll
              for (int c = 0; c < DIM; ++c) t0 += Sm[b][c] * (-nu * qs[c]);
              if (b == 0) fa[0][j] = t0;
              else qt[(el * DIM + b) * NU + i] = t0;
            }
            const T qm = sqrt_(g2);
            const T p0 = (T)A.psi0[(e0 + el) * NU + i];
            chi[el * 2 * NU + i] = tanh_(p0 / fmax(qm, P.delta)) * ((T)1 - qm) * dj;
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const T* fl = qt + ((lel * NFLD + q) * DIM + a) * NU + base;
#pragma unroll
          for (int j = 0; j < N; ++j) fa[q][j] = fl[j * st];
        }
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int fld = q;
        const T* v = fa[q];
        T fp0 = 0, fp1 = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          fp0 += O.lend[0][j] * v[j];
          fp1 += O.lend[1][j] * v[j];
        }
        const int fo = (lel * NFLD + fld) * NF;
        const T c0 = cor[fo + k0] + fp0;   // F~ - f~perp with f~perp = -f~_a(-1)
        const T c1 = cor[fo + k1] - fp1;   // F~ - f~perp with f~perp = +f~_a(+1)
        T* dv = us + (lel * NFLD + fld) * NU + base;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          T acc = -O.gLd[j] * c0 + O.gRd[j] * c1;
#pragma unroll
          for (int m = 0; m < N; ++m) acc += O.D[j][m] * v[m];
          dv[j * st] = a == 0 ? acc : dv[j * st] + acc;
        }
      }
    }
    __syncthreads();
  }
  // ---- coalesced write of the partial divergence
  for (int idx = tid; idx < ne * NFLD * NU; idx += blockDim.x) {
    const int el = idx / (NFLD * NU), r = idx % (NFLD * NU), fld = r / NU, i = r % NU;
    T d = us[idx];
    if (MODE == 1) d -= chi[el * 2 * NU + i];
    rp[((e0 + el) * 2 + F0 + fld) * NU + i] = d;
  }
}

// kb_tensor: one block per tile of ET elements (the body above with the
// block's index; a group launch calls the same body, see k_group.cu)
template <int DIM, int N, typename T, int MODE, int TD = 1>
__global__ void __launch_bounds__(KBLayout<DIM, N, T, MODE, TD>::THREADS, KBLayout<DIM, N, T, MODE, TD>::MINB)
    kb_tensor(const KArgs A) {
  kb_tensor_body<DIM, N, T, MODE, TD>(A, blockIdx.x);
}

// ============================================================================
template <int DIM, int N, typename T, int MODE, int TD = 1>
struct KALayout {
  using S = TS<DIM, N>;
  static constexpr int NFLD = MODE == 0 ? 2 : 1;
  static constexpr int LN = S::NFP;
  // mixed path: float-float state, accumulator, w det J and the step's
  // mass-balance accumulator staged in shared memory as well, plus 2 NF
  // words per element that no array uses any more (the own fluxes now come
  // with the line-end loads): the tile size they give spreads the blocks
  // better over the SMs than the smaller footprint (measured)
  static constexpr bool PRE = sizeof(T) == 4 && MODE == 0;
  static constexpr int BYTES_EL = (NFLD * S::NU + S::NG + kMetricRec) * (int)sizeof(T) +
                                  (PRE ? 2 * S::NU * 8 + 2 * S::NU * 4 + S::NU * 8 + 2 * S::NF * 4 + 16 : 0);
  static constexpr int ET_T = 256 / LN < 1 ? 1 : 256 / LN;
  static constexpr int ET_S = 45056 / BYTES_EL < 1 ? 1 : 45056 / BYTES_EL;
  static constexpr int ET0 = warp_tile(ET_T < ET_S ? ET_T : ET_S, LN);
  static constexpr int ET = TD == 1 ? ET0 : (ET0 / TD < 1 ? 1 : warp_tile(ET0 / TD, LN));
  static constexpr int FS = FRP_FIELD_SPLIT ? NFLD : 1;  // fields split across threads
  static constexpr int LINES = ET * LN;
  static constexpr int THREADS = (LINES * FS + 31) / 32 * 32;  // whole warps; idle lanes inactive
  static constexpr int MINB = MinBlocks<THREADS, T>::v;
  // per-element RK constants and the mixed path's flux-balance work arrays
  // (beside the tile; not counted in the tile-size budget above)
  static constexpr int EXTRA_EL = (int)sizeof(RKConstF) + (PRE ? 2 * LN * 8 + 2 * 8 + 4 * 4 : 0);
  static constexpr size_t SMEM = (size_t)ET * (BYTES_EL + EXTRA_EL) + 16 * 13;  // + region alignment
};

// ka_tensor: R-side lift, du/dt, RK4 update, next-stage traces; line passes
// as in kb_tensor, the last of which also applies the update to its line.  stage -1 writes du/dt to A.out (fp64) and leaves the
// state alone; stage 0 only recomputes the traces of ustg.
// SF: the RK stage as a compile-time constant (1..4), or -2 to read it
// from A.stage; a fixed stage removes the per-point stage switch and the
// code of the other stages.
template <int DIM, int N, typename T, int MODE, int TD = 1, int SF = -2>
__device__ __forceinline__ void ka_tensor_body(const KArgs& A, const int blk) {
  using S = TS<DIM, N>;
  using LY = KALayout<DIM, N, T, MODE, TD>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG, NFP = S::NFP, NFLD = LY::NFLD, ET = LY::ET, LN = LY::LN;
  constexpr int FS = LY::FS, NQ = NFLD / FS;
  constexpr int F0 = MODE == 0 ? 0 : 1;
  if (MODE == 1 && *(volatile int32_t*)&A.status[ST_PSEUDO_DONE]) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  constexpr bool PRE = LY::PRE;
  SmemCarve sc{smem_raw};
  T* ys = sc.take<T>(ET * NFLD * NU);  // [ET][NFLD][NU]
  T* gs = sc.take<T>(ET * NG);         // [ET][NG]
  T* mcs = sc.take<T>(ET * kMetricRec);  // metric records
  float2* u2s = sc.take<float2>(PRE ? ET * 2 * NU : 0);  // float-float state, tile order
  float* acs = sc.take<float>(PRE ? ET * 2 * NU : 0);    // RK accumulator
  float2* wds = sc.take<float2>(PRE ? ET * NU : 0);      // w det J (float-float)
  double* tas = sc.take<double>(PRE ? ET * 2 : 0);       // mass-balance accumulator
  RKConstF* rks = sc.take<RKConstF>(ET);                 // RK constants per element (batches)
  float2* fb = sc.take<float2>(PRE ? 2 * ET * LN : 0);   // flux balances, per line
  double* tgt = sc.take<double>(PRE ? 2 * ET : 0);       // target mass change per element and field
  float* dlt = sc.take<float>(PRE ? 4 * ET : 0);         // uniform shift (float-float)

  const int64_t e0 = (int64_t)blk * ET;
  const int ne = (int)min((int64_t)ET, A.E - e0);
  T* ustg = reinterpret_cast<T*>(A.ustg);
  T* tr = reinterpret_cast<T*>(A.tr);
  const T* fc = reinterpret_cast<const T*>(A.fc);
  const T* rp = reinterpret_cast<const T*>(A.rp);
  const int tid = threadIdx.x;
  const int stage = SF >= -1 ? SF : A.stage;
  const TensorOpsT<T>& O = bulk<T>(A).ops;
  // line-pass role: line (lel, ll) of the fields fsel + q FS, q < NQ
  const int fsel = tid / LY::LINES, lin = tid % LY::LINES;
  const int lel = lin / LN, ll = lin % LN;
  const bool lact = lel < ne && fsel < FS;  // false on the idle lanes of a padded last warp

  // prefetch the partner fluxes of this line's R ends (0 on L ends) and, for
  // the mixed path's flux balance, this element's own L-end fluxes
  constexpr bool kCons = sizeof(T) == 4 && MODE == 0;
  const bool cons = kCons && A.tacc != nullptr && stage >= 1;
  // This element's own transformed common flux at its L points and the
  // partner's at its R points: with FluxScatter both sit in the own slots
  // (one independent load per line end), else the R value is gathered from
  // the partner's slot.
  // Hexahedra read one face word per line end (face_link), decoded below
  // once the tile copies are issued; wpre then holds the flags (bit 0 L
  // side, bit 1 wall).
  T fpre[DIM][2][NQ];
  int32_t wpre[DIM][2];
  [[maybe_unused]] int2 fwr[DIM][2];
  if (lact) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int k = (2 * a + sd) * NFP + ll;
        if constexpr (DIM == 3) {
          fwr[a][sd] = __ldg(A.ffw + (e0 + lel) * 6 + 2 * a + sd);
        } else {
          wpre[a][sd] = A.fnbr[(e0 + lel) * NF + k];
          // with FaceScatter both values sit in the own slot
          if (stage != 0 && FaceScatter<DIM>::v)
#pragma unroll
            for (int q = 0; q < NQ; ++q) fpre[a][sd][q] = fc[((e0 + lel) * 2 + F0 + fsel + q * FS) * NF + k];
        }
      }
  }
  // contiguous tiles, all in flight together with the connectivity loads
  constexpr int TH = LY::THREADS;
  if (MODE == 0) {
    tile_rows_async<2 * NU * (int)sizeof(T), ET, TH>(ys, (stage == 0 ? ustg : rp) + e0 * 2 * NU, ne);
  } else {
    for (int idx = tid; idx < ne * NU; idx += blockDim.x) {
      const int el = idx / NU, i = idx % NU;
      const int64_t g = ((e0 + el) * 2 + F0) * NU + i;
      ys[idx] = stage == 0 ? ustg[g] : rp[g];
    }
  }
  if (stage != 0) {
    tile_rows_async<NG * (int)sizeof(T), ET, TH>(gs, geo_of<T>(A) + e0 * NG, ne);
    tile_rows_async<kMetricRec * (int)sizeof(T), ET, TH>(mcs, reinterpret_cast<const T*>(A.mcg) + e0 * kMetricRec, ne);
  }
  if (PRE && stage >= 1) {
    tile_rows_async<2 * NU * 8, ET, TH>(u2s, reinterpret_cast<const float2*>(A.u) + e0 * 2 * NU, ne);
    if (stage >= 2) tile_rows_async<2 * NU * 4, ET, TH>(acs, reinterpret_cast<const float*>(A.acc) + e0 * 2 * NU, ne);
    if (cons) {
      if (stage >= 2) tile_rows_async<2 * 8, ET, TH>(tas, A.tacc + e0 * 2, ne);
      if (stage == 4) tile_rows_async<NU * 8, ET, TH>(wds, A.wdetf + e0 * NU, ne);
    }
  }
  if constexpr (DIM == 3) {
    if (lact) {
      // one load per line end: the own slot at L ends, the partner's at R ends
      const int fi = ll % N, fj = ll / N;
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          int32_t fl;
          const int32_t po = face_link<N, NF>(A, fwr[a][sd], e0 + lel, 2 * a + sd, fi, fj, fl);
          wpre[a][sd] = fl;
          if (stage != 0) {
            // slot offsets fit 31 bits (E 2 Nf < 2^31, checked at mesh creation)
            const int32_t own = (int32_t)((e0 + lel) * 2 * NF + (2 * a + sd) * NFP + ll);
            const int32_t o = (fl & 1) ? own : po;
#pragma unroll
            for (int q = 0; q < NQ; ++q) fpre[a][sd][q] = fc[o + (F0 + fsel + q * FS) * NF];
          }
        }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  double sq = 0.0;
  // RK constants: one set, or one per element for batched instances
  const RKConstF& rk0 = A.rk;
  if (A.ep) {
    for (int el = tid; el < ne; el += blockDim.x) rks[el] = MODE == 0 ? A.ep[e0 + el].rk : A.ep[e0 + el].rkp;
    __syncthreads();
  }
  auto rkc_el = [&](int el) -> const RKConstF& { return A.ep ? rks[el] : rk0; };
  // mixed path: element flux balances (float-float partial sums per line)
  if (stage != 0) {
    // ---- lift of the R-side common fluxes: minus L's transformed flux, one
    //      pass per axis
    float2 bal[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) bal[q] = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (lact) {
        const int st = ipow(N, a);
        const int base = line_base<DIM, N>(a, ll);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int fld = fsel + q * FS;
          // R ends lift minus the partner's F~; L ends were lifted in kb_tensor
          const bool L0 = wpre[a][0] & 1, L1 = wpre[a][1] & 1;
          const T c0 = L0 ? (T)0 : -fpre[a][0][q], c1 = L1 ? (T)0 : -fpre[a][1][q];
          if (cons) {
            // outward transformed flux at both ends: own F~ (L ends) or
            // -partner F~ (R ends)
            const float2 wf = O.wff[ll];
            const T o0 = L0 ? fpre[a][0][q] : c0, o1 = L1 ? fpre[a][1][q] : c1;
            bal[q] = ff_add(bal[q], ff_mul(wf, (float)o0));
            bal[q] = ff_add(bal[q], ff_mul(wf, (float)o1));
          }
          if (c0 == (T)0 && c1 == (T)0) continue;
          T* yl = ys + (lel * NFLD + fld) * NU + base;
#pragma unroll
          for (int j = 0; j < N; ++j) yl[j * st] += -O.gLd[j] * c0 + O.gRd[j] * c1;
        }
        if (a == DIM - 1) {
          // every contribution to this line's points is in: du/dt and the
          // RK4 register update, by the line's own thread
          const RKConstF& rkc = rkc_el(lel);
          LineMetric<DIM, T> em;
          em.load(gs + lel * NG, mcs + lel * kMetricRec);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const int i = base + j * st;
            T xi[3], Sm[3][3];
            upt_xi<DIM, N>(i, O.x, xi);
            T rdj;
            em.at(xi, Sm, &rdj);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              const int fld = fsel + q * FS;
              const int li = (lel * NFLD + fld) * NU + i;  // tile index
              const T R = -ys[li] * rdj;
              const int64_t g = ((e0 + lel) * 2 + F0 + fld) * NU + i;
              if (stage < 0) {
                A.out[(int64_t)fld * A.E * NU + (e0 + lel) * NU + i] = (double)R;
                continue;
              }
              if (kCons && cons && stage == 4) {
                // float-float update now (kept in shared memory), the
                // element's uniform correction below
                const float2 u = u2s[li];
                const float inc = rkc.dt6 * (acs[li] + (float)R);
                const float s2 = u.x + inc;
                const float e2 = two_sum_lo(u.x, inc, s2) + u.y;
                const float hi = s2 + e2;
                u2s[li] = make_float2(hi, e2 - (hi - s2));
                ys[li] = (T)inc;
                continue;
              }
              T yt;
              if constexpr (PRE) {
                float2 un;
                yt = rk_apply_v(A, stage, g, R, rkc, u2s[li], stage >= 2 ? acs[li] : 0.f, nullptr, &un);
                if (stage == 4) reinterpret_cast<float2*>(A.u)[g] = un;
              } else {
                yt = rk_apply(A, stage, g, R, rkc, (MODE == 1 && stage == 4) ? &sq : nullptr);
              }
              if (!isfinite(yt)) atomicExch(&A.status[ST_STATUS], -4);
              ustg[g] = yt;
              ys[li] = yt;
            }
          }
        }
      }
      __syncthreads();
    }
    if (cons) {
      if (lact)
#pragma unroll
        for (int q = 0; q < NQ; ++q) fb[(lel * 2 + fsel + q * FS) * LN + ll] = bal[q];
      __syncthreads();
      // element mass rate = -sum_k w_f F~_out,k, accumulated with the RK4
      // weights; stage 4 turns it into the step's target mass change
      for (int t = tid; t < 2 * ne; t += blockDim.x) {
        float2 sm = make_float2(0.f, 0.f);
        for (int l = 0; l < LN; ++l) sm = ff_add(sm, fb[t * LN + l]);
        const double Te = -((double)sm.x + (double)sm.y);
        const int64_t gt = e0 * 2 + t;
        if (stage == 1) A.tacc[gt] = Te;
        else if (stage < 4) A.tacc[gt] = tas[t] + 2.0 * Te;
        else tgt[t] = rkc_el(t / 2).ddt6 * (tas[t] + Te);
      }
    }
    if (kCons && cons && stage == 4) {
      __syncthreads();  // the element sums above have read fb
      // per line: sum of w det J * increment, float-float
      if (lact) {
        const int base = line_base<DIM, N>(0, ll);
        const float2* wd = wds + lel * NU + base;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int fld = fsel + q * FS;
          float2 sl = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < N; ++j)
            sl = ff_add(sl, ff_mul(wd[j], (float)ys[(lel * NFLD + fld) * NU + base + j]));
          fb[(lel * 2 + fld) * LN + ll] = sl;
        }
      }
      __syncthreads();
      for (int t = tid; t < 2 * ne; t += blockDim.x) {
        const int el = t / 2;
        float2 S2 = make_float2(0.f, 0.f);
        for (int l = 0; l < LN; ++l) S2 = ff_add(S2, fb[t * LN + l]);
        const T* mc = mcs + el * kMetricRec;
        const double S = (double)S2.x + (double)S2.y, rW = (double)mc[12] + (double)mc[13];
        const double d = (tgt[t] - S) * rW;
        const float dh = (float)d;
        dlt[2 * t] = dh;
        dlt[2 * t + 1] = (float)(d - (double)dh);
      }
      __syncthreads();
      for (int idx = tid; idx < ne * NFLD * NU; idx += blockDim.x) {
        const int el = idx / (NFLD * NU), r = idx % (NFLD * NU), fld = r / NU, i = r % NU;
        const int64_t g = ((e0 + el) * 2 + F0 + fld) * NU + i;
        float2* U = reinterpret_cast<float2*>(A.u);
        const float2 u = u2s[idx];
        const float dh = dlt[2 * (el * 2 + fld)], dl = dlt[2 * (el * 2 + fld) + 1];
        const float s2 = u.x + dh;
        const float e2 = two_sum_lo(u.x, dh, s2) + (u.y + dl);
        const float hi = s2 + e2;
        U[g] = make_float2(hi, e2 - (hi - s2));
        if (!isfinite(hi)) atomicExch(&A.status[ST_STATUS], -4);
        ustg[g] = (T)hi;
        ys[idx] = (T)hi;
      }
      __syncthreads();
    }
  }
  if (stage >= 0 && lact) {
    // ---- flux-point traces of the new stage input (Step 1 of the next stage)
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int st = ipow(N, a);
      const int base = line_base<DIM, N>(a, ll);
      const int k0 = (2 * a) * NFP + ll, k1 = k0 + NFP;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int fld = fsel + q * FS;
        const T* yl = ys + (lel * NFLD + fld) * NU + base;
        T t0 = 0, t1 = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T v = yl[j * st];
          t0 += O.lend[0][j] * v;
          t1 += O.lend[1][j] * v;
        }
        if constexpr (FaceScatter<DIM>::v) {
          // each trace goes where kb_tensor reads it: the L-side partner's
          // slot at R points, the own slot at walls (own partner); at
          // interior L points no one reads it
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            const int32_t w = wpre[a][sd];
            const int64_t og = (e0 + lel) * NF + (sd ? k1 : k0);
            const int64_t pg = (int64_t)partner<NF>(A, w, (int32_t)og);
            if (!(w & 1) || pg == og) tr[((pg / NF) * 2 + F0 + fld) * NF + pg % NF] = sd ? t1 : t0;
          }
        } else {
          // owner slots: only the traces a partner's kb gathers, at R ends
          // (the partner is L there) and at walls (the own partner)
          T* trl = tr + ((e0 + lel) * 2 + F0 + fld) * NF;
          const int32_t w0 = wpre[a][0], w1 = wpre[a][1];
          if (!(w0 & 1) || (w0 & 2)) trl[k0] = t0;
          if (!(w1 & 1) || (w1 & 2)) trl[k1] = t1;
        }
      }
    }
  }
  if (MODE == 0 && stage == 4 && A.use_dev_time && blk == 0 && tid == 0)
    A.dstate[DS_TIME] = A.dstate[DS_TIME] + A.dt;
  if (MODE == 0 && stage == 4 && A.use_dev_time && A.ep)
    for (int el = tid; el < ne; el += blockDim.x) A.ep[e0 + el].t += A.ep[e0 + el].dt;
  if (MODE == 1 && stage == 4) pseudo_rms_finish(A, block_sum(sq, red_sh), red_sh, A.E * NU);
}

template <int DIM, int N, typename T, int MODE, int TD = 1, int SF = -2>
__global__ void __launch_bounds__(KALayout<DIM, N, T, MODE, TD>::THREADS, KALayout<DIM, N, T, MODE, TD>::MINB)
    ka_tensor(const KArgs A) {
  ka_tensor_body<DIM, N, T, MODE, TD, SF>(A, blockIdx.x);
}

// Update kernels compiled once per RK stage: the physical step of mixed
// hexahedral fields (the large 3D workloads); other fields read the stage
// from their arguments.
template <int DIM, typename T, int MODE>
struct StageKA {
  static constexpr bool v = DIM == 3 && sizeof(T) == 4 && MODE == 0;
};

// Spatial velocity factor v(x) (g = 1) at the solution and flux points of
// every element, evaluated once in double and stored in the bulk type.
template <int DIM, int N, typename T>
__global__ void k_vel_cache(const KArgs A) {
  using S = TS<DIM, N>;
  constexpr int NU = S::NU, NF = S::NF, NG = S::NG;
  const int64_t n = A.E * (NU + NF);
  const TensorOpsT<double>& O = A.cd.ops;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / (NU + NF);
    const int r = (int)(g % (NU + NF));
    double xi[3], x[3], v[3];
    if (r < NU) upt_xi<DIM, N>(r, O.x, xi);
    else fpt_xi<DIM, N>(r - NU, O.x, xi);
    map_point<S::ET_, double>(A.geo + e * NG, xi, x);
    velocity<DIM, double>(A.cd.vel, x, 1.0, v);
    if (r < NU) {
      T* o = reinterpret_cast<T*>(const_cast<void*>(A.vsu)) + e * DIM * NU + r;
      for (int c = 0; c < DIM; ++c) o[c * NU] = (T)v[c];
    } else {
      T* o = reinterpret_cast<T*>(const_cast<void*>(A.vsf)) + e * DIM * NF + (r - NU);
      for (int c = 0; c < DIM; ++c) o[c * NF] = (T)v[c];
    }
  }
}

}  // namespace frp
