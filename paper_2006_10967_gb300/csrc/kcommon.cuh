// Device-side shared definitions of libfrpcpf: kernel arguments, analytic
// velocity fields, the pointwise fluxes and small reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "geom.cuh"
#include "refel.hpp"

namespace frp {

constexpr int kMaxModes = 32;
constexpr int kThreads = 256;

// status words (int32) in the workspace
enum { ST_STATUS = 0, ST_PSEUDO_DONE = 1, ST_PSEUDO_ITERS = 2, ST_COUNTER = 3, ST_BAD_INDEX = 4, ST_WORDS = 8 };
constexpr int kStatusBounds = -7;  // FR_EBOUNDS
// double slots in the workspace
enum { DS_TIME = 0, DS_PSEUDO_RMS = 1, DS_MASS = 2, DS_MASS_C = 3, DS_WORDS = 8 };

// Velocity constants in the kernel's bulk precision R (the time factor
// g(t) is evaluated once per block in double and passed in).
template <typename R>
struct VelDescT {
  int kind, n_modes;
  R a[3];
  R kx[kMaxModes], ky[kMaxModes], A[kMaxModes], B[kMaxModes];
};

// Physical parameters in the bulk precision (double copies for the host-side
// and reduction logic live in PhysPrm).
template <typename R>
struct PrmT {
  R gamma, eps, tau, tau_psi, tau_pseudo, delta;
  int nphi;    // 1: the sharpening normal comes from phi's gradient (unpreconditioned CPF)
  int noflux;  // 1: zero common normal flux of the physical system at wall flux points
};

struct PhysPrm {
  double gamma, eps, tau, tau_psi, tau_pseudo, delta, s0, kappa, nu_max, pseudo_tol;
  int pseudo_fixed;
  double T;   // period of the velocity time factor (<= 0: none)
  double rT;  // 1 / T (0 when T <= 0)
};

// 1D tensor operators; kernels stage them into shared memory.
template <typename R>
struct TensorOpsT {
  R x[kMaxN], w[kMaxN], lend[2][kMaxN], D[kMaxN][kMaxN], gLd[kMaxN], gRd[kMaxN], Vinv[kMaxN][kMaxN];
  float2 wff[kMaxN * kMaxN];  // face quadrature weights (products of GL weights) as float-float pairs
};
typedef TensorOpsT<double> TensorOps;

// Bulk-precision constants of one field, in both precisions.
template <typename R>
struct BulkConst {
  VelDescT<R> vel;
  PrmT<R> prm;
  TensorOpsT<R> ops;
};

// Dense triangle operators live in device memory (one copy per precision).
template <typename R>
struct TriOpsT {
  const R* xu;   // nu x 2
  const R* xf;   // nf x 2
  const R* nref; // nf x 2
  const R* L;    // nf x nu
  const R* Dr;   // nu x nu
  const R* Ds;   // nu x nu
  const R* LIFT; // nu x nf
  const R* Vinv; // nu x nu
  const uint8_t* high;
};

// RK4 step constants (filled on the host for uniform fields; per element for
// batched instances)
// Values per element in the tensor kernels' metric records (bulk type).
constexpr int kMetricRec = 16;

struct RKConstF {
  float half_dt, dt, dt6;
  double rdt, ddt, ddt6;
};

__host__ __device__ __forceinline__ RKConstF rk_const(double dt) {
  RKConstF c;
  c.half_dt = (float)(0.5 * dt);
  c.dt = (float)dt;
  c.dt6 = (float)(dt / 6.0);
  c.rdt = 1.0 / dt;
  c.ddt = dt;
  c.ddt6 = dt / 6.0;
  return c;
}

// Per-element parameters of a batch of independent instances (one union
// mesh): each instance keeps its own time step, time, eps and nu_max.
struct ElemPar {
  double dt, dtau;  // physical and pseudo time steps
  double t;         // physical time at the start of the current step
  double eps, nu_max;
  RKConstF rk, rkp;  // RK4 constants of dt and dtau
};

struct KArgs {
  int64_t E;
  const double* geo;     // E x dim x ncoef (fp64)
  const float* geof;     // E x dim x ncoef (fp32 copy for the mixed path)
  const int32_t* fnbr;   // E x nf
  const int2* ffw;       // hexahedra: E x 6 face words (face_link), or nullptr
  void* ustg;            // T   E x 2 x nu  stage input
  double* u;             // E x 2 x nu     solution (RK base)
  double* acc;           // E x 2 x nu     RK accumulator
  void* rp;              // T   E x 2 x nu  partial transformed divergence
  void* tr;              // T   E x 2 x nf  flux-point traces of the stage input
  void* fc;              // T   E x 2 x nf  common normal flux out of L (physical), at L points
  double* psi0;          // E x nu
  const double* wdet;    // E x nu
  int32_t* status;       // ST_WORDS
  double* dstate;        // DS_WORDS
  double* red;           // reduction partials (one per block)
  double* out;           // fr_rhs output (2 x E x nu) or nullptr
  const void* vsu;       // T E x dim x nu: spatial velocity factor at solution points (or nullptr)
  const void* vsf;       // T E x dim x nf: spatial velocity factor at flux points (or nullptr)
  double* tacc;          // E x 2: RK accumulation of the element flux balances (mixed path) or nullptr
  ElemPar* ep;           // E per-element parameters (batched instances) or nullptr (uniform)
  const float2* wdetf;   // E x nu: w_i det J_i as float-float pairs (mixed path)
  void* mcg;             // tensor elements: E x 16 metric records (bulk type)
  const float2* wphys;   // triangles: E x nf physical flux-point weights (float-float), equal on both sides
  int stage;             // 1..4 RK stage, -1: write the rate into out
  int use_dev_time;      // KB: t = dstate[DS_TIME] + c_s dt
  double t;              // KB: stage time when !use_dev_time
  double dt;             // physical dt or pseudo dtau
  RKConstF rk;           // rk_const(dt), set on the host with dt
  PhysPrm prm;
  BulkConst<double> cd;
  BulkConst<float> cf;
  TriOpsT<double> trid;
  TriOpsT<float> trif;
};

// Partner flux point of a connectivity word w (bit 0: the L flag, bits 1-31:
// the global flux-point index, E Nf < 2^30 checked at mesh creation).  In a
// build with FR_BOUNDS_CHECK defined (the library's checked build) every such
// index is checked against E Nf before it is used: an index out of range
// records FR_EBOUNDS and the connectivity word in the status words, and the
// caller's own flux point (always in range) is used instead, so no access
// leaves the arrays.  Without the flag this is the plain shift.
template <int NF>
__device__ __forceinline__ int32_t partner(const KArgs& A, int32_t w, int32_t own) {
  const int32_t p = w >> 1;
#ifdef FR_BOUNDS_CHECK
  if (p < 0 || (int64_t)p >= A.E * NF) {
    atomicExch(&A.status[ST_STATUS], kStatusBounds);
    atomicExch(&A.status[ST_BAD_INDEX], w);
    return own;
  }
#else
  (void)A;
  (void)own;
#endif
  return p;
}

// Hexahedra carry one word pair per face (KArgs.ffw) in place of one
// connectivity word per flux point.  Face point (i, j) (the line index
// i + N j of the two other axes, lowest fastest) meets the partner's face
// point face_perm(o, i, j) for one orientation o of the shared face: o & 4
// exchanges i and j, then o & 1 reverses the first index and o & 2 the
// second; the eight values of o are the eight symmetries of the N x N point
// grid of a face.  That index is affine in (i, j), c0 + ci i + cj j with
// ci, cj in {+-1, +-N}, so the word pair stores x = the offset of the
// partner's point (0, 0)-image in an E x 2 x NF array (field 0), plus c0,
// and y = bit 0 L side, bit 1 wall (the face is its own partner), bits 2-11
// ci and bits 12-21 cj as signed 10-bit fields.  The host derives the words
// from the per-point connectivity with face_perm.
constexpr int kFwL = 1, kFwWall = 2;

__host__ __device__ __forceinline__ int face_perm(int o, int i, int j, int N) {
  const int a = (o & 4) ? j : i, b = (o & 4) ? i : j;
  return ((o & 1) ? N - 1 - a : a) + N * ((o & 2) ? N - 1 - b : b);
}

// Decodes the face word pair w of face f of element e for face point
// (i, j): returns the offset of the partner flux point's slot in an
// E x 2 x NF array (field 0; E 2 NF < 2^31 since E NF < 2^30) and sets
// flags (bit 0 L side, bit 1 wall).  With FR_BOUNDS_CHECK an offset outside
// the array or off the field-0 rows records FR_EBOUNDS and the word, and the
// face is treated as a wall (its own partner).
template <int N, int NF>
__device__ __forceinline__ int32_t face_link(const KArgs& A, int2 w, int64_t e, int f, int i, int j,
                                             int32_t& flags) {
  const int32_t ci = (int32_t)((uint32_t)w.y << 20) >> 22, cj = (int32_t)((uint32_t)w.y << 10) >> 22;
  const int32_t off = w.x + ci * i + cj * j;
  flags = w.y & 3;
#ifdef FR_BOUNDS_CHECK
  if (off < 0 || (int64_t)off >= A.E * 2 * NF || off % (2 * NF) >= NF) {
    atomicExch(&A.status[ST_STATUS], kStatusBounds);
    atomicExch(&A.status[ST_BAD_INDEX], w.x);
    flags = kFwL | kFwWall;
    return (int32_t)(e * 2 * NF + f * N * N + i + N * j);
  }
#else
  (void)A;
  (void)e;
  (void)f;
#endif
  return off;
}

template <typename T> __device__ __forceinline__ const BulkConst<T>& bulk(const KArgs& A);
template <> __device__ __forceinline__ const BulkConst<double>& bulk<double>(const KArgs& A) { return A.cd; }
template <> __device__ __forceinline__ const BulkConst<float>& bulk<float>(const KArgs& A) { return A.cf; }
template <typename T> __device__ __forceinline__ const TriOpsT<T>& tri_of(const KArgs& A);
template <> __device__ __forceinline__ const TriOpsT<double>& tri_of<double>(const KArgs& A) { return A.trid; }
template <> __device__ __forceinline__ const TriOpsT<float>& tri_of<float>(const KArgs& A) { return A.trif; }
template <typename T> __device__ __forceinline__ const T* geo_of(const KArgs& A);
template <> __device__ __forceinline__ const double* geo_of<double>(const KArgs& A) { return A.geo; }
template <> __device__ __forceinline__ const float* geo_of<float>(const KArgs& A) { return A.geof; }

// Time factor g(t) = cos(pi t / T) of the modulated velocity fields, in double.
__device__ __forceinline__ double time_factor(const KArgs& A, double t) {
  return A.prm.T > 0.0 ? cospi(t / A.prm.T) : 1.0;
}
// The bulk-precision time factor: the FP64 path as above; the float path
// evaluates cos(pi t / T) in float from t / T rounded to float (the time
// itself stays FP64), which keeps the slow FP64 pipe out of the kernels.
template <typename T> __device__ __forceinline__ T time_factor_t(const KArgs& A, double t);
template <> __device__ __forceinline__ double time_factor_t<double>(const KArgs& A, double t) {
  return time_factor(A, t);
}
template <> __device__ __forceinline__ float time_factor_t<float>(const KArgs& A, double t) {
  return A.prm.T > 0.0 ? cospif((float)(t * A.prm.rT)) : 1.0f;
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ double spi(double x) { return sinpi(x); }
__device__ __forceinline__ float spi(float x) { return sinpif(x); }
__device__ __forceinline__ double cpi(double x) { return cospi(x); }
__device__ __forceinline__ float cpi(float x) { return cospif(x); }
__device__ __forceinline__ void scpi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void scpi(float x, float* s, float* c) { sincospif(x, s, c); }
// Velocity sin/cos of pi*x: the FP64 path keeps sincospi; the float path uses
// the special-function unit (__sincosf of pi*x, absolute error ~4e-7 for the
// coordinates of the unit domain).
__device__ __forceinline__ void vscpi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void vscpi(float x, float* s, float* c) { __sincosf(3.14159265358979f * x, s, c); }
__device__ __forceinline__ double tanh_(double x) { return tanh(x); }
__device__ __forceinline__ float tanh_(float x) { return tanhf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }

// Analytic velocity (Sections 4.1-4.3); time modulation g(t) = cos(pi t / T).
template <int DIM, typename R>
__device__ __forceinline__ void velocity(const VelDescT<R>& V, const R* x, R g, R* v) {
  switch (V.kind) {
    case 0:  // uniform, a g(t)
      for (int c = 0; c < DIM; ++c) v[c] = V.a[c] * g;
      break;
    case 1: {  // Rider-Kothe; sin(2 pi a) = 2 sin(pi a) cos(pi a)
      R sx, cx, sy, cy;
      vscpi(x[0], &sx, &cx);
      vscpi(x[1], &sy, &cy);
      v[0] = -sx * sx * ((R)2 * sy * cy) * g;
      v[1] = ((R)2 * sx * cx) * sy * sy * g;
      if (DIM == 3) v[DIM - 1] = 0;
      break;
    }
    case 2: {  // LeVeque 3D deformation
      if (DIM == 3) {
        R sx, cx, sy, cy, sz, cz;
        vscpi(x[0], &sx, &cx);
        vscpi(x[1], &sy, &cy);
        vscpi(x[DIM - 1], &sz, &cz);
        const R s2x = (R)2 * sx * cx, s2y = (R)2 * sy * cy, s2z = (R)2 * sz * cz;
        v[0] = (R)2 * sx * sx * s2y * s2z * g;
        v[1] = -s2x * sy * sy * s2z * g;
        v[DIM - 1] = -s2x * s2y * sz * sz * g;
      } else {
        v[0] = v[1] = 0;
      }
      break;
    }
    case 3: {  // stream function
      R u0 = 0, u1 = 0;
      for (int m = 0; m < V.n_modes; ++m) {
        const R kx = V.kx[m], ky = V.ky[m];
        const R arg = (R)2 * (kx * x[0] + ky * x[1]);
        const R d = (R)(2.0 * M_PI) * (V.A[m] * cpi(arg) - V.B[m] * spi(arg));
        u0 += ky * d;
        u1 -= kx * d;
      }
      v[0] = u0 * g;
      v[1] = u1 * g;
      if (DIM == 3) v[DIM - 1] = 0;
      break;
    }
    default:  // solid-body rotation about (a[0], a[1])
      v[0] = V.a[1] - x[1];
      v[1] = x[0] - V.a[0];
      if (DIM == 3) v[DIM - 1] = 0;
  }
}

// Separable velocity fields on elements whose map is affine with a diagonal
// Jacobian (x_c depends on xi_c alone): every factor of the uniform,
// Rider-Kothe, LeVeque and rotation fields is a function of one coordinate,
// so an element needs them only at the N solution coordinates of each axis
// and at the two ends.  Table layout per element: tab[(c (N + 2) + j) 2 + m],
// j < N the solution coordinate j, N the end xi = -1, N + 1 the end xi = +1;
// m = 0: sin^2(pi x_c) (rotation: x_c itself), m = 1: sin(2 pi x_c).
__host__ __device__ constexpr bool vel_separable(int kind) { return kind == 0 || kind == 1 || kind == 2 || kind == 4; }

template <typename R>
__device__ __forceinline__ void vel_tab_entry(int kind, R x, R* e) {
  if (kind == 4) {
    e[0] = x;
    e[1] = 0;
    return;
  }
  R s, c;
  scpi(x, &s, &c);
  e[0] = s * s;
  e[1] = (R)2 * s * c;
}

// Velocity at the point with per-axis table indices j[0..DIM-1].
template <int DIM, int NT, typename R>
__device__ __forceinline__ void velocity_tab(const VelDescT<R>& V, const R* tab, const int* j, R g, R* v) {
  auto A = [&](int c) { return tab[(c * NT + j[c]) * 2]; };
  auto B = [&](int c) { return tab[(c * NT + j[c]) * 2 + 1]; };
  switch (V.kind) {
    case 0:
      for (int c = 0; c < DIM; ++c) v[c] = V.a[c] * g;
      break;
    case 1:  // u = -sin^2(pi x) sin(2 pi y) g, v = sin(2 pi x) sin^2(pi y) g
      v[0] = -A(0) * B(1) * g;
      v[1] = B(0) * A(1) * g;
      if (DIM == 3) v[DIM - 1] = 0;
      break;
    case 2:
      if (DIM == 3) {
        v[0] = (R)2 * A(0) * B(1) * B(DIM - 1) * g;
        v[1] = -B(0) * A(1) * B(DIM - 1) * g;
        v[DIM - 1] = -B(0) * B(1) * A(DIM - 1) * g;
      } else {
        v[0] = v[1] = 0;
      }
      break;
    default:  // rotation about (a[0], a[1]); the table holds the coordinates
      v[0] = V.a[1] - A(1);
      v[1] = A(0) - V.a[0];
      if (DIM == 3) v[DIM - 1] = 0;
  }
}

template <typename R>
__device__ __forceinline__ bool finite_(R x) { return isfinite(x); }

// RK4 stage nodes c_s (classical RK4)
__device__ __forceinline__ double rk_c(int s) { return s == 1 ? 0.0 : (s == 4 ? 1.0 : 0.5); }

// Classical RK4 register update for stage s with rate R.  Returns the next
// stage input (or the new solution at s = 4).
__device__ __forceinline__ double rk_update(int s, double dt, double R, double& u, double& acc) {
  switch (s) {
    case 1: acc = R; return u + 0.5 * dt * R;
    case 2: acc += 2.0 * R; return u + 0.5 * dt * R;
    case 3: acc += 2.0 * R; return u + dt * R;
    default: {
      const double un = u + dt / 6.0 * (acc + R);
      u = un;
      return un;
    }
  }
}

// RK4 stage update of value g in the FP64 path: u, acc double.  Returns the
// next stage input; adds the squared pseudo residual to *sq when asked.
__device__ __forceinline__ double rk_apply_d(const KArgs& A, int stage, int64_t g, double R, double dt, double* sq) {
  double uu = A.u[g], aa = stage == 1 ? 0.0 : A.acc[g];
  const double uold = uu;
  const double y = rk_update(stage, dt, R, uu, aa);
  if (stage < 4) A.acc[g] = aa;
  else A.u[g] = uu;
  if (sq) {
    const double d = (uu - uold) / dt;
    *sq += d * d;
  }
  return y;
}

// Mixed path: the solution u is a float-float pair (hi, lo) (48-bit
// significand) so that float stage increments accumulate without FP64
// instructions; acc = sum_s b_s k_s and the stage values are float.


__device__ __forceinline__ float two_sum_lo(float a, float b, float s) {
  const float bb = s - a;
  return (a - (s - bb)) + (b - bb);
}

// float-float arithmetic (pairs (hi, lo), |lo| <= ulp(hi)/2)
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float e = two_sum_lo(a.x, b.x, s) + (a.y + b.y);
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}
// (pair) x (float), exact product of the high parts by FMA
__device__ __forceinline__ float2 ff_mul(float2 a, float b) {
  const float p = a.x * b;
  const float e = fmaf(a.x, b, -p) + a.y * b;
  const float hi = p + e;
  return make_float2(hi, e - (hi - p));
}

// Float-float register update with the state u and the accumulator value
// already at hand (acc is read only from stage 2 on).  Writes the accumulator
// and, at stage 4, the state to global memory unless keep_u is set.
__device__ __forceinline__ float rk_apply_v(const KArgs& A, int stage, int64_t g, float R, const RKConstF& c,
                                            float2 u, float acc, double* sq, float2* unew) {
  float* Acc = reinterpret_cast<float*>(A.acc);
  switch (stage) {
    case 1: Acc[g] = R; return u.x + fmaf(c.half_dt, R, u.y);
    case 2: Acc[g] = fmaf(2.0f, R, acc); return u.x + fmaf(c.half_dt, R, u.y);
    case 3: Acc[g] = fmaf(2.0f, R, acc); return u.x + fmaf(c.dt, R, u.y);
    default: {
      const float inc = c.dt6 * (acc + R);
      const float s = u.x + inc;
      const float e = two_sum_lo(u.x, inc, s) + u.y;
      const float hi = s + e;
      const float lo = e - (hi - s);
      *unew = make_float2(hi, lo);
      if (sq) {
        const double d = (((double)hi - (double)u.x) + ((double)lo - (double)u.y)) * c.rdt;
        *sq += d * d;
      }
      return hi;
    }
  }
}

__device__ __forceinline__ float rk_apply(const KArgs& A, int stage, int64_t g, float R, const RKConstF& c,
                                          double* sq) {
  float2* U = reinterpret_cast<float2*>(A.u);
  const float acc = stage > 1 ? reinterpret_cast<const float*>(A.acc)[g] : 0.f;
  float2 un;
  const float y = rk_apply_v(A, stage, g, R, c, U[g], acc, sq, &un);
  if (stage >= 4) U[g] = un;
  return y;
}

__device__ __forceinline__ double rk_apply(const KArgs& A, int stage, int64_t g, double R, const RKConstF& c,
                                           double* sq) {
  return rk_apply_d(A, stage, g, R, c.ddt, sq);
}

// ---- asynchronous global -> shared copies (cp.async; completed by
//      cp_async_wait_all followed by a block barrier) -------------------------
__device__ __forceinline__ void cp_async_4(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Block-wide copy of nbytes (a multiple of 4) of contiguous global memory into
// shared memory, issued without waiting: 16-byte granules when both ends are
// 16-byte aligned, 4-byte granules otherwise.
__device__ __forceinline__ void tile_async(void* sdst, const void* gsrc, int nbytes) {
  const char* s = static_cast<const char*>(gsrc);
  char* d = static_cast<char*>(sdst);
  int done = 0;
  if (((reinterpret_cast<uintptr_t>(s) | (uintptr_t)__cvta_generic_to_shared(d)) & 15) == 0) {
    const int n16 = nbytes >> 4;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) cp_async_16(d + 16 * i, s + 16 * i);
    done = n16 << 4;
  }
  for (int i = (done >> 2) + threadIdx.x; i < (nbytes >> 2); i += blockDim.x) cp_async_4(d + 4 * i, s + 4 * i);
}

// tile_async for a tile of ne elements of ELB bytes each, with ET elements in
// a full tile, copied by the first TH threads of the block (a block may have
// more, as in a group launch): a full tile of rows that are whole 16-byte
// granules (every workspace region starts on a 256-byte boundary and every
// shared region on a 16-byte one) is copied in a loop of compile-time length
// without the alignment test; other tiles take tile_async.
template <int ELB, int ET, int TH>
__device__ __forceinline__ void tile_rows_async(void* sdst, const void* gsrc, int ne) {
  if constexpr (ELB % 16 == 0) {
    if (ne == ET) {
      constexpr int n16 = ELB * ET / 16;
      const char* s = static_cast<const char*>(gsrc);
      char* d = static_cast<char*>(sdst);
      if ((int)threadIdx.x < TH) {
#pragma unroll
        for (int r = 0; r < (n16 + TH - 1) / TH; ++r) {
          const int i = r * TH + (int)threadIdx.x;
          if (i < n16) cp_async_16(d + 16 * i, s + 16 * i);
        }
      }
      return;
    }
  }
  tile_async(sdst, gsrc, ne * ELB);
}

// Carves 16-byte aligned regions out of dynamic shared memory.
struct SmemCarve {
  unsigned char* p;
  template <typename U>
  __device__ __forceinline__ U* take(int count) {
    U* r = reinterpret_cast<U*>(p);
    p += ((size_t)count * sizeof(U) + 15) & ~(size_t)15;
    return r;
  }
};

// Block-wide sum of one double (all threads get the result).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += sh[i];
  __syncthreads();
  return t;
}

// Last-block-done finalisation of the pseudo-time RMS (fixed summation order).
__device__ __forceinline__ void pseudo_rms_finish(const KArgs& A, double partial, double* sh, int64_t ndof) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    A.red[blockIdx.x] = partial;
    __threadfence();
    const int prev = atomicAdd(&A.status[ST_COUNTER], 1);
    last = (prev == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += ((volatile double*)A.red)[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double rms = sqrt(s / (double)ndof);
    A.dstate[DS_PSEUDO_RMS] = rms;
    A.status[ST_PSEUDO_ITERS] += 1;
    if (!A.prm.pseudo_fixed && rms <= A.prm.pseudo_tol) A.status[ST_PSEUDO_DONE] = 1;
    if (!isfinite(rms)) atomicExch(&A.status[ST_STATUS], -4);
    A.status[ST_COUNTER] = 0;
  }
}

}  // namespace frp
