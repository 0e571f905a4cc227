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
enum { ST_STATUS = 0, ST_PSEUDO_DONE = 1, ST_PSEUDO_ITERS = 2, ST_COUNTER = 3, ST_WORDS = 8 };
// double slots in the workspace
enum { DS_TIME = 0, DS_PSEUDO_RMS = 1, DS_MASS = 2, DS_MASS_C = 3, DS_WORDS = 8 };

struct VelDesc {
  int kind, n_modes;
  double T;
  double a[3];
  double kx[kMaxModes], ky[kMaxModes], A[kMaxModes], B[kMaxModes];
};

struct PhysPrm {
  double gamma, eps, tau, tau_psi, tau_pseudo, delta, s0, kappa, nu_max, pseudo_tol;
  int pseudo_fixed;
};

// 1D tensor operators (double); kernels stage them into shared memory.
struct TensorOps {
  double x[kMaxN], lend[2][kMaxN], D[kMaxN][kMaxN], gLd[kMaxN], gRd[kMaxN], Vinv[kMaxN][kMaxN];
};

// Dense triangle operators live in device memory (double).
struct TriOps {
  const double* xu;   // nu x 2
  const double* xf;   // nf x 2
  const double* nref; // nf x 2
  const double* L;    // nf x nu
  const double* Dr;   // nu x nu
  const double* Ds;   // nu x nu
  const double* LIFT; // nu x nf
  const double* Vinv; // nu x nu
  const uint8_t* high;
};

struct KArgs {
  int64_t E;
  const double* geo;     // E x dim x ncoef
  const int32_t* fnbr;   // E x nf
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
  int stage;             // 1..4 RK stage, -1: write the rate into out
  int use_dev_time;      // KB: t = dstate[DS_TIME] + c_s dt
  double t;              // KB: stage time when !use_dev_time
  double dt;             // physical dt or pseudo dtau
  VelDesc vel;
  PhysPrm prm;
  TensorOps ops;
  TriOps tri;
};

// ---------------------------------------------------------------------------
__device__ __forceinline__ double spi(double x) { return sinpi(x); }
__device__ __forceinline__ float spi(float x) { return sinpif(x); }
__device__ __forceinline__ double cpi(double x) { return cospi(x); }
__device__ __forceinline__ float cpi(float x) { return cospif(x); }
__device__ __forceinline__ double tanh_(double x) { return tanh(x); }
__device__ __forceinline__ float tanh_(float x) { return tanhf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }

// Analytic velocity (Sections 4.1-4.3); time modulation g(t) = cos(pi t / T).
template <int DIM, typename R>
__device__ __forceinline__ void velocity(const VelDesc& V, const R* x, double t, R* v) {
  const R g = V.T > 0.0 ? (R)cospi(t / V.T) : (R)1;
  switch (V.kind) {
    case 0:  // uniform
      for (int c = 0; c < DIM; ++c) v[c] = (R)V.a[c];
      break;
    case 1: {  // Rider-Kothe
      const R sx = spi(x[0]), sy = spi(x[1]);
      v[0] = -sx * sx * spi((R)2 * x[1]) * g;
      v[1] = spi((R)2 * x[0]) * sy * sy * g;
      if (DIM == 3) v[DIM - 1] = 0;
      break;
    }
    case 2: {  // LeVeque 3D deformation
      if (DIM == 3) {
        const R sx = spi(x[0]), sy = spi(x[1]), sz = spi(x[DIM - 1]);
        const R s2x = spi((R)2 * x[0]), s2y = spi((R)2 * x[1]), s2z = spi((R)2 * x[DIM - 1]);
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
        const R kx = (R)V.kx[m], ky = (R)V.ky[m];
        const R arg = (R)2 * (kx * x[0] + ky * x[1]);
        const R d = (R)(2.0 * M_PI) * ((R)V.A[m] * cpi(arg) - (R)V.B[m] * spi(arg));
        u0 += ky * d;
        u1 -= kx * d;
      }
      v[0] = u0 * g;
      v[1] = u1 * g;
      if (DIM == 3) v[DIM - 1] = 0;
      break;
    }
    default:  // solid-body rotation
      v[0] = (R)0.5 - x[1];
      v[1] = x[0] - (R)0.5;
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
