// Two forms of the same element-local operator applies on hexahedra, for
// measuring one against the other (fr_probe_hex_apply).  For every column
// (element, field) of N^3 solution-point values u, both forms compute
//   the flux-point traces u^f = L u (Section 3.1, Step 1, Eq. extrapolateSoln),
//     6 N^2 values: face 2a + sd, face point l in the residual kernel's line
//     order (line l along axis a ends at point l of faces (a, -) and (a, +));
//   the reference derivatives D_a u (Step 3, Eq. continuousGrad, without the
//     correction terms), 3 N^3 values: axis a, then solution point i.
// Form 0 applies the 1D operators along solution-point lines (sum
// factorisation, as the residual kernel does): per line 2 N + N^2 FMAs.
// Form 1 applies the dense operators, the (6 N^2 + 3 N^3) x N^3 matrix
// [L; D_0; D_1; D_2], on the tensor cores: mma.sync m16n8k8 in three-term
// TF32 (mma_tf32.cuh) with FP32 accumulation, the operator's fragments
// resident in shared memory for a persistent block.  p = 3 only (N = 4:
// 288 x 64, 18 row tiles of 16 and 8 inner steps of 8).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fr_pcpf.h"
#include "mma_tf32.cuh"
#include "refel.hpp"

namespace frp {
namespace {

constexpr int PN = 4;                // points per line (p = 3)
constexpr int PNU = PN * PN * PN;    // 64 solution points
constexpr int PNFP = PN * PN;        // 16 points per face
constexpr int PNF = 6 * PNFP;        // 96 flux points
constexpr int PM = PNF + 3 * PNU;    // 288 values per column
constexpr int PTH = 512;             // threads per block, both forms

struct ProbeOps {
  float lend[2][PN];  // l_j(-1), l_j(+1)
  float D[PN][PN];    // D[i][j] = l_j'(x_i)
};

__host__ __device__ constexpr int pstride(int a) { return a == 0 ? 1 : (a == 1 ? PN : PN * PN); }

// first solution point of line l along axis a (the other two coordinates,
// lower axis fastest, encode l)
__device__ __forceinline__ int pline_base(int a, int l) {
  const int r0 = l % PN, r1 = l / PN;
  return a == 0 ? PN * r0 + PN * PN * r1 : (a == 1 ? r0 + PN * PN * r1 : r0 + PN * r1);
}

__device__ __forceinline__ int pcoord(int i, int a) { return (i / pstride(a)) % PN; }

// ---- form 0: one thread per solution-point line of an element, both fields,
//      the three axes in turn (PTH / N^2 = 32 elements per block)
constexpr int SF_ET = PTH / PNFP;

__global__ void __launch_bounds__(PTH) k_probe_sf(const float* __restrict__ u, int64_t E, float* __restrict__ out,
                                                  int reduce, const ProbeOps ops) {
  __shared__ __align__(16) float us[SF_ET * 2 * PNU];
  const int64_t e0 = (int64_t)blockIdx.x * SF_ET;
  const int ne = (int)min((int64_t)SF_ET, E - e0);
  const int tid = threadIdx.x;
  const float4* src = reinterpret_cast<const float4*>(u + e0 * 2 * PNU);
  for (int i = tid; i < ne * 2 * PNU / 4; i += PTH) reinterpret_cast<float4*>(us)[i] = __ldg(src + i);
  __syncthreads();
  const int lel = tid / PNFP, ll = tid % PNFP;
  float s[2] = {0.f, 0.f};
  if (lel < ne) {
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      const float* ue = us + (lel * 2 + fld) * PNU;
      float* oe = out + ((e0 + lel) * 2 + fld) * PM;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int st = pstride(a), base = pline_base(a, ll);
        float v[PN];
#pragma unroll
        for (int j = 0; j < PN; ++j) v[j] = ue[base + j * st];
        float f0 = 0.f, f1 = 0.f;
#pragma unroll
        for (int j = 0; j < PN; ++j) {
          f0 = fmaf(ops.lend[0][j], v[j], f0);
          f1 = fmaf(ops.lend[1][j], v[j], f1);
        }
        float d[PN];
#pragma unroll
        for (int i = 0; i < PN; ++i) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < PN; ++m) acc = fmaf(ops.D[i][m], v[m], acc);
          d[i] = acc;
        }
        if (reduce) {
          s[fld] += f0 + f1;
#pragma unroll
          for (int i = 0; i < PN; ++i) s[fld] += d[i];
        } else {
          oe[(2 * a) * PNFP + ll] = f0;
          oe[(2 * a + 1) * PNFP + ll] = f1;
#pragma unroll
          for (int i = 0; i < PN; ++i) oe[PNF + a * PNU + base + i * st] = d[i];
        }
      }
    }
  }
  if (reduce) {
    // an element's 16 lines are 16 consecutive lanes of one warp
#pragma unroll
    for (int o = PNFP / 2; o >= 1; o >>= 1) {
      s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
      s[1] += __shfl_xor_sync(0xffffffffu, s[1], o);
    }
    if (lel < ne && ll == 0) {
      out[(e0 + lel) * 2] = s[0];
      out[(e0 + lel) * 2 + 1] = s[1];
    }
  }
}

// ---- form 1: dense operators on the tensor cores
constexpr int DN_ET = 64;               // elements per tile
constexpr int DN_COLS = 2 * DN_ET;      // 128 columns: one group of 8 per warp
constexpr int DN_LD = PNU + 4;          // padded column stride: the B-fragment loads hit 32 banks
constexpr int MT = PM / 16, KT = PNU / 8;
static_assert(PM % 32 == 0 && PNU % 8 == 0, "two row tiles per pass, whole inner steps");
static_assert(DN_COLS == 8 * (PTH / 32), "one column group per warp");
constexpr size_t DN_AFR = (size_t)MT * KT * 2 * 32 * sizeof(uint4);  // hi and lo A fragments
constexpr size_t DN_SMEM = DN_AFR + (size_t)DN_COLS * DN_LD * sizeof(float);

// entry (r, c) of [L; D_0; D_1; D_2]: output r, input solution point c
__device__ float dense_entry(const ProbeOps& ops, int r, int c) {
  if (r < PNF) {
    const int fa = r / PNFP, l = r % PNFP, a = fa >> 1, sd = fa & 1;
    const int ca = pcoord(c, a);
    return c - ca * pstride(a) == pline_base(a, l) ? ops.lend[sd][ca] : 0.f;
  }
  const int a = (r - PNF) / PNU, i = (r - PNF) % PNU;
  const int ia = pcoord(i, a), ca = pcoord(c, a);
  return i - ia * pstride(a) == c - ca * pstride(a) ? ops.D[ia][ca] : 0.f;
}

__global__ void __launch_bounds__(PTH, 1) k_probe_dense(const float* __restrict__ u, int64_t E,
                                                        float* __restrict__ out, int reduce, const ProbeOps ops) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint4* afr = reinterpret_cast<uint4*>(smem);                  // [MT][KT][hi, lo][32 lanes]
  float* us = reinterpret_cast<float*>(smem + DN_AFR);          // [DN_COLS][DN_LD]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  for (int idx = tid; idx < MT * KT * 32; idx += PTH) {
    const int ln = idx % 32, mk = idx / 32, k = mk % KT, m = mk / KT;
    const int gg = ln >> 2, tt = ln & 3;
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      split_tf32(dense_entry(ops, 16 * m + gg + 8 * (q & 1), 8 * k + tt + 4 * (q >> 1)), h[q], l[q]);
    afr[(mk * 2) * 32 + ln] = make_uint4(h[0], h[1], h[2], h[3]);
    afr[(mk * 2 + 1) * 32 + ln] = make_uint4(l[0], l[1], l[2], l[3]);
  }
  const int64_t ntiles = (E + DN_ET - 1) / DN_ET;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();  // fragments written; the previous tile's columns read
    const int64_t e0 = tile * DN_ET;
    const int ne = (int)min((int64_t)DN_ET, E - e0);
    const int ncols = 2 * ne;
    const float4* src = reinterpret_cast<const float4*>(u + e0 * 2 * PNU);
    for (int i = tid; i < ncols * PNU / 4; i += PTH) {
      const int col = i / (PNU / 4), w = i % (PNU / 4);
      *reinterpret_cast<float4*>(us + col * DN_LD + 4 * w) = __ldg(src + i);
    }
    __syncthreads();
    if (8 * warp >= ncols) continue;  // warp-uniform: no columns in this group
    const int col = 8 * warp + g;     // this lane's B column
    uint32_t bh[KT][2], bl[KT][2];
#pragma unroll
    for (int k = 0; k < KT; ++k)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float v = col < ncols ? us[col * DN_LD + 8 * k + t + 4 * q] : 0.f;
        split_tf32(v, bh[k][q], bl[k][q]);
      }
    const int c0 = 8 * warp + 2 * t;  // this lane's two C columns
    float cs0 = 0.f, cs1 = 0.f;
    for (int m = 0; m < MT; m += 2) {
      // two row tiles, three independent accumulator chains each
      float dl[2][4] = {}, dm[2][4] = {}, dh[2][4] = {};
#pragma unroll
      for (int k = 0; k < KT; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint4 a4 = afr[(((m + h) * KT + k) * 2) * 32 + lane];
          const uint4 b4 = afr[(((m + h) * KT + k) * 2 + 1) * 32 + lane];
          const uint32_t ah[4] = {a4.x, a4.y, a4.z, a4.w}, al[4] = {b4.x, b4.y, b4.z, b4.w};
          mma_tf32(dl[h], al, bh[k]);
          mma_tf32(dm[h], ah, bl[k]);
          mma_tf32(dh[h], ah, bh[k]);
        }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float d[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = (dl[h][q] + dm[h][q]) + dh[h][q];
        if (reduce) {
          cs0 += d[0] + d[2];
          cs1 += d[1] + d[3];
        } else if (c0 < ncols) {  // ncols and c0 are even: column c0 + 1 exists too
          const int r0 = 16 * (m + h) + g;
          float* o0 = out + (e0 * 2 + c0) * PM;
          o0[r0] = d[0];
          o0[r0 + 8] = d[2];
          o0[PM + r0] = d[1];
          o0[PM + r0 + 8] = d[3];
        }
      }
    }
    if (reduce) {
#pragma unroll
      for (int o = 4; o <= 16; o <<= 1) {
        cs0 += __shfl_xor_sync(0xffffffffu, cs0, o);
        cs1 += __shfl_xor_sync(0xffffffffu, cs1, o);
      }
      if (g == 0 && c0 < ncols) {
        out[e0 * 2 + c0] = cs0;
        out[e0 * 2 + c0 + 1] = cs1;
      }
    }
  }
}

}  // namespace
}  // namespace frp

extern "C" int fr_probe_hex_apply(int order, int form, int reduce, const float* u_dev, int64_t n_elems,
                                  float* out_dev, int64_t out_len, void* stream) {
  using namespace frp;
  if (order != 3) return FR_EUNSUPPORTED;
  if ((form != 0 && form != 1) || n_elems < 0) return FR_EINVAL;
  if (n_elems > ((int64_t)1 << 31) * SF_ET - SF_ET) return FR_EINVAL;  // form 0 grid limit
  if (n_elems == 0) return FR_OK;
  if (!u_dev || !out_dev || (reinterpret_cast<uintptr_t>(u_dev) & 15) != 0) return FR_EINVAL;
  const int64_t need = reduce ? n_elems * 2 : n_elems * 2 * PM;
  if (out_len < need) return FR_EINVAL;
  Tensor1D t1;
  build_tensor1d(order, t1);
  ProbeOps ops;
  for (int j = 0; j < PN; ++j) {
    ops.lend[0][j] = (float)t1.lend[0][j];
    ops.lend[1][j] = (float)t1.lend[1][j];
    for (int i = 0; i < PN; ++i) ops.D[i][j] = (float)t1.D[i][j];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (form == 0) {
    const int64_t grid = (n_elems + SF_ET - 1) / SF_ET;
    k_probe_sf<<<(unsigned)grid, PTH, 0, s>>>(u_dev, n_elems, out_dev, reduce, ops);
  } else {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FR_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FR_ECUDA;
    if (cudaFuncSetAttribute(k_probe_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DN_SMEM) !=
        cudaSuccess)
      return FR_ECUDA;
    const int64_t ntiles = (n_elems + DN_ET - 1) / DN_ET;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    k_probe_dense<<<grid, PTH, DN_SMEM, s>>>(u_dev, n_elems, out_dev, reduce, ops);
  }
  return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ECUDA;
}
