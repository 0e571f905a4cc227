// Warp-level tensor-core contraction for the small dense FR operators of the
// float path (triangles): Y[c][r] = sum_k Op[r][k] X[c][k] over a tile of
// columns c (element-field pairs) held in shared memory.
//
// Each product runs on mma.sync m16n8k8 with TF32 inputs and FP32
// accumulation, in the compensated three-term form: with a = a_h + a_l and
// x = x_h + x_l split into TF32 parts (a_h the TF32 rounding of a, a_l the
// TF32 value of the remainder), a x ~ a_l x_h + a_h x_l + a_h x_h, dropping
// a_l x_l (relative 2^-22).  The result carries FP32 accuracy (parity with
// the scalar FP32 kernels to round-off) at tensor-core throughput.
//
// Fragment layout of m16n8k8 (.tf32): lane = 4 g + t.  A (16 x 8, row
// major): a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4).  B
// (8 x 8, column major): b0 (t, g), b1 (t + 4, g).  C/D (16 x 8): c0 (g, 2t),
// c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace frp {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

// (hi, lo) TF32 parts of x
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Y = Op X for M operator rows, K inner indices and ncols columns, by the
// warps of the block.  opf(r, k) returns Op[r][k] (called only for r < M,
// k < K), xf(c, k) returns X[c][k] (c < ncols, k < K), yf(c, r, v) stores
// Y[c][r] (c < ncols, r < M).  Work items are (16-row tile, 8-column group)
// pairs; a warp loads its row tile's operator fragments once.
template <int M, int K, typename OpF, typename XF, typename YF>
__device__ __forceinline__ void warp_gemm_3xtf32(int ncols, OpF opf, XF xf, YF yf) {
  constexpr int MT = (M + 15) / 16, KT = (K + 7) / 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ng = (ncols + 7) / 8;
  for (int m = 0; m < MT; ++m) {
    if (warp >= ng) break;
    uint32_t ah[KT][4], al[KT][4];
#pragma unroll
    for (int k = 0; k < KT; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = 16 * m + g + 8 * (q & 1), c = 8 * k + t + 4 * (q >> 1);
        const float v = (r < M && c < K) ? opf(r, c) : 0.f;
        split_tf32(v, ah[k][q], al[k][q]);
      }
    for (int cg = warp; cg < ng; cg += nw) {
      const int col = 8 * cg + g;  // this lane's B column
      uint32_t bh[KT][2], bl[KT][2];
#pragma unroll
      for (int k = 0; k < KT; ++k)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int kk = 8 * k + t + 4 * q;
          const float v = (col < ncols && kk < K) ? xf(col, kk) : 0.f;
          split_tf32(v, bh[k][q], bl[k][q]);
        }
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < KT; ++k) {
        mma_tf32(d, al[k], bh[k]);
        mma_tf32(d, ah[k], bl[k]);
      }
#pragma unroll
      for (int k = 0; k < KT; ++k) mma_tf32(d, ah[k], bh[k]);
      const int r0 = 16 * m + g, c0 = 8 * cg + 2 * t;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + 8 * (q >> 1), c = c0 + (q & 1);
        if (r < M && c < ncols) yf(c, r, d[q]);
      }
    }
  }
}

}  // namespace frp
