// emd_corr.cuh -- device code shared by the direct-form kernels (the fused
// CTA-pair kernel and the halo-exchange kernel): an FP64 block sum, and the
// register-blocked FP32 correlation, where a thread accumulates an RY x RX
// block of outputs
//     acc[p][c] += sum_{a < Kc, b < KP} k[a][b] src[oy + p + a][ox + c + b]
// from a shared-memory plane, one 16-byte kernel quad and a (RX + 4)-float
// window of the source row at a time.
#pragma once

#include <cuda_runtime.h>

namespace emd {

struct SPlane {
  float* base;
  int pitch;
  int shift;  // row R starts at base + R*pitch + 4*(R >> shift)
};

__device__ __forceinline__ float* srow(const SPlane& p, int R) {
  return p.base + R * p.pitch + ((R >> p.shift) << 2);
}

template <int RY, int RX, bool CHECK>
__device__ __forceinline__ void corr_row(float (&acc)[RY][RX], const float* __restrict__ row,
                                         const float* __restrict__ ks, int KP, int Kc, int s) {
  const float4* row4 = reinterpret_cast<const float4*>(row);
#pragma unroll 2
  for (int bq = 0; bq < (KP >> 2); ++bq) {
    float xv[RX + 4];
#pragma unroll
    for (int m = 0; m < RX / 4 + 1; ++m) {
      const float4 v = row4[bq + m];
      xv[4 * m + 0] = v.x;
      xv[4 * m + 1] = v.y;
      xv[4 * m + 2] = v.z;
      xv[4 * m + 3] = v.w;
    }
#pragma unroll
    for (int p = 0; p < RY; ++p) {
      const int a = s - p;
      if (!CHECK || (a >= 0 && a < Kc)) {
        const float4 kv = reinterpret_cast<const float4*>(ks + a * KP)[bq];
        // one tap at a time across the 16 outputs: each accumulator still
        // takes its taps in order, consecutive FMAs share the kernel operand
#pragma unroll
        for (int c = 0; c < RX; ++c) acc[p][c] = fmaf(kv.x, xv[c + 0], acc[p][c]);
#pragma unroll
        for (int c = 0; c < RX; ++c) acc[p][c] = fmaf(kv.y, xv[c + 1], acc[p][c]);
#pragma unroll
        for (int c = 0; c < RX; ++c) acc[p][c] = fmaf(kv.z, xv[c + 2], acc[p][c]);
#pragma unroll
        for (int c = 0; c < RX; ++c) acc[p][c] = fmaf(kv.w, xv[c + 3], acc[p][c]);
      }
    }
  }
}

template <int RY, int RX>
__device__ __forceinline__ void corr_tile(float (&acc)[RY][RX], const SPlane& src, int oy,
                                          int ox, const float* __restrict__ ks, int KP,
                                          int Kc) {
#pragma unroll 1
  for (int s = 0; s < Kc + RY - 1; ++s) {
    const float* row = srow(src, oy + s) + ox;
    if (s >= RY - 1 && s < Kc)
      corr_row<RY, RX, false>(acc, row, ks, KP, Kc, s);
    else
      corr_row<RY, RX, true>(acc, row, ks, KP, Kc, s);
  }
}

// Sum of v over the CTA, in FP64 (warp shuffles, then the warps in order).
__device__ __forceinline__ double block_sum_f64(double v, double* red /* >= 8 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;  // valid in thread 0
}

}  // namespace emd
