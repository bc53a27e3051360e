// emd_tc.cuh -- declarations of the tensor-core path (csrc/emd_tc.cu), kept
// apart from emd_internal.cuh so that changes here leave the direct
// kernel's sources untouched.
#pragma once

#include <cuda.h>

#include "emd_internal.cuh"

namespace emd {

struct TcShape {
  int mode, fp16, nprod;
  int NW;           // tile columns (128) = MMA N; tile rows 128 = MMA M
  int Kd;           // K extent of a band: dlt + 128 + 2 hc, rounded up to 16
  int dlt;          // hc mod 8: band columns before the window (16-byte aligned start)
  int XRp;          // band rows: 128 + 2 hc rounded up to 8
  int Sd;           // Hankel core matrices per filter row
  int gxt, gyt;     // tiles
  int stage_bytes;  // one ring stage (hi + lo)
  int hank_block;   // bytes of the Hankel block of one (t, phi, a): forward, adjoint
  size_t smem;
};

struct TcLaunch {
  const float* x;
  float* xn;
  const float* N;
  float* Den;
  const float* u;
  uint16_t* xb;          // [2 ping-pong][2 hi/lo][R2] 16-bit planes
  uint16_t* wb;          // [2 hi/lo][n] 16-bit planes of w = u z (zero outside the image)
  const uint16_t* hank;  // Hankel blocks
  int pp;                // ping-pong slot of the current x
  const float* scales;   // device {z, w, Den, x} scales (all 1 for BF16)
  int write_xb;
  int* err;
};

bool make_tc_shape(const Shape& s, int mode, TcShape* t, const char** why);
size_t tc_buffer_bytes(const Shape& s, const TcShape& t);
size_t tc_w_offset(const Shape& s, const TcShape& t);  // byte offset of the w planes
int make_plane_tensormap(const Shape& s, const TcShape& t, void* base, int planes,
                         CUtensorMap* map);
cudaError_t launch_build_hankel(const Shape& s, const TcShape& t, const float* kf, const float* ka,
                                uint16_t* hank, float gscale, cudaStream_t st);
cudaError_t launch_split_x(const Shape& s, const TcShape& t, const float* x, uint16_t* xb, int pp,
                           const float* scales, cudaStream_t st);
cudaError_t launch_max_nonneg(const float* v, long long count, unsigned int* out, cudaStream_t st);
cudaError_t launch_fp16_scales(const unsigned int* xmax_bits, float gscale, float umax, float fsum,
                               float* scales, cudaStream_t st);
// the forward kernel (x bands through xmap; w planes written) and the
// adjoint-and-update kernel (w bands through wmap), stream-ordered
cudaError_t launch_tc_iter(const Shape& s, const TcShape& t, const TcLaunch& L,
                           const CUtensorMap& xmap, const CUtensorMap& wmap, cudaStream_t st);

}  // namespace emd
