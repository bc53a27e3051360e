// emd_fft.cuh -- declarations of the FFT form (csrc/emd_fft.cu), kept apart
// from emd_internal.cuh so that changes here leave the direct kernel's
// sources untouched.
#pragma once

#include "emd_internal.cuh"

namespace emd {

// FFT path: overlap-save on 128 x 128 tiles
struct FftLaunch {
  const float* x;       // current iterate (padded plane)
  float* xn;            // next iterate
  const float* N;       // numerator
  const float* u;       // n weight planes
  float* w;             // n planes of u_t z_t (written by the forward pass)
  const float2* spec;   // n R2 half spectra of the phase kernels, 65 columns x 128 rows each
  float2* scratch;      // r > 1: per tile, R2 half spectra (x^ of the phases, then the
                        // adjoint's accumulators); unused for r = 1
};
size_t fft_buffer_bytes(const Shape& s);
size_t fft_smem_bytes();
int fft_tile_side(const Shape& s);
size_t fft_scratch_offset(const Shape& s);  // bytes before the scratch in the FFT buffer
cudaError_t launch_fft_spectra(const Shape& s, const float* ka, float2* spec, cudaStream_t st);
cudaError_t launch_fft_iter(const Shape& s, const FftLaunch& a, cudaStream_t st);

}  // namespace emd
