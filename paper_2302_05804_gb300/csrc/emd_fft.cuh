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
  float2* scratch;      // per tile (r > 1 or Student-t): R2 half spectra of the phases
                        // of x, then the adjoint's accumulators (R2, or 2 R2 for
                        // Student-t: Den then N'); unused for r = 1 Gaussian
  const float* y;       // Student-t: n data planes (masked pixels 0)
  float* w2;            // Student-t: n planes of u'_t y_t
  float nu;             // Student-t degrees of freedom; 0 = Gaussian
  // split launch (r = 1, at least split_ctas tiles): split_ctas persistent
  // CTAs take equal ranges of the (tile, exposure) units; an adjoint tile
  // cut between two CTAs passes its head's accumulator through the head
  // CTA's slot (partials, one per CTA) and the tile's flag (counters).
  // split_ctas = 0: one CTA per tile.
  float2* partials;
  int* counters;
  int split_ctas;
  int* err;  // device error word (a bounded wait that gives up sets kErrTimeout)
};
// bytes of the FFT buffer; split_ctas > 0 adds the split launch's partial
// accumulators and counters (r = 1 Gaussian)
size_t fft_buffer_bytes(const Shape& s, bool student, int split_ctas = 0);
size_t fft_split_offset(const Shape& s, bool student);     // bytes before the partials
size_t fft_counters_offset(const Shape& s, bool student, int split_ctas);
size_t fft_smem_bytes();
int fft_tile_side(const Shape& s);
size_t fft_w2_offset(const Shape& s);                      // bytes before the w2 planes
size_t fft_scratch_offset(const Shape& s, bool student);  // bytes before the scratch
cudaError_t launch_fft_spectra(const Shape& s, const float* ka, float2* spec, cudaStream_t st);
cudaError_t launch_fft_iter(const Shape& s, const FftLaunch& a, cudaStream_t st);

// batch of FFT jobs: persistent forward and adjoint kernels over (job, tile)
struct FftBatchJob {
  Shape s;
  FftLaunch a[2];  // with x = buffer c, xn = buffer c^1, for c = cur
  int cur;
  int remaining;   // iterations still to run (0: skipped)
  int gxt;         // FFT tiles per row
};
int fft_tiles_x(const Shape& s);
int fft_tiles_total(const Shape& s);
cudaError_t launch_fft_batch(const FftBatchJob* jobs, int njobs, const int2* items,
                             const int* n_items, int* counters, int ctas, cudaStream_t st);

}  // namespace emd
