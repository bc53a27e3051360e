// emd_internal.cuh -- shared declarations of the CUDA library (not part of
// the public ABI). Data layout in HBM:
//
//   * every image plane (one exposure's u or y, one polyphase component of
//     x, N or Den) is stored padded: the coarse pixel (i, j) lives at
//     plane[(B + i) * P + (B + j)], with a zero border of B = 2*hc pixels on
//     the top/left and enough zero rows/columns on the bottom/right for the
//     last tile's halo reads. P is a multiple of 8 floats, so rows start on
//     32-byte boundaries and the x staging copies of the fused kernel start
//     16-byte aligned.
//   * the latent (rH) x (rW) image is stored as r^2 polyphase planes of
//     H x W: plane phi = py*r + px holds x[r*I + py][r*J + px]. With that
//     layout Eq. (3)'s D^r(h * x) is a sum over phases of H x W
//     convolutions with Kc x Kc kernels, Kc = 2*hc + 1,
//     hc = floor(((K-1)/2 + r - 1) / r), and its transpose is one
//     correlation per phase. r = 1 is the single plane of Eq. (1).
//   * per exposure t and phase phi two Kc x KP kernels (KP = Kc rounded up
//     to 4, zero columns on the right): kf = the convolution kernel flipped
//     (the forward model as a correlation) and ka = unflipped (the adjoint).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "emd.h"

namespace emd {

constexpr int kTile = 128;      // Den tile side handled by one CTA pair
constexpr int kHalf = 64;       // Den rows per CTA of the pair
constexpr int kThreads = 256;   // threads per CTA of the direct kernels
constexpr int kRedBlocks = 1024;  // fixed grid of the FP64 reductions

// device error word bits
constexpr int kErrData = 1;
constexpr int kErrTimeout = 2;

struct Geom {
  int H, W;       // coarse (exposure) size
  int B;          // zero border before the image, rows and columns
  int P;          // row pitch in floats
  int PH;         // rows per plane
  long long plane;  // floats per plane (PH * P)
};

// Shapes derived from (K, r) that every kernel uses.
struct Shape {
  int H, W, n, K, r, R2;
  int hc, Kc, KP;
  int gx, gy;          // 128 x 128 tiles
  int Rh;              // forward-region rows per CTA of the pair
  int MXf;             // forward-region columns / 16
  int xrows, xpitch;   // staged x tile (per CTA)
  int wrows, wpitch;   // w tile (per CTA, own rows + halo rows)
  size_t smem_fused;   // dynamic shared memory of the fused kernel
  Geom g;
};

bool make_shape(int H, int W, int n, int K, int r, Shape* s, const char** why);

struct FusedArgs {
  const float* x;     // R2 planes (current iterate)
  float* xn;          // R2 planes (next iterate)
  const float* u;     // n planes
  const float* y;     // n planes (numerator mode)
  const float* kf;    // n * R2 kernels Kc x KP (flipped)
  const float* ka;    // n * R2 kernels Kc x KP
  const float* N;     // R2 planes (input of mode 0)
  float* Nw;          // R2 planes (output of mode 1)
  float* Den;         // R2 planes (scratch between exposures)
  int* err;
  int t0, t1;         // exposures [t0, t1) of this launch (all: 0, n)
  float nu;           // Student-t degrees of freedom; 0 = Gaussian noise
};

struct SetupArgs {
  const uint8_t* mask;  // n x H x W uint8 (natural layout, device), or null
  float* u;             // in: v (copied into the u planes); out: u
  float* y;             // in/out: y; masked pixels become 0
  double* part;         // kRedBlocks x 4 partial sums
  int* err;
};

// one job of a batch (device-side table entry)
struct BatchJob {
  Shape s;
  FusedArgs a[2];  // arguments with x = buffer c, xn = buffer c^1, for c = cur
  int cur;         // current x buffer
  int remaining;   // iterations still to run (0: skipped)
};

size_t batch_smem_bytes();
int batch_max_clusters(size_t smem);
// memset(counter) + persistent kernel + advance, all on st (graph-capturable)
cudaError_t launch_batch(const BatchJob* jobs, int njobs, const int2* items, const int* n_items,
                         int* counter, int* err, int clusters, size_t smem, cudaStream_t st);

// sets the thread-local message returned by emd_last_error (emd_api.cu)
void set_error_message(const char* msg);

// Raises a kernel's dynamic shared-memory limit to the most the current
// device allows it (the opt-in maximum per block less the kernel's static
// shared memory), once per kernel and device. The limit is never set to one
// launch's size: host threads launching one kernel for problems of different
// shapes would race, one thread's smaller setting failing another's launch.
cudaError_t allow_max_dynamic_smem(const void* func);

// kernels (emd_direct.cu)
cudaError_t launch_setup(const Shape& s, const SetupArgs& a, cudaStream_t st);
cudaError_t launch_reduce_final(const double* part, int nblocks, int ncols,
                                double* out, cudaStream_t st);
cudaError_t launch_build_kernels(const Shape& s, const float* f_raw, float* kf,
                                 float* ka, cudaStream_t st);
// mode 0: one EM iteration a.x -> a.xn; mode 1: numerator into a.Nw;
// mode 2: chi-square partial sums into part[fused_blocks(s)].
cudaError_t launch_fused(const Shape& s, const FusedArgs& a, int mode, double* part,
                         cudaStream_t st);
int fused_blocks(const Shape& s);
// one CTA waiting (bounded by `limit` polls) on an mbarrier nothing arrives on
cudaError_t launch_wait_selftest(uint32_t limit, int* err, cudaStream_t st);
cudaError_t launch_fill_latent(const Shape& s, float* x, float c,
                               cudaStream_t st);
cudaError_t launch_scatter_latent(const Shape& s, const float* nat, float* planes,
                                  int clamp_neg, cudaStream_t st);
cudaError_t launch_gather_latent(const Shape& s, const float* planes, float* nat,
                                 cudaStream_t st);

}  // namespace emd
