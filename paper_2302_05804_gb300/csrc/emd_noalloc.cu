// emd_noalloc.cu -- the one entry point of the library that allocates no
// device memory: per-exposure frame statistics in FP64.
//
// Some callers cannot call cudaMalloc: code that issues work while a stream
// is being captured into a CUDA graph (an allocation there either breaks the
// capture or has to be hoisted out of it), real-time pipelines that reserve
// all device memory up front, and frameworks whose device memory belongs to
// their own caching allocator. For them, emd_frame_stats_noalloc reads
// caller-owned device buffers and writes a caller-owned device output; its
// only scratch is a fixed-size array compiled into the library's device
// image (g_stats_part below), which every GPU that loads the library holds
// until the process exits.
//
// It computes, per exposure, the same quantities emd_set_frames derives
// for a context: the log-likelihood constant sum log(2 pi v), the sums
// sum u y and sum u behind the default start, and the count of valid pixels
// whose v or y is unusable -- with the same per-pixel arithmetic (u = 1/v in
// FP32 on valid pixels, FP64 sums), reading natural n x H x W layouts.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "emd_internal.cuh"

namespace {

constexpr int kNaBlocks = 64;     // blocks per exposure
constexpr int kNaThreads = 256;   // threads per block
constexpr int kNaMaxDevices = 64;

// Scratch: FP64 partial sums per (exposure, block): {log term, u y, u, bad}.
// Fully rewritten by every call, so nothing has to be cleared in between.
static __device__ __align__(256) double
    g_stats_part[EMD_NOALLOC_MAX_EXPOSURES * kNaBlocks * 4];

std::mutex g_mu;
double* g_part_dev[kNaMaxDevices];  // device address of g_stats_part, per device

__device__ __forceinline__ double na_block_sum(double v, double* red) {
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

__global__ void __launch_bounds__(kNaThreads) stats_partial_kernel(
    const float* __restrict__ y, const float* __restrict__ v, const uint8_t* __restrict__ mask,
    long long hw, double* __restrict__ part) {
  __shared__ double red[kNaThreads / 32];
  const int t = blockIdx.y;
  const long long base = (long long)t * hw;
  double ld = 0.0, suy = 0.0, su = 0.0, bad = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < hw;
       i += (long long)gridDim.x * blockDim.x) {
    const bool valid = mask ? (mask[base + i] != 0) : true;
    if (!valid) continue;
    const float vv = v[base + i], yv = y[base + i];
    if (!(vv > 0.f) || !isfinite(vv) || !isfinite(yv)) {
      bad += 1.0;
      continue;
    }
    const float u = 1.0f / vv;
    ld += log(6.283185307179586 * (double)vv);
    suy += (double)u * (double)yv;
    su += (double)u;
  }
  double* out = part + ((long long)t * gridDim.x + blockIdx.x) * 4;
  const double s0 = na_block_sum(ld, red);
  const double s1 = na_block_sum(suy, red);
  const double s2 = na_block_sum(su, red);
  const double s3 = na_block_sum(bad, red);
  if (threadIdx.x == 0) {
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
    out[3] = s3;
  }
}

// out[t][k] = sum over the blocks of exposure t, in block order
__global__ void stats_final_kernel(const double* __restrict__ part, int nblocks,
                                   double* __restrict__ out) {
  const int t = blockIdx.x, k = threadIdx.x;
  if (k >= 4) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[((long long)t * nblocks + b) * 4 + k];
  out[t * 4 + k] = s;
}

int na_fail(int code, const char* msg) {
  char m[256];
  snprintf(m, sizeof(m), "emd_frame_stats_noalloc: %s", msg);
  emd::set_error_message(m);
  return code;
}

// True for device memory of the current device `dev` and for managed
// memory. Device memory of another GPU is refused: the kernels would read it
// through peer addressing, which may not be enabled.
bool device_accessible(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int emd_frame_stats_noalloc(const float* y, const float* v, const uint8_t* mask,
                                       int H, int W, int n, double* out, void* stream) {
  if (!y || !v || !out) return na_fail(EMD_EINVAL, "y, v and out must not be NULL");
  if (H < 1 || W < 1 || n < 1) return na_fail(EMD_EINVAL, "H, W and n must be >= 1");
  if (n > EMD_NOALLOC_MAX_EXPOSURES) {
    char m[128];
    snprintf(m, sizeof(m), "n = %d exceeds the maximum of %d exposures", n,
             EMD_NOALLOC_MAX_EXPOSURES);
    return na_fail(EMD_EINVAL, m);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
    return na_fail(EMD_ECUDA, "no usable current device");
  if (!device_accessible(y, dev) || !device_accessible(v, dev) || !device_accessible(out, dev) ||
      (mask && !device_accessible(mask, dev)))
    return na_fail(EMD_EINVAL, "y, v, mask and out must be device pointers of the current device");
  double* part = nullptr;
  {
    // set-up, once per device with that device current: the host-side name
    // g_stats_part is not a device address, so look the address up
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_part_dev[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_stats_part);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return na_fail(EMD_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_part_dev[dev] = static_cast<double*>(p);
    }
    part = g_part_dev[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  stats_partial_kernel<<<dim3(kNaBlocks, n), kNaThreads, 0, st>>>(y, v, mask, (long long)H * W,
                                                                  part);
  stats_final_kernel<<<n, 32, 0, st>>>(part, kNaBlocks, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(EMD_ECUDA, cudaGetErrorString(e));
  return EMD_OK;
}
