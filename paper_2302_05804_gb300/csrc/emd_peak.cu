// emd_peak.cu -- measured FP32 FMA rate of this GPU: independent FMA chains
// in every thread of a grid that fills the SMs, timed with CUDA events. The
// roofline of the direct FP32 kernel is reported against it (beside the
// rate derived from the unit counts and the maximum clock).
#include <stdio.h>

#include "emd_internal.cuh"

namespace emd {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) fma_chain_kernel(float* __restrict__ out, int iters,
                                                        float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains alive, never true in practice
}

int peak_fail(int code, const char* msg) {
  char m[256];
  snprintf(m, sizeof(m), "emd_measure_fma_rate: %s", msg);
  set_error_message(m);
  return code;
}

}  // namespace
}  // namespace emd

extern "C" int emd_measure_fma_rate(int iters, double* tflops) {
  using namespace emd;
  if (!tflops || iters < 1) return peak_fail(EMD_EINVAL, "need tflops != NULL and iters >= 1");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return peak_fail(EMD_ECUDA, "no CUDA device");
  }
  const int blocks = sms * 8, threads = 256;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, blocks * sizeof(float));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    fma_chain_kernel<<<blocks, threads, 0, st>>>(out, iters / 4 + 1, 0.9999999f, 1e-7f);  // warm
    cudaEventRecord(e0, st);
    fma_chain_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return peak_fail(EMD_ECUDA, cudaGetErrorString(e));
  const double fmas = (double)blocks * threads * iters * kUnroll * kChains;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return EMD_OK;
}
