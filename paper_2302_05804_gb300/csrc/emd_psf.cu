// emd_psf.cu -- super-resolved PSFs of Eq. (4) on the GPU:
//   h_t = argmin_{h >= 0} sum_ij ([D^r(h * g)]_ij - f_t,ij)^2 + lambda (grad h)_ij^2
// solved by projected Adam (the solver Sec. 2 names), one CTA per PSF. h,
// h * g (then the gradient), the residual, f and g stay in shared memory for
// all iterations; each thread owns fixed elements of the Adam moments, which
// live in global memory (read and written once per iteration, coalesced).
//
// Grids: f is K x K (coarse); h has Kh = r (K-1) + 1 fine pixels per side,
// fine pixel P belonging to coarse pixel P div r; h * g is the zero-padded
// 'same' convolution on the Kh x Kh grid, zero-extended to rK x rK before
// the r x r block sum; (grad h)^2 sums the squared forward differences
// inside the grid. Default start: the coarse PSF spread evenly over each
// block, h0[P][Q] = f[P div r][Q div r] / r^2.
#include <math.h>
#include <stdio.h>

#include "emd_internal.cuh"

namespace emd {
namespace {

constexpr int kPsfThreads = 512;

__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;  // valid in thread 0
}

// q = h * g ('same', zero outside the Kh x Kh grid)
__device__ __forceinline__ void psf_conv(const float* h, const float* gs, int Kh, int Kg,
                                         float* q) {
  const int nh = Kh * Kh, hg = (Kg - 1) / 2;
  for (int e = threadIdx.x; e < nh; e += blockDim.x) {
    const int P = e / Kh, Q = e % Kh;
    float s = 0.f;
    for (int a = 0; a < Kg; ++a) {
      const int ii = P + hg - a;
      if (ii < 0 || ii >= Kh) continue;
      for (int b = 0; b < Kg; ++b) {
        const int jj = Q + hg - b;
        if (jj < 0 || jj >= Kh) continue;
        s = fmaf(gs[a * Kg + b], h[ii * Kh + jj], s);
      }
    }
    q[e] = s;
  }
}

// res = D^r(q zero-extended to rK x rK) - f; with RED, returns sum res^2 in
// thread 0 (every thread must call it then)
template <bool RED>
__device__ __forceinline__ float psf_residual(const float* q, const float* fs, int K, int r,
                                              int Kh, float* res, float* red) {
  float acc = 0.f;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e / K, j = e % K;
    float s = 0.f;
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) {
        const int P = r * i + a, Q = r * j + b;
        if (P < Kh && Q < Kh) s += q[P * Kh + Q];
      }
    const float d = s - fs[e];
    res[e] = d;
    acc = fmaf(d, d, acc);
  }
  return RED ? block_sum(acc, red) : 0.f;
}

__global__ void __launch_bounds__(kPsfThreads, 1)
    psf_fit_kernel(const float* __restrict__ f, int K, int r, const float* __restrict__ g, int Kg,
                   const float* __restrict__ h0, float lambda, float lr, int iters,
                   float* __restrict__ mom, float* __restrict__ hout, float* __restrict__ loss) {
  extern __shared__ float sm[];
  __shared__ float red[kPsfThreads / 32];
  const int Kh = r * (K - 1) + 1, nh = Kh * Kh, nk = K * K, hg = (Kg - 1) / 2;
  float* h = sm;
  float* q = h + nh;    // h * g, then the gradient
  float* res = q + nh;  // D^r(h * g) - f
  float* fs = res + nk;
  float* gs = fs + nk;
  float* mo = mom + (long long)blockIdx.x * 2 * nh;
  float* vo = mo + nh;
  const float* ft = f + (long long)blockIdx.x * nk;
  const int tid = threadIdx.x;
  for (int e = tid; e < nk; e += blockDim.x) fs[e] = ft[e];
  for (int e = tid; e < Kg * Kg; e += blockDim.x) gs[e] = g[e];
  __syncthreads();
  const float inv_r2 = 1.0f / (float)(r * r);
  for (int e = tid; e < nh; e += blockDim.x) {
    const int P = e / Kh, Q = e % Kh;
    h[e] = h0 ? h0[(long long)blockIdx.x * nh + e] : fs[(P / r) * K + Q / r] * inv_r2;
    mo[e] = 0.f;
    vo[e] = 0.f;
  }
  __syncthreads();
  double p1 = 1.0, p2 = 1.0;
  for (int k = 1; k <= iters; ++k) {
    psf_conv(h, gs, Kh, Kg, q);
    __syncthreads();
    psf_residual<false>(q, fs, K, r, Kh, res, red);
    __syncthreads();
    // gradient: 2 (g-correlation of the replicated residual) + smoothness
    for (int e = tid; e < nh; e += blockDim.x) {
      const int P = e / Kh, Q = e % Kh;
      float s = 0.f;
      for (int a = 0; a < Kg; ++a) {
        const int ii = P - hg + a;
        if (ii < 0 || ii >= Kh) continue;
        for (int b = 0; b < Kg; ++b) {
          const int jj = Q - hg + b;
          if (jj < 0 || jj >= Kh) continue;
          s = fmaf(gs[a * Kg + b], res[(ii / r) * K + jj / r], s);
        }
      }
      const float c = h[e];
      float d = 0.f;
      if (P >= 1) d += c - h[e - Kh];
      if (P + 1 < Kh) d -= h[e + Kh] - c;
      if (Q >= 1) d += c - h[e - 1];
      if (Q + 1 < Kh) d -= h[e + 1] - c;
      q[e] = 2.f * s + 2.f * lambda * d;
    }
    __syncthreads();
    // projected Adam step (Kingma & Ba, bias-corrected), h >= 0
    p1 *= 0.9;
    p2 *= 0.999;
    const float c1 = (float)(1.0 - p1), c2 = (float)(1.0 - p2);
    for (int e = tid; e < nh; e += blockDim.x) {
      const float gr = q[e];
      const float m = 0.9f * mo[e] + 0.1f * gr;
      const float v = 0.999f * vo[e] + 0.001f * gr * gr;
      mo[e] = m;
      vo[e] = v;
      h[e] = fmaxf(h[e] - lr * (m / c1) / (sqrtf(v / c2) + 1e-8f), 0.f);
    }
    __syncthreads();
  }
  float* ho = hout + (long long)blockIdx.x * nh;
  for (int e = tid; e < nh; e += blockDim.x) ho[e] = h[e];
  if (loss) {
    psf_conv(h, gs, Kh, Kg, q);
    __syncthreads();
    const float data = psf_residual<true>(q, fs, K, r, Kh, res, red);
    float acc = 0.f;
    for (int e = tid; e < nh; e += blockDim.x) {
      const int P = e / Kh, Q = e % Kh;
      if (P + 1 < Kh) { const float d = h[e + Kh] - h[e]; acc = fmaf(d, d, acc); }
      if (Q + 1 < Kh) { const float d = h[e + 1] - h[e]; acc = fmaf(d, d, acc); }
    }
    const float smooth = block_sum(acc, red);
    if (tid == 0) loss[blockIdx.x] = data + lambda * smooth;
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int psf_fail(int code, const char* msg) {
  char m[256];
  snprintf(m, sizeof(m), "emd_fit_psf: %s", msg);
  set_error_message(m);
  return code;
}

size_t psf_fit_smem_bytes(int K, int r, int Kg) {
  const size_t Kh = (size_t)r * (K - 1) + 1;
  return (2 * Kh * Kh + 2ull * K * K + (size_t)Kg * Kg) * sizeof(float);
}

}  // namespace
}  // namespace emd

extern "C" int emd_fit_psf(const float* f, int n, int K, int r, const float* g, int Kg,
                           const float* h0, float lambda, float lr, int iters, float* h_out,
                           float* loss_out) {
  using namespace emd;
  if (!f || !g || !h_out) return psf_fail(EMD_EINVAL, "f, g and h_out must not be NULL");
  if (n < 1 || K < 1 || (K % 2) == 0 || r < 1 || Kg < 1 || (Kg % 2) == 0 || iters < 0 ||
      !(lambda >= 0.f) || !(lr > 0.f))
    return psf_fail(EMD_EINVAL,
                    "need n >= 1, odd K, r >= 1, odd Kg, iters >= 0, lambda >= 0, lr > 0");
  if (r > 8 || K > EMD_PSF_MAX_COARSE || Kg > EMD_PSF_MAX_COARSE)
    return psf_fail(EMD_EINVAL, "need r <= 8 and K, Kg <= EMD_PSF_MAX_COARSE");
  const size_t smem = psf_fit_smem_bytes(K, r, Kg);
  if (smem > 200 * 1024) return psf_fail(EMD_EUNSUPPORTED, "fine PSF too large for one CTA");
  const int Kh = r * (K - 1) + 1;
  const size_t fb = (size_t)n * K * K * sizeof(float), gb = (size_t)Kg * Kg * sizeof(float),
               hb = (size_t)n * Kh * Kh * sizeof(float), lb = (size_t)n * sizeof(float);
  const bool fd = on_device(f), gd = on_device(g), hd = on_device(h_out);
  const bool h0d = h0 ? on_device(h0) : true, ld = loss_out ? on_device(loss_out) : true;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t need = up(2 * hb) + (fd ? 0 : up(fb)) + (gd ? 0 : up(gb)) + (hd ? 0 : up(hb)) +
                      (h0d ? 0 : up(hb)) + (ld ? 0 : up(lb));
  char* tmp = nullptr;
  if (cudaMalloc(&tmp, need) != cudaSuccess) {
    cudaGetLastError();
    return psf_fail(EMD_ENOMEM, "device allocation failed");
  }
  size_t off = 0;
  auto take = [&](size_t b) { char* p = tmp + off; off += up(b); return p; };
  float* mom = reinterpret_cast<float*>(take(2 * hb));
  const float* df = fd ? f : reinterpret_cast<float*>(take(fb));
  const float* dg = gd ? g : reinterpret_cast<float*>(take(gb));
  float* dh = hd ? h_out : reinterpret_cast<float*>(take(hb));
  const float* dh0 = h0d ? h0 : reinterpret_cast<float*>(take(hb));
  float* dl = ld ? loss_out : reinterpret_cast<float*>(take(lb));
  int rc = EMD_OK;
  cudaError_t e = cudaSuccess;
  if (!fd) e = cudaMemcpy(const_cast<float*>(df), f, fb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !gd)
    e = cudaMemcpy(const_cast<float*>(dg), g, gb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !h0d)
    e = cudaMemcpy(const_cast<float*>(dh0), h0, hb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(psf_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e == cudaSuccess) {
    psf_fit_kernel<<<n, kPsfThreads, smem>>>(df, K, r, dg, Kg, dh0, lambda, lr, iters, mom, dh,
                                             dl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess && !hd) e = cudaMemcpy(h_out, dh, hb, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && !ld) e = cudaMemcpy(loss_out, dl, lb, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = psf_fail(EMD_ECUDA, cudaGetErrorString(e));
  cudaFree(tmp);
  return rc;
}
