// emd_psf.cu -- super-resolved PSFs of Eq. (4) on the GPU:
//   h_t = argmin_{h >= 0} sum_ij ([D^r(h * g)]_ij - f_t,ij)^2 + lambda (grad h)_ij^2
// solved by projected Adam (the solver Sec. 2 names).
//
// Grids: f is K x K (coarse); h has Kh = r (K-1) + 1 fine pixels per side,
// fine pixel P belonging to coarse pixel P div r; h * g is the zero-padded
// 'same' convolution on the Kh x Kh grid, zero-extended to rK x rK before
// the r x r block sum; (grad h)^2 sums the squared forward differences
// inside the grid. Default start: the coarse PSF spread evenly over each
// block, h0[P][Q] = f[P div r][Q div r] / r^2.
//
// One thread-block cluster of C CTAs per PSF (C up to 8, chosen so that the
// clusters of all PSFs fill the SMs); CTA c owns the band of fine rows
// [c BR, (c+1) BR), BR a multiple of r, so every coarse row lies in one band.
// Each CTA keeps h and the replicated residual as full zero-haloed planes
// (hp, rp; halo hg = (Kg-1)/2) plus the coarse residual, f and g in shared
// memory, but computes only its band; the rows it needs from other bands
// (hg fine rows of h, the coarse residual rows under hg fine rows) are read
// from their owners' shared memory (DSMEM) after a cluster barrier. Both
// correlations of an iteration (h * g, then the adjoint g-correlation of the
// replicated residual) run as register strips of kStrip fine pixels along a
// row: a thread loads the strip's input row segment with 128-bit loads and
// reuses each filter tap, loaded as a 128-bit shared-memory broadcast,
// kStrip times. Consecutive threads take consecutive rows of one column
// block; the plane pitch is 4 mod 8 floats, so the eight threads of each
// 128-bit load phase hit distinct banks. The Adam moments and the new h of
// each step live in global memory (each element touched once per step).
//
// One iteration (CB = cluster barrier, sb = CTA barrier):
//   A  q = h * g on the band (q parked in the band's rows of rp)        sb
//   A2 res = D^r(q) - f on the band's coarse rows; data-loss partial     CB
//      pull the coarse residual rows other bands own                      sb
//   B  rp = rep(res) on the band and its hg-row halo                      sb
//   C  grad = 2 g-corr(rp) + 2 lambda (smoothness), Adam -> new h;
//      smoothness-loss partial; CTA partials                              CB
//   D  loss of h_k from all CTAs' partials (same order everywhere); keep
//      h_k if it is the best so far; band of hp <- new h                   CB
//      pull the hg halo rows of the new h from their owners               sb
// The fit returns the iterate of lowest Eq. (4) loss among h_0 .. h_iters
// (the first on ties): Adam at a fixed step is not monotone once its
// moments have decayed.
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>

#include "emd_internal.cuh"

namespace cg = cooperative_groups;

namespace emd {
namespace {

constexpr int kPsfThreads = 512;
constexpr int kPsfWarps = kPsfThreads / 32;
constexpr int kStrip = 4;
constexpr int kMaxCluster = 8;

__host__ __device__ constexpr int rup4(int v) { return (v + 3) & ~3; }

struct PsfGeom {
  int K, r, Kg, hg, Kh, ncb, XL, HC, HR, KGP, C, BR;
};

// C: CTAs per PSF requested (1..8); the band height BR and the final C
// (every band non-empty) follow.
__host__ __device__ inline PsfGeom psf_geom(int K, int r, int Kg, int C) {
  PsfGeom G;
  G.K = K;
  G.r = r;
  G.Kg = Kg;
  G.hg = (Kg - 1) / 2;
  G.Kh = r * (K - 1) + 1;
  G.ncb = (G.Kh + kStrip - 1) / kStrip;
  G.XL = rup4(kStrip + Kg - 1);           // input segment of a strip, whole float4s
  int hc = (G.ncb - 1) * kStrip + G.XL;   // last segment's end
  hc = (hc + 7) & ~7;
  G.HC = hc + 4;                          // pitch = 4 (mod 8) floats
  G.HR = G.Kh + Kg - 1;
  G.KGP = rup4(Kg);
  const int rows = (G.Kh + C - 1) / C;
  G.BR = ((rows + r - 1) / r) * r;
  G.C = (G.Kh + G.BR - 1) / G.BR;
  return G;
}

// floats of dynamic shared memory: hp, rp, g, g flipped, res, f
size_t psf_smem_floats(const PsfGeom& G) {
  return 2 * (size_t)G.HR * G.HC + 2 * (size_t)G.K * G.K + 2 * (size_t)G.Kg * G.KGP;
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// acc[c] = sum_{a,b} w[a][b] src[(P + a) HC + Q0 + c + b], c < kStrip;
// w rows padded to KGP floats
template <int KG>
__device__ __forceinline__ void corr_strip(const float* src, const float* w, int HC, int P,
                                           int Q0, float (&acc)[kStrip]) {
  constexpr int XL = rup4(kStrip + KG - 1), KGP = rup4(KG);
#pragma unroll
  for (int c = 0; c < kStrip; ++c) acc[c] = 0.f;
#pragma unroll 1
  for (int a = 0; a < KG; ++a) {
    const float4* row = reinterpret_cast<const float4*>(src + (P + a) * HC + Q0);
    float x[XL];
#pragma unroll
    for (int m = 0; m < XL / 4; ++m) {
      const float4 v = row[m];
      x[4 * m] = v.x;
      x[4 * m + 1] = v.y;
      x[4 * m + 2] = v.z;
      x[4 * m + 3] = v.w;
    }
    float wr[KGP];
    const float4* wrow = reinterpret_cast<const float4*>(w + a * KGP);
#pragma unroll
    for (int m = 0; m < KGP / 4; ++m) {
      const float4 v = wrow[m];
      wr[4 * m] = v.x;
      wr[4 * m + 1] = v.y;
      wr[4 * m + 2] = v.z;
      wr[4 * m + 3] = v.w;
    }
#pragma unroll
    for (int b = 0; b < KG; ++b)
#pragma unroll
      for (int c = 0; c < kStrip; ++c) acc[c] = fmaf(wr[b], x[c + b], acc[c]);
  }
}

template <int KG>
__global__ void __launch_bounds__(kPsfThreads, 1)
    psf_fit_kernel(const float* __restrict__ f, int K, int r, const float* __restrict__ g,
                   const float* __restrict__ h0, float lambda, float lr, int iters, int Creq,
                   float* mom, float* hnew, float* hout, float* __restrict__ loss) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float wpart[2][kPsfWarps];
  __shared__ float cta_part[2];
  cg::cluster_group cl = cg::this_cluster();
  const PsfGeom G = psf_geom(K, r, KG, Creq);
  const int crank = (int)cl.block_rank();
  const int psf = blockIdx.x / G.C;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nk = K * K, PS = G.HR * G.HC, nh = G.Kh * G.Kh;
  const int R0 = crank * G.BR, R1 = min(G.Kh, R0 + G.BR), nrows = R1 - R0;
  const int i0 = R0 / r, i1 = (R1 + r - 1) / r;  // the band's coarse rows
  float* hp = sm;  // planes and filters first: their float4 loads need 16-byte alignment
  float* rp = hp + PS;
  float* gs = rp + PS;
  float* gfs = gs + KG * G.KGP;
  float* res = gfs + KG * G.KGP;
  float* fs = res + nk;
  float* mo = mom + (long long)psf * 2 * nh;
  float* vo = mo + nh;
  float* hn = hnew + (long long)psf * nh;
  float* hb = hout + (long long)psf * nh;  // best iterate so far
  const float* ft = f + (long long)psf * nk;
  auto hpix = [&](float* plane, int P, int Q) -> float& {
    return plane[(P + G.hg) * G.HC + G.hg + Q];
  };

  for (int e = tid; e < 2 * PS; e += nt) hp[e] = 0.f;  // hp and rp with their halos
  for (int e = tid; e < nk; e += nt) fs[e] = ft[e];
  for (int e = tid; e < KG * G.KGP; e += nt) {
    const int a = e / G.KGP, b = e - a * G.KGP;
    gs[e] = b < KG ? g[a * KG + b] : 0.f;
    gfs[e] = b < KG ? g[(KG - 1 - a) * KG + (KG - 1 - b)] : 0.f;
  }
  __syncthreads();
  const float inv_r2 = 1.0f / (float)(r * r);
  for (int P = warp; P < G.Kh; P += kPsfWarps)  // every CTA holds all of h
    for (int Q = lane; Q < G.Kh; Q += 32)
      hpix(hp, P, Q) = h0 ? h0[(long long)psf * nh + P * G.Kh + Q] : fs[(P / r) * K + Q / r] * inv_r2;
  for (int P = R0 + warp; P < R1; P += kPsfWarps)
    for (int Q = lane; Q < G.Kh; Q += 32) {
      mo[P * G.Kh + Q] = 0.f;
      vo[P * G.Kh + Q] = 0.f;
    }
  __syncthreads();

  const int nstrip = nrows * G.ncb;
  // rows of the hg-row halo around the band, clipped to the grid (for h at
  // least one row: the smoothness term reads the rows next to the band)
  const int H0 = max(0, R0 - G.hg), H1 = min(G.Kh, R1 + G.hg);
  const int E0 = max(0, R0 - max(G.hg, 1)), E1 = min(G.Kh, R1 + max(G.hg, 1));

  // A + A2: q = h * g on the band, then the band's coarse residual rows;
  // returns this thread's share of sum res^2
  auto model_residual = [&]() -> float {
    for (int s = tid; s < nstrip; s += nt) {
      const int cb = s / nrows, P = R0 + (s - cb * nrows), Q0 = cb * kStrip;
      float acc[kStrip];
      corr_strip<KG>(hp, gfs, G.HC, P, Q0, acc);
      float* out = &hpix(rp, P, Q0);
#pragma unroll
      for (int c = 0; c < kStrip; ++c)
        if (Q0 + c < G.Kh) out[c] = acc[c];
    }
    __syncthreads();
    float dsum = 0.f;
    for (int e = tid; e < (i1 - i0) * K; e += nt) {
      const int i = i0 + e / K, j = e - (i - i0) * K;
      float s = 0.f;
      for (int a = 0; a < r; ++a) {
        const int P = r * i + a;
        if (P >= G.Kh) break;
        for (int b = 0; b < r; ++b) {
          const int Q = r * j + b;
          if (Q < G.Kh) s += hpix(rp, P, Q);
        }
      }
      const float d = s - fs[i * K + j];
      res[i * K + j] = d;
      dsum = fmaf(d, d, dsum);
    }
    return dsum;
  };
  // CTA partials of the two loss terms -> cta_part (thread 0), then a cluster
  // barrier; returns the loss summed over the cluster in CTA-rank order
  auto cluster_loss = [&](float dsum, float ssum) -> float {
    dsum = warp_sum(dsum);
    ssum = warp_sum(ssum);
    if (lane == 0) {
      wpart[0][warp] = dsum;
      wpart[1][warp] = ssum;
    }
    __syncthreads();
    if (tid == 0) {
      float d = 0.f, s = 0.f;
      for (int w = 0; w < kPsfWarps; ++w) {
        d += wpart[0][w];
        s += wpart[1][w];
      }
      cta_part[0] = d;
      cta_part[1] = s;
    }
    cl.sync();
    float d = 0.f, s = 0.f;
    for (int c = 0; c < G.C; ++c) {
      const float* pc = cl.map_shared_rank(cta_part, c);
      d += pc[0];
      s += pc[1];
    }
    return d + lambda * s;
  };

  double p1 = 1.0, p2 = 1.0;
  float best = 0.f;
  for (int k = 1; k <= iters; ++k) {
    const float dsum = model_residual();
    cl.sync();  // every band's residual rows are written
    for (int i = H0 / r + warp; i <= (H1 - 1) / r; i += kPsfWarps) {
      if (i >= i0 && i < i1) continue;
      const float* src = cl.map_shared_rank(res, (i * r) / G.BR);
      for (int j = lane; j < K; j += 32) res[i * K + j] = src[i * K + j];
    }
    __syncthreads();
    for (int P = H0 + warp; P < H1; P += kPsfWarps)  // B: replicate the residual
      for (int Q = lane; Q < G.Kh; Q += 32) hpix(rp, P, Q) = res[(P / r) * K + Q / r];
    __syncthreads();
    // C: gradient and projected Adam step (Kingma & Ba, bias-corrected)
    p1 *= 0.9;
    p2 *= 0.999;
    const float ic1 = (float)(1.0 / (1.0 - p1)), ic2 = (float)(1.0 / (1.0 - p2));
    float ssum = 0.f;
    for (int s = tid; s < nstrip; s += nt) {
      const int cb = s / nrows, P = R0 + (s - cb * nrows), Q0 = cb * kStrip;
      const int nq = min(kStrip, G.Kh - Q0), e0 = P * G.Kh + Q0;
      float m0[kStrip], v0[kStrip];
#pragma unroll
      for (int c = 0; c < kStrip; ++c) {  // moments in flight during the correlation
        m0[c] = c < nq ? mo[e0 + c] : 0.f;
        v0[c] = c < nq ? vo[e0 + c] : 0.f;
      }
      float acc[kStrip];
      corr_strip<KG>(rp, gs, G.HC, P, Q0, acc);
      const float* hrow = &hpix(hp, P, 0);
#pragma unroll
      for (int c = 0; c < kStrip; ++c) {
        if (c >= nq) break;
        const int Q = Q0 + c;
        const float h = hrow[Q];
        float d = 0.f;
        if (P >= 1) d += h - hrow[Q - G.HC];
        if (P + 1 < G.Kh) {
          const float t = hrow[Q + G.HC] - h;
          d -= t;
          ssum = fmaf(t, t, ssum);
        }
        if (Q >= 1) d += h - hrow[Q - 1];
        if (Q + 1 < G.Kh) {
          const float t = hrow[Q + 1] - h;
          d -= t;
          ssum = fmaf(t, t, ssum);
        }
        const float gr = 2.f * acc[c] + 2.f * lambda * d;
        const float m = 0.9f * m0[c] + 0.1f * gr;
        const float v = 0.999f * v0[c] + 0.001f * gr * gr;
        mo[e0 + c] = m;
        vo[e0 + c] = v;
        hn[e0 + c] = fmaxf(h - lr * (m * ic1) / (sqrtf(v * ic2) + 1e-8f), 0.f);
      }
    }
    // D: loss of h_k; keep h_k if it is the best so far, then h_k <- h_{k+1}
    const float L = cluster_loss(dsum, ssum);
    const bool improved = (k == 1) || (L < best);
    if (improved) best = L;
    for (int P = R0 + warp; P < R1; P += kPsfWarps)
      for (int Q = lane; Q < G.Kh; Q += 32) {
        float& c = hpix(hp, P, Q);
        if (improved) hb[P * G.Kh + Q] = c;
        c = hn[P * G.Kh + Q];
      }
    cl.sync();  // every band of h_{k+1} is in place
    for (int P = E0 + warp; P < E1; P += kPsfWarps) {
      if (P >= R0 && P < R1) continue;
      const float* src = &hpix(cl.map_shared_rank(hp, P / G.BR), P, 0);
      float* dst = &hpix(hp, P, 0);
      for (int Q = lane; Q < G.Kh; Q += 32) dst[Q] = src[Q];
    }
    __syncthreads();
  }

  // loss of the last iterate; it is returned when it beats the best earlier one
  const float dsum = model_residual();
  float ssum = 0.f;
  for (int P = R0 + warp; P < R1; P += kPsfWarps)
    for (int Q = lane; Q < G.Kh; Q += 32) {
      const float* c = &hpix(hp, P, Q);
      if (P + 1 < G.Kh) { const float d = c[G.HC] - c[0]; ssum = fmaf(d, d, ssum); }
      if (Q + 1 < G.Kh) { const float d = c[1] - c[0]; ssum = fmaf(d, d, ssum); }
    }
  const float L = cluster_loss(dsum, ssum);
  if (iters == 0 || L < best) {
    for (int P = R0 + warp; P < R1; P += kPsfWarps)
      for (int Q = lane; Q < G.Kh; Q += 32) hb[P * G.Kh + Q] = hpix(hp, P, Q);
    best = L;
  }
  if (loss && crank == 0 && tid == 0) loss[psf] = best;
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Launch with the largest cluster (at most creq CTAs per PSF) for which all
// n clusters are resident at once; the dynamic shared memory does not
// depend on the cluster size.
template <int KG>
cudaError_t launch_fit(int n, int creq, int K, int r, size_t smem, const float* f,
                       const float* g, const float* h0, float lambda, float lr, int iters,
                       float* mom, float* hn, float* hout, float* loss) {
  cudaError_t e = allow_max_dynamic_smem((const void*)psf_fit_kernel<KG>);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kPsfThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = 0;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PsfGeom G = psf_geom(K, r, KG, 1);
  for (int c = creq; c >= 1; --c) {
    G = psf_geom(K, r, KG, c);
    if (G.C < c && c > 1) continue;  // that request gives a smaller cluster anyway
    attr[0].val.clusterDim.x = G.C;
    cfg.gridDim = dim3(n * G.C, 1, 1);
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, psf_fit_kernel<KG>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      active = 0;
    }
    if (active >= n || G.C == 1) break;
  }
  attr[0].val.clusterDim.x = G.C;
  cfg.gridDim = dim3(n * G.C, 1, 1);
  return cudaLaunchKernelEx(&cfg, psf_fit_kernel<KG>, f, K, r, g, h0, lambda, lr, iters, G.C,
                            mom, hn, hout, loss);
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
  if (r > 8 || K > EMD_PSF_MAX_COARSE || Kg > EMD_PSF_MAX_KG)
    return psf_fail(EMD_EINVAL, "need r <= 8, K <= EMD_PSF_MAX_COARSE, Kg <= EMD_PSF_MAX_KG");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return psf_fail(EMD_ECUDA, "no CUDA device");
  }
  // CTAs per PSF: enough clusters to cover the SMs, at most 8
  const int creq = std::max(1, std::min(kMaxCluster, sms / n));
  const PsfGeom G = psf_geom(K, r, Kg, 1);
  const size_t smem = psf_smem_floats(G) * sizeof(float);
  if (smem > 220 * 1024) return psf_fail(EMD_EUNSUPPORTED, "fine PSF too large for one CTA");
  const size_t nh = (size_t)G.Kh * G.Kh;
  const size_t fb = (size_t)n * K * K * sizeof(float), gb = (size_t)Kg * Kg * sizeof(float),
               hb = (size_t)n * nh * sizeof(float), lb = (size_t)n * sizeof(float);
  const bool fd = on_device(f), gd = on_device(g), hd = on_device(h_out);
  const bool h0d = h0 ? on_device(h0) : true, ld = loss_out ? on_device(loss_out) : true;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t need = up(2 * hb) + up(hb) + (fd ? 0 : up(fb)) + (gd ? 0 : up(gb)) +
                      (hd ? 0 : up(hb)) + (h0d ? 0 : up(hb)) + (ld ? 0 : up(lb));
  char* tmp = nullptr;
  if (cudaMalloc(&tmp, need) != cudaSuccess) {
    cudaGetLastError();
    return psf_fail(EMD_ENOMEM, "device allocation failed");
  }
  size_t off = 0;
  auto take = [&](size_t b) { char* p = tmp + off; off += up(b); return p; };
  float* mom = reinterpret_cast<float*>(take(2 * hb));
  float* hn = reinterpret_cast<float*>(take(hb));
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
  if (e == cudaSuccess) {
#define EMD_FIT_CASE(KG)                                                                    \
  case KG:                                                                                  \
    e = launch_fit<KG>(n, creq, K, r, smem, df, dg, dh0, lambda, lr, iters, mom, hn, dh, dl); \
    break;
    switch (Kg) {
      EMD_FIT_CASE(1)
      EMD_FIT_CASE(3)
      EMD_FIT_CASE(5)
      EMD_FIT_CASE(7)
      EMD_FIT_CASE(9)
      EMD_FIT_CASE(11)
      EMD_FIT_CASE(13)
      EMD_FIT_CASE(15)
      default:
        e = cudaErrorInvalidValue;
    }
#undef EMD_FIT_CASE
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e == cudaSuccess && !hd) e = cudaMemcpy(h_out, dh, hb, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && !ld) e = cudaMemcpy(loss_out, dl, lb, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = psf_fail(EMD_ECUDA, cudaGetErrorString(e));
  cudaFree(tmp);
  return rc;
}
