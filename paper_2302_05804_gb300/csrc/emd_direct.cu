// emd_direct.cu -- FP32 direct-convolution kernels of the EM update (Sec. 2,
// Eq. (2)), one GPU, sm_103a.
//
// The hot kernel (fused_kernel) computes, for one 128 x 128 tile of the
// latent grid and all exposures t in ascending order,
//     w_t = u_t . (F_t x)        on the tile plus a halo of hc pixels
//     Den += F_t^T w_t            on the tile
// and on the last exposure applies x' = Den > 0 ? x max(N,0)/Den : x. w_t
// lives only in shared memory; Den is carried in an L2-resident scratch
// plane between exposures, so no per-exposure image is written to HBM.
//
// A tile is handled by a CTA pair (thread-block cluster of 2): each CTA
// computes the forward model on half of the haloed region, the pair swaps
// the halo rows of w through distributed shared memory, and each CTA then
// runs the adjoint for 64 of the 128 rows. The x tile of each CTA (its half
// of the region plus the 2*hc convolution halo) is staged into shared
// memory with cp.async.bulk row copies completing on an mbarrier.
//
// Inner loops are register-blocked FP32 FMA: a thread owns a 4 x 16
// (forward) or 2 x 16 (adjoint) block of outputs; per input row and group
// of 4 taps it loads a 20-float window (five 16-byte loads) and one 16-byte
// kernel quad per output row (a warp-wide broadcast). Rows in shared memory
// carry a skew (4 floats every 4 rows for x, every 2 rows for w) so that the
// eight lanes of each 16-byte load phase hit distinct bank groups.
#include <cooperative_groups.h>
#include <math.h>

#include <mutex>
#include <set>
#include <utility>

#include "emd_corr.cuh"
#include "emd_internal.cuh"

namespace cg = cooperative_groups;

namespace emd {

static inline int rup(int a, int b) { return (a + b - 1) / b * b; }

cudaError_t allow_max_dynamic_smem(const void* func) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({func, dev})) return cudaSuccess;
  int optin = 0;
  cudaFuncAttributes fa;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes)) != cudaSuccess)
    return e;
  done.insert({func, dev});
  return cudaSuccess;
}

bool make_shape(int H, int W, int n, int K, int r, Shape* s, const char** why) {
  if (H < 1 || W < 1 || n < 1) { *why = "H, W and n must be >= 1"; return false; }
  if (K < 1 || (K % 2) == 0) { *why = "psf_k must be odd and >= 1"; return false; }
  if (r < 1 || r > 8) { *why = "r must be in [1, 8]"; return false; }
  if ((long long)H * r > (1 << 20) || (long long)W * r > (1 << 20)) {
    *why = "image too large"; return false;
  }
  const int h = (K - 1) / 2;
  const int hc = (h + r - 1) / r;
  if (hc > EMD_MAX_HC) { *why = "PSF footprint too large (hc > EMD_MAX_HC)"; return false; }
  s->H = H; s->W = W; s->n = n; s->K = K; s->r = r; s->R2 = r * r;
  s->hc = hc; s->Kc = 2 * hc + 1; s->KP = rup(s->Kc, 4);
  s->gx = (W + kTile - 1) / kTile;
  s->gy = (H + kTile - 1) / kTile;
  const int Rw = rup(kTile + 2 * hc, 8);
  s->Rh = Rw / 2;
  s->MXf = rup(kTile + 2 * hc, 16) / 16;
  s->xrows = s->Rh + 2 * hc;
  s->xpitch = rup(16 * s->MXf + s->KP, 8);
  s->wrows = (Rw - kHalf > kHalf + 2 * hc) ? Rw - kHalf : kHalf + 2 * hc;
  {
    int a = 16 * s->MXf, b = kTile + s->KP;
    s->wpitch = rup(a > b ? a : b, 16);
  }
  const size_t xs = (size_t)s->xrows * s->xpitch + 4 * ((s->xrows + 3) / 4);
  const size_t ws = (size_t)s->wrows * s->wpitch + 4 * ((s->wrows + 1) / 2);
  const size_t ks = 2 * (size_t)s->Kc * s->KP;
  s->smem_fused = (xs + ws + ks) * sizeof(float) + 16;
  if (s->smem_fused + 1024 > 227 * 1024) { *why = "shared memory budget exceeded"; return false; }
  if ((s->Rh / 4) * s->MXf > kThreads) { *why = "forward region exceeds one microtile per thread"; return false; }
  // padded plane geometry
  Geom& g = s->g;
  g.H = H; g.W = W; g.B = 2 * hc;
  int P = (s->gx - 1) * kTile + 16 * s->MXf + s->KP;
  if (P < g.B + W + 1) P = g.B + W + 1;
  g.P = rup(P, 8);
  int PH = (s->gy - 1) * kTile + 2 * s->Rh + 4 * hc + 8;
  if (PH < g.B + H + 1) PH = g.B + H + 1;
  // the halo-exchange kernel's last row of tiles (TH = 64, 48 or 32 rows)
  // reaches row ceil(H / TH) TH + hc - 1 <= H + 63 + hc of the image
  if (PH < H + 64 + 3 * hc) PH = H + 64 + 3 * hc;
  g.PH = PH;
  g.plane = (long long)g.PH * g.P;
  return true;
}

// ---------------------------------------------------------------------------
// small PTX helpers: mbarrier, bulk copy, cluster barrier
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after `limit` polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t limit = (1u << 22)) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// fused EM iteration / numerator / chi-square kernel
// ---------------------------------------------------------------------------
// mode 0: one EM iteration x -> xn (Eq. (2)).
// mode 1: N = sum_t F_t^T (u_t y_t) into a.N.
// mode 2: chi2 = sum_t sum_i u (y - F_t x)^2 of the tile into part[block].
// mode 3: N' = sum_t F_t^T (u'_t y_t) into a.Nw (heavy-tailed numerator).
// With a.nu > 0 (Student-t noise, nu degrees of freedom) the weights of
// modes 0 and 3 are u' = u (nu+1) / (nu + u (y - z)^2), z = F_t x, and mode 2
// sums (nu+1) log(1 + u (y - z)^2 / nu) instead of u (y - z)^2.
//
// Cluster barrier protocol of mode 0 (every thread of both CTAs, in order):
//   write own w rows (t) -> arrive+wait [A_t] -> copy peer halo rows ->
//   arrive [B_t] -> adjoint t -> forward t+1 -> wait [B_t] -> write own w
//   rows (t+1) ... and a final wait [B_{n-1}] before exit, so no CTA
//   overwrites or releases shared memory its peer may still be reading.

// One 128 x 128 tile (rows i0.., cols j0..) handled by CTA q of a pair; the
// caller owns the mbarrier, its phase, the timeout flag and the chi-square
// accumulator so a persistent kernel can run many tiles per CTA pair.
// STUDENT: heavy-tailed weights (a.nu > 0); compiled separately so that the
// Gaussian kernel carries none of that code.
template <bool STUDENT>
__device__ __forceinline__ void fused_tile(const Shape& s, const FusedArgs& a, const int mode,
                                           const int i0, const int j0, const int q, float* smem,
                                           uint64_t* mbar, uint32_t& phase, bool& timed_out,
                                           double& chi) {
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x;
  const Geom& g = s.g;
  const int hc = s.hc, Kc = s.Kc, KP = s.KP;

  const int xs_floats = s.xrows * s.xpitch + 4 * ((s.xrows + 3) >> 2);
  const int ws_floats = s.wrows * s.wpitch + 4 * ((s.wrows + 1) >> 1);
  float* xs_base = smem;
  float* ws_base = xs_base + xs_floats;
  float* ksf = ws_base + ws_floats;
  float* ksa = ksf + Kc * KP;
  const SPlane xs{xs_base, s.xpitch, 2};
  const SPlane ws{ws_base, s.wpitch, 1};

  for (int e = tid; e < ws_floats; e += kThreads) ws_base[e] = 0.f;
  __syncthreads();

  // forward microtile (4 x 16) of this thread in its CTA's half region
  const int MYf = s.Rh >> 2;
  const bool has_f = tid < MYf * s.MXf;
  const int fmy = tid % MYf, fmx = tid / MYf;
  // adjoint microtile (2 x 16) in the CTA's 64 x 128 block of Den
  const int wid = tid >> 5, lane = tid & 31;
  const int amy = (wid & 3) * 8 + (lane & 7);
  const int amx = (wid >> 2) * 4 + (lane >> 3);

  const int ccols = 16 * s.MXf;

  const int t0 = a.t0, t1 = a.t1;  // exposures of this launch, ascending
  const bool xchg = (mode == 0 || mode == 3);  // forward, weights, halo swap, adjoint
  for (int t = t0; t < t1; ++t) {
    const long long tplane = (long long)t * g.plane;
    if (mode != 1) {
      // ---------------- forward: z = sum_phi kf_phi (x) x_phi -----------------
      float acc[4][16];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[p][c] = 0.f;
      for (int phi = 0; phi < s.R2; ++phi) {
        const bool stage = (s.R2 > 1) || (t == t0);
        __syncthreads();  // earlier readers of xs / ksf are done
        if (stage && tid < 32) {
          const float* plane = a.x + (long long)phi * g.plane;
          const int row0 = i0 + q * s.Rh;  // padded row of staged row 0 (B = 2 hc)
          const uint32_t row_bytes = (uint32_t)(ccols + KP) * 4u;
          if (tid == 0) mbar_arrive_expect_tx(mbar, row_bytes * (uint32_t)s.xrows);
          __syncwarp();
          for (int R = tid; R < s.xrows; R += 32)
            bulk_g2s(srow(xs, R), plane + (long long)(row0 + R) * g.P + j0, row_bytes, mbar);
        }
        const float4* kg =
            reinterpret_cast<const float4*>(a.kf + ((long long)t * s.R2 + phi) * Kc * KP);
        for (int e = tid; e < (Kc * KP) >> 2; e += kThreads)
          reinterpret_cast<float4*>(ksf)[e] = kg[e];
        if (stage) {
          if (!mbar_wait_bounded(mbar, phase)) timed_out = true;
          phase ^= 1u;
        }
        __syncthreads();
        if (has_f && !timed_out) corr_tile<4, 16>(acc, xs, 4 * fmy, 16 * fmx, ksf, KP, Kc);
      }
      // ---------------- weights (modes 0, 3) or chi-square (mode 2) -------------
      if (xchg && t > t0) cluster_wait();  // [B_{t-1}]: peer done reading our w
      if (has_f) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int rr = q * s.Rh + 4 * fmy + p;  // region row
          const long long grow = tplane + (long long)(i0 + hc + rr) * g.P + j0 + hc;
          if (xchg) {
            float* wrow = srow(ws, rr - kHalf * q);
            if (STUDENT) {
              const float nu1 = a.nu + 1.f;
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int cc = 16 * fmx + c;
                const float uv = a.u[grow + cc], yv = a.y[grow + cc];
                const float d = yv - acc[p][c];
                const float us = uv > 0.f ? uv * nu1 / fmaf(uv * d, d, a.nu) : 0.f;
                wrow[cc] = us * (mode == 3 ? yv : acc[p][c]);
              }
            } else {
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int cc = 16 * fmx + c;
                wrow[cc] = a.u[grow + cc] * acc[p][c];
              }
            }
          } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int cc = 16 * fmx + c;
              const int i = i0 - hc + rr, j = j0 - hc + cc;
              const float uv = a.u[grow + cc];
              if (rr >= hc && rr < hc + kTile && cc >= hc && cc < hc + kTile && i < g.H &&
                  j < g.W && uv != 0.f) {
                const double d = (double)a.y[grow + cc] - (double)acc[p][c];
                if (STUDENT)
                  chi += ((double)a.nu + 1.0) * log1p((double)uv * d * d / (double)a.nu);
                else
                  chi += (double)uv * d * d;
              }
            }
          }
        }
      }
      if (mode == 2) continue;
      // ---------------- halo exchange with the peer CTA ------------------------
      cluster_arrive();
      cluster_wait();  // [A_t]: both CTAs wrote their own w rows
      {
        const float* peer_base = cluster.map_shared_rank(ws_base, q ^ 1);
        const SPlane pws{const_cast<float*>(peer_base), s.wpitch, 1};
        // region rows needed from the peer and the local-row offsets
        int r_lo, r_hi;
        if (q == 0) { r_lo = s.Rh; r_hi = kHalf + 2 * hc; }
        else { r_lo = kHalf; r_hi = s.Rh; }
        const int nrows = r_hi - r_lo;
        const int c4 = s.wpitch >> 2;
        for (int e = tid; e < nrows * c4; e += kThreads) {
          const int rr = r_lo + e / c4, k4 = e % c4;
          const int ldst = rr - kHalf * q, lsrc = rr - kHalf * (q ^ 1);
          reinterpret_cast<float4*>(srow(ws, ldst))[k4] =
              reinterpret_cast<const float4*>(srow(pws, lsrc))[k4];
        }
      }
      cluster_arrive();  // [B_t] arrive: done reading the peer's w
      __syncthreads();
    } else {
      // numerator: w = u_t y_t on the CTA's local rows (no forward model)
      __syncthreads();  // previous adjoint done reading ws
      const int lrows = kHalf + 2 * hc;
      for (int e = tid; e < lrows * ccols; e += kThreads) {
        const int L = e / ccols, cc = e % ccols;
        const int rr = kHalf * q + L;
        const long long gi = tplane + (long long)(i0 + hc + rr) * g.P + j0 + hc + cc;
        srow(ws, L)[cc] = a.u[gi] * a.y[gi];
      }
      __syncthreads();
    }
    // ---------------- adjoint: Den_phi += ka_phi (*) w --------------------------
    for (int phi = 0; phi < s.R2; ++phi) {
      if (phi > 0) __syncthreads();  // ksa readers of phi-1 are done
      const float4* kg =
          reinterpret_cast<const float4*>(a.ka + ((long long)t * s.R2 + phi) * Kc * KP);
      for (int e = tid; e < (Kc * KP) >> 2; e += kThreads)
        reinterpret_cast<float4*>(ksa)[e] = kg[e];
      __syncthreads();
      // each exposure's adjoint is summed from zero and then added to the
      // running Den: a per-exposure FMA chain of Kc^2 terms instead of one
      // chain of n Kc^2 terms keeps the FP32 rounding of Den near 1e-7
      float acc2[2][16];
      const long long pbase = (long long)phi * g.plane;
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc2[p][c] = 0.f;
      if (!timed_out) corr_tile<2, 16>(acc2, ws, 2 * amy, 16 * amx, ksa, KP, Kc);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int i = i0 + kHalf * q + 2 * amy + p;
        const long long grow = pbase + (long long)(g.B + i) * g.P + g.B + j0 + 16 * amx;
        if (t > t0) {
#pragma unroll
          for (int c = 0; c < 16; ++c) acc2[p][c] = a.Den[grow + c] + acc2[p][c];
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = j0 + 16 * amx + c;
          if (t + 1 < t1) {
            a.Den[grow + c] = acc2[p][c];
          } else if (i < g.H && j < g.W) {
            if (mode == 1 || mode == 3) {
              a.Nw[grow + c] = acc2[p][c];
            } else {
              const float d = acc2[p][c];
              const float xo = a.x[grow + c];
              float xv = xo;
              if (d > 0.f) {
                const float nv = fmaxf(a.N[grow + c], 0.f);
                if (d < 1e-30f)  // denominator near zero: guarded ratio in FP64
                  xv = (float)((double)xo * (double)nv / (double)d);
                else
                  xv = xo * nv / d;
              }
              a.xn[grow + c] = xv;
            }
          }
        }
      }
    }
  }
  if (xchg) cluster_wait();  // [B_{n-1}]
}

template <bool STUDENT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    fused_kernel(const Shape s, const FusedArgs a, const int mode, double* __restrict__ part) {
  extern __shared__ __align__(128) float smem[];
  __shared__ double red[kThreads / 32];
  __shared__ uint64_t mbar_s;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  if (threadIdx.x == 0) {
    mbar_init(&mbar_s, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  bool timed_out = false;
  double chi = 0.0;
  fused_tile<STUDENT>(s, a, mode, blockIdx.y * kTile, (blockIdx.x >> 1) * kTile, q, smem, &mbar_s,
                      phase, timed_out, chi);
  if (mode == 2) {
    const double tot = block_sum_f64(chi, red);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
  if (timed_out) {
    // give the staged copies a bounded chance to land before the CTA exits
    mbar_wait_bounded(&mbar_s, phase ^ 1u);
    if (threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
  }
}

template <bool STUDENT>
cudaError_t launch_fused_t(const Shape& s, const FusedArgs& a, int mode, double* part,
                           cudaStream_t st) {
  cudaError_t e = allow_max_dynamic_smem((const void*)fused_kernel<STUDENT>);
  if (e != cudaSuccess) return e;
  dim3 grid(2 * s.gx, s.gy), block(kThreads);
  fused_kernel<STUDENT><<<grid, block, s.smem_fused, st>>>(s, a, mode, part);
  return cudaGetLastError();
}

cudaError_t launch_fused(const Shape& s, const FusedArgs& a, int mode, double* part,
                         cudaStream_t st) {
  return a.nu > 0.f ? launch_fused_t<true>(s, a, mode, part, st)
                    : launch_fused_t<false>(s, a, mode, part, st);
}

int fused_blocks(const Shape& s) { return 2 * s.gx * s.gy; }

// ---------------------------------------------------------------------------
// persistent multi-job kernel: one EM iteration for every active job of a
// batch. CTA pairs claim (job, tile) items from a device counter until the
// work list is exhausted; items of jobs with no iterations left are skipped.
// ---------------------------------------------------------------------------

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    batch_kernel(const BatchJob* __restrict__ jobs, const int2* __restrict__ items,
                 const int* __restrict__ n_items, int* __restrict__ counter, int* err) {
  extern __shared__ __align__(128) float smem[];
  __shared__ uint64_t mbar_s;
  __shared__ int claim_s[2];
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  if (threadIdx.x == 0) {
    mbar_init(&mbar_s, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  bool timed_out = false;
  double chi = 0.0;
  const int total = *n_items;
  volatile int* leader_claim = cluster.map_shared_rank(claim_s, 0);
  for (int it = 0;; ++it) {
    if (q == 0 && threadIdx.x == 0) claim_s[it & 1] = atomicAdd(counter, 1);
    cluster_arrive();
    cluster_wait();  // the claim is visible to both CTAs
    const int item = leader_claim[it & 1];
    cluster_arrive();
    cluster_wait();  // both read it: the leader may move on (or exit)
    if (item >= total) break;
    const int2 w = items[item];
    const BatchJob& J = jobs[w.x];
    if (J.remaining <= 0) continue;
    const int tx = w.y % J.s.gx, ty = w.y / J.s.gx;
    fused_tile<false>(J.s, J.a[J.cur], 0, ty * kTile, tx * kTile, q, smem, &mbar_s, phase, timed_out,
               chi);
  }
  if (timed_out) {
    mbar_wait_bounded(&mbar_s, phase ^ 1u);
    if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
  }
}

// after a batch step: every job that ran advances one iteration
__global__ void batch_advance_kernel(BatchJob* __restrict__ jobs, int njobs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < njobs && jobs[j].remaining > 0) {
    jobs[j].remaining -= 1;
    jobs[j].cur ^= 1;
  }
}

size_t batch_smem_bytes() {
  // the largest fused-kernel footprint of any accepted shape (hc <= EMD_MAX_HC)
  size_t m = 0;
  for (int r = 1; r <= 2; ++r)
    for (int K = 1; K <= 2 * EMD_MAX_HC * r + 1; K += 2) {
      Shape s;
      const char* why;
      if (make_shape(256, 256, 1, K, r, &s, &why) && s.smem_fused > m) m = s.smem_fused;
    }
  return m;
}

int batch_max_clusters(size_t smem) {
  static int cached = -1;
  if (cached >= 0) return cached;
  if (allow_max_dynamic_smem((const void*)batch_kernel) != cudaSuccess) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, batch_kernel, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return -1;
  }
  cached = n;
  return n;
}

cudaError_t launch_batch(const BatchJob* jobs, int njobs, const int2* items, const int* n_items,
                         int* counter, int* err, int clusters, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_max_dynamic_smem((const void*)batch_kernel);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  batch_kernel<<<2 * clusters, kThreads, smem, st>>>(jobs, items, n_items, counter, err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_advance_kernel<<<(njobs + 127) / 128, 128, 0, st>>>(const_cast<BatchJob*>(jobs), njobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// self-test of the bounded waits: an mbarrier that nothing arrives on
// ---------------------------------------------------------------------------

__global__ void wait_selftest_kernel(uint32_t limit, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // the expected arrival never comes: the bounded wait must give up
  const bool ok = mbar_wait_bounded(&bar, 0, limit);
  if (!ok && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

cudaError_t launch_wait_selftest(uint32_t limit, int* err, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(limit, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// set-up: u = mask ? 1/v : 0 (in place over v), y sanitised, FP64 sums
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) setup_kernel(const Shape s, const SetupArgs a) {
  __shared__ double red[8];
  const Geom& g = s.g;
  const long long hw = (long long)g.H * g.W, total = hw * s.n;
  double ld = 0.0, suy = 0.0, su = 0.0, cnt = 0.0;
  int bad = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / hw);
    const long long rem = e - (long long)t * hw;
    const int i = (int)(rem / g.W), j = (int)(rem - (long long)i * g.W);
    const long long off = (long long)t * g.plane + (long long)(g.B + i) * g.P + g.B + j;
    const bool valid = a.mask ? (a.mask[e] != 0) : true;
    const float v = a.u[off], yv = a.y[off];
    float uo = 0.f, yo = 0.f;
    if (valid) {
      if (!(v > 0.f) || !isfinite(v) || !isfinite(yv)) {
        bad = 1;
      } else {
        uo = 1.0f / v;
        yo = yv;
        ld += log(6.283185307179586 * (double)v);
        suy += (double)uo * (double)yv;
        su += (double)uo;
        cnt += 1.0;
      }
    }
    a.u[off] = uo;
    a.y[off] = yo;
  }
  if (bad) atomicOr(a.err, kErrData);
  const double s0 = block_sum_f64(ld, red);
  const double s1 = block_sum_f64(suy, red);
  const double s2 = block_sum_f64(su, red);
  const double s3 = block_sum_f64(cnt, red);
  if (threadIdx.x == 0) {
    a.part[4 * blockIdx.x + 0] = s0;
    a.part[4 * blockIdx.x + 1] = s1;
    a.part[4 * blockIdx.x + 2] = s2;
    a.part[4 * blockIdx.x + 3] = s3;
  }
}

cudaError_t launch_setup(const Shape& s, const SetupArgs& a, cudaStream_t st) {
  setup_kernel<<<kRedBlocks, 256, 0, st>>>(s, a);
  return cudaGetLastError();
}

// out[c] = sum_b part[b * ncols + c], one block, fixed order
__global__ void __launch_bounds__(256) reduce_final_kernel(const double* __restrict__ part,
                                                           int nblocks, int ncols,
                                                           double* __restrict__ out) {
  __shared__ double red[8];
  for (int c = 0; c < ncols; ++c) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += part[(long long)b * ncols + c];
    const double tot = block_sum_f64(v, red);
    if (threadIdx.x == 0) out[c] = tot;
  }
}

cudaError_t launch_reduce_final(const double* part, int nblocks, int ncols, double* out,
                                cudaStream_t st) {
  reduce_final_kernel<<<1, 256, 0, st>>>(part, nblocks, ncols, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// polyphase PSF kernels: for phase (py, px) and offsets d in [-hc, hc]
//   c[dy][dx] = sum_{s,t < r} f[r dy + s + h - py][r dx + t + h - px]
// ka[a][b] = c[a - hc][b - hc] (adjoint, a correlation), kf = ka flipped
// (the forward convolution written as a correlation). r = 1: ka = f.
// ---------------------------------------------------------------------------

__global__ void build_kernels_kernel(const Shape s, const float* __restrict__ f,
                                     float* __restrict__ kf, float* __restrict__ ka) {
  const int Kc = s.Kc, KP = s.KP, K = s.K, r = s.r, hc = s.hc, h = (s.K - 1) / 2;
  const long long total = (long long)s.n * s.R2 * Kc * KP;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % KP);
    const int a = (int)((e / KP) % Kc);
    const int phi = (int)((e / ((long long)KP * Kc)) % s.R2);
    const int t = (int)(e / ((long long)KP * Kc * s.R2));
    const int py = phi / r, px = phi % r;
    const float* ft = f + (long long)t * K * K;
    float vka = 0.f, vkf = 0.f;
    if (b < Kc) {
      // ka at (a, b), kf at (a, b) = c at the flipped offsets
      for (int which = 0; which < 2; ++which) {
        const int dy = (which == 0 ? a : Kc - 1 - a) - hc;
        const int dx = (which == 0 ? b : Kc - 1 - b) - hc;
        float acc = 0.f;
        for (int sy = 0; sy < r; ++sy) {
          const int fa = r * dy + sy + h - py;
          if (fa < 0 || fa >= K) continue;
          for (int sx = 0; sx < r; ++sx) {
            const int fb = r * dx + sx + h - px;
            if (fb < 0 || fb >= K) continue;
            acc += ft[fa * K + fb];
          }
        }
        if (which == 0) vka = acc; else vkf = acc;
      }
    }
    ka[e] = vka;
    kf[e] = vkf;
  }
}

cudaError_t launch_build_kernels(const Shape& s, const float* f_raw, float* kf, float* ka,
                                 cudaStream_t st) {
  build_kernels_kernel<<<256, 256, 0, st>>>(s, f_raw, kf, ka);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// latent layout conversions: natural (rH x rW) <-> r^2 padded phase planes
// ---------------------------------------------------------------------------

__global__ void scatter_latent_kernel(const Shape s, const float* __restrict__ nat,
                                      float* __restrict__ planes, int clamp_neg, int fill,
                                      float c) {
  const Geom& g = s.g;
  const int r = s.r, Wf = r * g.W;
  const long long total = (long long)r * g.H * Wf;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int P_ = (int)(e / Wf), Q_ = (int)(e % Wf);
    const int phi = (P_ % r) * r + (Q_ % r);
    float v = fill ? c : nat[e];
    if (clamp_neg && !(v > 0.f)) v = 0.f;  // also maps NaN to 0
    planes[(long long)phi * g.plane + (long long)(g.B + P_ / r) * g.P + g.B + Q_ / r] = v;
  }
}

__global__ void gather_latent_kernel(const Shape s, const float* __restrict__ planes,
                                     float* __restrict__ nat) {
  const Geom& g = s.g;
  const int r = s.r, Wf = r * g.W;
  const long long total = (long long)r * g.H * Wf;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int P_ = (int)(e / Wf), Q_ = (int)(e % Wf);
    const int phi = (P_ % r) * r + (Q_ % r);
    nat[e] = planes[(long long)phi * g.plane + (long long)(g.B + P_ / r) * g.P + g.B + Q_ / r];
  }
}

cudaError_t launch_fill_latent(const Shape& s, float* x, float c, cudaStream_t st) {
  scatter_latent_kernel<<<1024, 256, 0, st>>>(s, nullptr, x, 0, 1, c);
  return cudaGetLastError();
}

cudaError_t launch_scatter_latent(const Shape& s, const float* nat, float* planes, int clamp_neg,
                                  cudaStream_t st) {
  scatter_latent_kernel<<<1024, 256, 0, st>>>(s, nat, planes, clamp_neg, 0, 0.f);
  return cudaGetLastError();
}

cudaError_t launch_gather_latent(const Shape& s, const float* planes, float* nat,
                                 cudaStream_t st) {
  gather_latent_kernel<<<1024, 256, 0, st>>>(s, planes, nat);
  return cudaGetLastError();
}

}  // namespace emd
