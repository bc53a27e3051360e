// emd_tc.cu -- tensor-core form of the EM iteration of Eq. (2) for sm_103a:
// both convolutions of every exposure run as banded-Toeplitz GEMMs on
// tcgen05 (BF16 or FP16 operands, FP32 accumulation in tensor memory),
// optionally with a hi+lo split (x = x_hi + x_lo, f = f_hi + f_lo, three
// products x_hi f_hi + x_hi f_lo + x_lo f_hi).
//
// Toeplitz form. For one filter row a, the forward model restricted to the
// image rows of an M-tile is a GEMM
//     Z[m][n] += sum_k X[m + a][k] * T_a[k][n],   T_a[k][n] = kf[a][k - n],
// m = image row (M = 128, tensor-memory lane), n = output column, k = input
// column. X rows shifted by a are the A operand read straight from the
// staged x tile: in the no-swizzle K-major layout ([8-column group][row][8])
// a row shift is a 16-byte shift of the descriptor's start address. T_a is
// banded; its transposed, column-reversed form is a Hankel matrix whose 8x8
// core matrices depend only on (k-group + n-group), so a descriptor with
// leading and stride byte offsets both 128 walks one compressed array of
// (Kdim + N)/8 - 1 core matrices. The adjoint is the same GEMM with w rows
// as A and the unflipped kernel ka. Tensor-memory column n of the result
// holds output column N-1-n.
//
// Two kernels per iteration, each on 128 x 128 tiles (M = N = 128):
//   tc_fwd_kernel: one CTA per tile of the exposure grid, every exposure:
//     z_t on exactly the tile (no halo is recomputed), w_t = u_t z_t encoded
//     as 16-bit hi (and lo) planes in device memory (zero outside the image);
//   tc_adj_kernel: one CTA per tile of the latent planes: for every exposure
//     the w_t band around the tile (rows and columns -hc .. 128 + hc) by TMA,
//     its adjoint GEMM into a tensor-memory partial, added in FP32 to the
//     running Den in exposure order; the last exposure applies the update.
// A band starts 16-byte aligned: dlt = hc mod 8 columns before the window
// it needs, which the Hankel operands absorb (their index carries -dlt).
// Warp roles in both: warp 0 issues TMA / bulk copies, warp 1 allocates
// tensor memory and issues MMAs, warps 2-5 run the epilogue. Every mbarrier
// wait is bounded; a timeout raises the error word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>

#include "emd_internal.cuh"
#include "emd_tc.cuh"

namespace emd {

namespace {

constexpr int kTcRows = 128;    // tile rows = MMA M
constexpr int kTcCols = 128;    // tile columns = MMA N
constexpr int kTcThreads = 192; // 6 warps
constexpr int kTcStages = 4;    // B (Hankel) ring depth
constexpr uint32_t kSpin = 1u << 22;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; once any thread of the CTA gave up (*abort set), later waits
// return at once so every role reaches the exit.
__device__ __forceinline__ void bar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  for (uint32_t i = 0; i < kSpin; ++i) {
    if (bar_try(b, parity)) return;
    if (*abort) return;
  }
  *abort = 1;
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                       uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(su32(b))
      : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b))
      : "memory");
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16-bit encodings of the operand type
__device__ __forceinline__ uint16_t enc16(float v, int fp16) {
  if (fp16) {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
  }
  __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ float dec16(uint16_t u, int fp16) {
  if (fp16) {
    __half h = *reinterpret_cast<__half*>(&u);
    return __half2float(h);
  }
  __nv_bfloat16 b = *reinterpret_cast<__nv_bfloat16*>(&u);
  return __bfloat162float(b);
}

}  // namespace

// ---------------------------------------------------------------------------
// shapes
// ---------------------------------------------------------------------------

static inline int rup(int a, int b) { return (a + b - 1) / b * b; }

bool make_tc_shape(const Shape& s, int mode, TcShape* t, const char** why) {
  if (s.R2 > 4) { *why = "tensor-core path supports r <= 2"; return false; }
  t->mode = mode;
  t->fp16 = (mode == EMD_PREC_FP16 || mode == EMD_PREC_SPLIT_FP16);
  t->nprod = (mode == EMD_PREC_SPLIT_BF16 || mode == EMD_PREC_SPLIT_FP16) ? 3 : 1;
  t->NW = kTcCols;
  t->dlt = s.hc & 7;
  t->Kd = rup(kTcCols + 2 * s.hc + t->dlt, 16);
  t->XRp = rup(kTcRows + 2 * s.hc, 8);
  t->Sd = t->Kd / 8 + kTcCols / 8 - 1;
  t->gxt = (s.W + kTcCols - 1) / kTcCols;
  t->gyt = (s.H + kTcRows - 1) / kTcRows;
  t->stage_bytes = 2 * t->Sd * 128;
  t->hank_block = 2 * t->stage_bytes;  // forward (hi, lo), adjoint (hi, lo)
  const size_t band = 2ull * t->XRp * t->Kd * 2;
  t->smem = band + kTcStages * (size_t)t->stage_bytes;
  if (t->smem > 227 * 1024 - 1024) { *why = "tensor-core tile exceeds shared memory"; return false; }
  // one CTA per SM: a second resident CTA would wait in tcgen05.alloc for
  // the tensor-memory columns of the first
  if (t->smem < 120 * 1024) t->smem = 120 * 1024;
  // the epilogues' plane accesses (rows < gyt 128, columns < gxt 128 of the
  // image) stay in the padded planes; TMA loads outside them read zeros
  const Geom& g = s.g;
  if (g.B + t->gxt * kTcCols > g.P || g.B + t->gyt * kTcRows > g.PH) {
    *why = "padded geometry too small for the tensor-core tiles";
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------

// Hankel core matrices of every (t, phi, a): block = [F_hi | F_lo | A_hi | A_lo],
// each Sd x 8 x 8 entries g[8s + r + e - (NW - 1) - dlt] of row a of kf (F)
// or ka (A); lo = rounding residue of the scaled value.
__global__ void build_hankel_kernel(const Shape s, const TcShape t, const float* __restrict__ kf,
                                    const float* __restrict__ ka, uint16_t* __restrict__ hank,
                                    float gscale) {
  const int per_op = t.Sd * 64;
  const long long per = 2LL * per_op;
  const long long total = (long long)s.n * s.R2 * s.Kc * per;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / per;
    const int within = (int)(e - blk * per);
    const int a = (int)(blk % s.Kc);
    const long long tp = blk / s.Kc;  // t * R2 + phi
    const bool fwd = within < per_op;
    const int w = fwd ? within : within - per_op;
    const int sidx = w / 64, r = (w / 8) % 8, c = w % 8;
    const int idx = 8 * sidx + r + c - (t.NW - 1) - t.dlt;
    const float* krow = (fwd ? kf : ka) + (tp * s.Kc + a) * s.KP;
    const float g = (idx >= 0 && idx < s.Kc) ? krow[idx] * gscale : 0.f;
    const uint16_t hi = enc16(g, t.fp16);
    const uint16_t lo = enc16(g - dec16(hi, t.fp16), t.fp16);
    uint16_t* part = hank + blk * (long long)(t.hank_block / 2) + (fwd ? 0 : 2 * per_op);
    part[w] = hi;
    part[per_op + w] = lo;
  }
}

// x (fp32 planes) -> 16-bit hi and lo planes at ping-pong slot pp:
// xb[((pp * 2 + hl) * R2 + phi) * plane + offset]
__global__ void split_x_kernel(const Shape s, int fp16, const float* __restrict__ x,
                               uint16_t* __restrict__ xb, int pp, const float* __restrict__ scales) {
  const Geom& g = s.g;
  const float xscale = scales[3];
  const long long tot = (long long)s.R2 * g.plane;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long phi = e / g.plane, off = e - phi * g.plane;
    const float v = x[e] * xscale;
    const uint16_t hi = enc16(v, fp16);
    const uint16_t lo = enc16(v - dec16(hi, fp16), fp16);
    xb[((long long)(pp * 2 + 0) * s.R2 + phi) * g.plane + off] = hi;
    xb[((long long)(pp * 2 + 1) * s.R2 + phi) * g.plane + off] = lo;
  }
}

// ---------------------------------------------------------------------------
// the iteration kernel
// ---------------------------------------------------------------------------

struct TcArgs {
  const float* x;        // R2 fp32 planes (current)
  float* xn;             // R2 fp32 planes (next)
  const float* N;        // R2 planes
  float* Den;            // R2 planes: running sum of the exposures' partials
  const float* u;        // n planes
  uint16_t* xb;          // [2][2][R2] 16-bit planes
  uint16_t* wb;          // [2 hi/lo][n] 16-bit planes of w = u z
  const uint16_t* hank;  // Hankel blocks
  int pp;                // ping-pong slot of the current x in xb
  const float* scales;   // device: {forward acc -> z, w -> operand, adjoint acc -> Den, x -> operand}
  int write_xb;          // epilogue writes the next x's 16-bit planes (BF16 modes)
  int* err;
};

// CTA set-up shared by both kernels: barriers (count per entry of `counts`),
// tensor memory (`cols` columns, a power of two), abort flag.
__device__ __forceinline__ uint32_t tc_setup(uint64_t* bars, const uint32_t* counts, int nbars,
                                             uint32_t* tmem_base_s, int* abort_s, uint32_t cols) {
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    *abort_s = 0;
    for (int i = 0; i < nbars; ++i) bar_init(&bars[i], counts[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_base_s)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *tmem_base_s;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t cols, int abort_s, int* err) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
  }
  if (threadIdx.x == 0 && abort_s) atomicOr(err, kErrTimeout);
}

// instruction descriptor: FP32 accumulate, BF16 or FP16 operands, M = 128, N = 128
__device__ __forceinline__ uint32_t tc_idesc(int fp16) {
  return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) |
         ((uint32_t)(kTcCols >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

// One filter row's GEMM of a band (rows shifted by a) with the Hankel operand
// of a ring stage: Kd / 16 k-steps, 1 or 3 products (hi hi, hi lo, lo hi).
template <int NPROD>
__device__ __forceinline__ void tc_row_gemm(uint32_t dacc, uint32_t band_a, uint32_t bandplane,
                                            uint32_t lbo, uint32_t bst, int Sd, int ksteps,
                                            int a, uint32_t idesc, uint32_t& accum) {
  uint64_t ah = sdesc(band_a + a * 16, lbo, 128);
  uint64_t al = ah + (bandplane >> 4);
  uint64_t bh = sdesc(bst, 128, 128);
  uint64_t bl = bh + ((uint32_t)(Sd * 128) >> 4);
  const uint64_t astep = (2u * lbo) >> 4, bstep = 256u >> 4;
#pragma unroll 2
  for (int kk = 0; kk < ksteps; ++kk) {
    mma(dacc, ah, bh, idesc, accum);
    if (NPROD == 3) {
      mma(dacc, ah, bl, idesc, 1u);
      mma(dacc, al, bh, idesc, 1u);
    }
    accum = 1;
    ah += astep;
    al += astep;
    bh += bstep;
    bl += bstep;
  }
}

// Forward model of one 128 x 128 tile for every exposure: z_t = sum over the
// phases and the Kc filter rows of (x band rows shifted by a) x Hankel(kf),
// then w_t = u_t z_t into the 16-bit w planes (hi, and lo for the split).
// Tensor memory: two accumulators of 128 columns (exposure t in t & 1).
template <int NPROD>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_fwd_kernel(const Shape s, const TcShape t, const TcArgs A,
                  const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t bars[6 + 2 * kTcStages];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * kTcRows, j0 = blockIdx.x * kTcCols;
  const Geom& g = s.g;
  const int hc = s.hc, Kc = s.Kc, R2 = s.R2;
  constexpr int nslots = NPROD == 3 ? 2 : 1;
  const uint32_t bandplane = (uint32_t)t.XRp * t.Kd * 2;
  uint8_t* band = sm;
  uint8_t* ring = band + 2 * bandplane;
  uint64_t* x_full = &bars[0];
  uint64_t* x_empty = &bars[1];
  uint64_t* acc_full = &bars[2];   // [2]
  uint64_t* acc_empty = &bars[4];  // [2]
  uint64_t* b_full = &bars[6];
  uint64_t* b_empty = &bars[6 + kTcStages];
  uint32_t counts[6 + 2 * kTcStages];
  counts[0] = 1; counts[1] = 1; counts[2] = 1; counts[3] = 1; counts[4] = 128; counts[5] = 128;
  for (int i = 0; i < 2 * kTcStages; ++i) counts[6 + i] = 1;
  const uint32_t tmem = tc_setup(bars, counts, 6 + 2 * kTcStages, &tmem_base_s, &abort_s, 256);
  volatile int* abort = &abort_s;
  const float zscale = A.scales[0], wscale = A.scales[1];
  const int ksteps = t.Kd / 16;
  const int cs = j0 + hc - t.dlt;  // padded column of band column 0 (a multiple of 8)

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------ producer
      uint32_t xe_phase = 1, be_phase = 1;
      int stage = 0;
      const uint32_t hbytes = (uint32_t)(nslots * t.Sd * 128);
      for (int tt = 0; tt < s.n && !*abort; ++tt) {
        for (int phi = 0; phi < R2; ++phi) {
          if (R2 > 1 || tt == 0) {  // r = 1: the band stays resident for all exposures
            bar_wait(x_empty, xe_phase, abort);
            xe_phase ^= 1u;
            bar_expect_tx(x_full, nslots * bandplane);
            for (int hl = 0; hl < nslots; ++hl) {
              const int plane = (A.pp * 2 + hl) * R2 + phi;
              for (int c = 0; c < t.Kd / 8; ++c)
                tma_3d(band + hl * bandplane + c * t.XRp * 16, &xmap, cs + 8 * c, i0 + hc, plane,
                       x_full);
            }
          }
          for (int a = 0; a < Kc; ++a) {
            bar_wait(&b_empty[stage], be_phase, abort);
            const uint8_t* src = reinterpret_cast<const uint8_t*>(A.hank) +
                                 (((long long)tt * R2 + phi) * Kc + a) * t.hank_block;
            bar_expect_tx(&b_full[stage], hbytes);
            bulk_copy(ring + stage * t.stage_bytes, src, hbytes, &b_full[stage]);
            if (++stage == kTcStages) { stage = 0; be_phase ^= 1u; }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------ MMA issuer
      const uint32_t idesc = tc_idesc(t.fp16);
      const uint32_t band_a = su32(band), ring_a = su32(ring);
      const uint32_t lbo = (uint32_t)t.XRp * 16;
      uint32_t xf_phase = 0, bf_phase = 0;
      uint32_t ae_phase[2] = {1u, 1u};
      int stage = 0;
      for (int tt = 0; tt < s.n && !*abort; ++tt) {
        const int buf = tt & 1;
        bar_wait(&acc_empty[buf], ae_phase[buf], abort);
        ae_phase[buf] ^= 1u;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(128 * buf);
        uint32_t accum = 0;
        for (int phi = 0; phi < R2; ++phi) {
          if (R2 > 1 || tt == 0) {
            bar_wait(x_full, xf_phase, abort);
            xf_phase ^= 1u;
            tc_fence_after();
          }
          for (int a = 0; a < Kc; ++a) {
            bar_wait(&b_full[stage], bf_phase, abort);
            tc_fence_after();
            tc_row_gemm<NPROD>(dacc, band_a, bandplane, lbo, ring_a + stage * t.stage_bytes,
                               t.Sd, ksteps, a, idesc, accum);
            mma_commit(&b_empty[stage]);
            if (++stage == kTcStages) { stage = 0; bf_phase ^= 1u; }
          }
          if (R2 > 1) mma_commit(x_empty);
        }
        mma_commit(&acc_full[buf]);
      }
    }
  } else {
    // ------------------------------ epilogue (warps 2-5): w = u z
    const int quad = warp & 3;
    const int m = 32 * quad + lane;  // tile row of this thread
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    const int i = i0 + m;
    const bool row_ok = i < g.H;
    uint32_t af_phase[2] = {0u, 0u};
    const int fp16 = t.fp16;
    for (int tt = 0; tt < s.n; ++tt) {
      const int buf = tt & 1;
      bar_wait(&acc_full[buf], af_phase[buf], abort);
      af_phase[buf] ^= 1u;
      tc_fence_after();
      const long long roff = (long long)(g.B + i) * g.P + g.B + j0;  // tile column 0 of row i
      const float* urow = A.u + (long long)tt * g.plane + roff;
      uint16_t* wh = A.wb + (long long)tt * g.plane + roff;
      uint16_t* wl = A.wb + (long long)(s.n + tt) * g.plane + roff;
      // tensor-memory column q holds tile column 127 - q; chunk cb: columns
      // c0 .. c0 + 15 with c0 = 112 - 16 cb (B is even: 8-byte aligned u pairs,
      // 4-byte aligned w pairs)
      for (int cb = 0; cb < kTcCols / 16; ++cb) {
        float z[16];
        tmem_ld16(tmem + lane_off + (uint32_t)(128 * buf + 16 * cb), z);
        const int c0 = kTcCols - 16 - 16 * cb;
        if (row_ok && !*abort) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int jc = c0 + 2 * q;  // tile columns jc, jc + 1
            if (j0 + jc >= g.W) break;
            const float2 uv = *reinterpret_cast<const float2*>(urow + jc);
            const float w0 = uv.x * z[15 - 2 * q] * zscale * wscale;
            const float w1 = (j0 + jc + 1 < g.W) ? uv.y * z[14 - 2 * q] * zscale * wscale : 0.f;
            const uint16_t h0 = enc16(w0, fp16), h1 = enc16(w1, fp16);
            *reinterpret_cast<uint32_t*>(wh + jc) = h0 | ((uint32_t)h1 << 16);
            if (NPROD == 3) {
              const uint16_t l0 = enc16(w0 - dec16(h0, fp16), fp16);
              const uint16_t l1 = enc16(w1 - dec16(h1, fp16), fp16);
              *reinterpret_cast<uint32_t*>(wl + jc) = l0 | ((uint32_t)l1 << 16);
            }
          }
        }
      }
      tc_fence_before();
      bar_arrive(&acc_empty[buf]);
    }
  }
  tc_teardown(tmem, 256, abort_s, A.err);
}

// Adjoint and update of one 128 x 128 tile of the latent planes: for every
// exposure the w band (hi, lo) by TMA, per phase the Kc filter rows of
// (band rows shifted by a) x Hankel(ka) into a tensor-memory partial, which
// the epilogue adds in FP32 to the running Den (exposures in ascending
// order); the last exposure applies x' = Den > 0 ? x max(N, 0) / Den : x.
// Tensor memory: R2 partials of 128 columns, double-buffered when R2 = 1.
template <int NPROD>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_adj_kernel(const Shape s, const TcShape t, const TcArgs A,
                  const __grid_constant__ CUtensorMap wmap) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t bars[6 + 2 * kTcStages];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * kTcRows, j0 = blockIdx.x * kTcCols;
  const Geom& g = s.g;
  const int hc = s.hc, Kc = s.Kc, R2 = s.R2;
  constexpr int nslots = NPROD == 3 ? 2 : 1;
  const int nbuf = R2 == 1 ? 2 : 1;
  const uint32_t bandplane = (uint32_t)t.XRp * t.Kd * 2;
  uint8_t* band = sm;
  uint8_t* ring = band + 2 * bandplane;
  uint64_t* w_full = &bars[0];
  uint64_t* w_empty = &bars[1];
  uint64_t* den_full = &bars[2];   // [2]
  uint64_t* den_empty = &bars[4];  // [2]
  uint64_t* b_full = &bars[6];
  uint64_t* b_empty = &bars[6 + kTcStages];
  uint32_t counts[6 + 2 * kTcStages];
  counts[0] = 1; counts[1] = 1; counts[2] = 1; counts[3] = 1; counts[4] = 128; counts[5] = 128;
  for (int i = 0; i < 2 * kTcStages; ++i) counts[6 + i] = 1;
  const uint32_t tmem = tc_setup(bars, counts, 6 + 2 * kTcStages, &tmem_base_s, &abort_s, 512);
  volatile int* abort = &abort_s;
  const float dscale = A.scales[2], xscale = A.scales[3];
  const int ksteps = t.Kd / 16;
  const int cs = j0 + hc - t.dlt;

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------ producer
      uint32_t we_phase = 1, be_phase = 1;
      int stage = 0;
      const uint32_t hbytes = (uint32_t)(nslots * t.Sd * 128);
      for (int tt = 0; tt < s.n && !*abort; ++tt) {
        bar_wait(w_empty, we_phase, abort);
        we_phase ^= 1u;
        bar_expect_tx(w_full, nslots * bandplane);
        for (int hl = 0; hl < nslots; ++hl)
          for (int c = 0; c < t.Kd / 8; ++c)
            tma_3d(band + hl * bandplane + c * t.XRp * 16, &wmap, cs + 8 * c, i0 + hc,
                   hl * s.n + tt, w_full);
        for (int phi = 0; phi < R2; ++phi) {
          for (int a = 0; a < Kc; ++a) {
            bar_wait(&b_empty[stage], be_phase, abort);
            const uint8_t* src = reinterpret_cast<const uint8_t*>(A.hank) +
                                 (((long long)tt * R2 + phi) * Kc + a) * t.hank_block +
                                 t.stage_bytes;
            bar_expect_tx(&b_full[stage], hbytes);
            bulk_copy(ring + stage * t.stage_bytes, src, hbytes, &b_full[stage]);
            if (++stage == kTcStages) { stage = 0; be_phase ^= 1u; }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------ MMA issuer
      const uint32_t idesc = tc_idesc(t.fp16);
      const uint32_t band_a = su32(band), ring_a = su32(ring);
      const uint32_t lbo = (uint32_t)t.XRp * 16;
      uint32_t wf_phase = 0, bf_phase = 0;
      uint32_t de_phase[2] = {1u, 1u};
      int stage = 0;
      for (int tt = 0; tt < s.n && !*abort; ++tt) {
        const int buf = nbuf == 2 ? (tt & 1) : 0;
        bar_wait(&den_empty[buf], de_phase[buf], abort);
        de_phase[buf] ^= 1u;
        bar_wait(w_full, wf_phase, abort);
        wf_phase ^= 1u;
        tc_fence_after();
        for (int phi = 0; phi < R2; ++phi) {
          const uint32_t dden = tmem + (uint32_t)(128 * (R2 * buf + phi));
          uint32_t accum = 0;
          for (int a = 0; a < Kc; ++a) {
            bar_wait(&b_full[stage], bf_phase, abort);
            tc_fence_after();
            tc_row_gemm<NPROD>(dden, band_a, bandplane, lbo, ring_a + stage * t.stage_bytes,
                               t.Sd, ksteps, a, idesc, accum);
            mma_commit(&b_empty[stage]);
            if (++stage == kTcStages) { stage = 0; bf_phase ^= 1u; }
          }
        }
        mma_commit(w_empty);
        mma_commit(&den_full[buf]);
      }
    }
  } else {
    // ------------------------------ epilogue (warps 2-5): Den, update
    const int quad = warp & 3;
    const int m = 32 * quad + lane;
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    const int i = i0 + m;
    const bool row_ok = i < g.H;
    uint32_t df_phase[2] = {0u, 0u};
    const int fp16 = t.fp16;
    for (int tt = 0; tt < s.n; ++tt) {
      const int buf = nbuf == 2 ? (tt & 1) : 0;
      bar_wait(&den_full[buf], df_phase[buf], abort);
      df_phase[buf] ^= 1u;
      tc_fence_after();
      const bool last = (tt + 1 == s.n);
      for (int phi = 0; phi < R2; ++phi) {
        const long long pb = (long long)phi * g.plane + (long long)(g.B + i) * g.P + g.B + j0;
        for (int cb = 0; cb < kTcCols / 16; ++cb) {
          float dv[16];
          tmem_ld16(tmem + lane_off + (uint32_t)(128 * (R2 * buf + phi) + 16 * cb), dv);
          if (!row_ok || *abort) continue;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int jc = kTcCols - 1 - (16 * cb + e);  // tile column of dv[e]
            if (j0 + jc >= g.W) continue;
            const long long off = pb + jc;
            float d = dv[e] * dscale;
            if (tt > 0) d = A.Den[off] + d;
            if (!last) {
              A.Den[off] = d;
              continue;
            }
            const float xo = A.x[off];
            float xv = xo;
            if (d > 0.f) {
              const float nv = fmaxf(A.N[off], 0.f);
              if (d < 1e-30f)  // denominator near zero: guarded ratio in FP64
                xv = (float)((double)xo * (double)nv / (double)d);
              else
                xv = xo * nv / d;
            }
            A.xn[off] = xv;
            if (A.write_xb) {
              const float sv = xv * xscale;
              const uint16_t h = enc16(sv, fp16);
              const long long o2 = off - (long long)phi * g.plane;
              A.xb[((long long)((A.pp ^ 1) * 2 + 0) * R2 + phi) * g.plane + o2] = h;
              A.xb[((long long)((A.pp ^ 1) * 2 + 1) * R2 + phi) * g.plane + o2] =
                  enc16(sv - dec16(h, fp16), fp16);
            }
          }
        }
      }
      tc_fence_before();
      bar_arrive(&den_empty[buf]);
    }
  }
  tc_teardown(tmem, 512, abort_s, A.err);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// layout: 16-bit x planes [2][2][R2], Hankel blocks, 16-bit w planes [2][n],
// then 512 bytes of scales and maxima
size_t tc_buffer_bytes(const Shape& s, const TcShape& t) {
  return tc_w_offset(s, t) + ((2ull * s.n * s.g.plane * sizeof(uint16_t) + 255) & ~(size_t)255) +
         512;
}

size_t tc_w_offset(const Shape& s, const TcShape& t) {
  const size_t xb = 4ull * s.R2 * s.g.plane * sizeof(uint16_t);
  const size_t hk = (size_t)s.n * s.R2 * s.Kc * t.hank_block;
  return ((xb + 255) & ~(size_t)255) + ((hk + 255) & ~(size_t)255);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 3-D map over `planes` 16-bit padded planes (the x planes or the w planes):
// boxes of 8 columns x XRp rows of one plane
int make_plane_tensormap(const Shape& s, const TcShape& t, void* base, int planes,
                         CUtensorMap* map) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        !p || q != cudaDriverEntryPointSuccess)
      return -1;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  const Geom& g = s.g;
  cuuint64_t dims[3] = {(cuuint64_t)g.P, (cuuint64_t)g.PH, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)g.P * 2, (cuuint64_t)g.plane * 2};
  cuuint32_t box[3] = {8, (cuuint32_t)t.XRp, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

cudaError_t launch_build_hankel(const Shape& s, const TcShape& t, const float* kf, const float* ka,
                                uint16_t* hank, float gscale, cudaStream_t st) {
  build_hankel_kernel<<<1024, 256, 0, st>>>(s, t, kf, ka, hank, gscale);
  return cudaGetLastError();
}

cudaError_t launch_split_x(const Shape& s, const TcShape& t, const float* x, uint16_t* xb, int pp,
                           const float* scales, cudaStream_t st) {
  split_x_kernel<<<1024, 256, 0, st>>>(s, t.fp16, x, xb, pp, scales);
  return cudaGetLastError();
}

// max of non-negative values (the float bit patterns order like the integers)
__global__ void max_nonneg_kernel(const float* __restrict__ v, long long count,
                                  unsigned int* __restrict__ out) {
  float m = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, v[e]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

cudaError_t launch_max_nonneg(const float* v, long long count, unsigned int* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  max_nonneg_kernel<<<1024, 256, 0, st>>>(v, count, out);
  return cudaGetLastError();
}

// FP16 operand scales, all powers of two: x -> 2^ex x with max x scaled to
// <= 2^14, PSF taps by gscale (fixed per frame set), w by a bound:
// |w| <= max u * max x * fsum (fsum = largest sum of |taps| of a forward
// model). scales = {1/(xs gs), ws, 1/(ws gs), xs}.
__global__ void fp16_scales_kernel(const unsigned int* __restrict__ xmax_bits, float gscale,
                                   float umax, float fsum, float* __restrict__ scales) {
  const float xmax = fmaxf(__uint_as_float(*xmax_bits), 1e-30f);
  const float xs = exp2f(floorf(log2f(16384.f / xmax)));
  const float wb = fmaxf(umax * xmax * fsum, 1e-30f);
  const float ws = exp2f(floorf(log2f(16384.f / wb)));
  scales[0] = 1.f / (xs * gscale);
  scales[1] = ws;
  scales[2] = 1.f / (ws * gscale);
  scales[3] = xs;
}

cudaError_t launch_fp16_scales(const unsigned int* xmax_bits, float gscale, float umax, float fsum,
                               float* scales, cudaStream_t st) {
  fp16_scales_kernel<<<1, 1, 0, st>>>(xmax_bits, gscale, umax, fsum, scales);
  return cudaGetLastError();
}

cudaError_t launch_tc_iter(const Shape& s, const TcShape& t, const TcLaunch& L,
                           const CUtensorMap& xmap, const CUtensorMap& wmap, cudaStream_t st) {
  const bool split = t.nprod == 3;
  cudaError_t e = allow_max_dynamic_smem(split ? (const void*)tc_fwd_kernel<3>
                                               : (const void*)tc_fwd_kernel<1>);
  if (e == cudaSuccess)
    e = allow_max_dynamic_smem(split ? (const void*)tc_adj_kernel<3>
                                     : (const void*)tc_adj_kernel<1>);
  if (e != cudaSuccess) return e;
  TcArgs a;
  a.x = L.x;
  a.xn = L.xn;
  a.N = L.N;
  a.Den = L.Den;
  a.u = L.u;
  a.xb = L.xb;
  a.wb = L.wb;
  a.hank = L.hank;
  a.pp = L.pp;
  a.scales = L.scales;
  a.write_xb = L.write_xb;
  a.err = L.err;
  dim3 grid(t.gxt, t.gyt);
  if (split)
    tc_fwd_kernel<3><<<grid, kTcThreads, t.smem, st>>>(s, t, a, xmap);
  else
    tc_fwd_kernel<1><<<grid, kTcThreads, t.smem, st>>>(s, t, a, xmap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (split)
    tc_adj_kernel<3><<<grid, kTcThreads, t.smem, st>>>(s, t, a, wmap);
  else
    tc_adj_kernel<1><<<grid, kTcThreads, t.smem, st>>>(s, t, a, wmap);
  return cudaGetLastError();
}

}  // namespace emd
