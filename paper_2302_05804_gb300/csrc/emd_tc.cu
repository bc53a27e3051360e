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
// One CTA computes a 128 x 64 tile of Den for all exposures (Den stays in
// tensor memory for the whole iteration), recomputing the forward model on
// the tile plus a halo of hc (two 128-row M-tiles of up to 112 columns),
// and applies the multiplicative update at the end. Warp roles: warp 0
// issues TMA / bulk copies, warp 1 allocates tensor memory and issues MMAs,
// warps 2-5 run the epilogues (weighting by u into shared memory, update).
// Every mbarrier wait is bounded; a timeout raises the error word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>

#include "emd_internal.cuh"
#include "emd_tc.cuh"

namespace emd {

namespace {

constexpr int kTcRows = 128;    // Den rows per CTA = MMA M
constexpr int kTcCols = 64;     // Den columns per CTA = adjoint N
constexpr int kTcThreads = 192; // 6 warps
constexpr int kTcStages = 3;    // B (Hankel) ring depth
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
  t->TC = kTcCols;
  t->Nf = rup(kTcCols + 2 * s.hc, 16);
  t->Kf = rup(t->Nf + 2 * s.hc, 16);
  t->Ka = t->Nf;
  t->XRp = rup(kTcRows + 2 * s.hc, 8);
  t->WRp = rup(kTcRows + 2 * s.hc, 8);
  t->Sf = t->Kf / 8 + t->Nf / 8 - 1;
  t->Sa = t->Ka / 8 + kTcCols / 8 - 1;
  t->gxt = (s.W + kTcCols - 1) / kTcCols;
  t->gyt = (s.H + kTcRows - 1) / kTcRows;
  if (t->Nf > 128) { *why = "PSF footprint too large for the tensor-core tile"; return false; }
  const size_t xs = 2ull * t->XRp * t->Kf * 2;
  const size_t ws = 2ull * t->WRp * t->Ka * 2;
  const size_t stage = 2ull * t->Sf * 128;
  t->stage_bytes = (int)stage;
  t->hank_block = 2 * (t->Sf + t->Sa) * 128;
  t->smem = xs + ws + kTcStages * stage + 256;
  if (t->smem > 227 * 1024 - 1024) { *why = "tensor-core tile exceeds shared memory"; return false; }
  // one CTA per SM: a second resident CTA would wait in tcgen05.alloc for
  // the 512 tensor-memory columns of the first
  if (t->smem < 120 * 1024) t->smem = 120 * 1024;
  // the epilogue's u reads (region rows < 128 + 2hc, columns < Nf) stay in
  // the padded planes; TMA loads outside the planes read zeros
  const Geom& g = s.g;
  if ((t->gxt - 1) * kTcCols + s.hc + t->Nf > g.P ||
      (t->gyt - 1) * kTcRows + 3 * s.hc + kTcRows > g.PH) {
    *why = "padded geometry too small for the tensor-core tiles";
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------

// Hankel core matrices of every (t, phi, a): block = [F_hi | F_lo | A_hi | A_lo],
// F: Sf x 8 x 8 entries g[8s + r + e - (Nf - 1)] of kf row a; A: the same with
// ka and N = TC. lo = rounding residue of the scaled value.
__global__ void build_hankel_kernel(const Shape s, const TcShape t, const float* __restrict__ kf,
                                    const float* __restrict__ ka, uint16_t* __restrict__ hank,
                                    float gscale) {
  const long long per = (long long)(t.Sf + t.Sa) * 64;
  const long long total = (long long)s.n * s.R2 * s.Kc * per;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / per;
    const int within = (int)(e - blk * per);
    const int a = (int)(blk % s.Kc);
    const long long tp = blk / s.Kc;  // t * R2 + phi
    const bool fwd = within < t.Sf * 64;
    const int w = fwd ? within : within - t.Sf * 64;
    const int sidx = w / 64, r = (w / 8) % 8, c = w % 8;
    const int N = fwd ? t.Nf : t.TC;
    const int idx = 8 * sidx + r + c - (N - 1);
    const float* krow = (fwd ? kf : ka) + (tp * s.Kc + a) * s.KP;
    const float g = (idx >= 0 && idx < s.Kc) ? krow[idx] * gscale : 0.f;
    const uint16_t hi = enc16(g, t.fp16);
    const uint16_t lo = enc16(g - dec16(hi, t.fp16), t.fp16);
    uint16_t* base = hank + blk * (long long)(t.hank_block / 2);
    const int S = fwd ? t.Sf : t.Sa;
    uint16_t* part = base + (fwd ? 0 : 2 * t.Sf * 64);
    part[w] = hi;
    part[S * 64 + w] = lo;
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
  const uint16_t* hank;  // Hankel blocks
  int pp;                // ping-pong slot of the current x in xb
  const float* scales;   // device: {forward acc -> z, w -> operand, adjoint acc -> Den, x -> operand}
  int write_xb;          // epilogue writes the next x's 16-bit planes (BF16 modes)
  int* err;
};

template <int NPROD>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_iter_kernel(const Shape s, const TcShape t, const TcArgs A,
                   const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t bars[9 + 2 * kTcStages];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * kTcRows, j0 = blockIdx.x * kTcCols;
  const Geom& g = s.g;
  const int hc = s.hc, Kc = s.Kc, R2 = s.R2;

  const uint32_t xplane_b = (uint32_t)t.XRp * t.Kf * 2;  // bytes of one x band plane
  const uint32_t wplane_b = (uint32_t)t.WRp * t.Ka * 2;
  uint8_t* xs = sm;
  uint8_t* ws = xs + 2 * xplane_b;
  uint8_t* ring = ws + 2 * wplane_b;
  uint64_t* x_full = &bars[0];
  uint64_t* x_empty = &bars[1];
  uint64_t* acc_full = &bars[2];   // [2]
  uint64_t* acc_empty = &bars[4];  // [2]
  uint64_t* w_full = &bars[6];
  uint64_t* den_full = &bars[7];
  uint64_t* den_empty = &bars[8];
  uint64_t* b_full = &bars[9];
  uint64_t* b_empty = &bars[9 + kTcStages];
  volatile int* abort = &abort_s;

  if (threadIdx.x == 0) {
    abort_s = 0;
    bar_init(x_full, 1);
    bar_init(x_empty, 1);
    for (int i = 0; i < 2; ++i) {
      bar_init(&acc_full[i], 1);
      bar_init(&acc_empty[i], 128);
    }
    bar_init(w_full, 128);
    bar_init(den_full, 1);
    bar_init(den_empty, 128);
    for (int i = 0; i < kTcStages; ++i) {
      bar_init(&b_full[i], 1);
      bar_init(&b_empty[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        su32(&tmem_base_s)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  constexpr int nprod = NPROD;
  const float zscale = A.scales[0], wscale = A.scales[1], dscale = A.scales[2],
              xscale = A.scales[3];
  const int KSf = t.Kf / 16, KSa = t.Ka / 16;

  if (warp == 0) {
    // ------------------------------ producer ------------------------------
    if (lane == 0) {
      uint32_t xe_phase = 1;  // x_empty: the first wait passes
      int stage = 0;
      uint32_t be_phase = 1;
      const long long hb = t.hank_block;
      for (int tt = 0; tt < s.n && !*abort; ++tt) {
        // split products: one pass per forward M-tile with its hi and lo x
        // bands; one product: a single pass with both M-tiles' bands resident
        // (the lo slot holds the second band), so consecutive MMAs share B
        for (int pass = 0; pass < (nprod == 1 ? 1 : 2); ++pass) {
          for (int phi = 0; phi < R2; ++phi) {
            bar_wait(x_empty, xe_phase, abort);
            xe_phase ^= 1u;
            bar_expect_tx(x_full, 2 * xplane_b);
            for (int slot = 0; slot < 2; ++slot) {
              const int hl = (nprod == 1) ? 0 : slot;
              const int mt = (nprod == 1) ? slot : pass;
              const int plane = (A.pp * 2 + hl) * R2 + phi;
              for (int c = 0; c < t.Kf / 8; ++c)
                tma_3d(xs + slot * xplane_b + c * t.XRp * 16, &xmap, j0 + 8 * c, i0 + kTcRows * mt,
                       plane, x_full);
            }
            for (int a = 0; a < Kc; ++a) {
              bar_wait(&b_empty[stage], be_phase, abort);
              const uint8_t* src =
                  reinterpret_cast<const uint8_t*>(A.hank) + (((long long)tt * R2 + phi) * Kc + a) * hb;
              const uint32_t bytes = 2u * t.Sf * 128u;
              bar_expect_tx(&b_full[stage], bytes);
              bulk_copy(ring + stage * t.stage_bytes, src, bytes, &b_full[stage]);
              if (++stage == kTcStages) { stage = 0; be_phase ^= 1u; }
            }
          }
        }
        for (int phi = 0; phi < R2; ++phi) {
          for (int a = 0; a < Kc; ++a) {
            bar_wait(&b_empty[stage], be_phase, abort);
            const uint8_t* src = reinterpret_cast<const uint8_t*>(A.hank) +
                                 (((long long)tt * R2 + phi) * Kc + a) * hb + 2ll * t.Sf * 128;
            const uint32_t bytes = 2u * t.Sa * 128u;
            bar_expect_tx(&b_full[stage], bytes);
            bulk_copy(ring + stage * t.stage_bytes, src, bytes, &b_full[stage]);
            if (++stage == kTcStages) { stage = 0; be_phase ^= 1u; }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer -----------------------------
    if (lane == 0) {
      const uint32_t idesc_base = (1u << 4) | ((t.fp16 ? 0u : 1u) << 7) | ((t.fp16 ? 0u : 1u) << 10) |
                                  ((uint32_t)(kTcRows >> 4) << 24);
      const uint32_t idesc_f = idesc_base | ((uint32_t)(t.Nf >> 3) << 17);
      const uint32_t idesc_a = idesc_base | ((uint32_t)(t.TC >> 3) << 17);
      const uint32_t xs_a = su32(xs), ws_a = su32(ws), ring_a = su32(ring);
      const uint32_t x_lbo = (uint32_t)t.XRp * 16, w_lbo = (uint32_t)t.WRp * 16;
      uint32_t xf_phase = 0, wf_phase = 0, bf_phase = 0, de_phase = 1;
      uint32_t ae_phase[2] = {1u, 1u};
      int stage = 0;
      for (int tt = 0; tt < s.n && !*abort; ++tt) {
        for (int pass = 0; pass < (nprod == 1 ? 1 : 2); ++pass) {
          const int mt0 = (nprod == 1) ? 0 : pass;
          const int mt1 = (nprod == 1) ? 1 : pass;
          for (int mt = mt0; mt <= mt1; ++mt) {
            bar_wait(&acc_empty[mt], ae_phase[mt], abort);
            ae_phase[mt] ^= 1u;
          }
          tc_fence_after();
          const uint32_t dacc = tmem + (uint32_t)(128 * mt0);
          uint32_t accum = 0;
          for (int phi = 0; phi < R2; ++phi) {
            bar_wait(x_full, xf_phase, abort);
            xf_phase ^= 1u;
            tc_fence_after();
            for (int a = 0; a < Kc; ++a) {
              bar_wait(&b_full[stage], bf_phase, abort);
              tc_fence_after();
              const uint32_t bst = ring_a + stage * t.stage_bytes;
              // descriptor bases; a k-step advances the start-address field.
              // Split: ah/al = x_hi/x_lo of this M-tile. One product: ah/al =
              // x of M-tile 0 / M-tile 1.
              uint64_t ah = sdesc(xs_a + a * 16, x_lbo, 128);
              uint64_t al = ah + (xplane_b >> 4);
              uint64_t bh = sdesc(bst, 128, 128);
              uint64_t bl = bh + ((uint32_t)(t.Sf * 128) >> 4);
              const uint64_t astep = (2u * x_lbo) >> 4, bstep = 256u >> 4;
#pragma unroll 2
              for (int kk = 0; kk < KSf; ++kk) {
                if (nprod == 3) {
                  mma(dacc, ah, bh, idesc_f, accum);
                  mma(dacc, ah, bl, idesc_f, 1u);
                  mma(dacc, al, bh, idesc_f, 1u);
                } else {
                  mma(dacc, ah, bh, idesc_f, accum);
                  mma(dacc + 128u, al, bh, idesc_f, accum);
                }
                accum = 1;
                ah += astep;
                al += astep;
                bh += bstep;
                bl += bstep;
              }
              mma_commit(&b_empty[stage]);
              if (++stage == kTcStages) { stage = 0; bf_phase ^= 1u; }
            }
            mma_commit(x_empty);
          }
          for (int mt = mt0; mt <= mt1; ++mt) mma_commit(&acc_full[mt]);
        }
        // adjoint of this exposure into the Den partial (tensor-memory
        // columns 256 + 64 phi), once the epilogue has taken the last one
        bar_wait(w_full, wf_phase, abort);
        wf_phase ^= 1u;
        bar_wait(den_empty, de_phase, abort);
        de_phase ^= 1u;
        tc_fence_after();
        for (int phi = 0; phi < R2; ++phi) {
          const uint32_t dden = tmem + 256u + (uint32_t)(t.TC * phi);
          for (int a = 0; a < Kc; ++a) {
            bar_wait(&b_full[stage], bf_phase, abort);
            tc_fence_after();
            const uint32_t bst = ring_a + stage * t.stage_bytes;
            uint64_t ah = sdesc(ws_a + a * 16, w_lbo, 128);
            uint64_t al = ah + (wplane_b >> 4);
            uint64_t bh = sdesc(bst, 128, 128);
            uint64_t bl = bh + ((uint32_t)(t.Sa * 128) >> 4);
            const uint64_t astep = (2u * w_lbo) >> 4, bstep = 256u >> 4;
            uint32_t acc = (a > 0) ? 1u : 0u;
#pragma unroll 2
            for (int kk = 0; kk < KSa; ++kk) {
              mma(dden, ah, bh, idesc_a, acc);
              acc = 1u;
              if (nprod == 3) {
                mma(dden, ah, bl, idesc_a, 1u);
                mma(dden, al, bh, idesc_a, 1u);
              }
              ah += astep;
              al += astep;
              bh += bstep;
              bl += bstep;
            }
            mma_commit(&b_empty[stage]);
            if (++stage == kTcStages) { stage = 0; bf_phase ^= 1u; }
          }
        }
        mma_commit(den_full);
      }
    }
  } else {
    // ------------------------------ epilogue (warps 2-5) -------------------
    const int quad = warp & 3;           // tensor-memory lane quadrant of this warp
    const int m = 32 * quad + lane;      // row within an M-tile
    const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
    uint32_t af_phase[2] = {0u, 0u};
    uint32_t df_phase = 0;
    const int fp16 = t.fp16;
    for (int tt = 0; tt < s.n; ++tt) {
      const float* ut = A.u + (long long)tt * g.plane;
      for (int mt = 0; mt < 2; ++mt) {
        const int rr = kTcRows * mt + m;  // region row (0 = coarse row i0 - hc)
        const bool valid = rr < kTcRows + 2 * hc;
        const bool warp_valid = kTcRows * mt + 32 * quad < kTcRows + 2 * hc;
        const float* urow = ut + (long long)(i0 + hc + rr) * g.P + (j0 + hc);
        const int nch = t.Nf / 16;
        if (warp_valid) {
          // tensor-memory columns 16cb..16cb+15 hold region columns
          // Nf-1-16cb down to Nf-16-16cb; u of the next chunk is loaded while
          // the current one is converted
          float un[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) un[e] = valid ? urow[t.Nf - 1 - e] : 0.f;
          for (int cb = 0; cb < nch; ++cb) {
            float uc[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) uc[e] = un[e];
            if (cb + 1 < nch) {
#pragma unroll
              for (int e = 0; e < 16; ++e) un[e] = valid ? urow[t.Nf - 17 - 16 * cb - e] : 0.f;
            }
            float z[16];
            if (cb == 0) {
              bar_wait(&acc_full[mt], af_phase[mt], abort);
              tc_fence_after();
            }
            tmem_ld16(tmem + lane_off + (uint32_t)(128 * mt + 16 * cb), z);
            if (valid) {
              const int c_hi = t.Nf - 16 * cb - 1;  // region column of z[0]
              uint16_t hv[16], lv[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float w = uc[e] * z[e] * zscale * wscale;
                const uint16_t h = enc16(w, fp16);
                hv[15 - e] = h;
                lv[15 - e] = enc16(w - dec16(h, fp16), fp16);
              }
              const int c0 = c_hi - 15;  // lowest region column of the chunk (multiple of 8)
#pragma unroll
              for (int half = 0; half < 2; ++half) {
                const int grp = (c0 >> 3) + half;
                uint4 ph, pl;
                ph.x = hv[8 * half + 0] | ((uint32_t)hv[8 * half + 1] << 16);
                ph.y = hv[8 * half + 2] | ((uint32_t)hv[8 * half + 3] << 16);
                ph.z = hv[8 * half + 4] | ((uint32_t)hv[8 * half + 5] << 16);
                ph.w = hv[8 * half + 6] | ((uint32_t)hv[8 * half + 7] << 16);
                *reinterpret_cast<uint4*>(ws + (size_t)grp * t.WRp * 16 + rr * 16) = ph;
                if (nprod == 3) {
                  pl.x = lv[8 * half + 0] | ((uint32_t)lv[8 * half + 1] << 16);
                  pl.y = lv[8 * half + 2] | ((uint32_t)lv[8 * half + 3] << 16);
                  pl.z = lv[8 * half + 4] | ((uint32_t)lv[8 * half + 5] << 16);
                  pl.w = lv[8 * half + 6] | ((uint32_t)lv[8 * half + 7] << 16);
                  *reinterpret_cast<uint4*>(ws + wplane_b + (size_t)grp * t.WRp * 16 + rr * 16) = pl;
                }
              }
            }
          }
        } else {
          bar_wait(&acc_full[mt], af_phase[mt], abort);
          tc_fence_after();
        }
        af_phase[mt] ^= 1u;
        tc_fence_before();
        bar_arrive(&acc_empty[mt]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_arrive(w_full);
      // ---- this exposure's Den partial: summed into the running Den (FP32,
      // exposures in ascending order); the last exposure applies
      // x' = Den > 0 ? x max(N,0) / Den : x instead of storing
      bar_wait(den_full, df_phase, abort);
      df_phase ^= 1u;
      tc_fence_after();
      const int i = i0 + m;
      const bool last = (tt + 1 == s.n);
      for (int phi = 0; phi < R2; ++phi) {
        const long long pb = (long long)phi * g.plane;
        for (int cb = 0; cb < t.TC / 16; ++cb) {
          float dv[16];
          tmem_ld16(tmem + lane_off + 256u + (uint32_t)(t.TC * phi + 16 * cb), dv);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int jj = t.TC - 1 - (16 * cb + e);
            const int j = j0 + jj;
            if (i < g.H && j < g.W && !*abort) {
              const long long off = pb + (long long)(g.B + i) * g.P + g.B + j;
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
                if (d < 1e-30f)
                  xv = (float)((double)xo * (double)nv / (double)d);
                else
                  xv = xo * nv / d;
              }
              A.xn[off] = xv;
              if (A.write_xb) {
                const float sv = xv * xscale;
                const uint16_t h = enc16(sv, fp16);
                const long long plane_hi = ((long long)((A.pp ^ 1) * 2 + 0) * R2 + phi) * g.plane;
                const long long plane_lo = ((long long)((A.pp ^ 1) * 2 + 1) * R2 + phi) * g.plane;
                const long long o2 = (long long)(g.B + i) * g.P + g.B + j;
                A.xb[plane_hi + o2] = h;
                A.xb[plane_lo + o2] = enc16(sv - dec16(h, fp16), fp16);
              }
            }
          }
        }
      }
      tc_fence_before();
      bar_arrive(den_empty);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
  if (threadIdx.x == 0 && abort_s) atomicOr(A.err, kErrTimeout);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

size_t tc_buffer_bytes(const Shape& s, const TcShape& t) {
  const size_t xb = 4ull * s.R2 * s.g.plane * sizeof(uint16_t);
  const size_t hk = (size_t)s.n * s.R2 * s.Kc * t.hank_block;
  return ((xb + 255) & ~(size_t)255) + ((hk + 255) & ~(size_t)255) + 512;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int make_x_tensormap(const Shape& s, const TcShape& t, void* xb, CUtensorMap* map) {
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
  cuuint64_t dims[3] = {(cuuint64_t)g.P, (cuuint64_t)g.PH, (cuuint64_t)(4 * s.R2)};
  cuuint64_t strides[2] = {(cuuint64_t)g.P * 2, (cuuint64_t)g.plane * 2};
  cuuint32_t box[3] = {8, (cuuint32_t)t.XRp, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, xb, dims, strides, box, estr,
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
                           const CUtensorMap& map, cudaStream_t st) {
  {
    cudaError_t e = allow_max_dynamic_smem(t.nprod == 3 ? (const void*)tc_iter_kernel<3>
                                                       : (const void*)tc_iter_kernel<1>);
    if (e != cudaSuccess) return e;
  }
  TcArgs a;
  a.x = L.x;
  a.xn = L.xn;
  a.N = L.N;
  a.Den = L.Den;
  a.u = L.u;
  a.xb = L.xb;
  a.hank = L.hank;
  a.pp = L.pp;
  a.scales = L.scales;
  a.write_xb = L.write_xb;
  a.err = L.err;
  dim3 grid(t.gxt, t.gyt);
  if (t.nprod == 3)
    tc_iter_kernel<3><<<grid, kTcThreads, t.smem, st>>>(s, t, a, map);
  else
    tc_iter_kernel<1><<<grid, kTcThreads, t.smem, st>>>(s, t, a, map);
  return cudaGetLastError();
}

}  // namespace emd
