// emd_fft.cu -- the forward model and the adjoint of Eq. (2) by FFT
// (overlap-save on 128 x 128 tiles), an alternative to the direct FP32
// kernel. Same arithmetic type (FP32), different rounding. For r > 1 every
// operator below acts on the polyphase planes with the Kc x Kc phase
// kernels (hc in place of h), summed over the phases in the forward model.
//
// For an output tile with origin (i0, j0) and side B = 128 - 2 hc (hc =
// (K-1)/2), the input region is rows/cols [i0 - hc, i0 - hc + 128) of the
// image, zero outside it. With k the K x K PSF at the top-left of a zero
// 128 x 128 array, the circular convolution of the region with k holds
// z(i0 + p, j0 + q) at circular index (p + 2hc, q + 2hc), and the circular
// correlation of the w region with k holds Den(i0 + p, j0 + q) at (p, q),
// for p, q < B: no wrapped term reaches those indices. In Fourier space the
// convolution multiplies by k^ and the correlation by conj(k^) (k is real).
//
// 2D real transforms in shared memory, in place, each 128-point FFT done by
// one warp in registers (radix-2 butterflies; four values per lane; the
// cross-lane stages exchange half of a lane's values with its partner lane):
//   forward (R2C): two real rows packed as one complex row; 64 row FFTs by
//     decimation in frequency (natural in; frequency 32 q + rev5(l) out in
//     slot q of lane l, stored at 32 q + l); the packed spectra split into
//     the half spectra (65 bins) of the two rows; 65 column FFTs, again by
//     decimation in frequency, stored the same way. Result: row frequency
//     permuted, column frequency 0..64 natural. The PSF spectra are made by
//     the same code, so products never need a reordering.
//   inverse (C2R): 65 column FFTs by decimation in time with conjugate
//     twiddles (the permuted order in, natural out); the half spectra of row
//     pairs merged into one packed full spectrum (Hermitian symmetry),
//     written in the permuted order; 64 row FFTs by decimation in time; real
//     part = even row, imaginary part = odd row; scaled by 1/128^2 (exact).
// A half-spectrum buffer is 128 rows x kFP complex; the packed row pair k
// occupies the 2 kFP slots from 2k kFP, so splitting and merging stay in
// place (each pair is one warp's, with a warp barrier between its reads and
// its writes).
//
// Per iteration: fft_forward_kernel (per tile: x^ once, then for each
// exposure z = IFFT(x^ k_t^), w_t = u_t z written to a plane) and
// fft_adjoint_kernel (per tile: sum_t FFT(w_t) conj(k_t^), one inverse
// transform, the update of Eq. (2)), one CTA per tile; or, for r = 1
// Gaussian with at least as many tiles as SMs, their split forms
// (fft_forward_split_kernel, fft_adjoint_split_kernel: one persistent CTA
// per SM, whole waves of tiles, then the last wave's tiles cut into
// exposure ranges across all CTAs).
#include <math.h>

#include "emd_internal.cuh"
#include "emd_fft.cuh"

namespace emd {
namespace {

constexpr int kFT = 128;                 // tile side
constexpr int kFP = 67;                  // half-spectrum row pitch (complex, odd:
                                         // a warp's column loads hit distinct banks)
constexpr int kFBins = 65;               // half-spectrum columns
constexpr int kFBuf = kFT * kFP;         // float2 per transform buffer
constexpr int kFThreads = 512;
constexpr float kFScale = 1.0f / (kFT * kFT);

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ int rev5(int m) { return (int)(__brev((unsigned)m) >> 27); }

// Twiddles exp(-2 pi i k / 128), laid out so that the 32 lanes of a warp
// read consecutive entries at every stage (no bank conflicts):
//   w[k]        k < 64 (first stage: lane l, value q reads w[32 q + l])
//   lane2[l]    w[2 l] (second stage)
//   xs[k][l]    the twiddle of the cross-lane stage on lane bit k (span
//               2^k): w[(l mod 2^k) 64 / 2^k], negated on the lanes whose bit
//               k is set (see warp_fft_dif and warp_ifft_dit)
struct TwTab {
  float2 w[64];
  float2 lane2[32];
  float2 xs[5][32];
};

__device__ __forceinline__ float2 twiddle(int k) {
  float sn, cs;
  sincospif((float)k / 64.f, &sn, &cs);
  return make_float2(cs, -sn);
}

__device__ __forceinline__ void init_twiddles(TwTab& T) {
  for (int e = threadIdx.x; e < 64 + 32 + 5 * 32; e += blockDim.x) {
    if (e < 64) {
      T.w[e] = twiddle(e);
    } else if (e < 96) {
      T.lane2[e - 64] = twiddle(2 * (e - 64));
    } else {
      const int k = (e - 96) >> 5, l = (e - 96) & 31, S = 1 << k;
      const float2 w = twiddle((l & (S - 1)) * (64 >> k));
      T.xs[k][l] = (l & S) ? make_float2(-w.x, -w.y) : w;
    }
  }
  __syncthreads();
}

// J independent 128-point FFTs per warp, in registers. A lane holds four
// values per transform; slot q = 2 s1 + s0 and lane l address element
// e = 32 q + l of the natural input. Decimation in frequency: the spans 64
// and 32 pair a lane's own slots (s1, then s0). Each shorter span 2^k pairs
// the lanes l and l ^ 2^k: the two exchange the halves of their slot pairs
// that the other needs -- lane bit k trades places with a slot bit whose
// element bit is already done (s1, s0, s1, s0, s1 for k = 4 .. 0) -- so
// every lane holds whole butterflies: per stage it sends two values of the
// four and runs two butterflies, (m + o, (m - o) t) with its own value m,
// the received o and t negated on the upper lane (the lower lane's a - b is
// the upper lane's b - a). Output: lane l, slot q holds the spectrum at
// 32 q + rev5(l). The J transforms share the twiddle loads and overlap each
// other's latency (J = 2 in the row and column passes).
template <int J, int K, int SB>  // lane bit K, slot bit SB
__device__ __forceinline__ void dif_exchange_stage(float2 (&v)[J][4], const TwTab& T, int lane) {
  const bool lower = ((lane >> K) & 1) == 0;
  const float2 t = K == 0 ? make_float2(lower ? 1.f : -1.f, 0.f) : T.xs[K][lane];
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    const int q0 = SB == 1 ? pr : 2 * pr, q1 = q0 | (1 << SB);
    float2 mine[J], snd[J], o[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      mine[j] = lower ? v[j][q0] : v[j][q1];
      snd[j] = lower ? v[j][q1] : v[j][q0];
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
      o[j].x = __shfl_xor_sync(0xffffffffu, snd[j].x, 1 << K);
      o[j].y = __shfl_xor_sync(0xffffffffu, snd[j].y, 1 << K);
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
      v[j][q0] = cadd(mine[j], o[j]);
      v[j][q1] = K == 0 ? make_float2(t.x * (mine[j].x - o[j].x), t.x * (mine[j].y - o[j].y))
                        : cmul(csub(mine[j], o[j]), t);
    }
  }
}

template <int J>
__device__ __forceinline__ void warp_fft_dif(float2 (&v)[J][4], const TwTab& T, int lane) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float2 t = T.w[32 * q + lane];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float2 a = v[j][q], b = v[j][q + 2];
      v[j][q] = cadd(a, b);
      v[j][q + 2] = cmul(csub(a, b), t);
    }
  }
  const float2 t1 = T.lane2[lane];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float2 a = v[j][2 * p], b = v[j][2 * p + 1];
      v[j][2 * p] = cadd(a, b);
      v[j][2 * p + 1] = cmul(csub(a, b), t1);
    }
  dif_exchange_stage<J, 4, 1>(v, T, lane);
  dif_exchange_stage<J, 3, 0>(v, T, lane);
  dif_exchange_stage<J, 2, 1>(v, T, lane);
  dif_exchange_stage<J, 1, 0>(v, T, lane);
  dif_exchange_stage<J, 0, 1>(v, T, lane);
}

// The inverse stage of dif_exchange_stage (conjugate twiddle t*, unscaled):
// the butterfly on the lane's own slot pair, (a + b t*, a - b t*), then the
// same exchange of lane bit K with slot bit SB, which undoes itself. With
// the signed twiddle s (= -t on the upper lane) and c = b s*, the lower lane
// holds (a + c, a - c) and the upper (a - c, a + c): every lane keeps a + c,
// sends a - c, and puts the received value in its other slot.
template <int J, int K, int SB>
__device__ __forceinline__ void dit_exchange_stage(float2 (&v)[J][4], const TwTab& T, int lane) {
  const bool lower = ((lane >> K) & 1) == 0;
  const float2 sc = K == 0 ? make_float2(lower ? 1.f : -1.f, 0.f) : conjf2(T.xs[K][lane]);
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    const int q0 = SB == 1 ? pr : 2 * pr, q1 = q0 | (1 << SB);
    float2 keep[J], o[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float2 b = v[j][q1];
      const float2 c = K == 0 ? make_float2(sc.x * b.x, sc.x * b.y) : cmul(b, sc);
      const float2 a = v[j][q0];
      keep[j] = cadd(a, c);
      const float2 snd = csub(a, c);
      o[j].x = __shfl_xor_sync(0xffffffffu, snd.x, 1 << K);
      o[j].y = __shfl_xor_sync(0xffffffffu, snd.y, 1 << K);
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
      v[j][q0] = lower ? keep[j] : o[j];
      v[j][q1] = lower ? o[j] : keep[j];
    }
  }
}

// Inverse (conjugate twiddles), unscaled: input in the layout warp_fft_dif
// leaves (lane l, slot q: frequency 32 q + rev5(l)), output natural
// (lane l, slot q: element 32 q + l).
template <int J>
__device__ __forceinline__ void warp_ifft_dit(float2 (&v)[J][4], const TwTab& T, int lane) {
  dit_exchange_stage<J, 0, 1>(v, T, lane);
  dit_exchange_stage<J, 1, 0>(v, T, lane);
  dit_exchange_stage<J, 2, 1>(v, T, lane);
  dit_exchange_stage<J, 3, 0>(v, T, lane);
  dit_exchange_stage<J, 4, 1>(v, T, lane);
  const float2 t1 = conjf2(T.lane2[lane]);
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float2 a = v[j][2 * p], b = cmul(v[j][2 * p + 1], t1);
      v[j][2 * p] = cadd(a, b);
      v[j][2 * p + 1] = csub(a, b);
    }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float2 t = conjf2(T.w[32 * q + lane]);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float2 a = v[j][q], b = cmul(v[j][q + 2], t);
      v[j][q] = cadd(a, b);
      v[j][q + 2] = csub(a, b);
    }
  }
}

// Position, in a row stored from the registers of warp_fft_dif (slot q of
// lane l at 32 q + l), of frequency m: 32 (m div 32) + rev5(m mod 32).
__device__ __forceinline__ int fpos(int m) { return (m & 96) | rev5(m & 31); }

// Shared-memory slot of position i of such a row: bit 0 flipped by bits 4
// and 5, so that a half-warp's 8-byte accesses in register order (32 q + l)
// and in frequency order (fpos) both fall on 16 distinct bank pairs.
__device__ __forceinline__ int rsw(int i) { return i ^ (((i >> 4) ^ (i >> 5)) & 1); }

// packed row spectrum of a pair (stored as warp_fft_dif leaves it, at r) -> half spectra of the
// even row (r[0..64]) and the odd row (r[kFP .. kFP+64]); one warp
__device__ __forceinline__ void split_pair(float2* r, int lane) {
  float2 e[3], o[3];
  const int ms[3] = {lane, lane + 32, 64};
  const int cnt = lane == 0 ? 3 : 2;
  for (int q = 0; q < cnt; ++q) {
    const int m = ms[q];
    const float2 cm = r[rsw(fpos(m))], cn = conjf2(r[rsw(fpos((128 - m) & 127))]);
    e[q] = make_float2(0.5f * (cm.x + cn.x), 0.5f * (cm.y + cn.y));
    const float2 d = csub(cm, cn);  // (cm - conj(c_-m)) / (2i) = -i d / 2
    o[q] = make_float2(0.5f * d.y, -0.5f * d.x);
  }
  __syncwarp();
  for (int q = 0; q < cnt; ++q) {
    r[ms[q]] = e[q];
    r[kFP + ms[q]] = o[q];
  }
  __syncwarp();
}

// half spectra of a row pair -> packed full spectrum in the input layout of
// warp_ifft_dit (frequency m at rsw(fpos(m))); one warp
__device__ __forceinline__ void merge_pair(float2* r, int lane) {
  float2 d[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = lane + 32 * q;
    float2 e, o;
    if (m <= 64) {
      e = r[m];
      o = r[kFP + m];
    } else {
      e = conjf2(r[128 - m]);
      o = conjf2(r[kFP + 128 - m]);
    }
    d[q] = make_float2(e.x - o.y, e.y + o.x);  // e + i o
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 4; ++q) r[rsw(32 * q + rev5(lane))] = d[q];  // frequency lane + 32 q
  __syncwarp();
}

// The column passes are split between the warps: warp w owns the column
// slots w + 16 c (c < 4). Slot 0 carries two columns: the bins 0 and 64 of
// a row's half spectrum are real (those of a real row), so columns 0 and 64
// travel as one complex column, c0 + i c64, and one FFT serves both (the
// two spectra are separated by Hermitian symmetry, C(k) = A(k) + i B(k)
// with conj(C(-k)) = A(k) - i B(k)); every warp runs four column FFTs. A PSF
// spectrum is stored column by column (column m: 128 rows, contiguous), so
// a warp loads the values of its columns coalesced into registers:
// kr[c][q] = spectrum(row 32 q + lane, column w + 16 c), c < 4, and on warp
// 0 kr[4] = column 64.
constexpr int kWarps = kFThreads / 32;
constexpr int kColsPerWarp = (kFBins + kWarps - 1) / kWarps;  // 5
using SpecRegs = float2[kColsPerWarp][4];

// The spectra A (column 0) and B (column 64) from C = FFT(c0 + i c64) in
// the layout of warp_fft_dif (lane l, slot q: frequency 32 q + rev5(l)).
// The frequency -k of k = 32 q + s sits in slot 3 - q of the lane holding
// 32 - s (s > 0), or in slot (4 - q) mod 4 of lane 0 (s = 0).
__device__ __forceinline__ void split_dc_nyquist(const float2 (&v)[4], float2 (&a)[4],
                                                 float2 (&b)[4], int lane) {
  const int src = rev5((32 - rev5(lane)) & 31);
  float2 p[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    p[q].x = __shfl_sync(0xffffffffu, v[3 - q].x, src);
    p[q].y = __shfl_sync(0xffffffffu, v[3 - q].y, src);
  }
  if (lane == 0) {  // the shuffle brought v[3 - q]; the partner is v[(4 - q) mod 4]
    p[0] = v[0];
    p[1] = v[3];
    p[2] = v[2];
    p[3] = v[1];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    a[q] = make_float2(0.5f * (v[q].x + p[q].x), 0.5f * (v[q].y - p[q].y));
    const float2 d = make_float2(v[q].x - p[q].x, v[q].y + p[q].y);  // C(k) - conj(C(-k))
    b[q] = make_float2(0.5f * d.y, -0.5f * d.x);
  }
}

// c0 + i c64 for complex c0, c64
__device__ __forceinline__ float2 pack_dc_nyquist(float2 c0, float2 c64) {
  return make_float2(c0.x - c64.y, c0.y + c64.x);
}

// Visits (p, q) of a B x B output region, warp w taking the rows w, w + 16,
// ... and its lanes the columns lane, lane + 32, ... (row addresses are
// computed once per row; no division by B per element).
template <class F>
__device__ __forceinline__ void for_region(int B, F&& f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < B; p += kWarps)
    for (int q = lane; q < B; q += 32) f(p, q);
}

__device__ __forceinline__ void load_spec_cols(SpecRegs& kr, const float2* kt) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) {
    const int m = warp + kWarps * c;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      kr[c][q] = m < kFBins ? kt[m * kFT + 32 * q + lane] : make_float2(0.f, 0.f);
  }
}

// forward 2D transform, rows: 64 packed row FFTs and the split, two rows per
// warp at a time (each warp owns row pairs warp + 16 i)
__device__ void r2c_rows(float2* buf, const TwTab& T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < 64; k += 2 * kWarps) {
    float2* r[2] = {buf + 2 * k * kFP, buf + 2 * (k + kWarps) * kFP};
    float2 v[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) v[j][q] = r[j][32 * q + lane];
    warp_fft_dif<2>(v, T, lane);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) r[j][rsw(32 * q + lane)] = v[j][q];
    __syncwarp();
    split_pair(r[0], lane);
    split_pair(r[1], lane);
  }
  __syncthreads();
}

// J column FFTs (columns m[0..J)) of buf in place; with DN, m[0] = 0 is
// the slot of columns 0 and 64 (forward: their real values in, their two
// spectra out; inverse: their Hermitian spectra in, real values out)
template <int J, bool INVERSE, bool DN>
__device__ __forceinline__ void columns_inplace(float2* buf, const int (&m)[J], const TwTab& T,
                                                int lane) {
  float2 v[J][4];
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2* row = buf + (32 * q + lane) * kFP;
      if (DN && j == 0)
        v[j][q] = INVERSE ? pack_dc_nyquist(row[0], row[64]) : make_float2(row[0].x, row[64].x);
      else
        v[j][q] = row[m[j]];
    }
  if (INVERSE)
    warp_ifft_dit<J>(v, T, lane);
  else
    warp_fft_dif<J>(v, T, lane);
  if (DN && !INVERSE) {
    float2 a[4], b[4];
    split_dc_nyquist(v[0], a, b, lane);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[0][q] = a[q];
      buf[(32 * q + lane) * kFP + 64] = b[q];
    }
  }
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2* row = buf + (32 * q + lane) * kFP;
      if (DN && INVERSE && j == 0) {
        row[0] = make_float2(v[0][q].x, 0.f);
        row[64] = make_float2(v[0][q].y, 0.f);
      } else {
        row[m[j]] = v[j][q];
      }
    }
}

// the 65 column FFTs as 64 slots: warp w owns the slots w + 16 c (c < 4),
// two at a time; slot 0 (warp 0) holds columns 0 and 64
template <bool INVERSE>
__device__ __forceinline__ void all_columns(float2* buf, const TwTab& T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
  for (int c = 0; c < 4; c += 2) {
    const int m[2] = {warp + kWarps * c, warp + kWarps * (c + 1)};
    if (warp == 0 && c == 0)
      columns_inplace<2, INVERSE, true>(buf, m, T, lane);
    else
      columns_inplace<2, INVERSE, false>(buf, m, T, lane);
  }
}

// forward real 2D transform in place (see the file comment)
__device__ void r2c_2d(float2* buf, const TwTab& T) {
  r2c_rows(buf, T);
  all_columns<false>(buf, T);
  __syncthreads();
}

// column slots c0, c0 + 1 of this warp (m = warp + 16 c): acc += FFT(buf)
// conj(k^); with DN, slot 0 (columns 0 and 64)
template <bool DN>
__device__ __forceinline__ void columns_accumulate(const float2* buf, float2* acc,
                                                   const SpecRegs& kr, int c0, const TwTab& T,
                                                   int warp, int lane) {
  float2 v[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2* row = buf + (32 * q + lane) * kFP;
      v[j][q] = DN && j == 0 ? make_float2(row[0].x, row[64].x) : row[warp + kWarps * (c0 + j)];
    }
  warp_fft_dif<2>(v, T, lane);
  if (DN) {
    float2 a[4], b[4];
    split_dc_nyquist(v[0], a, b, lane);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[0][q] = a[q];
      float2* o = acc + (32 * q + lane) * kFP + 64;
      *o = cadd(*o, cmulc(b[q], kr[4][q]));
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2* o = acc + (32 * q + lane) * kFP + warp + kWarps * (c0 + j);
      *o = cadd(*o, cmulc(v[j][q], kr[c0 + j][q]));
    }
}

// forward transform of buf (destroyed) added, times conj(spectrum), into acc:
// acc += FFT(buf) conj(k^), the column FFTs never written back
// (no closing barrier: the caller's next barrier orders it)
__device__ void r2c_2d_accumulate(float2* buf, float2* acc, const SpecRegs& kr, const TwTab& T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  r2c_rows(buf, T);
  if (warp == 0)
    columns_accumulate<true>(buf, acc, kr, 0, T, warp, lane);
  else
    columns_accumulate<false>(buf, acc, kr, 0, T, warp, lane);
  columns_accumulate<false>(buf, acc, kr, 2, T, warp, lane);
}

// merge, inverse row FFTs of the J row pairs k[0..J)
template <int J>
__device__ __forceinline__ void rows_inverse(float2* buf, const int (&k)[J], const TwTab& T,
                                             int lane) {
  float2 v[J][4];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    float2* r = buf + 2 * k[j] * kFP;
    merge_pair(r, lane);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[j][q] = r[rsw(32 * q + lane)];
  }
  warp_ifft_dit<J>(v, T, lane);
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) buf[2 * k[j] * kFP + 32 * q + lane] = v[j][q];
}

// inverse transform, rows: merge and the packed row inverse FFTs of the row
// pairs [k0, k1) (the rows a caller reads; the others are left undone), up
// to three at a time per warp (43 pairs: one pass); sync = false leaves the
// closing barrier to the caller
__device__ void c2r_rows(float2* buf, const TwTab& T, int k0 = 0, int k1 = 64, bool sync = true) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = k0 + warp; k < k1; k += 3 * kWarps) {
    if (k + 2 * kWarps < k1) {
      const int kk[3] = {k, k + kWarps, k + 2 * kWarps};
      rows_inverse<3>(buf, kk, T, lane);
    } else if (k + kWarps < k1) {
      const int kk[2] = {k, k + kWarps};
      rows_inverse<2>(buf, kk, T, lane);
    } else {
      const int kk[1] = {k};
      rows_inverse<1>(buf, kk, T, lane);
    }
  }
  if (sync) __syncthreads();
}

// merge and inverse row FFTs of the J row pairs k[0..J), the results handed
// to f(k, column, value) (value: real part row 2k, imaginary part row
// 2k + 1; unscaled) instead of stored
template <int J, class F>
__device__ __forceinline__ void rows_inverse_apply(float2* buf, const int (&k)[J], const TwTab& T,
                                                   int lane, F& f) {
  float2 v[J][4];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    float2* r = buf + 2 * k[j] * kFP;
    merge_pair(r, lane);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[j][q] = r[rsw(32 * q + lane)];
  }
  warp_ifft_dit<J>(v, T, lane);
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) f(k[j], 32 * q + lane, v[j][q]);
}

// c2r_rows with the results handed to f (see rows_inverse_apply); no
// closing barrier
template <class F>
__device__ void c2r_rows_apply(float2* buf, const TwTab& T, int k0, int k1, F& f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = k0 + warp; k < k1; k += 3 * kWarps) {
    if (k + 2 * kWarps < k1) {
      const int kk[3] = {k, k + kWarps, k + 2 * kWarps};
      rows_inverse_apply<3>(buf, kk, T, lane, f);
    } else if (k + kWarps < k1) {
      const int kk[2] = {k, k + kWarps};
      rows_inverse_apply<2>(buf, kk, T, lane, f);
    } else {
      const int kk[1] = {k};
      rows_inverse_apply<1>(buf, kk, T, lane, f);
    }
  }
}

// inverse real 2D transform in place (unscaled); rows of the pairs [k0, k1)
__device__ void c2r_2d(float2* buf, const TwTab& T, int k0 = 0, int k1 = 64) {
  all_columns<true>(buf, T);
  __syncthreads();
  c2r_rows(buf, T, k0, k1);
}

// column slots c0, c0 + 1 of this warp: dst = IFFT(src . k^) along the
// column; with DN, slot 0 (columns 0 and 64, real after the transform)
template <bool DN>
__device__ __forceinline__ void columns_product(const float2* src, float2* dst,
                                                const SpecRegs& kr, int c0, const TwTab& T,
                                                int warp, int lane) {
  float2 v[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2* row = src + (32 * q + lane) * kFP;
      v[j][q] = DN && j == 0
                    ? pack_dc_nyquist(cmul(row[0], kr[0][q]), cmul(row[64], kr[4][q]))
                    : cmul(row[warp + kWarps * (c0 + j)], kr[c0 + j][q]);
    }
  warp_ifft_dit<2>(v, T, lane);
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2* row = dst + (32 * q + lane) * kFP;
      if (DN && j == 0) {
        row[0] = make_float2(v[0][q].x, 0.f);
        row[64] = make_float2(v[0][q].y, 0.f);
      } else {
        row[warp + kWarps * (c0 + j)] = v[j][q];
      }
    }
}

// the column pass of dst = C2R(src . k^): dst's columns = IFFT(src . k^)
// along the column; src is left intact; no closing barrier (the rows,
// c2r_rows_apply, follow the caller's barrier)
__device__ void columns_product_pass(const float2* src, float2* dst, const SpecRegs& kr,
                                     const TwTab& T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0)
    columns_product<true>(src, dst, kr, 0, T, warp, lane);
  else
    columns_product<false>(src, dst, kr, 0, T, warp, lane);
  columns_product<false>(src, dst, kr, 2, T, warp, lane);
}

// values of the tile pixels (P, Q) and (P, Q + 1) after c2r_2d (unscaled),
// Q even: one 16-byte load of the two packed row pairs' entries
__device__ __forceinline__ float2 tile_pair_at(const float2* buf, int P, int Q) {
  const float4 v = *reinterpret_cast<const float4*>(buf + (P >> 1) * 2 * kFP + Q);
  return (P & 1) ? make_float2(v.y, v.w) : make_float2(v.x, v.z);
}

// Visits (p, q) of a B x B output region by column pairs, q = 0, 2, ..., warp
// w taking the rows w, w + 16, ... and its lanes the pairs lane, lane + 32,
// ... (B is even)
template <class F>
__device__ __forceinline__ void for_region_pairs(int B, F&& f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < B; p += kWarps)
    for (int c = lane; c < B / 2; c += 32) f(p, 2 * c);
}

// value of tile pixel (P, Q) after c2r_2d (unscaled)
__device__ __forceinline__ float tile_at(const float2* buf, int P, int Q) {
  const float2 v = buf[(P >> 1) * 2 * kFP + Q];
  return (P & 1) ? v.y : v.x;
}

// asynchronous 4-byte global -> shared copies (no register staging)
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
}
// asynchronous 8-byte global -> shared copy (both addresses 8-byte aligned)
__device__ __forceinline__ void cp_async8(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// start copying the 128 x 128 region with origin (r0, c0) of a padded plane
// into stg (row-major, zero outside the H x W image)
__device__ void region_async(float* stg, const float* plane, const Geom& g, int r0, int c0) {
  // warp w copies the rows w, w + 16, ...; a row's address is formed once
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int P = warp; P < kFT; P += kFThreads / 32) {
    const int i = r0 + P;
    const bool row_in = i >= 0 && i < g.H;
    const float* src = plane + (long long)(g.B + i) * g.P + g.B + c0;
    float* dst = stg + P * kFT;
#pragma unroll
    for (int c = 0; c < kFT / 32; ++c) {
      const int Q = lane + 32 * c, j = c0 + Q;
      if (row_in && j >= 0 && j < g.W)
        cp_async4(dst + Q, src + Q);
      else
        dst[Q] = 0.f;
    }
  }
  cp_async_commit();
}

// start copying the 128 x 128 region with origin (r0, c0) of a padded plane
// straight into the packed row-pair layout of buf (rows 2k and 2k + 1 as the
// real and imaginary parts of buf[2k kFP + j]; zero outside the image);
// complete after cp_async_wait_all and a CTA barrier
__device__ void region_async_packed(float2* buf, const float* plane, const Geom& g, int r0,
                                    int c0) {
  // warp w copies the row pairs w, w + 16, ...; lane 2 c + e takes row
  // 2k + e, column c (+ 16 per step), so a warp writes 32 consecutive words
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* bf = reinterpret_cast<float*>(buf);
  for (int k = warp; k < kFT / 2; k += kWarps) {
    const int P = 2 * k + (lane & 1), i = r0 + P;
    const bool row_in = i >= 0 && i < g.H;
    const float* src = plane + (long long)(g.B + i) * g.P + g.B + c0;
    float* dst = bf + 2 * (2 * k * kFP) + (lane & 1);
#pragma unroll 8
    for (int c = 0; c < kFT / 16; ++c) {
      const int Q = (lane >> 1) + 16 * c, j = c0 + Q;
      if (row_in && j >= 0 && j < g.W)
        cp_async4(dst + 2 * Q, src + Q);
      else
        dst[2 * Q] = 0.f;
    }
  }
  cp_async_commit();
}

// wait for the copies, then pack row pairs of stg into buf
__device__ void pack_region(float2* buf, const float* stg) {
  cp_async_wait_all();
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * kFT; e += blockDim.x) {
    const int k = e >> 7, j = e & (kFT - 1);
    buf[2 * k * kFP + j] = make_float2(stg[2 * k * kFT + j], stg[(2 * k + 1) * kFT + j]);
  }
  __syncthreads();
}

// one block per (exposure, phase): the Kc x Kc phase kernel (row pitch KP;
// for r = 1 the PSF itself) at the top-left of a zero 128 x 128 tile
__global__ void __launch_bounds__(kFThreads, 1)
    fft_spectra_kernel(const float* __restrict__ ka, int Kc, int KP, float2* __restrict__ spec) {
  extern __shared__ float2 fsm[];
  __shared__ TwTab T;
  float2* buf = fsm;
  init_twiddles(T);
  const float* ft = ka + (long long)blockIdx.x * Kc * KP;
  for (int e = threadIdx.x; e < 64 * kFT; e += blockDim.x) {
    const int k = e >> 7, j = e & (kFT - 1);
    const int i = 2 * k;
    const float a = (i < Kc && j < Kc) ? ft[i * KP + j] : 0.f;
    const float b = (i + 1 < Kc && j < Kc) ? ft[(i + 1) * KP + j] : 0.f;
    buf[2 * k * kFP + j] = make_float2(a, b);
  }
  __syncthreads();
  r2c_2d(buf, T);
  // column by column: out[m][row]
  float2* out = spec + (long long)blockIdx.x * kFT * kFBins;
  for (int e = threadIdx.x; e < kFT * kFBins; e += blockDim.x) {
    const int m = e >> 7, rr = e & (kFT - 1);
    out[e] = buf[rr * kFP + m];
  }
}

// column slot m of phase_sum_columns (DN: slot 0, columns 0 and 64)
template <bool DN>
__device__ __forceinline__ void phase_sum_column(const float2* xs, const float2* kt, int R2,
                                                 float2* dst, const TwTab& T, int m, int lane) {
  const int per = kFT * kFBins;
  float2 v[1][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[0][q] = make_float2(0.f, 0.f);
  for (int ph = 0; ph < R2; ++ph) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = ph * per + m * kFT + 32 * q + lane;
      if (DN) {
        const int o64 = o + 64 * kFT;
        v[0][q] = cadd(v[0][q], pack_dc_nyquist(cmul(xs[o], kt[o]), cmul(xs[o64], kt[o64])));
      } else {
        v[0][q] = cadd(v[0][q], cmul(xs[o], kt[o]));
      }
    }
  }
  warp_ifft_dit<1>(v, T, lane);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2* row = dst + (32 * q + lane) * kFP;
    if (DN) {
      row[0] = make_float2(v[0][q].x, 0.f);
      row[64] = make_float2(v[0][q].y, 0.f);
    } else {
      row[m] = v[0][q];
    }
  }
}

// r > 1: the column pass of dst = C2R(sum_phi x^_phi . k^_phi) with both
// spectra read from global memory (x^ from this tile's scratch,
// L2-resident), column by column; no closing barrier (the rows,
// c2r_rows_apply, follow the caller's barrier)
__device__ void phase_sum_columns(const float2* xs, const float2* kt, int R2, float2* dst,
                                  const TwTab& T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = warp; m < 64; m += kWarps) {  // column slots; slot 0: columns 0 and 64
    if (m == 0)
      phase_sum_column<true>(xs, kt, R2, dst, T, m, lane);
    else
      phase_sum_column<false>(xs, kt, R2, dst, T, m, lane);
  }
}

// the forward pass of one tile (tile index `tile` = ty gx + tx of its job)
// for the exposures [t_begin, t_end); starts and ends at a CTA barrier, so
// a persistent CTA can run many. STUDENT = false compiles the Gaussian
// weights only (the split launch, which never runs the heavy-tailed model).
template <bool STUDENT = true>
__device__ void fft_forward_tile(const Shape& s, const FftLaunch& a, int ty, int tx, int tile,
                                 float2* fsm, const TwTab& T, int t_begin, int t_end) {
  float2* xh = fsm;
  float2* wk = fsm + kFBuf;
  float* stg = reinterpret_cast<float*>(fsm + 2 * kFBuf);  // 128 x 128 floats
  const Geom& g = s.g;
  const int hc = s.hc, B = kFT - 2 * hc, R2 = s.R2;
  const int i0 = ty * B, j0 = tx * B;
  const int per = kFT * kFBins;
  // this tile's scratch block (sized for the adjoint's accumulators)
  float2* xs = a.scratch + (long long)tile * (a.nu > 0.f ? 2 * R2 : R2) * per;
  SpecRegs kr;
  if (R2 == 1) {
    load_spec_cols(kr, a.spec + (long long)t_begin * per);
    region_async(stg, a.x, g, i0 - hc, j0 - hc);
    pack_region(xh, stg);
    r2c_2d(xh, T);
  } else {
    // the phases' spectra, column by column, into this tile's scratch
    for (int ph = 0; ph < R2; ++ph) {
      region_async(stg, a.x + (long long)ph * g.plane, g, i0 - hc, j0 - hc);
      pack_region(xh, stg);
      r2c_2d(xh, T);
      for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const int m = e >> 7, rr = e & (kFT - 1);
        xs[ph * per + e] = xh[rr * kFP + m];
      }
      __syncthreads();
    }
  }
  for (int t = t_begin; t < t_end; ++t) {
    // u of this exposure (B x B, row-major in stg) arrives during the
    // inverse transform, by column pairs: the border (2 hc), the pitch (a
    // multiple of 8) and the tile origins (multiples of B) are even, so a
    // pair is 8-byte aligned; the last pair of an edge tile may read column
    // W, inside the padded row (pitch > border + W) and never used
    const long long tplane = (long long)t * g.plane;
    {
      const float* ut = a.u + tplane + (long long)(g.B + i0) * g.P + g.B + j0;
      const int pmax = min(B, g.H - i0), qmax = min(B, g.W - j0);
      for_region_pairs(B, [&](int p, int q) {
        if (p < pmax && q < qmax) cp_async8(stg + p * B + q, ut + (long long)p * g.P + q);
      });
    }
    cp_async_commit();
    if (R2 == 1)
      columns_product_pass(xh, wk, kr, T);
    else
      phase_sum_columns(xs, a.spec + (long long)t * R2 * per, R2, wk, T);
    const int pmax = min(B, g.H - i0), qmax = min(B, g.W - j0);
    const long long base = tplane + (long long)(g.B + i0) * g.P + g.B + j0;
    if (STUDENT && a.nu > 0.f) {
      // heavy-tailed weights u' = u (nu+1) / (nu + u (y - z)^2): both u' z
      // (denominator) and u' y (numerator) go to planes. The rows are stored
      // (pairs [hc, 64): z at rows [2 hc, 128)) and the weights computed
      // after a barrier, by column pairs (the y loads of a fused form stall
      // the row pass)
      __syncthreads();
      c2r_rows(wk, T, hc, 64, false);
      // the next spectrum loads during the epilogue and the next column pass
      if (R2 == 1 && t + 1 < t_end) load_spec_cols(kr, a.spec + (long long)(t + 1) * per);
      cp_async_wait_all();
      __syncthreads();
      const float nu1 = a.nu + 1.f;
      for_region_pairs(B, [&](int p, int q) {
        if (p < pmax && q < qmax) {
          const long long gi = base + (long long)p * g.P + q;
          const bool two = q + 1 < qmax;
          const float2 zz = tile_pair_at(wk, p + 2 * hc, q + 2 * hc);
          const float2 uu = *reinterpret_cast<const float2*>(stg + p * B + q);
          const float2 yy = two ? *reinterpret_cast<const float2*>(a.y + gi)
                                : make_float2(a.y[gi], 0.f);
          float wv[2], w2v[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float z = (e ? zz.y : zz.x) * kFScale, uv = e ? uu.y : uu.x;
            const float yv = e ? yy.y : yy.x, d = yv - z;
            const float us = uv > 0.f ? uv * nu1 / fmaf(uv * d, d, a.nu) : 0.f;
            wv[e] = us * z;
            w2v[e] = us * yv;
          }
          if (two) {
            *reinterpret_cast<float2*>(a.w + gi) = make_float2(wv[0], wv[1]);
            *reinterpret_cast<float2*>(a.w2 + gi) = make_float2(w2v[0], w2v[1]);
          } else {
            a.w[gi] = wv[0];
            a.w2[gi] = w2v[0];
          }
        }
      });
    } else {
      // this warp's columns are done: the next spectrum loads during the rows
      if (R2 == 1 && t + 1 < t_end) load_spec_cols(kr, a.spec + (long long)(t + 1) * per);
      cp_async_wait_all();
      __syncthreads();  // every column done, u landed
      // the inverse rows of the pairs [hc, 64) (z at rows [2 hc, 128)) go
      // straight from registers to the w plane: z(p, q) is row 2k + e - 2 hc,
      // column c - 2 hc of the value (k, c) (e = 0 real part, 1 imaginary)
      float* wt = a.w + base;
      auto out = [&](int k, int c, float2 v) {
        const int q = c - 2 * hc;
        if (q < 0 || q >= qmax) return;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int p = 2 * k + e - 2 * hc;
          if (p < pmax) wt[(long long)p * g.P + q] = stg[p * B + q] * ((e ? v.y : v.x) * kFScale);
        }
      };
      c2r_rows_apply(wk, T, hc, 64, out);
    }
    __syncthreads();  // wk and stg are free for the next exposure
  }
}

__global__ void __launch_bounds__(kFThreads, 1)
    fft_forward_kernel(const Shape s, const FftLaunch a) {
  extern __shared__ float2 fsm[];
  __shared__ TwTab T;
  init_twiddles(T);
  fft_forward_tile(s, a, blockIdx.y, blockIdx.x, blockIdx.y * gridDim.x + blockIdx.x, fsm, T, 0,
                   s.n);
}

// column slot m of r2c_2d_accumulate_phases (DN: slot 0, columns 0 and 64)
template <bool DN>
__device__ __forceinline__ void accumulate_phases_column(const float2* buf, float2* acc,
                                                         const float2* kt, int R2,
                                                         const TwTab& T, int m, int lane) {
  const int per = kFT * kFBins;
  float2 v[1][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2* row = buf + (32 * q + lane) * kFP;
    v[0][q] = DN ? make_float2(row[0].x, row[64].x) : row[m];
  }
  warp_fft_dif<1>(v, T, lane);
  if (DN) {
    float2 a[4], b[4];
    split_dc_nyquist(v[0], a, b, lane);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[0][q] = a[q];
    for (int ph = 0; ph < R2; ++ph) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = ph * per + 64 * kFT + 32 * q + lane;
        acc[o] = cadd(acc[o], cmulc(b[q], kt[o]));
      }
    }
  }
  for (int ph = 0; ph < R2; ++ph) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = ph * per + m * kFT + 32 * q + lane;
      acc[o] = cadd(acc[o], cmulc(v[0][q], kt[o]));
    }
  }
}

// r > 1: acc_phi += FFT(buf) conj(k^_phi) for every phase, accumulators in
// this tile's scratch (column by column, each element one lane's)
__device__ void r2c_2d_accumulate_phases(float2* buf, float2* acc, const float2* kt, int R2,
                                         const TwTab& T) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  r2c_rows(buf, T);
  for (int m = warp; m < 64; m += kWarps) {  // column slots; slot 0: columns 0 and 64
    if (m == 0)
      accumulate_phases_column<true>(buf, acc, kt, R2, T, m, lane);
    else
      accumulate_phases_column<false>(buf, acc, kt, R2, T, m, lane);
  }
  __syncthreads();
}

// Den of one phase (in sh after the inverse transform) -> the update; the
// numerator is a.N, or (Student-t) the transformed tile num
__device__ void update_phase(const float2* sh, const float2* num, const FftLaunch& a,
                             const Geom& g, long long off, int i0, int j0, int B) {
  const long long base = off + (long long)(g.B + i0) * g.P + g.B + j0;
  const int pmax = min(B, g.H - i0), qmax = min(B, g.W - j0);
  for_region(B, [&](int p, int q) {
    if (p < pmax && q < qmax) {
      const long long gi = base + (long long)p * g.P + q;
      const float d = tile_at(sh, p, q) * kFScale;
      const float xo = a.x[gi], nraw = a.N[gi];
      const float nt = num ? tile_at(num, p, q) * kFScale : nraw;
      float xv = xo;
      // The transform leaves a rounding floor (~1e-7 of the tile's weighted
      // model) where the exact denominator is 0; N, from the direct kernel,
      // is exactly 0 when no valid pixel lies in the footprint, which is
      // then the sign of a zero denominator (x unchanged, as for Den = 0);
      // with Student-t weights too, since u' = 0 exactly where u = 0.
      if (d > 0.f && nraw != 0.f) {
        const float nv = fmaxf(nt, 0.f);
        if (d < 1e-30f)  // denominator near zero: guarded ratio in FP64
          xv = (float)((double)xo * (double)nv / (double)d);
        else
          xv = xo * nv / d;
      }
      a.xn[gi] = xv;
    }
  });
}

// Equal ranges: CTA b of P takes the units [b U / P, (b+1) U / P) of U.
__device__ __forceinline__ long long split_start(long long U, int P, int b) {
  return (long long)b * U / P;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
constexpr unsigned kPartPolls = 1u << 23;  // x ~0.3 us per poll: seconds, not a hang

// A tile cut into parts (consecutive exposure ranges) on different CTAs
// of a split launch: part q > 0 waits (bounded) for the tile's flag to
// reach q, starts from the accumulator part q - 1 left in its CTA's slot,
// and, unless it is the last part, leaves its own in this CTA's slot and
// raises the flag to q + 1; the last part finishes the tile and resets the
// flag. The exposures are summed in the order a whole-tile CTA sums them
// (the same bits). A wait that gives up sets the timeout bit of the error
// word and starts from zero.
__device__ void adjoint_publish_part(const FftLaunch& a, int tile, const float2* sh, int q) {
  float2* slot = a.partials + (long long)blockIdx.x * kFBuf;
  for (int e = threadIdx.x; e < kFBuf; e += blockDim.x) slot[e] = sh[e];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) st_release_gpu(a.counters + tile, q + 1);
}

__device__ void adjoint_resume_part(const FftLaunch& a, int tile, float2* sh, int q, int prev_cta,
                                    bool last) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    unsigned i = 0;
    while (i < kPartPolls && ld_acquire_gpu(a.counters + tile) < q) {
      __nanosleep(200);
      ++i;
    }
    ok = i < kPartPolls;
    if (!ok)
      atomicOr(a.err, kErrTimeout);
    else if (last)
      a.counters[tile] = 0;  // ready for the next launch
  }
  __syncthreads();
  const float2* slot = a.partials + (long long)prev_cta * kFBuf;
  for (int e = threadIdx.x; e < kFBuf; e += blockDim.x)
    sh[e] = ok ? __ldcg(slot + e) : make_float2(0.f, 0.f);
}

// the adjoint pass and the update of one tile; starts and ends at a CTA
// barrier. r = 1 Gaussian: one accumulator in shared memory. Otherwise the
// accumulators live in the tile's scratch: R2 for Den, and for Student-t R2
// more for N' (the w2 planes, transformed the same way). A split launch
// (r = 1 Gaussian) runs part q of a cut tile: the sources [k_begin, k_end),
// resumed from CTA prev_cta's part q - 1 (prev_cta < 0: from zero), then
// the update if it is the last part, else published for part q + 1.
__device__ void fft_adjoint_tile(const Shape& s, const FftLaunch& a, int ty, int tx, int tile,
                                 float2* fsm, const TwTab& T, int k_begin = 0, int k_end = -1,
                                 int q = 0, int prev_cta = -1, bool last = true) {
  float2* sh = fsm;
  float2* wk = fsm + kFBuf;
  // the w regions arrive straight in the packed layout, alternating between
  // two work buffers: one is transformed while the next region lands in the other
  float2* wbuf[2] = {fsm + kFBuf, fsm + 2 * kFBuf};
  const Geom& g = s.g;
  const int hc = s.hc, B = kFT - 2 * hc, R2 = s.R2;
  const int i0 = ty * B, j0 = tx * B;
  const int per = kFT * kFBins;
  const bool student = a.nu > 0.f;
  const bool in_smem = R2 == 1 && !student;
  const int nacc = student ? 2 * R2 : R2;
  float2* acc = a.scratch + (long long)tile * nacc * per;
  // sources in order: w_0 (, w2_0), w_1 (, w2_1), ...
  const int nsrc = student ? 2 * s.n : s.n;
  if (k_end < 0) k_end = nsrc;
  auto src_plane = [&](int k) -> const float* {
    return student ? ((k & 1) ? a.w2 : a.w) + (long long)(k >> 1) * g.plane
                   : a.w + (long long)k * g.plane;
  };
  SpecRegs kr;
  if (in_smem) {
    if (prev_cta >= 0)
      adjoint_resume_part(a, tile, sh, q, prev_cta, last);
    else
      for (int e = threadIdx.x; e < kFBuf; e += blockDim.x) sh[e] = make_float2(0.f, 0.f);
    load_spec_cols(kr, a.spec + (long long)k_begin * per);
  } else {
    for (int e = threadIdx.x; e < nacc * per; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
  }
  region_async_packed(wbuf[k_begin & 1], src_plane(k_begin), g, i0 - hc, j0 - hc);
  for (int k = k_begin; k < k_end; ++k) {
    float2* cur = wbuf[k & 1];
    cp_async_wait_all();
    __syncthreads();  // region k landed; every reader of the other buffer is done
    // the next source's region arrives during this transform
    if (k + 1 < k_end)
      region_async_packed(wbuf[(k + 1) & 1], src_plane(k + 1), g, i0 - hc, j0 - hc);
    if (in_smem) {
      r2c_2d_accumulate(cur, sh, kr, T);  // the next loop-top barrier orders it
      if (k + 1 < k_end) load_spec_cols(kr, a.spec + (long long)(k + 1) * per);
    } else {
      const int t = student ? k >> 1 : k, base = student ? (k & 1) * R2 : 0;
      r2c_2d_accumulate_phases(cur, acc + (long long)base * per, a.spec + (long long)t * R2 * per,
                               R2, T);
    }
  }
  if (in_smem) {
    __syncthreads();  // the last accumulation is complete
    if (!last) {
      adjoint_publish_part(a, tile, sh, q);
    } else {
      c2r_2d(sh, T, 0, (B + 1) / 2);  // Den is read at rows [0, B)
      update_phase(sh, nullptr, a, g, 0, i0, j0, B);
    }
  } else {
    for (int ph = 0; ph < R2; ++ph) {
      for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const int m = e >> 7, rr = e & (kFT - 1);
        sh[rr * kFP + m] = acc[ph * per + e];
        if (student) wk[rr * kFP + m] = acc[(R2 + ph) * per + e];
      }
      __syncthreads();
      c2r_2d(sh, T, 0, (B + 1) / 2);
      if (student) c2r_2d(wk, T, 0, (B + 1) / 2);
      update_phase(sh, student ? wk : nullptr, a, g, (long long)ph * g.plane, i0, j0, B);
      __syncthreads();
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kFThreads, 1)
    fft_adjoint_kernel(const Shape s, const FftLaunch a) {
  extern __shared__ float2 fsm[];
  __shared__ TwTab T;
  init_twiddles(T);
  fft_adjoint_tile(s, a, blockIdx.y, blockIdx.x, blockIdx.y * gridDim.x + blockIdx.x, fsm, T);
}

// Split forms (r = 1 Gaussian, at least as many tiles as CTAs): P =
// a.split_ctas persistent CTAs. The Wf = tiles / P whole waves run as one
// CTA per tile would (CTA b takes the tiles b + P i, neighbours side by
// side, so their overlapping regions share the L2); the R = tiles - Wf P
// tiles of the last, partial wave are spread so that no SM idles through it.
// Forward: the R n (tile, exposure) units of the last wave in equal ranges
// over all CTAs (tile-major; a CTA recomputes x^ for each tile it touches).
__global__ void __launch_bounds__(kFThreads, 1)
    fft_forward_split_kernel(const Shape s, const FftLaunch a, int gxt, int tiles) {
  extern __shared__ float2 fsm[];
  __shared__ TwTab T;
  init_twiddles(T);
  const int P = a.split_ctas, n = s.n, b = blockIdx.x;
  const int Wf = tiles / P, R = tiles - Wf * P;
  for (int i = 0; i < Wf; ++i) {
    const int tile = b + P * i;
    fft_forward_tile<false>(s, a, tile / gxt, tile % gxt, tile, fsm, T, 0, n);
  }
  const long long U = (long long)R * n, base = (long long)Wf * P * n;
  const long long u_end = split_start(U, P, b + 1);
  for (long long u = split_start(U, P, b); u < u_end;) {
    const int tile = (int)((base + u) / n), t0 = (int)((base + u) % n);
    const int t1 = (int)min((long long)n, t0 + (u_end - u));
    fft_forward_tile<false>(s, a, tile / gxt, tile % gxt, tile, fsm, T, t0, t1);
    u += t1 - t0;
  }
}

// Adjoint: last-wave tile j is cut into k = min(n, P / R) parts of
// consecutive exposures, part q on CTA q R + j, which runs it after
// q Wf / (k - 1) of its whole tiles (part 0 first, part k - 1 last), so
// each part finds its predecessor done waves earlier and the last wave
// costs 1 / k of a tile.
__global__ void __launch_bounds__(kFThreads, 1)
    fft_adjoint_split_kernel(const Shape s, const FftLaunch a, int gxt, int tiles) {
  extern __shared__ float2 fsm[];
  __shared__ TwTab T;
  init_twiddles(T);
  const int P = a.split_ctas, n = s.n, b = blockIdx.x;
  const int Wf = tiles / P, R = tiles - Wf * P;
  const int k = R > 0 ? max(1, min(n, P / R)) : 0;
  const int has = b < k * R, q = has ? b / R : 0, j = has ? b % R : 0;
  const int pos = !has ? -1 : (k == 1 ? Wf : q * Wf / (k - 1));  // whole tiles before the part
  for (int it = 0; it < Wf + has; ++it) {
    int tile, k0 = 0, k1 = n, qq = 0, prev = -1;
    bool last = true;
    if (has && it == pos) {
      tile = Wf * P + j, k0 = q * n / k, k1 = (q + 1) * n / k, qq = q;
      prev = q > 0 ? (q - 1) * R + j : -1, last = q == k - 1;
    } else {
      tile = b + P * (it - (has && it > pos));
    }
    fft_adjoint_tile(s, a, tile / gxt, tile % gxt, tile, fsm, T, k0, k1, qq, prev, last);
  }
}

// Persistent forms for a batch of FFT jobs: every CTA claims (job, tile)
// items from a device counter until the list is exhausted; jobs whose
// iterations are done are skipped. One launch for the forward passes of all
// jobs, then one for the adjoints (the adjoint reads its neighbours' w).
__device__ __forceinline__ int claim_item(int* counter, int* slot) {
  __syncthreads();  // the previous item's readers of *slot are done
  if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
  __syncthreads();
  return *slot;
}

__global__ void __launch_bounds__(kFThreads, 1)
    fft_batch_forward_kernel(const FftBatchJob* __restrict__ jobs, const int2* __restrict__ items,
                             const int* __restrict__ n_items, int* __restrict__ counter) {
  extern __shared__ float2 fsm[];
  __shared__ TwTab T;
  __shared__ int slot;
  init_twiddles(T);
  const int total = *n_items;
  for (;;) {
    const int item = claim_item(counter, &slot);
    if (item >= total) break;
    const int2 w = items[item];
    const FftBatchJob& J = jobs[w.x];
    if (J.remaining <= 0) continue;
    fft_forward_tile(J.s, J.a[J.cur], w.y / J.gxt, w.y % J.gxt, w.y, fsm, T, 0, J.s.n);
  }
}

__global__ void __launch_bounds__(kFThreads, 1)
    fft_batch_adjoint_kernel(const FftBatchJob* __restrict__ jobs, const int2* __restrict__ items,
                             const int* __restrict__ n_items, int* __restrict__ counter) {
  extern __shared__ float2 fsm[];
  __shared__ TwTab T;
  __shared__ int slot;
  init_twiddles(T);
  const int total = *n_items;
  for (;;) {
    const int item = claim_item(counter, &slot);
    if (item >= total) break;
    const int2 w = items[item];
    const FftBatchJob& J = jobs[w.x];
    if (J.remaining <= 0) continue;
    fft_adjoint_tile(J.s, J.a[J.cur], w.y / J.gxt, w.y % J.gxt, w.y, fsm, T);
  }
}

__global__ void fft_batch_advance_kernel(FftBatchJob* __restrict__ jobs, int njobs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < njobs && jobs[j].remaining > 0) {
    jobs[j].remaining -= 1;
    jobs[j].cur ^= 1;
  }
}

}  // namespace

static size_t fft_tiles(const Shape& s) {
  const int B = kFT - 2 * s.hc;
  return (size_t)((s.g.W + B - 1) / B) * ((s.g.H + B - 1) / B);
}

// layout of the FFT buffer: PSF spectra (n R2), w planes (n), for Student-t
// the w2 planes (n), then the per-tile scratch (r > 1: tiles R2 spectra;
// Student-t: tiles 2 R2)
size_t fft_w2_offset(const Shape& s) {
  const size_t spec = ((size_t)s.n * s.R2 * kFT * kFBins * sizeof(float2) + 255) & ~(size_t)255;
  const size_t wpl = ((size_t)s.n * s.g.plane * sizeof(float) + 255) & ~(size_t)255;
  return spec + wpl;
}

size_t fft_scratch_offset(const Shape& s, bool student) {
  const size_t wpl = ((size_t)s.n * s.g.plane * sizeof(float) + 255) & ~(size_t)255;
  return fft_w2_offset(s) + (student ? wpl : 0);
}

size_t fft_split_offset(const Shape& s, bool student) {
  const int nacc = student ? 2 * s.R2 : (s.R2 > 1 ? s.R2 : 0);
  const size_t scratch = fft_tiles(s) * nacc * kFT * kFBins * sizeof(float2);
  return (fft_scratch_offset(s, student) + scratch + 255) & ~(size_t)255;
}

static bool fft_splits_adjoint(const Shape& s, bool student) { return s.R2 == 1 && !student; }

size_t fft_counters_offset(const Shape& s, bool student, int split_ctas) {
  const size_t parts = fft_splits_adjoint(s, student) && split_ctas > 0
                           ? (size_t)split_ctas * kFBuf * sizeof(float2)
                           : 0;
  return fft_split_offset(s, student) + parts;
}

size_t fft_buffer_bytes(const Shape& s, bool student, int split_ctas) {
  const size_t counters =
      fft_splits_adjoint(s, student) && split_ctas > 0 ? fft_tiles(s) * sizeof(int) : 0;
  return fft_counters_offset(s, student, split_ctas) + counters;
}

// two transform buffers and a 128 x 128 float staging area
// three transform buffers (the adjoint: accumulator and two work buffers;
// the forward: x^, work buffer and a 128 x 128 float staging area)
size_t fft_smem_bytes() { return 3 * (size_t)kFBuf * sizeof(float2); }

int fft_tile_side(const Shape& s) { return kFT - 2 * s.hc; }

cudaError_t launch_fft_spectra(const Shape& s, const float* ka, float2* spec, cudaStream_t st) {
  const size_t smem = (size_t)kFBuf * sizeof(float2);
  cudaError_t e = allow_max_dynamic_smem((const void*)fft_spectra_kernel);
  if (e != cudaSuccess) return e;
  fft_spectra_kernel<<<s.n * s.R2, kFThreads, smem, st>>>(ka, s.Kc, s.KP, spec);
  return cudaGetLastError();
}

int fft_tiles_x(const Shape& s) {
  const int B = kFT - 2 * s.hc;
  return (s.g.W + B - 1) / B;
}

int fft_tiles_total(const Shape& s) { return (int)fft_tiles(s); }

cudaError_t launch_fft_batch(const FftBatchJob* jobs, int njobs, const int2* items,
                             const int* n_items, int* counters, int ctas, cudaStream_t st) {
  const size_t smem = fft_smem_bytes();
  cudaError_t e = allow_max_dynamic_smem((const void*)fft_batch_forward_kernel);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)fft_batch_adjoint_kernel);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  fft_batch_forward_kernel<<<ctas, kFThreads, smem, st>>>(jobs, items, n_items, counters);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  fft_batch_adjoint_kernel<<<ctas, kFThreads, smem, st>>>(jobs, items, n_items, counters + 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  fft_batch_advance_kernel<<<(njobs + 127) / 128, 128, 0, st>>>(const_cast<FftBatchJob*>(jobs),
                                                                njobs);
  return cudaGetLastError();
}

cudaError_t launch_fft_iter(const Shape& s, const FftLaunch& a, cudaStream_t st) {
  const size_t smem = fft_smem_bytes();
  cudaError_t e = allow_max_dynamic_smem((const void*)fft_forward_kernel);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)fft_adjoint_kernel);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)fft_forward_split_kernel);
  if (e == cudaSuccess) e = allow_max_dynamic_smem((const void*)fft_adjoint_split_kernel);
  if (e != cudaSuccess) return e;
  const int B = fft_tile_side(s);
  const dim3 grid((s.g.W + B - 1) / B, (s.g.H + B - 1) / B);
  // the split forms: r = 1 (the forward pass of r > 1 keeps x^ in the
  // tile's scratch), Gaussian (the partial slots), at least as many tiles
  // as CTAs
  const bool split = s.R2 == 1 && a.nu <= 0.f && a.split_ctas > 0 && a.partials &&
                     a.counters && a.err && (long long)fft_tiles(s) >= a.split_ctas;
  if (split)
    fft_forward_split_kernel<<<a.split_ctas, kFThreads, smem, st>>>(s, a, (int)grid.x,
                                                                     (int)fft_tiles(s));
  else
    fft_forward_kernel<<<grid, kFThreads, smem, st>>>(s, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (split)
    fft_adjoint_split_kernel<<<a.split_ctas, kFThreads, smem, st>>>(s, a, (int)grid.x,
                                                                     (int)fft_tiles(s));
  else
    fft_adjoint_kernel<<<grid, kFThreads, smem, st>>>(s, a);
  return cudaGetLastError();
}

}  // namespace emd
