// emd_halo.cu -- the FP32 direct EM iteration of Sec. 2, Eq. (2) (Eq. (3)
// for r > 1) as one persistent kernel over two kinds of work items:
//
//   forward item (t, tile)   w_t = u_t . (F_t x) on the 64 x 128 tile,
//                            stored in one slot of a ring of tile buffers
//   adjoint item (t, tile)   Den += F_t^T w_t on the tile, reading w_t of the
//                            tile and of its 8 neighbours from the ring; the
//                            last exposure applies the update of Eq. (2)
//
// Every forward pixel is computed once. The CTA-pair kernel of
// emd_direct.cu keeps w in shared memory instead and so recomputes a 2*hc
// halo around each tile (176^2 forward outputs per 128^2 tile at K = 43:
// 1.48x the algorithmic FMAs overall against 1.0x here). What this costs is
// w passing through global memory: a ring of R tile buffers (about 1030 at
// 4096^2, 34 MB), written and read again within a few hundred items, so it
// stays in L2; no per-exposure image is kept.
//
// Tiles are TH rows x 128 columns, one per CTA of 128 threads (an RY x 16
// block of outputs per thread, TH = 16 RY), several CTAs per SM: when one
// waits at a barrier or on its staging loads, the others keep the FMA pipes
// busy. Three tile shapes are built (TileCfg below) and the library's
// autotuner picks one per problem shape: 64-row tiles (4 x 16 outputs per
// thread, two CTAs per SM), 48-row tiles (3 x 16, at most 168 registers, three
// CTAs per SM) and 32-row tiles (2 x 16, four CTAs per SM where the shared
// memory allows). All give the same iterates bit for bit: every output's
// taps are summed in the same order whatever block it falls in.
//
// Item order. One atomic counter hands out a fixed sequence: the first L
// forward items, then adjoint and forward items alternately, then the last
// L adjoint items (adjoint item a is claimed just before forward item
// a + L). Ids count exposure-major: id = e * T + tile, e = t - t0. Waits:
//   adjoint (e, k) needs the forward items (e, k') of its 3 x 3 neighbours
//     (id distance <= dmax < L, so claimed earlier) and adjoint (e-1, k)
//     (Den is read-modify-written in exposure order);
//   forward f reuses ring slot f mod R, written last by forward f - R; it
//     needs the adjoint items that read that tile done, ids <= f - R + dmax,
//     claimed earlier because R > L + dmax.
// A CTA only ever waits on an item claimed before its own, held by a running
// CTA, so the kernel completes with any number of co-resident CTAs. Each
// wait is bounded; one that gives up raises an abort flag that ends every
// later wait at once, and the host sees EMD_ETIMEOUT through the error word.
//
// The arithmetic (tap order of each output, w = u z, Den + sum, the guarded
// ratio) is the CTA-pair kernel's, so both give bit-identical iterates.
#include "emd_corr.cuh"
#include "emd_halo.cuh"

namespace emd {

namespace {

constexpr int kHT = 128;   // threads per CTA: 16 thread rows x 8 thread columns
constexpr uint32_t kPollLimit = 1u << 23;  // x ~0.3 us per poll: seconds, not a hang
constexpr int kGather = 8;             // 16-byte loads in flight per thread while staging

// Tile shapes: TH rows (16 thread rows of RY outputs) x 128 columns (8 thread
// columns of 16 outputs), MINB CTAs per SM requested from the compiler (which
// caps registers at 65536 / (128 MINB)). CTAS caps the grid (>= MINB x the
// SMs of one GB300) and, with it, the claim lag and the ring.
template <int CFG> struct TileCfg;
template <> struct TileCfg<0> { static constexpr int TH = 64, RY = 4, MINB = 2, CTAS = 320; };
template <> struct TileCfg<1> { static constexpr int TH = 48, RY = 3, MINB = 3, CTAS = 480; };
template <> struct TileCfg<2> { static constexpr int TH = 32, RY = 2, MINB = 4, CTAS = 640; };

__host__ __device__ constexpr int cfg_rows(int cfg) { return cfg == 0 ? 64 : cfg == 1 ? 48 : 32; }
constexpr int cfg_ctas(int cfg) { return cfg == 0 ? 320 : cfg == 1 ? 480 : 640; }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct HaloShape {
  int rows;   // staged rows: TH + 2 hc
  int cols;   // staged columns: kTile + KP
  int pitch;  // floats per staged row; rows also carry a skew of 4 floats every 4 rows
  int buf;    // floats of the staged window
  int ks;     // floats of one Kc x KP kernel
};

__host__ __device__ inline HaloShape halo_shape(const Shape& s, int TH) {
  HaloShape h;
  h.rows = TH + 2 * s.hc;
  h.cols = kTile + s.KP;
  h.pitch = h.cols;  // a multiple of 4: rows start 16-byte aligned; even: the
                     // 8 lanes of a load phase (rows 4 apart) hit distinct bank groups
  h.buf = h.rows * h.pitch + 4 * ((h.rows + 3) >> 2);
  h.ks = s.Kc * s.KP;
  return h;
}

size_t halo_smem_bytes(const Shape& s, int TH) {
  const HaloShape h = halo_shape(s, TH);
  return (size_t)(h.buf + h.ks) * sizeof(float);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait for *p >= v. Gives up after `limit` polls (raising the
// abort flag ctrl[2]) or at once when another CTA has already given up.
__device__ bool wait_geq(const int* p, int v, unsigned long long* ctrl,
                         uint32_t limit = kPollLimit) {
  const volatile unsigned long long* abort_flag = ctrl + 2;
  for (uint32_t i = 0; i < limit; ++i) {
    if (ld_acquire(p) >= v) return true;
    if (*abort_flag) return false;
    __nanosleep(200);
  }
  atomicExch(ctrl + 2, 1ull);
  return false;
}

// Writes the four floats of v into the staged row at columns C .. C+3,
// skipping columns outside [0, cols).
__device__ __forceinline__ void put4(float* row, int C, int cols, const float4 v) {
  if (C >= 0 && C + 3 < cols) {
    row[C] = v.x;
    row[C + 1] = v.y;
    row[C + 2] = v.z;
    row[C + 3] = v.w;
  } else {
    if (C >= 0 && C < cols) row[C] = v.x;
    if (C + 1 >= 0 && C + 1 < cols) row[C + 1] = v.y;
    if (C + 2 >= 0 && C + 2 < cols) row[C + 2] = v.z;
    if (C + 3 >= 0 && C + 3 < cols) row[C + 3] = v.w;
  }
}

// Forward item: the x window of rows [i0 - hc, i0 + TH + hc) and columns
// [j0 - hc, j0 - hc + cols) of one padded latent plane (read-only during
// the launch), through 16-byte loads on the plane's 16-byte grid.
__device__ void gather_plane(const Shape& s, const HaloShape& hs, const SPlane& sp,
                             const float* __restrict__ plane, int i0, int j0) {
  const int c0 = j0 + s.hc;  // padded column of window column 0 (border B = 2 hc)
  const int q0 = c0 >> 2;
  const int nq = ((c0 + hs.cols - 1) >> 2) - q0 + 1;
  const int total = hs.rows * nq;
  const float* base = plane + (long long)(i0 + s.hc) * s.g.P;
  for (int e0 = threadIdx.x; e0 < total; e0 += kHT * kGather) {
    float4 v[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      const int e = e0 + q * kHT;
      if (e < total) {
        const int R = e / nq, m = e - R * nq;
        v[q] = __ldg(reinterpret_cast<const float4*>(base + (long long)R * s.g.P + ((q0 + m) << 2)));
      }
    }
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      const int e = e0 + q * kHT;
      if (e < total) {
        const int R = e / nq, m = e - R * nq;
        put4(srow(sp, R), ((q0 + m) << 2) - c0, hs.cols, v[q]);
      }
    }
  }
}

// Adjoint item: the w window of rows [i0 - hc, i0 + TH + hc) and columns
// [j0 - hc, j0 - hc + cols) from the ring slots of the tile and its
// neighbours (nb[3 * (dy + 1) + (dx + 1)], null outside the tile grid: w = 0
// there), `off` floats into each slot. Tile column origins are multiples of
// 128, so the 16-byte image-column grid is each slot's own. Loads bypass L1
// (the slots are rewritten by other SMs during the launch).
template <int TH>
__device__ void gather_ring(const HaloShape& hs, const SPlane& sp, const float* const* nb,
                            int off, int hc, int i0, int j0) {
  const int c0 = j0 - hc;   // image column of window column 0
  const int q0 = c0 >> 2;   // floor
  const int nq = ((c0 + hs.cols - 1) >> 2) - q0 + 1;
  const int total = hs.rows * nq;
  const int ti = i0 / TH, tj = j0 >> 7;
  for (int e0 = threadIdx.x; e0 < total; e0 += kHT * kGather) {
    float4 v[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      const int e = e0 + q * kHT;
      v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < total) {
        const int R = e / nq, m = e - R * nq;
        const int ii = i0 - hc + R, cc = (q0 + m) << 2;
        const int tr = ii >= 0 ? ii / TH : -1, tc = cc >> 7;  // floor: neighbour tile row / column
        const float* src = nb[3 * (tr - ti + 1) + (tc - tj + 1)];
        if (src)
          v[q] = __ldcg(reinterpret_cast<const float4*>(src + off + (ii - tr * TH) * kTile +
                                                         (cc - (tc << 7))));
      }
    }
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      const int e = e0 + q * kHT;
      if (e < total) {
        const int R = e / nq, m = e - R * nq;
        put4(srow(sp, R), ((q0 + m) << 2) - c0, hs.cols, v[q]);
      }
    }
  }
}

// Position sq of the claim sequence -> (forward?, item id).
__device__ __forceinline__ bool decode_item(long long sq, long long NT, long long L,
                                            long long* id) {
  if (sq < L) {
    *id = sq;
    return true;
  }
  if (sq < 2 * NT - L) {
    const long long j = sq - L;
    *id = (j & 1) ? L + (j >> 1) : (j >> 1);
    return (j & 1) != 0;
  }
  *id = sq - NT;
  return false;
}

__device__ __forceinline__ void prefetch_l2(const float* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One warp: L2 prefetch of rows [r0, r0 + nrows), floats [c0, c0 + ncols) of
// a padded plane (rows start 32-byte aligned; each row's range is widened to
// the 16-byte grid the bulk prefetch wants).
__device__ void prefetch_rect(const float* plane, int P, int r0, int nrows, int c0, int ncols,
                              int lane) {
  const int a0 = c0 & ~3;
  const uint32_t bytes = (uint32_t)(((c0 + ncols - a0 + 3) & ~3) * sizeof(float));
  for (int R = lane; R < nrows; R += 32) prefetch_l2(plane + (long long)(r0 + R) * P + a0, bytes);
}

// One warp, at the start of the item before it: brings into L2 what item sq
// reads from DRAM (u, x and Den are each touched once per exposure, so they
// are not in L2 any more): a forward item's x window and u tile, an adjoint
// item's Den tile (and x and N for the update of the last exposure).
template <int TH>
__device__ void prefetch_item(const Shape& s, const FusedArgs& a, const HaloShape& hs,
                              const HaloPlan& pl, long long sq, int lane) {
  long long id;
  const bool fwd = decode_item(sq, pl.NT, pl.L, &id);
  const int e = (int)(id / pl.T), k = (int)(id - (long long)e * pl.T);
  const int i0 = (k / s.gx) * TH, j0 = (k % s.gx) * kTile;
  const Geom& g = s.g;
  const int t = a.t0 + e, ne = a.t1 - a.t0;
  if (fwd) {
    for (int phi = 0; phi < s.R2; ++phi)
      prefetch_rect(a.x + (long long)phi * g.plane, g.P, i0 + s.hc, hs.rows, j0 + s.hc, hs.cols,
                    lane);
    prefetch_rect(a.u + (long long)t * g.plane, g.P, g.B + i0, TH, g.B + j0, kTile, lane);
    if (a.nu > 0.f)
      prefetch_rect(a.y + (long long)t * g.plane, g.P, g.B + i0, TH, g.B + j0, kTile, lane);
  } else {
    for (int phi = 0; phi < s.R2; ++phi) {
      const long long pb = (long long)phi * g.plane;
      if (e > 0) prefetch_rect(a.Den + pb, g.P, g.B + i0, TH, g.B + j0, kTile, lane);
      if (e > 0 && a.nu > 0.f)
        prefetch_rect(a.Nw + pb, g.P, g.B + i0, TH, g.B + j0, kTile, lane);
      if (e + 1 == ne) {
        prefetch_rect(a.x + pb, g.P, g.B + i0, TH, g.B + j0, kTile, lane);
        prefetch_rect(a.N + pb, g.P, g.B + i0, TH, g.B + j0, kTile, lane);
      }
    }
  }
}

// STUDENT: heavy-tailed weights u' = u (nu+1) / (nu + u (y - z)^2); each
// forward item then stores two tiles per slot, w = u' z and w2 = u' y, and
// each adjoint item correlates both: Den and the numerator N' (a.Nw) of the
// generalised EM step, in one launch per iteration.
//
// One work item: position sq of a job's claim sequence, run by the whole
// CTA. claim_next() is called once, after the item's window is staged (the
// caller takes its next claim there and prefetches for it). nb_s: 9 shared
// pointers. A wait that gives up sets timed_out.
template <int CFG, bool STUDENT, class ClaimNext>
__device__ __forceinline__ void halo_item(const Shape& s, const HaloLaunch& h, const HaloPlan& pl,
                                          long long sq, float* smem, const float** nb_s,
                                          bool& timed_out, ClaimNext&& claim_next) {
  constexpr int TH = TileCfg<CFG>::TH, RY = TileCfg<CFG>::RY;
  constexpr int kTileFloats = TH * kTile;
  const FusedArgs& a = h.a;
  const Geom& g = s.g;
  const HaloShape hs = halo_shape(s, TH);
  const SPlane sp{smem, hs.pitch, 2};
  float* ks = smem + hs.buf;
  const int tid = threadIdx.x;
  const int my = tid & 15, mx = tid >> 4;  // this thread's RY x 16 outputs: rows RY my, cols 16 mx
  const int T = pl.T;
  const long long NT = pl.NT, L = pl.L, RS = pl.R;
  const int ne = a.t1 - a.t0;
  const int kq = hs.ks >> 2;
  constexpr long long kSlot = STUDENT ? 2LL * kTileFloats : kTileFloats;  // floats per ring slot
  long long id;
  const bool fwd = decode_item(sq, NT, L, &id);
  const int e = (int)(id / T), k = (int)(id - (long long)e * T);
  const int ti = k / s.gx, tj = k - ti * s.gx;
  const int i0 = ti * TH, j0 = tj * kTile;
  const int t = a.t0 + e;
  bool ok = true;
  float acc[RY][16];
#pragma unroll
  for (int p = 0; p < RY; ++p)
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[p][c] = 0.f;

  // Both kinds of item run one loop of steps, each staging a window and a
  // kernel and correlating them at ONE call site: the two CTAs of an SM may
  // be in different kinds of item, and one copy of the unrolled loop keeps
  // both in the instruction cache. Forward: R2 steps (the phases of x,
  // accumulated into z); adjoint: passes x R2 steps, each summed from zero
  // and then added into its running sum (pass 0: Den from w; heavy-tailed
  // pass 1: N' from w2 = u' y).
  const long long slot = fwd ? id % RS : 0;
  // Forward: the slot's previous tile (forward id - R) must have been read by
  // its adjoint readers before this item's w is stored: probe their counters
  // now (relaxed), settle after staging (a fence, or a bounded wait).
  const int* probe = nullptr;
  int need = 0, seen = 0;
  if (fwd) {
    if (id >= RS && tid < 9) {
      const long long prev = id - RS;
      const int pe = (int)(prev / T), pk = (int)(prev - (long long)pe * T);
      const int nti = pk / s.gx + tid / 3 - 1, ntj = pk % s.gx + tid % 3 - 1;
      if (nti >= 0 && nti < pl.T / s.gx && ntj >= 0 && ntj < s.gx) {
        probe = h.adone + nti * s.gx + ntj;
        need = pe + 1;
        seen = ld_relaxed(probe);
      }
    }
  } else {
    // adjoint: the forward items of the 3 x 3 neighbours, and adjoint (e - 1, k)
    if (tid < 9) {
      const int nti = ti + tid / 3 - 1, ntj = tj + tid % 3 - 1;
      const float* src = nullptr;
      if (nti >= 0 && nti < pl.T / s.gx && ntj >= 0 && ntj < s.gx) {
        const long long fid = (long long)e * T + nti * s.gx + ntj;
        const long long fslot = fid % RS;
        ok = wait_geq(h.fflag + fslot, (int)(fid + 1), h.ctrl);
        src = h.ring + fslot * kSlot;
      }
      nb_s[tid] = src;
    } else if (tid == 9 && e > 0) {
      ok = wait_geq(h.adone + k, e, h.ctrl);  // adjoint (e - 1, k) has written Den
    }
    __syncthreads();
  }
  const int nsteps = fwd ? s.R2 : (STUDENT ? 2 : 1) * s.R2;
  for (int step = 0; step < nsteps; ++step) {
    const int pass = step / s.R2, phi = step - pass * s.R2;
    if (step > 0) __syncthreads();  // readers of the previous step's window and kernel are done
    if (fwd) {
      gather_plane(s, hs, sp, a.x + (long long)phi * g.plane, i0, j0);
    } else {
      if (phi == 0) gather_ring<TH>(hs, sp, nb_s, pass * kTileFloats, s.hc, i0, j0);
      if (step > 0) {
#pragma unroll
        for (int p = 0; p < RY; ++p)
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[p][c] = 0.f;
      }
    }
    const float4* kg = reinterpret_cast<const float4*>((fwd ? a.kf : a.ka) +
                                                       ((long long)t * s.R2 + phi) * hs.ks);
    for (int q = tid; q < kq; q += kHT) reinterpret_cast<float4*>(ks)[q] = kg[q];
    if (step == 0) {
      claim_next();
      if (probe) {
        if (seen >= need)
          __threadfence();  // acquire: the readers' loads precede our stores
        else
          ok = wait_geq(probe, need, h.ctrl);
      }
    }
    __syncthreads();  // also orders the slot check above before the stores below
    corr_tile<RY, 16>(acc, sp, RY * my, 16 * mx, ks, s.KP, s.Kc);
    if (fwd) continue;
    // ---------------- adjoint epilogue: running sum, or the update ----------------
    float* run = pass == 0 ? a.Den : a.Nw;  // running sum over the exposures
    const long long pbase = (long long)phi * g.plane;
#pragma unroll
    for (int p = 0; p < RY; ++p) {
      const int i = i0 + RY * my + p;
      const long long grow = pbase + (long long)(g.B + i) * g.P + g.B + j0 + 16 * mx;
      float2* run2 = reinterpret_cast<float2*>(run + grow);
      if (e > 0) {
#pragma unroll
        for (int c2 = 0; c2 < 8; ++c2) {
          const float2 dv = __ldcg(run2 + c2);
          acc[p][2 * c2] = dv.x + acc[p][2 * c2];
          acc[p][2 * c2 + 1] = dv.y + acc[p][2 * c2 + 1];
        }
      }
      // not the last exposure; or the heavy-tailed Den, kept for pass 1
      // (read back below by the thread that wrote it)
      if (e + 1 < ne || (STUDENT && pass == 0)) {
#pragma unroll
        for (int c2 = 0; c2 < 8; ++c2)
          run2[c2] = make_float2(acc[p][2 * c2], acc[p][2 * c2 + 1]);
        continue;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int j = j0 + 16 * mx + c;
        if (i < g.H && j < g.W) {
          const float d = STUDENT ? __ldcg(a.Den + grow + c) : acc[p][c];
          const float xo = a.x[grow + c];
          float xv = xo;
          if (d > 0.f) {
            const float nv = fmaxf(STUDENT ? acc[p][c] : a.N[grow + c], 0.f);
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
  if (fwd) {
    // ---------------- forward epilogue: w_t = u_t . z into the ring slot ----------------
    float* wt = h.ring + slot * kSlot;
    const float* up = a.u + (long long)t * g.plane;
#pragma unroll
    for (int p = 0; p < RY; ++p) {
      // B and P are even: each row of the tile starts 8-byte aligned
      const long long grow = (long long)(g.B + i0 + RY * my + p) * g.P + g.B + j0 + 16 * mx;
      const float2* u2 = reinterpret_cast<const float2*>(up + grow);
      float4* dst = reinterpret_cast<float4*>(wt + (RY * my + p) * kTile + 16 * mx);
      if (STUDENT) {
        const float2* y2 = reinterpret_cast<const float2*>(a.y + (long long)t * g.plane + grow);
        float4* dst2 = reinterpret_cast<float4*>(wt + kTileFloats + (RY * my + p) * kTile + 16 * mx);
        const float nu1 = a.nu + 1.f;
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          const float2 ua = __ldg(u2 + 2 * c4), ub = __ldg(u2 + 2 * c4 + 1);
          const float2 ya = __ldg(y2 + 2 * c4), yb = __ldg(y2 + 2 * c4 + 1);
          const float uv[4] = {ua.x, ua.y, ub.x, ub.y}, yv[4] = {ya.x, ya.y, yb.x, yb.y};
          float w[4], w2[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float z = acc[p][4 * c4 + q];
            const float d = yv[q] - z;
            const float us = uv[q] > 0.f ? uv[q] * nu1 / fmaf(uv[q] * d, d, a.nu) : 0.f;
            w[q] = us * z;
            w2[q] = us * yv[q];
          }
          dst[c4] = make_float4(w[0], w[1], w[2], w[3]);
          dst2[c4] = make_float4(w2[0], w2[1], w2[2], w2[3]);
        }
      } else {
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          const float2 ua = __ldg(u2 + 2 * c4), ub = __ldg(u2 + 2 * c4 + 1);
          float4 w;
          w.x = ua.x * acc[p][4 * c4 + 0];
          w.y = ua.y * acc[p][4 * c4 + 1];
          w.z = ub.x * acc[p][4 * c4 + 2];
          w.w = ub.y * acc[p][4 * c4 + 3];
          dst[c4] = w;
        }
      }
    }
    if (__syncthreads_or(!ok)) timed_out = true;  // every w store of the CTA is issued
    if (tid == 0) {
      __threadfence();
      st_release(h.fflag + slot, (int)(id + 1));
    }
  } else {
    if (__syncthreads_or(!ok)) timed_out = true;  // all reads of the ring and Den are done
    if (tid == 0) {
      __threadfence();
      st_release(h.adone + k, e + 1);
    }
  }
}

// One launch per EM iteration of one context (exposures [a.t0, a.t1)).
template <int CFG, bool STUDENT>
__global__ void __launch_bounds__(kHT, TileCfg<CFG>::MINB)
    halo_kernel(const Shape s, const HaloLaunch h, const HaloPlan pl) {
  extern __shared__ __align__(128) float smem[];
  __shared__ long long item_s;
  __shared__ const float* nb_s[9];
  __shared__ int last_s;
  const HaloShape hs = halo_shape(s, TileCfg<CFG>::TH);
  const int tid = threadIdx.x;
  const long long total = 2 * pl.NT;
  bool timed_out = false;

  // Each CTA claims one item ahead: warp 0 takes the next position and
  // prefetches its data into L2 while the CTA works on the current one. (A
  // CTA then holds two claims; the one it has not started is later than the
  // one it is running, so every wait still ends: the earliest unfinished
  // claim is always running and waits only on finished ones.)
  if (tid == 0) item_s = (long long)atomicAdd(&h.ctrl[0], 1ull);
  __syncthreads();
  long long sq = item_s;
  while (sq < total) {
    __syncthreads();  // every thread has read item_s
    // the next claim is taken now and used after this item's window is staged,
    // so the atomic's round trip overlaps the staging loads
    unsigned long long nx_raw = 0;
    if (tid == 0) nx_raw = atomicAdd(&h.ctrl[0], 1ull);
    auto claim_next = [&]() {
      if (tid < 32) {
        const long long nx = (long long)__shfl_sync(0xffffffffu, nx_raw, 0);
        if (tid == 0) item_s = nx;
        if (nx < total) prefetch_item<TileCfg<CFG>::TH>(s, h.a, hs, pl, nx, tid);
      }
    };
    halo_item<CFG, STUDENT>(s, h, pl, sq, smem, nb_s, timed_out, claim_next);
    __syncthreads();  // readers of this item's window and kernel are done; item_s is set
    sq = item_s;
  }

  // The last CTA to finish resets the flags and counters for the next launch
  // (stream order makes the reset visible to it).
  __syncthreads();
  if (tid == 0) {
    if (timed_out) atomicOr(h.a.err, kErrTimeout);
    __threadfence();
    last_s = atomicAdd(&h.ctrl[1], 1ull) == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (last_s) {
    __threadfence();
    for (long long i = tid; i < pl.R; i += kHT) h.fflag[i] = 0;
    for (int i = tid; i < pl.T; i += kHT) h.adone[i] = 0;
    if (tid == 0) {
      h.ctrl[0] = 0ull;
      h.ctrl[1] = 0ull;
      h.ctrl[2] = 0ull;
    }
  }
}

// A batch step: the claim sequences of several contexts (one EM iteration
// each), merged into one work list of (job, position) entries that keeps
// each job's own order, so every wait is still on an earlier entry. Each
// job has its own ring, flags and abort flag; the list's claim counter and
// the finished-CTA count are the batch's. The last CTA resets the flags of
// every job that ran.
template <int CFG>
__global__ void __launch_bounds__(kHT, TileCfg<CFG>::MINB)
    halo_batch_kernel(const HaloBatchJob* __restrict__ jobs, int njobs,
                      const int2* __restrict__ items, const int* __restrict__ n_items,
                      unsigned long long* ctrl, int* err) {
  extern __shared__ __align__(128) float smem[];
  __shared__ long long item_s;
  __shared__ const float* nb_s[9];
  __shared__ int last_s;
  const int tid = threadIdx.x;
  const long long total = *n_items;
  bool timed_out = false;
  if (tid == 0) item_s = (long long)atomicAdd(&ctrl[0], 1ull);
  __syncthreads();
  long long q = item_s;
  while (q < total) {
    __syncthreads();  // every thread has read item_s
    unsigned long long nx_raw = 0;
    if (tid == 0) nx_raw = atomicAdd(&ctrl[0], 1ull);
    const int2 it = items[q];
    const HaloBatchJob& J = jobs[it.x];
    const Shape s = J.s;
    const HaloLaunch h = J.h[J.cur];
    const HaloPlan pl = J.pl;
    auto claim_next = [&]() {
      if (tid < 32) {
        const long long nx = (long long)__shfl_sync(0xffffffffu, nx_raw, 0);
        if (tid == 0) item_s = nx;
        if (nx < total) {
          const int2 nit = items[nx];
          const HaloBatchJob& NJ = jobs[nit.x];
          prefetch_item<TileCfg<CFG>::TH>(NJ.s, NJ.h[NJ.cur].a, halo_shape(NJ.s, TileCfg<CFG>::TH),
                                          NJ.pl, nit.y, tid);
        }
      }
    };
    if (J.remaining > 0) halo_item<CFG, false>(s, h, pl, it.y, smem, nb_s, timed_out, claim_next);
    else claim_next();
    __syncthreads();
    q = item_s;
  }
  __syncthreads();
  if (tid == 0) {
    if (timed_out) atomicOr(err, kErrTimeout);
    __threadfence();
    last_s = atomicAdd(&ctrl[1], 1ull) == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (last_s) {
    __threadfence();
    for (int j = 0; j < njobs; ++j) {
      const HaloBatchJob& J = jobs[j];
      if (J.remaining <= 0) continue;
      const HaloLaunch& h = J.h[0];  // ring, flags and counters are shared by h[0], h[1]
      for (long long i = tid; i < J.pl.R; i += kHT) h.fflag[i] = 0;
      for (int i = tid; i < J.pl.T; i += kHT) h.adone[i] = 0;
      if (tid == 0) h.ctrl[2] = 0ull;
    }
    if (tid == 0) {
      ctrl[0] = 0ull;
      ctrl[1] = 0ull;
    }
  }
}

// The data term of the log-likelihood (Eq. (1); the Student-t term with
// STUDENT): sum over valid pixels of u (y - z)^2, z = F_t x, in FP64 -- the
// forward model alone, each pixel once. Items (tile, group of exposures)
// are taken in a fixed stride by a persistent grid and each writes its own
// partial sum, so the total (a fixed-order sum of the partials) does not
// depend on scheduling. For r = 1 the x window is staged once per item.
template <bool STUDENT>
__global__ void __launch_bounds__(kHT, 2)
    halo_chi2_kernel(const Shape s, const FusedArgs a, const int groups,
                     double* __restrict__ part) {
  constexpr int kTH = TileCfg<0>::TH;  // 64-row tiles, 4 x 16 outputs per thread
  extern __shared__ __align__(128) float smem[];
  __shared__ double red[kHT / 32];
  const Geom& g = s.g;
  const HaloShape hs = halo_shape(s, kTH);
  const SPlane sp{smem, hs.pitch, 2};
  float* ks = smem + hs.buf;
  const int tid = threadIdx.x;
  const int my = tid & 15, mx = tid >> 4;
  const int kq = hs.ks >> 2;
  const int nitems = s.gx * ((s.H + kTH - 1) / kTH) * groups;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int k = item / groups, grp = item - k * groups;
    const int ti = k / s.gx, tj = k - ti * s.gx;
    const int i0 = ti * kTH, j0 = tj * kTile;
    const int t0 = (int)((long long)s.n * grp / groups);
    const int t1 = (int)((long long)s.n * (grp + 1) / groups);
    double chi = 0.0;
    for (int t = t0; t < t1; ++t) {
      float acc[4][16];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[p][c] = 0.f;
      for (int phi = 0; phi < s.R2; ++phi) {
        __syncthreads();  // readers of the previous window and kernel are done
        if (s.R2 > 1 || t == t0) gather_plane(s, hs, sp, a.x + (long long)phi * g.plane, i0, j0);
        const float4* kg =
            reinterpret_cast<const float4*>(a.kf + ((long long)t * s.R2 + phi) * hs.ks);
        for (int q = tid; q < kq; q += kHT) reinterpret_cast<float4*>(ks)[q] = kg[q];
        if (tid < 32 && phi == 0 && t + 1 < t1) {  // the next exposure's u and y into L2
          prefetch_rect(a.u + (long long)(t + 1) * g.plane, g.P, g.B + i0, kTH, g.B + j0,
                        kTile, tid);
          prefetch_rect(a.y + (long long)(t + 1) * g.plane, g.P, g.B + i0, kTH, g.B + j0,
                        kTile, tid);
        }
        __syncthreads();
        corr_tile<4, 16>(acc, sp, 4 * my, 16 * mx, ks, s.KP, s.Kc);
      }
      const long long tp = (long long)t * g.plane;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int i = i0 + 4 * my + p;
        const long long grow = tp + (long long)(g.B + i) * g.P + g.B + j0 + 16 * mx;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = j0 + 16 * mx + c;
          const float uv = a.u[grow + c];
          if (i < g.H && j < g.W && uv != 0.f) {
            const double d = (double)a.y[grow + c] - (double)acc[p][c];
            if (STUDENT)
              chi += ((double)a.nu + 1.0) * log1p((double)uv * d * d / (double)a.nu);
            else
              chi += (double)uv * d * d;
          }
        }
      }
    }
    const double tot = block_sum_f64(chi, red);
    if (tid == 0) part[item] = tot;
  }
}

// Self-test of the flag waits (no fault, no hang): the first wait is for a
// counter nothing increments and must give up after `limit` polls, raising
// the abort flag; the second, with the kernel's own poll limit, must then
// return at once. Only if both behave is the timeout recorded in *err.
__global__ void flag_wait_selftest_kernel(uint32_t limit, int* flags, unsigned long long* ctrl,
                                          int* err) {
  if (threadIdx.x != 0) return;
  const bool first = wait_geq(flags, 1, ctrl, limit);
  const bool second = wait_geq(flags + 1, 1, ctrl);
  if (!first && !second && *reinterpret_cast<volatile unsigned long long*>(ctrl + 2) != 0ull)
    atomicOr(err, kErrTimeout);
}

}  // namespace

cudaError_t launch_flag_wait_selftest(uint32_t limit, void* scratch, int* err, cudaStream_t st) {
  // scratch: 64 zeroed bytes: two counters, then the three control words
  int* flags = static_cast<int*>(scratch);
  unsigned long long* ctrl = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + 8);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 64, st);
  if (e != cudaSuccess) return e;
  flag_wait_selftest_kernel<<<1, 32, 0, st>>>(limit, flags, ctrl, err);
  return cudaGetLastError();
}

HaloPlan halo_plan(const Shape& s, int ne, int cfg) {
  HaloPlan p;
  p.cfg = cfg;
  p.TH = cfg_rows(cfg);
  const int gyh = (s.H + p.TH - 1) / p.TH;
  p.T = s.gx * gyh;
  p.dmax = (gyh > 1 ? s.gx : 0) + (s.gx > 1 ? 1 : 0);
  p.NT = (long long)ne * p.T;
  const int cap = cfg_ctas(cfg);
  p.L = p.dmax + 2LL * cap;
  if (p.L > p.NT) p.L = p.NT;
  p.R = p.L + p.dmax + 1 + cap;
  if (p.R > p.NT) p.R = p.NT;
  return p;
}

namespace {
// The buffer of one context, shared by every tile shape: the control words,
// the slot flags and tile counters (each shape uses a prefix of them; all are
// zero between launches, so the shape may change from one launch to the
// next), then the ring.
struct HaloBufLayout {
  size_t flags, adone, ring, total;
  long long Rmax;
  int Tmax;
};

HaloBufLayout halo_layout(const Shape& s, bool student) {
  HaloBufLayout b{};
  size_t ring = 0;
  for (int cfg = 0; cfg < kHaloTileConfigs; ++cfg) {
    const HaloPlan p = halo_plan(s, s.n, cfg);
    if (p.R > b.Rmax) b.Rmax = p.R;
    if (p.T > b.Tmax) b.Tmax = p.T;
    const size_t slot = (student ? 2 : 1) * (size_t)p.TH * kTile * sizeof(float);
    if ((size_t)p.R * slot > ring) ring = (size_t)p.R * slot;
  }
  b.flags = 256;
  b.adone = b.flags + align256((size_t)b.Rmax * sizeof(int));
  b.ring = b.adone + align256((size_t)b.Tmax * sizeof(int));
  b.total = b.ring + align256(ring);
  return b;
}
}  // namespace

size_t halo_buffer_bytes(const Shape& s, bool student) {
  // 32-bit item ids for every tile shape
  for (int cfg = 0; cfg < kHaloTileConfigs; ++cfg) {
    const HaloPlan p = halo_plan(s, s.n, cfg);
    if (2 * p.NT + 2LL * cfg_ctas(cfg) >= (1LL << 31)) return 0;
  }
  return halo_layout(s, student).total;
}

void halo_bind(const Shape& s, bool student, void* buf, HaloLaunch* h) {
  const HaloBufLayout b = halo_layout(s, student);
  char* base = static_cast<char*>(buf);
  h->ctrl = reinterpret_cast<unsigned long long*>(base);
  h->fflag = reinterpret_cast<int*>(base + b.flags);
  h->adone = reinterpret_cast<int*>(base + b.adone);
  h->ring = reinterpret_cast<float*>(base + b.ring);
}

namespace {

template <class Kern>
cudaError_t resident_ctas(Kern kern, size_t smem, int cap, int* out) {
  cudaError_t e = allow_max_dynamic_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kHT, smem)) != cudaSuccess)
    return e;
  long long grid = (long long)sms * (occ > 0 ? occ : 1);
  if (grid > cap) grid = cap;
  *out = (int)grid;
  return cudaSuccess;
}

template <int CFG, bool STUDENT>
cudaError_t launch_halo_t(const Shape& s, const HaloLaunch& h, const HaloPlan& pl,
                          cudaStream_t st) {
  const size_t smem = halo_smem_bytes(s, TileCfg<CFG>::TH);
  int grid = 0;
  cudaError_t e = resident_ctas(halo_kernel<CFG, STUDENT>, smem, TileCfg<CFG>::CTAS, &grid);
  if (e != cudaSuccess) return e;
  if (grid > 2 * pl.NT) grid = (int)(2 * pl.NT);
  halo_kernel<CFG, STUDENT><<<grid, kHT, smem, st>>>(s, h, pl);
  return cudaGetLastError();
}

// dynamic shared memory of the batch kernels: the largest accepted footprint
size_t halo_batch_smem_bytes(int TH) {
  size_t m = 0;
  for (int hc = 0; hc <= EMD_MAX_HC; ++hc) {
    Shape s{};
    s.hc = hc;
    s.Kc = 2 * hc + 1;
    s.KP = (s.Kc + 3) / 4 * 4;
    const size_t b = halo_smem_bytes(s, TH);
    if (b > m) m = b;
  }
  return m;
}

__global__ void halo_batch_advance_kernel(HaloBatchJob* __restrict__ jobs, int njobs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < njobs && jobs[j].remaining > 0) {
    jobs[j].remaining -= 1;
    jobs[j].cur ^= 1;
  }
}

template <int CFG>
int halo_batch_ctas_t() {
  int grid = 0;
  if (resident_ctas(halo_batch_kernel<CFG>, halo_batch_smem_bytes(TileCfg<CFG>::TH),
                    TileCfg<CFG>::CTAS, &grid) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return grid;
}

template <int CFG>
cudaError_t launch_halo_batch_t(const HaloBatchJob* jobs, int njobs, const int2* items,
                                const int* n_items, unsigned long long* ctrl, int* err, int ctas,
                                cudaStream_t st) {
  const size_t smem = halo_batch_smem_bytes(TileCfg<CFG>::TH);
  cudaError_t e = allow_max_dynamic_smem((const void*)halo_batch_kernel<CFG>);
  if (e != cudaSuccess) return e;
  if (ctas > TileCfg<CFG>::CTAS) ctas = TileCfg<CFG>::CTAS;
  halo_batch_kernel<CFG><<<ctas, kHT, smem, st>>>(jobs, njobs, items, n_items, ctrl, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  halo_batch_advance_kernel<<<(njobs + 127) / 128, 128, 0, st>>>(const_cast<HaloBatchJob*>(jobs),
                                                                 njobs);
  return cudaGetLastError();
}

}  // namespace

int halo_batch_ctas(int cfg) {
  switch (cfg) {
    case 0: return halo_batch_ctas_t<0>();
    case 1: return halo_batch_ctas_t<1>();
    case 2: return halo_batch_ctas_t<2>();
  }
  return 0;
}

cudaError_t launch_halo_batch(int cfg, const HaloBatchJob* jobs, int njobs, const int2* items,
                              const int* n_items, unsigned long long* ctrl, int* err, int ctas,
                              cudaStream_t st) {
  switch (cfg) {
    case 0: return launch_halo_batch_t<0>(jobs, njobs, items, n_items, ctrl, err, ctas, st);
    case 1: return launch_halo_batch_t<1>(jobs, njobs, items, n_items, ctrl, err, ctas, st);
    case 2: return launch_halo_batch_t<2>(jobs, njobs, items, n_items, ctrl, err, ctas, st);
  }
  return cudaErrorInvalidValue;
}

int halo_tile_ctas_per_sm(const Shape& s, int cfg) {
  int occ = 0;
  const size_t smem = halo_smem_bytes(s, cfg_rows(cfg));
  cudaError_t e = cudaErrorInvalidValue;
  switch (cfg) {
    case 0:
      e = allow_max_dynamic_smem((const void*)halo_kernel<0, false>);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, halo_kernel<0, false>, kHT, smem);
      break;
    case 1:
      e = allow_max_dynamic_smem((const void*)halo_kernel<1, false>);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, halo_kernel<1, false>, kHT, smem);
      break;
    case 2:
      e = allow_max_dynamic_smem((const void*)halo_kernel<2, false>);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, halo_kernel<2, false>, kHT, smem);
      break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

int launch_halo_chi2(const Shape& s, const FusedArgs& a, double* part, int max_parts,
                     cudaStream_t st, cudaError_t* err) {
  constexpr int kTH = TileCfg<0>::TH;
  const int T = s.gx * ((s.H + kTH - 1) / kTH);
  int groups = max_parts / T;
  if (groups > s.n) groups = s.n;
  if (groups < 1) {
    *err = cudaErrorInvalidValue;
    return 0;
  }
  const size_t smem = halo_smem_bytes(s, kTH);
  auto kern = a.nu > 0.f ? halo_chi2_kernel<true> : halo_chi2_kernel<false>;
  int grid = 0;
  cudaError_t e = resident_ctas(kern, smem, 1 << 30, &grid);
  if (e != cudaSuccess) {
    *err = e;
    return 0;
  }
  if (grid > T * groups) grid = T * groups;
  kern<<<grid, kHT, smem, st>>>(s, a, groups, part);
  *err = cudaGetLastError();
  return T * groups;
}

cudaError_t launch_halo_iter(const Shape& s, const HaloLaunch& h, int cfg, cudaStream_t st) {
  const int ne = h.a.t1 - h.a.t0;
  if (ne <= 0 || ne > s.n || cfg < 0 || cfg >= kHaloTileConfigs) return cudaErrorInvalidValue;
  const HaloPlan pl = halo_plan(s, ne, cfg);
  const bool st_ = h.a.nu > 0.f;
  switch (cfg) {
    case 0: return st_ ? launch_halo_t<0, true>(s, h, pl, st) : launch_halo_t<0, false>(s, h, pl, st);
    case 1: return st_ ? launch_halo_t<1, true>(s, h, pl, st) : launch_halo_t<1, false>(s, h, pl, st);
    default: return st_ ? launch_halo_t<2, true>(s, h, pl, st) : launch_halo_t<2, false>(s, h, pl, st);
  }
}

}  // namespace emd
