// emd_halo.cuh -- the halo-exchange form of the FP32 direct EM iteration
// (declarations; the kernel is in emd_halo.cu).
#pragma once

#include "emd_internal.cuh"

namespace emd {

// Tile shapes of the kernel (all 128 columns wide, 128 threads per CTA):
//   0: 64 rows, 4 x 16 outputs per thread, two CTAs per SM
//   1: 48 rows, 3 x 16 outputs per thread, three CTAs per SM
//   2: 32 rows, 2 x 16 outputs per thread, four CTAs per SM (shared memory
//      permitting)
// Every shape gives the same iterates bit for bit.
constexpr int kHaloTileConfigs = 3;
// CTAs of the shape's (Gaussian) kernel resident per SM for this problem (0 on error)
int halo_tile_ctas_per_sm(const Shape& s, int cfg);

// Work plan of one launch over the exposures [t0, t1) with tile shape cfg:
// ne = t1 - t0, T = gx * ceil(H / TH) tiles, NT = ne * T forward items and NT
// adjoint items.
struct HaloPlan {
  int cfg;        // tile shape
  int TH;         // tile rows
  int T;          // tiles per exposure
  int dmax;       // largest item-index distance between neighbouring tiles
  long long NT;   // forward (= adjoint) items
  long long L;    // adjoint items trail forward items by L
  long long R;    // w ring slots (tile-sized)
};

HaloPlan halo_plan(const Shape& s, int ne, int cfg);
// device bytes of the ring, its flags and the work counters for up to n
// exposures per launch and any tile shape (0 when the shape is too large for
// 32-bit item ids); student: two tiles per slot (w = u' z and w2 = u' y)
size_t halo_buffer_bytes(const Shape& s, bool student);

struct HaloLaunch {
  FusedArgs a;                 // x, xn, u, kf, ka, N, Den, err, t0, t1; heavy-tailed
                               // (a.nu > 0): also y, and a.Nw holds the running N'
  float* ring;                 // R slots of TH x 128 floats (two tiles if heavy-tailed)
  int* fflag;                  // R: forward item id + 1 last published in each slot
  int* adone;                  // T: adjoint items finished per tile in this launch
  unsigned long long* ctrl;    // [0] claim counter, [1] CTAs finished, [2] abort flag
};

// carves the control words, flags, counters and the ring out of a zeroed
// buffer of halo_buffer_bytes(s, student) bytes (the same layout for every
// tile shape: the flags and counters are zero between launches)
void halo_bind(const Shape& s, bool student, void* buf, HaloLaunch* h);
// one EM iteration of the exposures [a.t0, a.t1) with tile shape cfg: a.x ->
// a.xn, Den scratch in a.Den; the Gaussian update of Eq. (2) with numerator
// a.N, or (a.nu > 0) the heavy-tailed step with N' accumulated in a.Nw
cudaError_t launch_halo_iter(const Shape& s, const HaloLaunch& h, int cfg, cudaStream_t st);
// one job of a batch step (device table entry): h[c] has x = buffer c and
// xn = buffer c^1 of the job's context; ring, flags and counters are the
// context's own, sized for n exposures
struct HaloBatchJob {
  Shape s;
  HaloLaunch h[2];
  HaloPlan pl;     // halo_plan(s, s.n, cfg) for the step's tile shape
  int cur;         // current x buffer
  int remaining;   // iterations still to run (0: skipped)
};
// CTAs of the persistent batch kernel of tile shape cfg that fit the device
// (its shared memory sized for any accepted PSF; 0 on error)
int halo_batch_ctas(int cfg);
// a batch step over items (job, position in the job's claim sequence), every
// job planned for tile shape cfg: persistent kernel, then the advance kernel
// of the jobs; on st, graph-capturable (ctrl: 2 words, zero before the first
// launch, left zero)
cudaError_t launch_halo_batch(int cfg, const HaloBatchJob* jobs, int njobs, const int2* items,
                              const int* n_items, unsigned long long* ctrl, int* err, int ctas,
                              cudaStream_t st);

// The log-likelihood's data term (mode 2 of the fused kernel) with each
// forward pixel computed once: partial sums into part[0 .. returned count),
// to be added in index order (at most max_parts; needs max_parts >= gx*gy).
int launch_halo_chi2(const Shape& s, const FusedArgs& a, double* part, int max_parts,
                     cudaStream_t st, cudaError_t* err);

// one thread waits on a counter nothing increments (bounded by `limit`
// polls), then once more after its abort flag is up; records the timeout in
// *err only if both waits gave up. scratch: 64 bytes of device memory.
cudaError_t launch_flag_wait_selftest(uint32_t limit, void* scratch, int* err, cudaStream_t st);

}  // namespace emd
