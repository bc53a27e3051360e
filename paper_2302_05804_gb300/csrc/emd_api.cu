// emd_api.cu -- the C ABI of include/emd.h: context life cycle, argument
// validation, host/device marshalling and the launch sequence of the EM
// iteration (Sec. 2, Eq. (2)). All device memory of a context is one
// allocation carved into the buffers described in emd_internal.cuh.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "emd_internal.cuh"
#include "emd_tc.cuh"
#include "emd_fft.cuh"
#include "emd_halo.cuh"

using emd::Shape;

namespace {

thread_local std::string g_err;

void set_err(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Layout {
  size_t x0, x1, N, Den, u, y, kf, ka, fraw, part, sums, err, total;
};

Layout make_layout(const Shape& s) {
  Layout L{};
  const size_t lat = (size_t)s.R2 * s.g.plane * sizeof(float);
  const size_t exp = (size_t)s.n * s.g.plane * sizeof(float);
  const size_t ker = (size_t)s.n * s.R2 * s.Kc * s.KP * sizeof(float);
  size_t parts = (size_t)emd::kRedBlocks * 4;
  if ((size_t)emd::fused_blocks(s) > parts) parts = emd::fused_blocks(s);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
  L.x0 = take(lat);
  L.x1 = take(lat);
  L.N = take(lat);
  L.Den = take(lat);
  L.u = take(exp);
  L.y = take(exp);
  L.kf = take(ker);
  L.ka = take(ker);
  L.fraw = take((size_t)s.n * s.K * s.K * sizeof(float));
  L.part = take(parts * sizeof(double));
  L.sums = take(8 * sizeof(double));
  L.err = take(sizeof(int));
  L.total = off;
  return L;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace emd {
void set_error_message(const char* msg) { g_err = msg; }
}  // namespace emd

struct emd_ctx {
  Shape s;
  Layout L;
  int device = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t handoff = nullptr;  // orders work across emd_set_stream
  char* arena = nullptr;
  float* x[2] = {nullptr, nullptr};
  int cur = 0;
  float *N = nullptr, *Den = nullptr, *u = nullptr, *y = nullptr;
  float *kf = nullptr, *ka = nullptr, *fraw = nullptr;
  double *part = nullptr, *sums = nullptr;
  int* err = nullptr;
  double logdet = 0.0, suy = 0.0, su = 0.0, nvalid = 0.0;
  // noise model: Gaussian (Eq. (1)) or Student-t with nu degrees of freedom
  int noise = EMD_NOISE_GAUSSIAN;
  double nu = 0.0;
  float* Ns = nullptr;  // heavy-tailed numerator (latent planes), allocated on first use
  // FFT path (allocated when EMD_PREC_FFT_FP32 is first selected)
  char* fft_arena = nullptr;
  size_t fft_bytes = 0;
  float2* fft_spec = nullptr;
  float* fft_w = nullptr;
  float* fft_w2 = nullptr;
  float2* fft_scratch = nullptr;
  float2* fft_partials = nullptr;  // split launch (r = 1 Gaussian): partial accumulators
  int* fft_counters = nullptr;     // and per-tile flags
  size_t fft_counters_bytes = 0;
  int fft_split_ctas = 0;          // persistent CTAs of the split launch (one per SM)
  int fft_bound = -1;              // noise model the pointers are laid out for (-1: none)
  bool fft_ready = false;
  bool frames = false;
  int prec = EMD_PREC_FP32;
  // tensor-core path (allocated when a tensor-core mode is first selected)
  emd::TcShape ts{};
  char* tc_arena = nullptr;
  size_t tc_bytes = 0;
  uint16_t* xb = nullptr;
  uint16_t* hank = nullptr;
  CUtensorMap xmap;
  CUtensorMap wmap;
  uint16_t* wb = nullptr;  // 16-bit w planes of the tensor-core form
  bool hank_ready = false;
  float* scales = nullptr;       // device {z, w, Den, x} operand scales
  unsigned int* xmax = nullptr;  // device max of x (FP16 modes)
  float gscale = 1.f, umax = 0.f, fsum = 0.f;
  // streaming EM: per-exposure numerators (allocated on first use)
  float* Nt = nullptr;
  bool nt_ready = false;
  // halo-exchange form of the FP32 direct iteration: w ring, flags and
  // counters (allocated on the first FP32 direct iteration; zeroed)
  char* halo_arena = nullptr;
  size_t halo_bytes = 0;
  bool halo_student = false;  // slots hold two tiles (heavy-tailed weights)
  emd::HaloLaunch halo{};
  // its tile shape: fixed by emd_set_tile_shape (-1: autotuned), and the
  // autotuner's trials on this context (candidates in launch order, events
  // around each launch)
  int tile_forced = -1;
  int tile_last = 0;
  std::vector<int> trial_cfg;
  std::vector<cudaEvent_t> trial_ev;
  size_t trials_issued = 0;
  bool trial_student = false;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_err("%s failed: %s", #call, cudaGetErrorString(e_));                     \
      return EMD_ECUDA;                                                            \
    }                                                                              \
  } while (0)

int check_ctx(emd_ctx* c, bool need_frames) {
  if (!c) {
    set_err("null context");
    return EMD_EINVAL;
  }
  if (need_frames && !c->frames) {
    set_err("no frames loaded (call emd_set_frames first)");
    return EMD_ESTATE;
  }
  return EMD_OK;
}

// read the device error word (synchronises the stream) and clear it
int check_device_error(emd_ctx* c) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (h) CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  if (h & emd::kErrTimeout) {
    // a split FFT launch whose wait gave up may have left tile flags raised:
    // clear them so that the next launch starts from a clean state
    if (c->fft_counters) CK(cudaMemsetAsync(c->fft_counters, 0, c->fft_counters_bytes, c->st));
    set_err("a bounded device-side wait gave up");
    return EMD_ETIMEOUT;
  }
  return EMD_OK;
}

emd::FusedArgs fused_args(emd_ctx* c) {
  emd::FusedArgs a{};
  a.x = c->x[c->cur];
  a.xn = c->x[c->cur ^ 1];
  a.u = c->u;
  a.y = c->y;
  a.kf = c->kf;
  a.ka = c->ka;
  a.N = c->N;
  a.Nw = c->N;
  a.Den = c->Den;
  a.err = c->err;
  a.t0 = 0;
  a.t1 = c->s.n;
  a.nu = c->noise == EMD_NOISE_STUDENT_T ? (float)c->nu : 0.f;
  return a;
}

// copy an (n x H x W) natural array into n padded planes
int put_planes(emd_ctx* c, float* planes, const float* src, int count) {
  const emd::Geom& g = c->s.g;
  for (int t = 0; t < count; ++t) {
    CK(cudaMemcpy2DAsync(planes + (size_t)t * g.plane + (size_t)g.B * g.P + g.B,
                         (size_t)g.P * sizeof(float), src + (size_t)t * g.H * g.W,
                         (size_t)g.W * sizeof(float), (size_t)g.W * sizeof(float), g.H,
                         cudaMemcpyDefault, c->st));
  }
  return EMD_OK;
}

int get_planes(emd_ctx* c, float* dst, const float* planes, int count) {
  const emd::Geom& g = c->s.g;
  for (int t = 0; t < count; ++t) {
    CK(cudaMemcpy2DAsync(dst + (size_t)t * g.H * g.W, (size_t)g.W * sizeof(float),
                         planes + (size_t)t * g.plane + (size_t)g.B * g.P + g.B,
                         (size_t)g.P * sizeof(float), (size_t)g.W * sizeof(float), g.H,
                         cudaMemcpyDefault, c->st));
  }
  return EMD_OK;
}

// latent planes -> natural (rH x rW) at out (host or device)
int latent_out(emd_ctx* c, const float* planes, float* out) {
  if (!out) {
    set_err("null output pointer");
    return EMD_EINVAL;
  }
  const size_t nat = (size_t)c->s.R2 * c->s.H * c->s.W;
  if (c->s.r == 1) {
    int rc = get_planes(c, out, planes, 1);
    if (rc) return rc;
  } else if (is_device_ptr(out)) {
    CK(emd::launch_gather_latent(c->s, planes, out, c->st));
  } else {
    // the Den scratch holds the natural image on its way to the host
    CK(emd::launch_gather_latent(c->s, planes, c->Den, c->st));
    CK(cudaMemcpyAsync(out, c->Den, nat * sizeof(float), cudaMemcpyDeviceToHost, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  return EMD_OK;
}

}  // namespace

extern "C" {

const char* emd_last_error(void) { return g_err.c_str(); }

size_t emd_ctx_bytes(int H, int W, int n, int psf_k, int r) {
  Shape s;
  const char* why = nullptr;
  if (!emd::make_shape(H, W, n, psf_k, r, &s, &why)) return 0;
  return make_layout(s).total;
}

namespace {

// SMs of the current device, 0 if there is none
int current_device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

}  // namespace

size_t emd_ctx_bytes_precision(int H, int W, int n, int psf_k, int r, int mode) {
  Shape s;
  const char* why = nullptr;
  if (!emd::make_shape(H, W, n, psf_k, r, &s, &why)) return 0;
  const size_t base = make_layout(s).total;
  if (mode == EMD_PREC_FP32) return base + emd::halo_buffer_bytes(s, false);
  if (mode == EMD_PREC_FP32_PAIR) return base;
  if (mode == EMD_PREC_FFT_FP32)
    return base + emd::fft_buffer_bytes(s, false, current_device_sms());
  if (mode < EMD_PREC_FP32 || mode > EMD_PREC_FFT_FP32) return 0;
  emd::TcShape t;
  if (!emd::make_tc_shape(s, mode, &t, &why)) return 0;
  return base + emd::tc_buffer_bytes(s, t);
}

emd_ctx* emd_create(int H, int W, int n, int psf_k, int r) {
  Shape s;
  const char* why = nullptr;
  if (!emd::make_shape(H, W, n, psf_k, r, &s, &why)) {
    set_err("emd_create: %s", why);
    return nullptr;
  }
  emd_ctx* c = new emd_ctx();
  c->s = s;
  c->L = make_layout(s);
  cudaGetDevice(&c->device);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, c->L.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_err("emd_create: cudaMalloc(%zu bytes) failed: %s", c->L.total, cudaGetErrorString(e));
    delete c;
    return nullptr;
  }
  c->arena = static_cast<char*>(p);
  // Zero the arena and wait for it here: a plain cudaMemset would be queued
  // on the legacy stream, which does not order against the non-blocking
  // stream the caller may set next, so later uploads could be overwritten.
  e = cudaMemsetAsync(c->arena, 0, c->L.total, cudaStreamPerThread);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
  if (e != cudaSuccess) {
    set_err("emd_create: cudaMemset failed: %s", cudaGetErrorString(e));
    cudaFree(p);
    delete c;
    return nullptr;
  }
  c->x[0] = reinterpret_cast<float*>(c->arena + c->L.x0);
  c->x[1] = reinterpret_cast<float*>(c->arena + c->L.x1);
  c->N = reinterpret_cast<float*>(c->arena + c->L.N);
  c->Den = reinterpret_cast<float*>(c->arena + c->L.Den);
  c->u = reinterpret_cast<float*>(c->arena + c->L.u);
  c->y = reinterpret_cast<float*>(c->arena + c->L.y);
  c->kf = reinterpret_cast<float*>(c->arena + c->L.kf);
  c->ka = reinterpret_cast<float*>(c->arena + c->L.ka);
  c->fraw = reinterpret_cast<float*>(c->arena + c->L.fraw);
  c->part = reinterpret_cast<double*>(c->arena + c->L.part);
  c->sums = reinterpret_cast<double*>(c->arena + c->L.sums);
  c->err = reinterpret_cast<int*>(c->arena + c->L.err);
  g_err.clear();
  return c;
}

void emd_destroy(emd_ctx* c) {
  if (!c) return;
  DeviceGuard dg(c->device);
  cudaStreamSynchronize(c->st);  // NULL: the legacy default stream
  for (cudaEvent_t e : c->trial_ev) cudaEventDestroy(e);
  cudaFree(c->arena);
  if (c->handoff) cudaEventDestroy(c->handoff);
  if (c->tc_arena) cudaFree(c->tc_arena);
  if (c->Nt) cudaFree(c->Nt);
  if (c->Ns) cudaFree(c->Ns);
  if (c->fft_arena) cudaFree(c->fft_arena);
  if (c->halo_arena) cudaFree(c->halo_arena);
  delete c;
}

int emd_set_stream(emd_ctx* c, void* stream) {
  if (int rc = check_ctx(c, false)) return rc;
  cudaStream_t ns = static_cast<cudaStream_t>(stream);
  if (ns != c->st) {
    // everything queued on the previous stream precedes what comes next
    DeviceGuard dg(c->device);
    if (!c->handoff) CK(cudaEventCreateWithFlags(&c->handoff, cudaEventDisableTiming));
    CK(cudaEventRecord(c->handoff, c->st));
    CK(cudaStreamWaitEvent(ns, c->handoff, 0));
  }
  c->st = ns;
  return EMD_OK;
}

namespace {

// the FFT form's buffers, sized and laid out for the context's noise model
// (the heavy-tailed form adds the w2 planes and a larger per-tile scratch;
// r = 1 Gaussian adds the split launch's partial accumulators, one per SM,
// and per-tile flags); a buffer that grows is re-made, one whose layout
// changes is re-bound (its flags cleared), and either way the PSF spectra
// are recomputed
int ensure_fft_arena(emd_ctx* c) {
  const bool student = c->noise == EMD_NOISE_STUDENT_T;
  if (c->fft_split_ctas == 0) c->fft_split_ctas = current_device_sms();
  const size_t need = emd::fft_buffer_bytes(c->s, student, c->fft_split_ctas);
  if (!c->fft_arena || c->fft_bytes < need) {
    if (c->fft_arena) {
      CK(cudaStreamSynchronize(c->st));
      cudaFree(c->fft_arena);
      c->fft_arena = nullptr;
      c->fft_bytes = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      set_err("cudaMalloc(%zu) for the FFT path failed", need);
      return EMD_ENOMEM;
    }
    CK(cudaMemsetAsync(p, 0, need, c->st));
    c->fft_arena = static_cast<char*>(p);
    c->fft_bytes = need;
    c->fft_bound = -1;
  }
  if (c->fft_bound == (int)student) return EMD_OK;
  const size_t spec =
      ((size_t)c->s.n * c->s.R2 * 128 * 65 * sizeof(float2) + 255) & ~(size_t)255;
  c->fft_spec = reinterpret_cast<float2*>(c->fft_arena);
  c->fft_w = reinterpret_cast<float*>(c->fft_arena + spec);
  c->fft_w2 = student ? reinterpret_cast<float*>(c->fft_arena + emd::fft_w2_offset(c->s)) : nullptr;
  c->fft_scratch =
      reinterpret_cast<float2*>(c->fft_arena + emd::fft_scratch_offset(c->s, student));
  const bool parts = emd::fft_buffer_bytes(c->s, student, c->fft_split_ctas) >
                     emd::fft_buffer_bytes(c->s, student, 0);
  c->fft_partials =
      parts ? reinterpret_cast<float2*>(c->fft_arena + emd::fft_split_offset(c->s, student))
            : nullptr;
  c->fft_counters = parts ? reinterpret_cast<int*>(c->fft_arena + emd::fft_counters_offset(
                                                                      c->s, student, c->fft_split_ctas))
                          : nullptr;
  c->fft_counters_bytes =
      c->fft_counters ? need - emd::fft_counters_offset(c->s, student, c->fft_split_ctas) : 0;
  if (c->fft_counters) CK(cudaMemsetAsync(c->fft_counters, 0, c->fft_counters_bytes, c->st));
  c->fft_bound = (int)student;
  c->fft_ready = false;
  return EMD_OK;
}

// The halo-exchange iteration's ring, flags and counters for the current
// noise model (re-sized when it needs two tiles per slot); *ok = false (no
// error) when the shape has too many work items for it (the CTA-pair
// kernel runs).
int ensure_halo_arena(emd_ctx* c, bool* ok) {
  *ok = false;
  const bool student = c->noise == EMD_NOISE_STUDENT_T;
  const size_t need = emd::halo_buffer_bytes(c->s, student);
  if (need == 0) return EMD_OK;
  if (c->halo_arena && c->halo_bytes >= need) {
    if (student != c->halo_student) {
      // same buffer, other slot layout: the flags and counters move, so
      // they (and everything else) start from zero again
      CK(cudaMemsetAsync(c->halo_arena, 0, c->halo_bytes, c->st));
      emd::halo_bind(c->s, student, c->halo_arena, &c->halo);
      c->halo_student = student;
    }
    *ok = true;
    return EMD_OK;
  }
  if (c->halo_arena) {
    CK(cudaStreamSynchronize(c->st));
    cudaFree(c->halo_arena);
    c->halo_arena = nullptr;
    c->halo_bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, need) != cudaSuccess) {
    cudaGetLastError();
    set_err("cudaMalloc(%zu) for the FP32 direct iteration failed", need);
    return EMD_ENOMEM;
  }
  CK(cudaMemsetAsync(p, 0, need, c->st));  // flags and counters start at zero
  c->halo_arena = static_cast<char*>(p);
  c->halo_bytes = need;
  c->halo_student = student;
  emd::halo_bind(c->s, student, p, &c->halo);
  *ok = true;
  return EMD_OK;
}

// ---------------------------------------------------------------------------
// Tile-shape autotuner of the halo-exchange kernel. A process-wide table,
// keyed by the problem (H, W, n, K, r, noise model), holds the decided tile
// shape. A context whose key is undecided times the candidate shapes on its
// own iterations: each candidate runs in turn, twice, with CUDA events
// around its launch on the context's stream, and the second round's times
// decide (the first round carries each kernel's first-launch costs). The
// events are polled without blocking (cudaEventQuery) at later calls, so the
// iterations stay asynchronous. Every shape gives the same iterates, so
// trials change nothing but time.
// ---------------------------------------------------------------------------
struct TileKey {
  int H, W, n, K, r, student;
  bool operator<(const TileKey& o) const {
    const int a[6] = {H, W, n, K, r, student}, b[6] = {o.H, o.W, o.n, o.K, o.r, o.student};
    return std::lexicographical_compare(a, a + 6, b, b + 6);
  }
};
std::mutex g_tile_mu;
std::map<TileKey, int> g_tile_decided;

TileKey tile_key(const emd_ctx* c, bool student) {
  return TileKey{c->s.H, c->s.W, c->s.n, c->s.K, c->s.r, student ? 1 : 0};
}

// Candidate shapes for this problem: 64-row tiles always; 48-row tiles when
// three CTAs fit an SM; 32-row tiles when four do.
std::vector<int> tile_candidates(const emd_ctx* c) {
  std::vector<int> v{0};
  if (emd::halo_tile_ctas_per_sm(c->s, 1) >= 3) v.push_back(1);
  if (emd::halo_tile_ctas_per_sm(c->s, 2) >= 4) v.push_back(2);
  return v;
}

// Reads the trial events if they are all done (no blocking) and records the
// decision.
void tile_trials_poll(emd_ctx* c) {
  if (c->trial_cfg.empty() || c->trials_issued < c->trial_cfg.size()) return;
  if (cudaEventQuery(c->trial_ev[2 * c->trials_issued - 1]) != cudaSuccess) {
    cudaGetLastError();  // not ready yet (cudaErrorNotReady is not sticky)
    return;
  }
  const size_t half = c->trial_cfg.size() / 2;
  int best = c->trial_cfg[half];
  float best_ms = 0.f;
  for (size_t i = half; i < c->trial_cfg.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->trial_ev[2 * i], c->trial_ev[2 * i + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (i == half || ms < best_ms) {
      best_ms = ms;
      best = c->trial_cfg[i];
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile_decided[tile_key(c, c->trial_student)] = best;
  }
  c->trial_cfg.clear();
  c->trials_issued = 0;
}

// Tile shape of the next full-iteration launch; *trial: index of the trial
// it runs (events to record), or -1.
int tile_for_launch(emd_ctx* c, bool student, int* trial) {
  *trial = -1;
  if (c->tile_forced >= 0) return c->tile_forced;
  tile_trials_poll(c);
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile_decided.find(tile_key(c, student));
    if (it != g_tile_decided.end()) return it->second;
  }
  if (c->trial_cfg.empty() || c->trial_student != student) {
    const std::vector<int> cand = tile_candidates(c);
    if (cand.size() < 2) {
      std::lock_guard<std::mutex> lk(g_tile_mu);
      g_tile_decided[tile_key(c, student)] = cand[0];
      return cand[0];
    }
    c->trial_cfg.clear();
    for (int round = 0; round < 2; ++round)
      for (int cfg : cand) c->trial_cfg.push_back(cfg);
    c->trials_issued = 0;
    c->trial_student = student;
    while (c->trial_ev.size() < 2 * c->trial_cfg.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        c->trial_cfg.clear();
        return 0;
      }
      c->trial_ev.push_back(e);
    }
  }
  if (c->trials_issued < c->trial_cfg.size()) {
    *trial = (int)c->trials_issued;
    return c->trial_cfg[c->trials_issued++];
  }
  return c->trial_cfg[0];  // all trials issued, not yet read
}

// One halo-exchange launch of a full iteration, with the autotuner's shape.
int halo_launch_full(emd_ctx* c, const emd::HaloLaunch& h, bool student) {
  int trial = -1;
  const int cfg = tile_for_launch(c, student, &trial);
  if (trial >= 0) CK(cudaEventRecord(c->trial_ev[2 * trial], c->st));
  CK(emd::launch_halo_iter(c->s, h, cfg, c->st));
  if (trial >= 0) CK(cudaEventRecord(c->trial_ev[2 * trial + 1], c->st));
  c->tile_last = cfg;
  return EMD_OK;
}

}  // namespace

int emd_set_precision(emd_ctx* c, int mode) {
  if (int rc = check_ctx(c, false)) return rc;
  if (mode == EMD_PREC_FP32 || mode == EMD_PREC_FP32_PAIR) {
    c->prec = mode;
    return EMD_OK;
  }
  if (mode < 0 || mode > EMD_PREC_FFT_FP32) {
    set_err("unknown precision mode %d", mode);
    return EMD_EINVAL;
  }
  DeviceGuard dg(c->device);
  if (mode == EMD_PREC_FFT_FP32) {
    if (int rc = ensure_fft_arena(c)) return rc;
    c->prec = mode;
    return EMD_OK;
  }
  if (c->noise != EMD_NOISE_GAUSSIAN) {
    set_err("emd_set_precision: the heavy-tailed update runs on the FP32 direct and FFT forms");
    return EMD_EUNSUPPORTED;
  }
  emd::TcShape t;
  const char* why = nullptr;
  if (!emd::make_tc_shape(c->s, mode, &t, &why)) {
    set_err("emd_set_precision: %s", why);
    return EMD_EUNSUPPORTED;
  }
  const size_t need = emd::tc_buffer_bytes(c->s, t);
  if (!c->tc_arena || c->tc_bytes < need) {
    if (c->tc_arena) {
      CK(cudaStreamSynchronize(c->st));
      cudaFree(c->tc_arena);
      c->tc_arena = nullptr;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_err("emd_set_precision: cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
      return EMD_ENOMEM;
    }
    CK(cudaMemsetAsync(p, 0, need, c->st));  // ordered before its first use on c->st
    c->tc_arena = static_cast<char*>(p);
    c->tc_bytes = need;
  }
  const size_t xb_bytes = (4ull * c->s.R2 * c->s.g.plane * sizeof(uint16_t) + 255) & ~(size_t)255;
  c->xb = reinterpret_cast<uint16_t*>(c->tc_arena);
  c->hank = reinterpret_cast<uint16_t*>(c->tc_arena + xb_bytes);
  c->wb = reinterpret_cast<uint16_t*>(c->tc_arena + emd::tc_w_offset(c->s, t));
  c->scales = reinterpret_cast<float*>(c->tc_arena + need - 256);
  c->xmax = reinterpret_cast<unsigned int*>(c->tc_arena + need - 128);
  if (emd::make_plane_tensormap(c->s, t, c->xb, 4 * c->s.R2, &c->xmap) != 0 ||
      emd::make_plane_tensormap(c->s, t, c->wb, 2 * c->s.n, &c->wmap) != 0) {
    set_err("emd_set_precision: cuTensorMapEncodeTiled failed");
    return EMD_ECUDA;
  }
  c->ts = t;
  c->prec = mode;
  c->hank_ready = false;
  return EMD_OK;
}

int emd_set_frames(emd_ctx* c, const float* y, const float* v, const float* f,
                   const uint8_t* mask) {
  if (int rc = check_ctx(c, false)) return rc;
  if (!y || !v || !f) {
    set_err("emd_set_frames: y, v and f must not be NULL");
    return EMD_EINVAL;
  }
  DeviceGuard dg(c->device);
  const Shape& s = c->s;
  c->frames = false;
  c->hank_ready = false;
  c->fft_ready = false;
  c->nt_ready = false;
  const size_t npix = (size_t)s.n * s.H * s.W;
  if (int rc = put_planes(c, c->y, y, s.n)) return rc;
  if (int rc = put_planes(c, c->u, v, s.n)) return rc;  // v, converted in place below
  CK(cudaMemcpyAsync(c->fraw, f, (size_t)s.n * s.K * s.K * sizeof(float), cudaMemcpyDefault,
                     c->st));
  const uint8_t* dmask = nullptr;
  void* tmp = nullptr;
  if (mask) {
    if (is_device_ptr(mask)) {
      dmask = mask;
    } else {
      CK(cudaMallocAsync(&tmp, npix, c->st));
      CK(cudaMemcpyAsync(tmp, mask, npix, cudaMemcpyHostToDevice, c->st));
      dmask = static_cast<const uint8_t*>(tmp);
    }
  }
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  emd::SetupArgs sa{dmask, c->u, c->y, c->part, c->err};
  CK(emd::launch_setup(s, sa, c->st));
  if (tmp) CK(cudaFreeAsync(tmp, c->st));
  CK(emd::launch_reduce_final(c->part, emd::kRedBlocks, 4, c->sums, c->st));
  CK(emd::launch_build_kernels(s, c->fraw, c->kf, c->ka, c->st));
  double h[4];
  int herr = 0;
  CK(cudaMemcpyAsync(h, c->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (herr & emd::kErrData) {
    CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
    set_err("emd_set_frames: a valid pixel has v <= 0 or a non-finite y or v");
    return EMD_EDATA;
  }
  c->logdet = h[0];
  c->suy = h[1];
  c->su = h[2];
  c->nvalid = h[3];
  // numerator N = sum_t F_t^T (u_t y_t)
  emd::FusedArgs a = fused_args(c);
  CK(emd::launch_fused(s, a, 1, c->part, c->st));
  // default strictly positive start
  double x0 = 1.0;
  if (c->su > 0.0) {
    const double cc = c->suy / c->su / ((double)s.r * s.r);
    if (cc > 0.0) x0 = cc;
  }
  CK(emd::launch_fill_latent(s, c->x[c->cur], (float)x0, c->st));
  c->frames = true;
  return check_device_error(c);
}

int emd_set_x(emd_ctx* c, const float* x0) {
  if (int rc = check_ctx(c, true)) return rc;
  if (!x0) {
    set_err("emd_set_x: null pointer");
    return EMD_EINVAL;
  }
  DeviceGuard dg(c->device);
  const Shape& s = c->s;
  const size_t nat = (size_t)s.R2 * s.H * s.W;
  const float* src = x0;
  if (!is_device_ptr(x0)) {
    CK(cudaMemcpyAsync(c->Den, x0, nat * sizeof(float), cudaMemcpyHostToDevice, c->st));
    src = c->Den;
  }
  CK(emd::launch_scatter_latent(s, src, c->x[c->cur], 1, c->st));
  CK(cudaStreamSynchronize(c->st));
  return EMD_OK;
}

int emd_iterate(emd_ctx* c, int k) {
  if (int rc = check_ctx(c, true)) return rc;
  if (k < 0) {
    set_err("emd_iterate: k must be >= 0");
    return EMD_EINVAL;
  }
  DeviceGuard dg(c->device);
  if (c->prec == EMD_PREC_FFT_FP32 && k > 0) {
    if (int rc = ensure_fft_arena(c)) return rc;  // grows if the noise model changed
    if (!c->fft_ready) {
      CK(emd::launch_fft_spectra(c->s, c->ka, c->fft_spec, c->st));
      c->fft_ready = true;
    }
    for (int it = 0; it < k; ++it) {
      emd::FftLaunch L{};
      L.x = c->x[c->cur];
      L.xn = c->x[c->cur ^ 1];
      L.N = c->N;
      L.u = c->u;
      L.w = c->fft_w;
      L.spec = c->fft_spec;
      L.scratch = c->fft_scratch;
      L.partials = c->fft_partials;
      L.counters = c->fft_counters;
      L.split_ctas = c->fft_split_ctas;
      L.err = c->err;
      if (c->noise == EMD_NOISE_STUDENT_T) {
        L.y = c->y;
        L.w2 = c->fft_w2;
        L.nu = (float)c->nu;
      }
      CK(emd::launch_fft_iter(c->s, L, c->st));
      c->cur ^= 1;
    }
    return EMD_OK;
  }
  if (c->prec != EMD_PREC_FP32 && c->prec != EMD_PREC_FP32_PAIR && k > 0) {
    // tensor-core path: 16-bit operands of the PSFs (once per frame set) and
    // of the current x, then one kernel launch per iteration
    const bool fp16 = c->ts.fp16 != 0;
    if (!c->hank_ready) {
      const Shape& s = c->s;
      c->gscale = 1.f;
      if (fp16) {
        // PSF scale and the bound on |z| / max x, from the kernels on the host
        const size_t nk = (size_t)s.n * s.R2 * s.Kc * s.KP;
        std::vector<float> kf(nk);
        CK(cudaMemcpyAsync(kf.data(), c->kf, nk * sizeof(float), cudaMemcpyDeviceToHost, c->st));
        CK(emd::launch_max_nonneg(c->u, (long long)s.n * s.g.plane, c->xmax, c->st));
        unsigned int ub = 0;
        CK(cudaMemcpyAsync(&ub, c->xmax, sizeof(ub), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        float gmax = 0.f, fsum = 0.f;
        for (int t = 0; t < s.n; ++t) {
          float tsum = 0.f;
          for (size_t e = (size_t)t * s.R2 * s.Kc * s.KP; e < (size_t)(t + 1) * s.R2 * s.Kc * s.KP; ++e) {
            gmax = fmaxf(gmax, fabsf(kf[e]));
            tsum += fabsf(kf[e]);
          }
          fsum = fmaxf(fsum, tsum);
        }
        memcpy(&c->umax, &ub, sizeof(float));
        c->fsum = fsum;
        if (gmax > 0.f) c->gscale = exp2f(floorf(log2f(16384.f / gmax)));
      } else {
        const float one[4] = {1.f, 1.f, 1.f, 1.f};
        CK(cudaMemcpyAsync(c->scales, one, sizeof(one), cudaMemcpyHostToDevice, c->st));
        CK(cudaStreamSynchronize(c->st));
      }
      CK(emd::launch_build_hankel(c->s, c->ts, c->kf, c->ka, c->hank, c->gscale, c->st));
      c->hank_ready = true;
    }
    for (int it = 0; it < k; ++it) {
      if (fp16 || it == 0) {
        if (fp16) {
          CK(emd::launch_max_nonneg(c->x[c->cur], (long long)c->s.R2 * c->s.g.plane, c->xmax,
                                    c->st));
          CK(emd::launch_fp16_scales(c->xmax, c->gscale, c->umax, c->fsum, c->scales, c->st));
        }
        CK(emd::launch_split_x(c->s, c->ts, c->x[c->cur], c->xb, c->cur, c->scales, c->st));
      }
      emd::TcLaunch L{};
      L.x = c->x[c->cur];
      L.xn = c->x[c->cur ^ 1];
      L.N = c->N;
      L.Den = c->Den;
      L.u = c->u;
      L.xb = c->xb;
      L.wb = c->wb;
      L.hank = c->hank;
      L.pp = c->cur;
      L.scales = c->scales;
      L.write_xb = fp16 ? 0 : 1;
      L.err = c->err;
      CK(emd::launch_tc_iter(c->s, c->ts, L, c->xmap, c->wmap, c->st));
      c->cur ^= 1;
    }
    return EMD_OK;
  }
  if (c->noise == EMD_NOISE_STUDENT_T) {
    // heavy-tailed EM: the numerator depends on x through the weights u' of
    // the current x. The halo-exchange kernel computes the forward model
    // once and both adjoints (Den' and N') in one launch; the CTA-pair
    // kernel (EMD_PREC_FP32_PAIR) runs N' (mode 3), then Den' and the update
    // (mode 0), each with its own forward pass. Same iterates either way.
    bool halo = false;
    if (c->prec == EMD_PREC_FP32 && k > 0)
      if (int rc = ensure_halo_arena(c, &halo)) return rc;
    for (int it = 0; halo && it < k; ++it) {
      emd::HaloLaunch h = c->halo;
      h.a = fused_args(c);
      h.a.Nw = c->Ns;
      if (int rc = halo_launch_full(c, h, true)) return rc;
      c->cur ^= 1;
    }
    for (int it = 0; !halo && it < k; ++it) {
      emd::FusedArgs a = fused_args(c);
      a.Nw = c->Ns;
      CK(emd::launch_fused(c->s, a, 3, c->part, c->st));
      a.N = c->Ns;
      CK(emd::launch_fused(c->s, a, 0, c->part, c->st));
      c->cur ^= 1;
    }
    return EMD_OK;
  }
  bool halo = false;
  if (c->prec == EMD_PREC_FP32 && k > 0)
    if (int rc = ensure_halo_arena(c, &halo)) return rc;
  for (int it = 0; it < k; ++it) {
    emd::FusedArgs a = fused_args(c);
    if (halo) {
      emd::HaloLaunch h = c->halo;
      h.a = a;
      if (int rc = halo_launch_full(c, h, false)) return rc;
    } else {
      CK(emd::launch_fused(c->s, a, 0, c->part, c->st));
    }
    c->cur ^= 1;
  }
  return EMD_OK;
}

int emd_set_noise(emd_ctx* c, int model, double nu) {
  if (int rc = check_ctx(c, false)) return rc;
  if (model == EMD_NOISE_GAUSSIAN) {
    c->noise = model;
    c->nu = 0.0;
    return EMD_OK;
  }
  if (model != EMD_NOISE_STUDENT_T) {
    set_err("emd_set_noise: unknown noise model %d", model);
    return EMD_EINVAL;
  }
  if (!(nu > 0.0) || !std::isfinite(nu) || nu > 1e30) {
    set_err("emd_set_noise: nu must be finite and in (0, 1e30]");
    return EMD_EINVAL;
  }
  if (c->prec != EMD_PREC_FP32 && c->prec != EMD_PREC_FP32_PAIR &&
      c->prec != EMD_PREC_FFT_FP32) {
    set_err("emd_set_noise: the heavy-tailed update runs on the FP32 direct and FFT forms");
    return EMD_EUNSUPPORTED;
  }
  if (!c->Ns) {
    DeviceGuard dg(c->device);
    void* p = nullptr;
    const size_t bytes = (size_t)c->s.R2 * c->s.g.plane * sizeof(float);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      set_err("emd_set_noise: cudaMalloc of the numerator planes failed");
      return EMD_ENOMEM;
    }
    CK(cudaMemsetAsync(p, 0, bytes, c->st));
    c->Ns = static_cast<float*>(p);
  }
  c->noise = model;
  c->nu = nu;
  return EMD_OK;
}

int emd_iterate_streaming(emd_ctx* c, int k, const int* order) {
  if (int rc = check_ctx(c, true)) return rc;
  const Shape& s = c->s;
  if (c->noise != EMD_NOISE_GAUSSIAN) {
    set_err("emd_iterate_streaming: Gaussian noise only");
    return EMD_EUNSUPPORTED;
  }
  if (k < 0) {
    set_err("emd_iterate_streaming: k must be >= 0");
    return EMD_EINVAL;
  }
  std::vector<int> ord(s.n);
  for (int t = 0; t < s.n; ++t) ord[t] = t;
  if (order) {
    std::vector<char> seen(s.n, 0);
    for (int t = 0; t < s.n; ++t) {
      const int e = order[t];
      if (e < 0 || e >= s.n || seen[e]) {
        set_err("emd_iterate_streaming: order must be a permutation of 0..n-1");
        return EMD_EINVAL;
      }
      seen[e] = 1;
      ord[t] = e;
    }
  }
  DeviceGuard dg(c->device);
  const size_t lat = (size_t)s.R2 * s.g.plane;
  if (!c->Nt) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, (size_t)s.n * lat * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_err("emd_iterate_streaming: cudaMalloc of the per-exposure numerators failed");
      return EMD_ENOMEM;
    }
    CK(cudaMemsetAsync(p, 0, (size_t)s.n * lat * sizeof(float), c->st));
    c->Nt = static_cast<float*>(p);
  }
  if (!c->nt_ready) {
    for (int t = 0; t < s.n; ++t) {
      emd::FusedArgs a = fused_args(c);
      a.Nw = c->Nt + (size_t)t * lat;
      a.t0 = t;
      a.t1 = t + 1;
      CK(emd::launch_fused(s, a, 1, c->part, c->st));
    }
    c->nt_ready = true;
  }
  // the halo-exchange kernel over the one-exposure range (the CTA-pair
  // kernel under EMD_PREC_FP32_PAIR): the same iterates either way
  bool halo = false;
  if (c->prec != EMD_PREC_FP32_PAIR && k > 0)
    if (int rc = ensure_halo_arena(c, &halo)) return rc;
  for (int it = 0; it < k; ++it) {
    for (int q = 0; q < s.n; ++q) {
      const int t = ord[q];
      emd::FusedArgs a = fused_args(c);
      a.N = c->Nt + (size_t)t * lat;
      a.t0 = t;
      a.t1 = t + 1;
      if (halo) {
        // one-exposure launches: the shape decided for the full iteration
        // (or fixed by the caller), without trials of their own
        int cfg = c->tile_forced;
        if (cfg < 0) {
          std::lock_guard<std::mutex> lk(g_tile_mu);
          auto f = g_tile_decided.find(tile_key(c, false));
          cfg = f != g_tile_decided.end() ? f->second : 0;
        }
        emd::HaloLaunch h = c->halo;
        h.a = a;
        CK(emd::launch_halo_iter(s, h, cfg, c->st));
      } else {
        CK(emd::launch_fused(s, a, 0, c->part, c->st));
      }
      c->cur ^= 1;
    }
  }
  return EMD_OK;
}

int emd_set_tile_shape(emd_ctx* c, int shape) {
  if (int rc = check_ctx(c, false)) return rc;
  if (shape < EMD_TILE_AUTO || shape > emd::kHaloTileConfigs) {
    set_err("emd_set_tile_shape: unknown tile shape %d", shape);
    return EMD_EINVAL;
  }
  c->tile_forced = shape - 1;  // -1: autotuned
  return EMD_OK;
}

int emd_get_tile_shape(emd_ctx* c, int* shape, int* decided) {
  if (int rc = check_ctx(c, false)) return rc;
  DeviceGuard dg(c->device);
  tile_trials_poll(c);
  int cfg = c->tile_forced, dec = 1;
  if (cfg < 0) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile_decided.find(tile_key(c, c->noise == EMD_NOISE_STUDENT_T));
    if (it != g_tile_decided.end()) {
      cfg = it->second;
    } else {
      cfg = c->tile_last;
      dec = 0;
    }
  }
  if (shape) *shape = cfg + 1;
  if (decided) *decided = dec;
  return EMD_OK;
}

int emd_get_x(emd_ctx* c, float* out) {
  if (int rc = check_ctx(c, true)) return rc;
  DeviceGuard dg(c->device);
  if (int rc = latent_out(c, c->x[c->cur], out)) return rc;
  return check_device_error(c);
}

int emd_selftest_wait_timeout(emd_ctx* c, int spins) {
  if (int rc = check_ctx(c, false)) return rc;
  if (spins < 1) {
    set_err("emd_selftest_wait_timeout: spins must be >= 1");
    return EMD_EINVAL;
  }
  DeviceGuard dg(c->device);
  // the mbarrier wait of the staging copies
  CK(emd::launch_wait_selftest((uint32_t)spins, c->err, c->st));
  const int rc = check_device_error(c);
  if (rc != EMD_ETIMEOUT) return rc;
  // the flag waits of the halo-exchange kernel, and their abort flag
  CK(emd::launch_flag_wait_selftest((uint32_t)spins, c->part, c->err, c->st));
  return check_device_error(c);
}

int emd_get_numerator(emd_ctx* c, float* out) {
  if (int rc = check_ctx(c, true)) return rc;
  DeviceGuard dg(c->device);
  return latent_out(c, c->N, out);
}

int emd_get_weights(emd_ctx* c, float* out) {
  if (int rc = check_ctx(c, true)) return rc;
  if (!out) {
    set_err("null output pointer");
    return EMD_EINVAL;
  }
  DeviceGuard dg(c->device);
  if (int rc = get_planes(c, out, c->u, c->s.n)) return rc;
  CK(cudaStreamSynchronize(c->st));
  return EMD_OK;
}

int emd_loglik(emd_ctx* c, double* out) { return emd_loglik_chi2(c, out, nullptr); }

int emd_loglik_chi2(emd_ctx* c, double* out, double* chi2) {
  if (int rc = check_ctx(c, true)) return rc;
  if (!out) {
    set_err("null output pointer");
    return EMD_EINVAL;
  }
  DeviceGuard dg(c->device);
  emd::FusedArgs a = fused_args(c);
  // the forward model once per pixel (the CTA-pair kernel's halo form under
  // EMD_PREC_FP32_PAIR); FP64 partial sums added in a fixed order
  const int max_parts = (int)((c->L.sums - c->L.part) / sizeof(double));
  int nparts = 0;
  if (c->prec != EMD_PREC_FP32_PAIR && max_parts >= c->s.gx * c->s.gy) {
    cudaError_t e = cudaSuccess;
    nparts = emd::launch_halo_chi2(c->s, a, c->part, max_parts, c->st, &e);
    CK(e);
  } else {
    CK(emd::launch_fused(c->s, a, 2, c->part, c->st));
    nparts = emd::fused_blocks(c->s);
  }
  CK(emd::launch_reduce_final(c->part, nparts, 1, c->sums + 4, c->st));
  double h = 0.0;
  CK(cudaMemcpyAsync(&h, c->sums + 4, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if (int rc = check_device_error(c)) return rc;
  if (c->noise == EMD_NOISE_STUDENT_T) {
    // sum over valid pixels of lgamma((nu+1)/2) - lgamma(nu/2) - 1/2 log(nu pi v)
    // - (nu+1)/2 log(1 + u r^2 / nu); h holds the last term's sum times 2
    const double nu = c->nu, kPi = 3.14159265358979323846, k2Pi = 6.28318530717958647692;
    const double sum_log_v = c->logdet - c->nvalid * std::log(k2Pi);
    *out = c->nvalid * (std::lgamma(0.5 * (nu + 1.0)) - std::lgamma(0.5 * nu) -
                        0.5 * std::log(nu * kPi)) -
           0.5 * sum_log_v - 0.5 * h;
  } else {
    *out = -0.5 * (h + c->logdet);
  }
  if (chi2) *chi2 = h;
  return EMD_OK;
}

}  // extern "C"

// ===========================================================================
// Batching: one persistent kernel per step over all active jobs
// ===========================================================================

namespace {

constexpr int kBatchItemCap = 1 << 20;  // (job, tile) work items per step
constexpr int kHaloItemCap = 1 << 22;   // (job, position) items of the halo kernel per step

struct TuneChoice {
  int clusters = 0;
  int order = 1;  // 0: job-major (halo form: round-robin over jobs), 1: most expensive jobs first
  int form = 0;   // FP32 jobs: 0 = halo-exchange kernel, 1 = CTA-pair kernel (same iterates)
  int tile = 0;   // halo-exchange kernel's tile shape (emd::halo_plan's cfg)
  bool same_table(const TuneChoice& o) const {
    return order == o.order && form == o.form && tile == o.tile;
  }
};

}  // namespace

struct emd_batch {
  int max_jobs = 0;
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<emd_ctx*> job;   // per slot; nullptr when free
  std::vector<int> remaining;  // host mirror of the device table
  char* arena = nullptr;
  emd::BatchJob* d_jobs = nullptr;
  int2* d_items = nullptr;
  int* d_nitems = nullptr;
  int* d_counter = nullptr;
  int* d_err = nullptr;
  size_t smem = 0;
  int max_clusters = 0;
  bool dirty = true;
  int njobs_table = 0;
  // FFT jobs: their own table, work list and counters (forward, adjoint)
  emd::FftBatchJob* d_fjobs = nullptr;
  int2* d_fitems = nullptr;
  int* d_fnitems = nullptr;
  int* d_fcounters = nullptr;
  int fft_ctas = 0;
  // FP32 jobs on the halo-exchange kernel: table, (job, position) list, claim counters
  emd::HaloBatchJob* d_hjobs = nullptr;
  int2* d_hitems = nullptr;
  int* d_hnitems = nullptr;
  unsigned long long* d_hctrl = nullptr;
  char* harena = nullptr;
  int halo_ctas[emd::kHaloTileConfigs] = {};  // resident CTAs of each tile shape's kernel
  bool has_direct = false, has_fft = false, has_halo = false;
  // captured step graphs, one per (cluster count, parts present)
  std::map<int, cudaGraphExec_t> graphs;
  // autotuner: decision per composition, and the candidates still to try
  std::map<std::string, TuneChoice> tuned;
  std::string sig;
  std::vector<TuneChoice> trying;
  std::vector<float> trial_ms;
  TuneChoice cur;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  long long steps = 0;
};

namespace {

std::string composition_signature(emd_batch* b) {
  std::vector<std::string> parts;
  for (size_t i = 0; i < b->job.size(); ++i) {
    emd_ctx* c = b->job[i];
    if (!c || b->remaining[i] <= 0) continue;
    int sb = 0;
    for (int v = c->s.H > c->s.W ? c->s.H : c->s.W; v > 1; v >>= 1) ++sb;
    char buf[64];
    snprintf(buf, sizeof(buf), "%d.%d.%d.%d.%d", sb, c->s.Kc, c->s.r, (c->s.n + 7) / 8, c->prec);
    parts.push_back(buf);
  }
  std::sort(parts.begin(), parts.end());
  std::string out;
  for (auto& p : parts) out += p + ";";
  return out;
}

int upload_table(emd_batch* b) {
  std::vector<emd::BatchJob> tab(b->job.size());
  std::vector<emd::FftBatchJob> ftab(b->job.size());
  std::vector<emd::HaloBatchJob> htab(b->job.size());
  struct Hj { long long cost; int job; long long len; };
  std::vector<Hj> hjobs;
  struct It { long long cost; int job, tile; };
  std::vector<It> its;
  std::vector<int2> fitems;
  for (size_t i = 0; i < b->job.size(); ++i) {
    emd_ctx* c = b->job[i];
    emd::BatchJob& J = tab[i];
    memset(&J, 0, sizeof(J));
    memset(&ftab[i], 0, sizeof(ftab[i]));
    memset(&htab[i], 0, sizeof(htab[i]));
    if (!c) continue;
    if (c->prec == EMD_PREC_FFT_FP32) {
      emd::FftBatchJob& F = ftab[i];
      F.s = c->s;
      for (int k = 0; k < 2; ++k) {
        emd::FftLaunch& L = F.a[k];
        L.x = c->x[k];
        L.xn = c->x[k ^ 1];
        L.N = c->N;
        L.u = c->u;
        L.w = c->fft_w;
        L.spec = c->fft_spec;
        L.scratch = c->fft_scratch;
      }
      F.cur = c->cur;
      F.remaining = b->remaining[i];
      F.gxt = emd::fft_tiles_x(c->s);
      if (F.remaining > 0)
        for (int t = 0; t < emd::fft_tiles_total(c->s); ++t) fitems.push_back(make_int2((int)i, t));
      continue;  // not in the direct table (remaining 0 there)
    }
    if (c->prec == EMD_PREC_FP32 && b->cur.form == 0 && c->halo_arena && b->remaining[i] > 0) {
      emd::HaloBatchJob& Hj = htab[i];
      Hj.s = c->s;
      for (int k = 0; k < 2; ++k) {
        const int save = c->cur;
        c->cur = k;
        Hj.h[k] = c->halo;
        Hj.h[k].a = fused_args(c);
        c->cur = save;
      }
      Hj.pl = emd::halo_plan(c->s, c->s.n, b->cur.tile);
      Hj.cur = c->cur;
      Hj.remaining = b->remaining[i];
      hjobs.push_back({(long long)c->s.n * c->s.R2 * c->s.Kc * c->s.Kc * Hj.pl.T, (int)i,
                       2 * Hj.pl.NT});
      continue;  // not in the CTA-pair table (remaining 0 there)
    }
    J.s = c->s;
    for (int k = 0; k < 2; ++k) {
      const int save = c->cur;
      c->cur = k;
      J.a[k] = fused_args(c);
      c->cur = save;
    }
    J.cur = c->cur;
    J.remaining = b->remaining[i];
    if (J.remaining <= 0) continue;
    const long long cost = (long long)c->s.n * c->s.R2 * c->s.Kc * c->s.Kc;
    for (int t = 0; t < c->s.gx * c->s.gy; ++t) its.push_back({cost, (int)i, t});
  }
  if (its.size() > (size_t)kBatchItemCap || fitems.size() > (size_t)kBatchItemCap) {
    set_err("emd_batch_step: more than %d tiles in one step", kBatchItemCap);
    return EMD_EINVAL;
  }
  if (b->cur.order == 1)
    std::stable_sort(its.begin(), its.end(), [](const It& x, const It& y) { return x.cost > y.cost; });
  std::vector<int2> items(its.size());
  for (size_t k = 0; k < its.size(); ++k) items[k] = make_int2(its[k].job, its[k].tile);
  const int n = (int)items.size();
  // halo-exchange jobs: each job's claim sequence in its own order, merged
  // round-robin (order 0) or job after job, most expensive first (order 1)
  std::vector<int2> hitems;
  {
    long long tot = 0;
    for (auto& j : hjobs) tot += j.len;
    if (tot > kHaloItemCap) {
      set_err("emd_batch_step: more than %d halo work items in one step", kHaloItemCap);
      return EMD_EINVAL;
    }
    hitems.reserve((size_t)tot);
    if (b->cur.order == 1) {
      std::stable_sort(hjobs.begin(), hjobs.end(),
                       [](const Hj& x, const Hj& y) { return x.cost > y.cost; });
      for (auto& j : hjobs)
        for (long long q = 0; q < j.len; ++q) hitems.push_back(make_int2(j.job, (int)q));
    } else {
      for (long long q = 0; (long long)hitems.size() < tot; ++q)
        for (auto& j : hjobs)
          if (q < j.len) hitems.push_back(make_int2(j.job, (int)q));
    }
  }
  const int nh = (int)hitems.size();
  CK(cudaMemcpyAsync(b->d_jobs, tab.data(), tab.size() * sizeof(emd::BatchJob),
                     cudaMemcpyHostToDevice, b->st));
  if (n) CK(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, b->st));
  CK(cudaMemcpyAsync(b->d_nitems, &n, sizeof(int), cudaMemcpyHostToDevice, b->st));
  const int nf = (int)fitems.size();
  CK(cudaMemcpyAsync(b->d_fjobs, ftab.data(), ftab.size() * sizeof(emd::FftBatchJob),
                     cudaMemcpyHostToDevice, b->st));
  if (nf) CK(cudaMemcpyAsync(b->d_fitems, fitems.data(), fitems.size() * sizeof(int2),
                             cudaMemcpyHostToDevice, b->st));
  CK(cudaMemcpyAsync(b->d_fnitems, &nf, sizeof(int), cudaMemcpyHostToDevice, b->st));
  CK(cudaMemcpyAsync(b->d_hjobs, htab.data(), htab.size() * sizeof(emd::HaloBatchJob),
                     cudaMemcpyHostToDevice, b->st));
  if (nh) CK(cudaMemcpyAsync(b->d_hitems, hitems.data(), hitems.size() * sizeof(int2),
                             cudaMemcpyHostToDevice, b->st));
  CK(cudaMemcpyAsync(b->d_hnitems, &nh, sizeof(int), cudaMemcpyHostToDevice, b->st));
  CK(cudaStreamSynchronize(b->st));
  b->njobs_table = (int)tab.size();
  b->has_direct = n > 0;
  b->has_fft = nf > 0;
  b->has_halo = nh > 0;
  return EMD_OK;
}

int get_graph(emd_batch* b, int clusters, cudaGraphExec_t* out) {
  // a step: the persistent direct kernel over the FP32 jobs' tiles, then the
  // persistent FFT forward and adjoint kernels over the FFT jobs' tiles
  const int key = clusters | (b->has_direct ? 1 << 20 : 0) | (b->has_fft ? 1 << 21 : 0) |
                  (b->has_halo ? 1 << 22 : 0) | (b->cur.tile << 23);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = it->second;
    return EMD_OK;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  if (b->has_direct)
    e = emd::launch_batch(b->d_jobs, b->max_jobs, b->d_items, b->d_nitems, b->d_counter, b->d_err,
                          clusters, b->smem, b->st);
  if (e == cudaSuccess && b->has_halo) {
    // the halo kernel's share of the CTAs follows the tuned cluster count
    int ctas = b->halo_ctas[b->cur.tile] * clusters / (b->max_clusters > 0 ? b->max_clusters : 1);
    if (ctas < 1) ctas = 1;
    e = emd::launch_halo_batch(b->cur.tile, b->d_hjobs, b->max_jobs, b->d_hitems, b->d_hnitems,
                               b->d_hctrl, b->d_err, ctas, b->st);
  }
  if (e == cudaSuccess && b->has_fft)
    e = emd::launch_fft_batch(b->d_fjobs, b->max_jobs, b->d_fitems, b->d_fnitems, b->d_fcounters,
                              b->fft_ctas, b->st);
  cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_err("batch graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return EMD_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_err("batch graph instantiate failed: %s", cudaGetErrorString(e));
    return EMD_ECUDA;
  }
  b->graphs[key] = ex;
  *out = ex;
  return EMD_OK;
}

int batch_check(emd_batch* b) {
  if (!b) {
    set_err("null batch");
    return EMD_EINVAL;
  }
  return EMD_OK;
}

}  // namespace

extern "C" {

emd_batch* emd_batch_create(int max_jobs) {
  if (max_jobs < 1 || max_jobs > 4096) {
    set_err("emd_batch_create: max_jobs must be in [1, 4096]");
    return nullptr;
  }
  emd_batch* b = new emd_batch();
  b->max_jobs = max_jobs;
  cudaGetDevice(&b->device);
  b->job.assign(max_jobs, nullptr);
  b->remaining.assign(max_jobs, 0);
  const size_t jb = (sizeof(emd::BatchJob) * max_jobs + 255) & ~(size_t)255;
  const size_t ib = (sizeof(int2) * (size_t)kBatchItemCap + 255) & ~(size_t)255;
  const size_t fjb = (sizeof(emd::FftBatchJob) * max_jobs + 255) & ~(size_t)255;
  const size_t total = jb + ib + 1024 + fjb + ib + 1024;
  void* p = nullptr;
  if (cudaMalloc(&p, total) != cudaSuccess) {
    cudaGetLastError();
    set_err("emd_batch_create: out of device memory");
    delete b;
    return nullptr;
  }
  b->arena = static_cast<char*>(p);
  b->d_jobs = reinterpret_cast<emd::BatchJob*>(b->arena);
  b->d_items = reinterpret_cast<int2*>(b->arena + jb);
  b->d_nitems = reinterpret_cast<int*>(b->arena + jb + ib);
  b->d_counter = reinterpret_cast<int*>(b->arena + jb + ib + 256);
  b->d_err = reinterpret_cast<int*>(b->arena + jb + ib + 512);
  char* fa = b->arena + jb + ib + 1024;
  b->d_fjobs = reinterpret_cast<emd::FftBatchJob*>(fa);
  b->d_fitems = reinterpret_cast<int2*>(fa + fjb);
  b->d_fnitems = reinterpret_cast<int*>(fa + fjb + ib);
  b->d_fcounters = reinterpret_cast<int*>(fa + fjb + ib + 256);
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->fft_ctas = sms > 0 ? sms : 1;  // one persistent FFT CTA per SM
  }
  b->smem = emd::batch_smem_bytes();
  b->max_clusters = emd::batch_max_clusters(b->smem);
  for (int cfg = 0; cfg < emd::kHaloTileConfigs; ++cfg) b->halo_ctas[cfg] = emd::halo_batch_ctas(cfg);
  if (b->max_clusters <= 0 || b->halo_ctas[0] <= 0) {
    set_err("emd_batch_create: the persistent kernels cannot be resident");
    cudaFree(b->arena);
    delete b;
    return nullptr;
  }
  {
    // halo-exchange jobs: table, work list, item count, claim counters
    const size_t hjb = (sizeof(emd::HaloBatchJob) * max_jobs + 255) & ~(size_t)255;
    const size_t hib = sizeof(int2) * (size_t)kHaloItemCap;
    void* hp = nullptr;
    if (cudaMalloc(&hp, hjb + hib + 512) != cudaSuccess) {
      cudaGetLastError();
      set_err("emd_batch_create: out of device memory");
      cudaFree(b->arena);
      delete b;
      return nullptr;
    }
    b->harena = static_cast<char*>(hp);
    b->d_hjobs = reinterpret_cast<emd::HaloBatchJob*>(b->harena);
    b->d_hitems = reinterpret_cast<int2*>(b->harena + hjb);
    b->d_hnitems = reinterpret_cast<int*>(b->harena + hjb + hib);
    b->d_hctrl = reinterpret_cast<unsigned long long*>(b->harena + hjb + hib + 256);
  }
  b->cur.clusters = b->max_clusters;
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
    set_err("emd_batch_create: stream creation failed");
    cudaFree(b->arena);
    cudaFree(b->harena);
    delete b;
    return nullptr;
  }
  b->own_stream = true;
  // zeroed on the batch's own stream, ahead of every table upload and step
  if (cudaMemsetAsync(b->arena, 0, total, b->st) != cudaSuccess ||
      cudaMemsetAsync(b->harena, 0, (size_t)(reinterpret_cast<char*>(b->d_hitems) - b->harena),
                      b->st) != cudaSuccess ||
      cudaMemsetAsync(b->d_hnitems, 0, 512, b->st) != cudaSuccess) {
    cudaGetLastError();
    set_err("emd_batch_create: memset failed");
    cudaStreamDestroy(b->st);
    cudaFree(b->arena);
    cudaFree(b->harena);
    delete b;
    return nullptr;
  }
  cudaEventCreate(&b->e0);
  cudaEventCreate(&b->e1);
  return b;
}

void emd_batch_destroy(emd_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  cudaStreamSynchronize(b->st);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  if (b->own_stream) cudaStreamDestroy(b->st);
  cudaEventDestroy(b->e0);
  cudaEventDestroy(b->e1);
  cudaFree(b->arena);
  cudaFree(b->harena);
  delete b;
}

int emd_batch_add(emd_batch* b, emd_ctx* c, int iterations) {
  if (int rc = batch_check(b)) return rc;
  if (int rc = check_ctx(c, true)) return rc;
  if (iterations < 0) {
    set_err("emd_batch_add: iterations must be >= 0");
    return EMD_EINVAL;
  }
  if ((c->prec != EMD_PREC_FP32 && c->prec != EMD_PREC_FP32_PAIR &&
       c->prec != EMD_PREC_FFT_FP32) ||
      c->noise != EMD_NOISE_GAUSSIAN) {
    set_err("emd_batch_add: batched jobs run the FP32 direct or FFT Gaussian-noise forms");
    return EMD_EUNSUPPORTED;
  }
  if (c->device != b->device) {
    set_err("emd_batch_add: job and batch are on different devices");
    return EMD_EINVAL;
  }
  for (int i = 0; i < b->max_jobs; ++i)
    if (b->job[i] == c) {
      set_err("emd_batch_add: job already in the batch");
      return EMD_EINVAL;
    }
  for (int i = 0; i < b->max_jobs; ++i) {
    if (!b->job[i]) {
      // the job's own stream work (set_frames, set_x, its PSF spectra) must
      // be done first
      DeviceGuard dg(c->device);
      if (c->prec == EMD_PREC_FFT_FP32 && !c->fft_ready) {
        CK(emd::launch_fft_spectra(c->s, c->ka, c->fft_spec, c->st));
        c->fft_ready = true;
      }
      if (c->prec == EMD_PREC_FP32) {
        bool ok = false;  // without a ring (too many items) the job runs the CTA-pair form
        if (int rc = ensure_halo_arena(c, &ok)) return rc;
      }
      CK(cudaStreamSynchronize(c->st));
      b->job[i] = c;
      b->remaining[i] = iterations;
      b->dirty = true;
      return i;
    }
  }
  set_err("emd_batch_add: no free slot (max_jobs = %d)", b->max_jobs);
  return EMD_ESTATE;
}

int emd_batch_remove(emd_batch* b, int slot) {
  if (int rc = batch_check(b)) return rc;
  if (slot < 0 || slot >= b->max_jobs || !b->job[slot]) {
    set_err("emd_batch_remove: no job in slot %d", slot);
    return EMD_EINVAL;
  }
  DeviceGuard dg(b->device);
  CK(cudaStreamSynchronize(b->st));
  b->job[slot] = nullptr;
  b->remaining[slot] = 0;
  b->dirty = true;
  return EMD_OK;
}

int emd_batch_remaining(emd_batch* b, int slot) {
  if (int rc = batch_check(b)) return rc;
  if (slot < 0 || slot >= b->max_jobs || !b->job[slot]) {
    set_err("emd_batch_remaining: no job in slot %d", slot);
    return EMD_EINVAL;
  }
  return b->remaining[slot];
}

int emd_batch_step(emd_batch* b, int* finished) {
  if (int rc = batch_check(b)) return rc;
  DeviceGuard dg(b->device);
  if (finished) *finished = 0;
  int active = 0;
  for (int i = 0; i < b->max_jobs; ++i)
    if (b->job[i] && b->remaining[i] > 0) ++active;
  if (!active) return EMD_OK;
  // autotuner: a new composition tries each candidate on one real step
  const std::string sig = composition_signature(b);
  bool timing = false;
  if (sig != b->sig) {
    b->sig = sig;
    b->trying.clear();
    b->trial_ms.clear();
    auto it = b->tuned.find(sig);
    if (it != b->tuned.end()) {
      if (!it->second.same_table(b->cur)) b->dirty = true;
      b->cur = it->second;
    } else {
      // candidates: the FP32 jobs' form (halo-exchange: round-robin or most
      // expensive job first, 64-row tiles; most expensive first on 48-row
      // tiles (three CTAs per SM); CTA pairs: all or 3/4 of the resident
      // pairs)
      const int full = b->max_clusters, part = b->max_clusters - b->max_clusters / 4;
      b->trying.push_back({full, 0, 0, 0});
      b->trying.push_back({full, 1, 0, 0});
      if (b->halo_ctas[1] > 0) b->trying.push_back({full, 1, 0, 1});
      b->trying.push_back({full, 1, 1, 0});
      b->trying.push_back({part, 1, 1, 0});
      b->dirty = true;
    }
  }
  if (!b->trying.empty()) {
    const TuneChoice next = b->trying[b->trial_ms.size()];
    if (!next.same_table(b->cur)) b->dirty = true;
    b->cur = next;
    timing = true;
  }
  if (b->dirty) {
    if (int rc = upload_table(b)) return rc;
    b->dirty = false;
  }
  cudaGraphExec_t ex;
  if (int rc = get_graph(b, b->cur.clusters, &ex)) return rc;
  if (timing) CK(cudaEventRecord(b->e0, b->st));
  CK(cudaGraphLaunch(ex, b->st));
  if (timing) {
    CK(cudaEventRecord(b->e1, b->st));
    CK(cudaEventSynchronize(b->e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->e0, b->e1);
    b->trial_ms.push_back(ms);
    if (b->trial_ms.size() == b->trying.size()) {
      size_t best = 0;
      for (size_t k = 1; k < b->trial_ms.size(); ++k)
        if (b->trial_ms[k] < b->trial_ms[best]) best = k;
      if (!b->trying[best].same_table(b->cur)) b->dirty = true;
      b->cur = b->trying[best];
      b->tuned[b->sig] = b->cur;
      b->trying.clear();
    }
  }
  ++b->steps;
  // host mirror of the advance kernel
  for (int i = 0; i < b->max_jobs; ++i) {
    emd_ctx* c = b->job[i];
    if (!c || b->remaining[i] <= 0) continue;
    b->remaining[i] -= 1;
    c->cur ^= 1;
    if (b->remaining[i] == 0) {
      if (finished) ++*finished;
      b->dirty = true;  // its tiles leave the work list
    }
  }
  return EMD_OK;
}

int emd_batch_sync(emd_batch* b) {
  if (int rc = batch_check(b)) return rc;
  DeviceGuard dg(b->device);
  int h = 0;
  CK(cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
  CK(cudaStreamSynchronize(b->st));
  if (h & emd::kErrTimeout) {
    CK(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st));
    set_err("a bounded device-side wait gave up");
    return EMD_ETIMEOUT;
  }
  return EMD_OK;
}

int emd_batch_config(emd_batch* b, int* clusters, int* order, int* max_clusters, int* form,
                     int* tile_shape) {
  if (int rc = batch_check(b)) return rc;
  if (clusters) *clusters = b->cur.clusters;
  if (order) *order = b->cur.order;
  if (max_clusters) *max_clusters = b->max_clusters;
  if (form) *form = b->cur.form;
  if (tile_shape) *tile_shape = b->cur.tile + 1;
  return EMD_OK;
}

}  // extern "C"
