/*
 * emd.h -- C ABI of the GB300 (sm_103a) EM multi-frame deconvolution library.
 *
 * The library runs the expectation-maximization update of Sec. 2 of
 * Sukurdeep, Navarro & Budavari (arXiv:2302.05804) on one GPU:
 *
 *   Eq. (1)  y_t = f_t * x + eta_t,   eta_t ~ N(0, v_t)        (r = 1)
 *   Eq. (3)  y_t = D^r(h_t * x) + eta_t                        (r > 1)
 *   Eq. (2)  x <- x . max(N, 0) / Den   where Den > 0 (x unchanged elsewhere)
 *              N   = sum_t F_t^T (u_t . y_t)      (once per frame set)
 *              Den = sum_t F_t^T (u_t . F_t x)    (every iteration)
 *            u_t = 1/v_t on valid pixels, 0 on masked pixels.
 *
 * "*" is the zero-padded "same" 2-D convolution with an odd K x K PSF
 * centred at ((K-1)/2, (K-1)/2); F_t^T is the matching correlation; D^r sums
 * r x r blocks of the fine grid and its transpose replicates a coarse pixel
 * over its block.
 *
 * Conventions shared by every call:
 *   - H, W are EXPOSURE sizes. The latent image x is (rH) x (rW).
 *   - All arrays are C order (row-major), densely packed:
 *       y, v   : n x H x W   float32
 *       mask   : n x H x W   uint8, 0 = masked, nonzero = valid (NULL: all valid)
 *       f      : n x K x K   float32 (fine-grid PSFs when r > 1)
 *       x      : (rH) x (rW) float32
 *   - Array arguments may be host or device pointers (CUDA unified
 *     addressing decides). The library copies inputs into device memory it
 *     owns; callers may reuse their buffers once the call returns.
 *   - Work is ordered on the context's stream (emd_set_stream; default: the
 *     legacy default stream). Calls that read back to the host, and calls
 *     given host pointers, synchronise that stream before returning.
 *   - Return codes: EMD_OK (0) or a negative EMD_E* code; emd_last_error()
 *     then describes the failure (thread-local).
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef EMD_H
#define EMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct emd_ctx emd_ctx;

enum emd_status {
    EMD_OK = 0,
    EMD_EINVAL = -1,      /* bad argument (sizes, parity of K, NULL, mode)   */
    EMD_ENOMEM = -2,      /* device allocation failed                        */
    EMD_ECUDA = -3,       /* a CUDA call or kernel failed                    */
    EMD_ESTATE = -4,      /* call out of order (e.g. iterate before frames)  */
    EMD_EDATA = -5,       /* a valid pixel has v <= 0 or a non-finite y or v */
    EMD_ETIMEOUT = -6,    /* a bounded device-side wait gave up              */
    EMD_EUNSUPPORTED = -7 /* configuration not built in this library         */
};

/* Arithmetic of the two convolutions of each iteration (Eq. (2)). */
enum emd_precision {
    EMD_PREC_FP32 = 0,        /* FP32 FMA direct convolution (default)        */
    EMD_PREC_BF16 = 1,        /* tensor cores, BF16 operands, FP32 accumulate */
    EMD_PREC_FP16 = 2,        /* tensor cores, FP16 operands, FP32 accumulate */
    EMD_PREC_SPLIT_BF16 = 3,  /* tensor cores, hi+lo BF16 split, 3 products   */
    EMD_PREC_SPLIT_FP16 = 4,  /* tensor cores, hi+lo FP16 split, 3 products   */
    EMD_PREC_FFT_FP32 = 5,    /* FP32 FFTs, overlap-save on 128 x 128 tiles   */
    EMD_PREC_FP32_PAIR = 6    /* FP32 direct, per-tile CTA-pair kernel        */
};

/* Largest PSF footprint the direct kernels accept: with
 * hc = floor(((K-1)/2 + r - 1) / r), hc must not exceed EMD_MAX_HC. */
#define EMD_MAX_HC 23

/*
 * emd_create -- new context for n exposures of H x W pixels, K x K PSFs
 * (K odd, on the fine grid when r > 1) and super-resolution factor r >= 1
 * (Eq. (3); r = 1 is Eq. (1)). Allocates all device memory the context
 * will use (emd_ctx_bytes reports how much) on the current device.
 * Returns NULL on error (emd_last_error explains): H, W, n < 1, K even or
 * < 1, r < 1, hc > EMD_MAX_HC, or out of device memory.
 */
emd_ctx *emd_create(int H, int W, int n, int psf_k, int r);

/* Device bytes a context of this shape holds (0 for invalid shapes). */
size_t emd_ctx_bytes(int H, int W, int n, int psf_k, int r);

/* The same plus the buffers the mode adds (EMD_PREC_FP32: the w ring of
 * the halo-exchange kernel; the tensor-core operands; the FFT form's
 * spectra, w planes and scratch; nothing for EMD_PREC_FP32_PAIR); 0 for an
 * invalid shape or a mode this shape does not support. Host only. */
size_t emd_ctx_bytes_precision(int H, int W, int n, int psf_k, int r, int mode);

/* Destroy a context and free its device memory. NULL is ignored. */
void emd_destroy(emd_ctx *ctx);

/* Thread-local description of the last error ("" if none). */
const char *emd_last_error(void);

/* Order all later work of ctx on `stream` (a cudaStream_t; NULL = legacy
 * default stream). Work already queued on the previous stream completes
 * before anything later queued on the new one (an event hand-off; the call
 * does not block). The library never synchronises the device, only this
 * stream. */
int emd_set_stream(emd_ctx *ctx, void *stream);

/*
 * emd_set_frames -- load a frame set (Sec. 2: exposures y, PSFs f and
 * variance maps v, plus per-pixel masks) and prepare the iteration:
 *   u_t = mask ? 1/v_t : 0,  N = sum_t F_t^T (u_t . y_t),
 *   the constant sum of log(2 pi v) of the log-likelihood, and the default
 *   start x^(0) = c with c = (sum u y / sum u) / r^2 when positive, else 1
 *   (Sec. 2 only asks for a strictly positive start).
 * y, v: n x H x W; f: n x K x K; mask: n x H x W or NULL. Masked pixels of y
 * and v may hold anything (NaN included); they are never read
 * arithmetically. A valid pixel with v <= 0 or non-finite y or v fails with
 * EMD_EDATA (the context keeps no frames then).
 */
int emd_set_frames(emd_ctx *ctx, const float *y, const float *v,
                   const float *f, const uint8_t *mask);

/* Replace the current iterate by x0 ((rH) x (rW)). Negative entries are
 * taken as 0. Requires frames. */
int emd_set_x(emd_ctx *ctx, const float *x0);

/* Run k >= 0 iterations of Eq. (2) on the current iterate (stream-ordered,
 * asynchronous). A bounded device-side wait that gives up (the FP32
 * halo-exchange kernel's dependency waits; the FFT form's split launch,
 * where part of a tile waits for the part before it) sets the context's
 * error word: the next emd_get_x or emd_loglik returns EMD_ETIMEOUT, and the
 * iterate is then not valid (set it again with emd_set_x); the context's
 * wait state is cleared for the next iterations. */
int emd_iterate(emd_ctx *ctx, int k);

/* Streaming (frame-by-frame) EM, the order-dependent alternative the paper
 * contrasts with its simultaneous update (Sec. 1 and the remarks after
 * Eq. (2), after Harmeling et al.): each of k passes updates x once per
 * exposure t, in the given order, with that exposure alone:
 *   x <- x . max(F_t^T(u_t y_t), 0) / F_t^T(u_t F_t x)
 * (x unchanged where the denominator is 0). order: a permutation of
 * 0..n-1, or NULL for ascending. The per-exposure numerators are computed
 * on the first call after emd_set_frames (n latent planes of device memory,
 * allocated then). Runs the FP32 direct halo-exchange kernel whatever the
 * precision (the CTA-pair kernel under EMD_PREC_FP32_PAIR; same iterates). */
int emd_iterate_streaming(emd_ctx *ctx, int k, const int *order);

/* Copy the current iterate to out ((rH) x (rW) float32). */
int emd_get_x(emd_ctx *ctx, float *out);

/*
 * emd_loglik -- log-likelihood of the current iterate under Eq. (1)/(3):
 *   l = -1/2 sum_{t,i valid} [ u (y - z)^2 + log(2 pi v) ],  z = D^r(f_t * x),
 * accumulated in FP64, into *out. Synchronises the stream.
 * emd_loglik_chi2 does the same and also returns the data term
 * sum u (y-z)^2 in *chi2 (when chi2 is not NULL).
 */
int emd_loglik(emd_ctx *ctx, double *out);
int emd_loglik_chi2(emd_ctx *ctx, double *out, double *chi2);

/* Select the convolution arithmetic (enum emd_precision). Modes not built
 * into this library return EMD_EUNSUPPORTED and leave the mode unchanged.
 * EMD_PREC_FFT_FP32 computes the forward model and the adjoint of each
 * iteration by FP32 FFTs (overlap-save: output tiles of 128 - 2 hc pixels,
 * hc = floor(((K-1)/2 + r - 1) / r), transformed as 128 x 128 real tiles
 * of the polyphase planes); it needs n extra exposure planes of device
 * memory for the weighted model images u_t z_t and, for r > 1, a per-tile
 * scratch of r^2 spectra (66.5 KB each), allocated on first selection.
 * EMD_PREC_FP32 (Gaussian noise) runs one persistent kernel per iteration
 * that computes each pixel's forward model once and passes the weighted
 * model images u_t z_t between 64 x 128 tiles through a ring of tile
 * buffers in device memory (about 1030 tiles of 32 KB at 4096^2, fewer for
 * smaller images; emd_ctx_bytes_precision counts them), allocated at the
 * first such iteration. EMD_PREC_FP32_PAIR gives the same iterates bit for
 * bit from the kernel that keeps u_t z_t in the shared memory of a CTA
 * pair per tile and recomputes the forward model on a 2 hc halo around it
 * (no extra memory, 1.48x the multiply-adds at K = 43). emd_loglik
 * computes the forward model once per pixel in every mode except
 * EMD_PREC_FP32_PAIR. */
int emd_set_precision(emd_ctx *ctx, int mode);

/*
 * Noise model of the likelihood (Sec. 3's outlook: heavier-tailed noise
 * terms for robustness to outliers such as satellite trails).
 * EMD_NOISE_GAUSSIAN (default): Eq. (1), update Eq. (2).
 * EMD_NOISE_STUDENT_T: y_t - D^r(f_t * x) = sqrt(v_t) e, e Student-t with nu
 * degrees of freedom. Each emd_iterate step is then a generalised EM step:
 * with z_t = D^r(f_t * x) and weights u' = u (nu+1) / (nu + u (y - z)^2)
 * (the expected precision scale of the Gaussian scale mixture),
 *   x <- x . max(sum_t F_t^T(u'_t y_t), 0) / sum_t F_t^T(u'_t z_t)
 * (x unchanged where the denominator is 0); it never lowers the Student-t
 * likelihood, and tends to Eq. (2) as nu grows. It costs one forward and
 * two adjoint passes per iteration (Eq. (2): one each; under
 * EMD_PREC_FP32_PAIR two of each). emd_loglik then
 * returns the Student-t log-likelihood
 *   sum_valid [lgamma((nu+1)/2) - lgamma(nu/2) - 1/2 log(nu pi v)
 *              - (nu+1)/2 log(1 + u (y - z)^2 / nu)]
 * and *chi2 = sum_valid (nu+1) log(1 + u (y - z)^2 / nu).
 * nu: finite, in (0, 1e30] (ignored for the Gaussian model). The heavy-tailed
 * model runs on the FP32 direct forms (EMD_PREC_FP32: its w ring then holds
 * two tiles per slot, re-allocated at the next emd_iterate) and the FFT form
 * (which then keeps n more exposure planes, of u'y, and a larger per-tile
 * scratch, allocated at the next emd_set_precision or emd_iterate):
 * EMD_EUNSUPPORTED with a tensor-core precision, in emd_iterate_streaming
 * and in emd_batch_add.
 */
enum emd_noise {
    EMD_NOISE_GAUSSIAN = 0,
    EMD_NOISE_STUDENT_T = 1
};
int emd_set_noise(emd_ctx *ctx, int model, double nu);

/* Tile shape of the FP32 halo-exchange iteration (EMD_PREC_FP32). Its 128
 * threads compute a tile of rows x 128 pixels, each thread a (rows/16) x 16
 * block of outputs:
 *   EMD_TILE_64         64 rows, two CTAs per SM
 *   EMD_TILE_48         48 rows, three CTAs per SM (at most 168 registers)
 *   EMD_TILE_32         32 rows, four CTAs per SM where the shared memory allows
 * EMD_TILE_AUTO (the default) lets the autotuner choose: the first
 * iterations of a problem shape (H, W, n, K, r, noise model) not seen before
 * in this process run each candidate twice, timed with CUDA events on the
 * context's stream and read without blocking at later calls, and the
 * fastest is kept for every context of that problem shape. All tile shapes
 * give the same iterates bit for bit (every output sums its taps in the same
 * order). EMD_EINVAL for another value. */
enum emd_tile_shape {
    EMD_TILE_AUTO = 0,
    EMD_TILE_64 = 1,
    EMD_TILE_48 = 2,
    EMD_TILE_32 = 3
};
int emd_set_tile_shape(emd_ctx *ctx, int shape);
/* The tile shape the next FP32 iteration uses (an emd_tile_shape other than
 * EMD_TILE_AUTO), and *decided = 1 once the autotuner has decided (or the
 * shape was fixed); either pointer may be NULL. */
int emd_get_tile_shape(emd_ctx *ctx, int *shape, int *decided);

/* Self-test of failure detection: launches, on ctx's stream, one CTA that
 * waits on an mbarrier nothing ever arrives on, with the same bounded-wait
 * code the kernels use but a limit of `spins` polls. The wait gives up, the
 * kernel records the timeout in the context's device error word and exits.
 * Then one thread waits, the same way as the halo-exchange kernel's
 * dependency waits, for a counter nothing increments (`spins` polls), and
 * once more after giving up: that second wait must return at once because
 * the first raised the kernel's abort flag. The call returns EMD_ETIMEOUT
 * (the expected outcome) when both behave, and clears the word, leaving the
 * context usable. EMD_OK would mean a wait did not give up. */
int emd_selftest_wait_timeout(emd_ctx *ctx, int spins);

/* Inspection: the numerator N ((rH) x (rW)) and the weights u (n x H x W)
 * prepared by emd_set_frames. */
int emd_get_numerator(emd_ctx *ctx, float *out);
int emd_get_weights(emd_ctx *ctx, float *out);

/* ---------------------------------------------------------------------------
 * Batching: many deconvolution jobs (contexts of any shapes) advance one EM
 * iteration per emd_batch_step. FP32 direct jobs run in ONE persistent
 * launch of the halo-exchange kernel whose work list merges every job's
 * (forward, adjoint) x (exposure, tile) items, each job keeping its own
 * order and w ring (EMD_PREC_FP32), or of the CTA-pair kernel, whose pairs
 * claim (job, 128 x 128 tile) items (EMD_PREC_FP32_PAIR); FFT-form jobs
 * run in persistent FFT forward and adjoint launches. The step (persistent
 * kernels, per-job advance) is captured once as a CUDA graph and replayed.
 * Jobs may join or leave between steps (continuous batching); a job gives
 * bit-for-bit the same iterates in a batch as with emd_iterate alone.
 *
 * An online autotuner picks, per job mix (a signature of the active jobs'
 * size class, Kc, r, exposure count and mode), the FP32 jobs' kernel form,
 * tile shape and work order and the resident CTA count: the first steps of
 * a new mix each run one candidate (halo-exchange kernel on 64-row tiles
 * with jobs interleaved round-robin or most expensive first, or on 48-row
 * tiles; CTA pairs, all or 3/4 resident), timed with CUDA events, and the
 * fastest is kept. Heavy-tailed noise is not batched.
 * -------------------------------------------------------------------------*/
typedef struct emd_batch emd_batch;

/* New batch with room for max_jobs (1..4096) jobs; NULL on error. The batch
 * runs on a stream of its own. */
emd_batch *emd_batch_create(int max_jobs);
void emd_batch_destroy(emd_batch *b);

/* Add a context that has frames (and, optionally, a start from emd_set_x)
 * to run `iterations` more iterations. Returns the slot (>= 0) or a negative
 * EMD_E* code. The context must not be iterated on its own while it is in
 * the batch. */
int emd_batch_add(emd_batch *b, emd_ctx *job, int iterations);

/* Remove the job in `slot` (finished or not); its context keeps the iterate
 * reached so far. */
int emd_batch_remove(emd_batch *b, int slot);

/* One iteration for every job that has iterations left (asynchronous on the
 * batch stream). *finished (may be NULL) receives the number of jobs that
 * ran their last iteration in this step. */
int emd_batch_step(emd_batch *b, int *finished);

/* Iterations left for the job in `slot` (0 when finished), or an error. */
int emd_batch_remaining(emd_batch *b, int slot);

/* Wait for all queued steps; call before reading a job's results with
 * emd_get_x / emd_loglik. EMD_ETIMEOUT if a bounded device wait gave up. */
int emd_batch_sync(emd_batch *b);

/* The autotuner's current choice: resident CTA pairs, work order (0 =
 * job-major, or round-robin over jobs in the halo-exchange form; 1 = most
 * expensive jobs first), the maximum pairs, the FP32 jobs' form (0 =
 * halo-exchange kernel, 1 = CTA-pair kernel) and the halo-exchange kernel's
 * tile shape (an emd_tile_shape). Any pointer may be NULL. */
int emd_batch_config(emd_batch *b, int *clusters, int *order, int *max_clusters, int *form,
                     int *tile_shape);

/*
 * emd_frame_stats_noalloc -- per-exposure FP64 frame statistics without any
 * device allocation. The paper has no counterpart: this exists for callers
 * that cannot call cudaMalloc (work issued during CUDA-graph stream capture,
 * real-time pipelines that reserve device memory up front, frameworks that
 * own all device memory through their own allocator).
 *
 * Inputs are caller-owned DEVICE buffers in natural layout: y, v (n x H x W
 * float32) and mask (n x H x W uint8, 0 = masked) or NULL. The output out
 * is a caller-owned DEVICE buffer of n x 4 doubles; for exposure t:
 *   out[4t+0] = sum over valid pixels of log(2 pi v)
 *   out[4t+1] = sum over valid pixels of u y,  u = 1/v (FP32 reciprocal)
 *   out[4t+2] = sum over valid pixels of u
 *   out[4t+3] = number of valid pixels with v <= 0 or non-finite y or v
 *               (they are left out of the three sums)
 * These are the statistics emd_set_frames computes for a context.
 *
 * Work is queued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * and the call returns without synchronising. Scratch lives in one
 * fixed-size array inside the library's device image (room for
 * EMD_NOALLOC_MAX_EXPOSURES exposures; every GPU that loads the library
 * holds it until the process exits). n > EMD_NOALLOC_MAX_EXPOSURES is
 * rejected with EMD_EINVAL, as are NULL or host pointers, device memory of a
 * GPU other than the current one, and sizes < 1. The C side cannot check
 * buffer sizes: y and v must hold n*H*W floats, mask n*H*W bytes and out
 * 4*n doubles.
 * The first call on a device looks up the scratch array's device address;
 * make that first call before any stream capture. All calls share the one
 * scratch array, so calls that overlap on the GPU (concurrent streams or
 * threads) race and must be serialised by the caller.
 */
#define EMD_NOALLOC_MAX_EXPOSURES 64
int emd_frame_stats_noalloc(const float *y, const float *v, const uint8_t *mask,
                            int H, int W, int n, double *out, void *stream);

/*
 * emd_fit_psf -- super-resolved PSFs of Eq. (4) (Sec. 2): for each of the n
 * coarse PSFs f_t (K x K, odd K) find the fine PSF
 *   h_t = argmin_{h >= 0} sum_ij ([D^r(h * g)]_ij - f_t,ij)^2
 *                         + lambda sum_ij (grad h)_ij^2
 * by `iters` steps of projected Adam (bias-corrected, beta1 0.9, beta2
 * 0.999, epsilon 1e-8, step `lr`; h is clipped to >= 0 after every step).
 * Adam at a fixed step is not monotone, so the result is the iterate of
 * lowest Eq. (4) loss among h_0 .. h_iters (the first on ties), with the
 * loss evaluated in FP32 on the device.
 * h_t has Kh = r (K-1) + 1 fine pixels per side (odd), fine pixel P lying
 * in coarse pixel P div r, so it is directly the K = Kh PSF of an r x r
 * super-resolution context (emd_create(..., Kh, r)). h * g is the
 * zero-padded 'same' convolution on the Kh x Kh grid, zero-extended to
 * rK x rK before the block sum D^r; (grad h)^2 is the sum of squared
 * forward differences inside the grid.
 *
 * f: n x K x K float32, row-major; g: Kg x Kg float32 (odd Kg, the
 * broadening kernel of Eq. (4), e.g. a Gaussian whose FWHM is one coarse
 * pixel); h0: n x Kh x Kh start, or NULL for the coarse PSF spread evenly
 * over each block (h0[P][Q] = f[P div r][Q div r] / r^2); h_out: n x Kh x Kh;
 * loss_out: n floats (the Eq. (4) loss at the returned h, FP32) or NULL.
 * h_out also serves as the store of the best iterate during the fit.
 * Every buffer may be host or device memory (caller-owned; host buffers are
 * staged through a temporary device allocation, which also holds the Adam
 * moments). One CTA fits one PSF, with h, the residual, f and g resident in
 * its shared memory for all iterations; the call runs on the legacy default
 * stream and returns when the fit is done.
 * Errors: EMD_EINVAL for NULL f/g/h_out, even K or Kg, r outside 1..8, K
 * above EMD_PSF_MAX_COARSE, Kg above EMD_PSF_MAX_KG, iters < 0, lambda < 0
 * or lr <= 0; EMD_EUNSUPPORTED when Kh is too large for one CTA's shared
 * memory (two zero-haloed planes of (Kh + Kg - 1)^2 floats plus 2 K^2 +
 * 2 Kg^2 floats above 220 KB; Kh up to about 160 fits, e.g. K = 43 with
 * r = 2 or 3); EMD_ENOMEM / EMD_ECUDA on device failures.
 */
#define EMD_PSF_MAX_COARSE 127
#define EMD_PSF_MAX_KG 15
int emd_fit_psf(const float *f, int n, int K, int r, const float *g, int Kg,
                const float *h0, float lambda, float lr, int iters, float *h_out,
                float *loss_out);

/*
 * emd_measure_fma_rate -- the FP32 FMA rate of the current GPU, measured:
 * independent FMA chains in 8 blocks of 256 threads per SM, `iters` rounds
 * of 128 FMAs per thread, one timed launch after a warm-up, on a private
 * stream (blocks until done). *tflops = 2 x FMAs / s / 1e12. The paper has
 * no counterpart: this is the denominator of the direct kernel's roofline.
 * EMD_EINVAL for NULL tflops or iters < 1; EMD_ECUDA on CUDA failures.
 */
int emd_measure_fma_rate(int iters, double *tflops);

#ifdef __cplusplus
}
#endif

#endif /* EMD_H */
