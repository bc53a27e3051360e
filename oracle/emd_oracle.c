/*
 * emd_oracle.c -- plain FP64 CPU oracle of the EM multi-frame deconvolution
 * update (Sukurdeep, Navarro & Budavari, "A Flexible Expectation
 * Maximization Framework for Fast, Scalable and High-fidelity Multi-frame
 * Astronomical Image Deconvolution", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY. This is the slow, obviously correct reference
 * that the CUDA library is checked against. Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark load it; the product path never
 * does. It shares no code, header, table or constant with the CUDA library.
 *
 * Every function is a direct transcription of a definition; there is no
 * blocking, fusion or reordering. Arrays are C order, double precision.
 *
 * Definitions (the readings of the paper are listed beside each function):
 *
 *   Eq. (1)   y_t = f_t * x + eta_t,  eta_t ~ N(0, v_t) per pixel.
 *             "*" is the zero-padded "same" 2-D convolution with an odd
 *             K x K kernel centred at (h, h), h = (K-1)/2:
 *               (f*x)[i][j] = sum_{a,b} f[a][b] x[i+h-a][j+h-b].
 *   F_t       the linear operator with F_t x = f_t * x (Sec. 2, after
 *             Eq. (2)); its transpose is the correlation
 *               (F^T w)[p][q] = sum_{a,b} f[a][b] w[p-h+a][q-h+b].
 *   Eq. (3)   super-resolution: y_t = D^r(h_t * x) + eta_t with x on an
 *             (rH) x (rW) grid and D^r the r x r block SUM; its transpose
 *             replicates a coarse pixel over its r x r block.
 *   Eq. (2)   multiplicative update with u_t = 1/v_t, read with the weights
 *             applied on the exposure grid between F_t and F_t^T:
 *               N   = sum_t F_t^T (u_t . y_t)
 *               Den = sum_t F_t^T (u_t . F_t x)
 *               x'  = Den > 0 ? x . max(N, 0) / Den : x
 *             (the literal placement, u_t outside F_t^T, is kept as
 *             oracle_em_step_literal for r = 1).
 *   masks     u_t = 0 where the mask is 0; masked pixels of y and v are
 *             never read arithmetically.
 *   log-lik   l(x) = -1/2 sum_{t,i: m != 0} [ u (y - z)^2 + log(2 pi v) ],
 *             z = D^r(f_t * x), from the Gaussian model of Eq. (1).
 *
 * Parity unpinned: none -- every function is pinned by the CPU tests
 * (library convolutions, adjoint identity, closed forms, fixed points,
 * monotone likelihood, NNLS limit, dense brute force).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ----------------------------------------------------------------------- */
/* Operators of Eq. (1) and Eq. (3)                                         */
/* ----------------------------------------------------------------------- */

/* (f*x)[i][j] = sum_{a,b} f[a][b] x[i+h-a][j+h-b]; x = 0 outside the image. */
void oracle_conv_same(const double *x, int H, int W, const double *f, int K,
                      double *out)
{
    const int h = (K - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; i++) {
        for (int j = 0; j < W; j++) {
            double s = 0.0;
            for (int a = 0; a < K; a++) {
                int ii = i + h - a;
                if (ii < 0 || ii >= H) continue;
                for (int b = 0; b < K; b++) {
                    int jj = j + h - b;
                    if (jj < 0 || jj >= W) continue;
                    s += f[a * K + b] * x[(long)ii * W + jj];
                }
            }
            out[(long)i * W + j] = s;
        }
    }
}

/* (F^T w)[p][q] = sum_{a,b} f[a][b] w[p-h+a][q-h+b]; w = 0 outside. */
void oracle_corr_same(const double *w, int H, int W, const double *f, int K,
                      double *out)
{
    const int h = (K - 1) / 2;
#pragma omp parallel for schedule(static)
    for (int p = 0; p < H; p++) {
        for (int q = 0; q < W; q++) {
            double s = 0.0;
            for (int a = 0; a < K; a++) {
                int ii = p - h + a;
                if (ii < 0 || ii >= H) continue;
                for (int b = 0; b < K; b++) {
                    int jj = q - h + b;
                    if (jj < 0 || jj >= W) continue;
                    s += f[a * K + b] * w[(long)ii * W + jj];
                }
            }
            out[(long)p * W + q] = s;
        }
    }
}

/* D^r: coarse (i,j) = sum_{s,t < r} fine (r i + s, r j + t). zf is rH x rW. */
void oracle_downsample(const double *zf, int H, int W, int r, double *out)
{
    const long Wf = (long)r * W;
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W; j++) {
            double s = 0.0;
            for (int a = 0; a < r; a++)
                for (int b = 0; b < r; b++)
                    s += zf[((long)r * i + a) * Wf + (long)r * j + b];
            out[(long)i * W + j] = s;
        }
}

/* (D^r)^T: fine (p,q) = coarse (p div r, q div r). out is rH x rW. */
void oracle_upsample(const double *w, int H, int W, int r, double *out)
{
    const long Wf = (long)r * W;
    for (long p = 0; p < (long)r * H; p++)
        for (long q = 0; q < Wf; q++)
            out[p * Wf + q] = w[(p / r) * W + q / r];
}

/* Forward model of one exposure: z = D^r(f * x); x is (rH) x (rW), z is
 * H x W. Eq. (1) for r = 1, Eq. (3) for r > 1. */
void oracle_forward(const double *x, int H, int W, int r, const double *f,
                    int K, double *z)
{
    if (r == 1) {
        oracle_conv_same(x, H, W, f, K, z);
        return;
    }
    double *zf = (double *)malloc(sizeof(double) * (size_t)r * r * H * W);
    oracle_conv_same(x, r * H, r * W, f, K, zf);
    oracle_downsample(zf, H, W, r, z);
    free(zf);
}

/* Transpose of the forward model: out = F^T (D^r)^T w; w is H x W, out is
 * (rH) x (rW). */
void oracle_adjoint(const double *w, int H, int W, int r, const double *f,
                    int K, double *out)
{
    if (r == 1) {
        oracle_corr_same(w, H, W, f, K, out);
        return;
    }
    double *wf = (double *)malloc(sizeof(double) * (size_t)r * r * H * W);
    oracle_upsample(w, H, W, r, wf);
    oracle_corr_same(wf, r * H, r * W, f, K, out);
    free(wf);
}

/* ----------------------------------------------------------------------- */
/* Weights, numerator, update (Eq. (2))                                     */
/* ----------------------------------------------------------------------- */

/* u = 1/v where mask != 0, u = 0 where mask == 0 (mask may be NULL: all
 * valid). Returns the number of valid pixels with v <= 0, v or y not finite
 * (y may be NULL). Those pixels get u = 0 as well. */
long oracle_weights(const double *v, const double *y,
                    const unsigned char *mask, long npix, double *u)
{
    long bad = 0;
    for (long i = 0; i < npix; i++) {
        int valid = mask ? (mask[i] != 0) : 1;
        if (!valid) {
            u[i] = 0.0;
            continue;
        }
        if (!(v[i] > 0.0) || !isfinite(v[i]) || (y && !isfinite(y[i]))) {
            bad++;
            u[i] = 0.0;
            continue;
        }
        u[i] = 1.0 / v[i];
    }
    return bad;
}

/* N = sum_t F_t^T (u_t . y_t), t ascending. y, u: n x H x W; f: n x K x K;
 * N: (rH) x (rW). Masked pixels (u = 0) contribute nothing and their y is
 * not read. */
void oracle_numerator(const double *y, const double *u, const double *f,
                      int n, int H, int W, int K, int r, double *N)
{
    const long np = (long)H * W, nf = (long)r * r * H * W;
    double *w = (double *)malloc(sizeof(double) * np);
    double *a = (double *)malloc(sizeof(double) * nf);
    memset(N, 0, sizeof(double) * nf);
    for (int t = 0; t < n; t++) {
        for (long i = 0; i < np; i++)
            w[i] = (u[t * np + i] != 0.0) ? u[t * np + i] * y[t * np + i] : 0.0;
        oracle_adjoint(w, H, W, r, f + (long)t * K * K, K, a);
        for (long i = 0; i < nf; i++) N[i] += a[i];
    }
    free(w);
    free(a);
}

/* Den = sum_t F_t^T (u_t . F_t x), t ascending. */
void oracle_denominator(const double *x, const double *u, const double *f,
                        int n, int H, int W, int K, int r, double *Den)
{
    const long np = (long)H * W, nf = (long)r * r * H * W;
    double *z = (double *)malloc(sizeof(double) * np);
    double *a = (double *)malloc(sizeof(double) * nf);
    memset(Den, 0, sizeof(double) * nf);
    for (int t = 0; t < n; t++) {
        const double *ft = f + (long)t * K * K;
        oracle_forward(x, H, W, r, ft, K, z);
        for (long i = 0; i < np; i++) z[i] *= u[t * np + i];
        oracle_adjoint(z, H, W, r, ft, K, a);
        for (long i = 0; i < nf; i++) Den[i] += a[i];
    }
    free(z);
    free(a);
}

/* x' = Den > 0 ? x max(N,0) / Den : x, element-wise. */
void oracle_apply_update(double *x, const double *N, const double *Den,
                         long nf)
{
    for (long i = 0; i < nf; i++)
        if (Den[i] > 0.0)
            x[i] = x[i] * fmax(N[i], 0.0) / Den[i];
}

/* One EM iteration of Eq. (2) in place on x ((rH) x (rW)); N from
 * oracle_numerator. Den is returned in den_out when it is not NULL. */
void oracle_em_step(double *x, const double *N, const double *u,
                    const double *f, int n, int H, int W, int K, int r,
                    double *den_out)
{
    const long nf = (long)r * r * H * W;
    double *Den = den_out ? den_out : (double *)malloc(sizeof(double) * nf);
    oracle_denominator(x, u, f, n, H, W, K, r, Den);
    oracle_apply_update(x, N, Den, nf);
    if (!den_out) free(Den);
}

/* k EM iterations. */
void oracle_em_run(double *x, const double *N, const double *u,
                   const double *f, int n, int H, int W, int K, int r, int k)
{
    for (int it = 0; it < k; it++)
        oracle_em_step(x, N, u, f, n, H, W, K, r, NULL);
}

/* Eq. (2) with the weights placed literally (outside F^T, r = 1 only):
 *   x' = x . sum_t u_t . (F_t^T y_t) / sum_t u_t . (F_t^T F_t x).
 * Masked y is taken as 0 inside F_t^T y_t. */
void oracle_em_step_literal(double *x, const double *y, const double *u,
                            const unsigned char *mask, const double *f,
                            int n, int H, int W, int K)
{
    const long np = (long)H * W;
    double *num = (double *)calloc(np, sizeof(double));
    double *den = (double *)calloc(np, sizeof(double));
    double *tmp = (double *)malloc(sizeof(double) * np);
    double *tmp2 = (double *)malloc(sizeof(double) * np);
    for (int t = 0; t < n; t++) {
        const double *ft = f + (long)t * K * K;
        for (long i = 0; i < np; i++) {
            int valid = mask ? (mask[t * np + i] != 0) : 1;
            tmp[i] = valid ? y[t * np + i] : 0.0;
        }
        oracle_corr_same(tmp, H, W, ft, K, tmp2);
        for (long i = 0; i < np; i++) num[i] += u[t * np + i] * tmp2[i];
        oracle_conv_same(x, H, W, ft, K, tmp);
        oracle_corr_same(tmp, H, W, ft, K, tmp2);
        for (long i = 0; i < np; i++) den[i] += u[t * np + i] * tmp2[i];
    }
    oracle_apply_update(x, num, den, np);
    free(num);
    free(den);
    free(tmp);
    free(tmp2);
}

/* Streaming (frame-by-frame) EM, the order-dependent scheme the paper
 * contrasts with Eq. (2) (Sec. 1 and the remarks after Eq. (2)): one pass
 * updates x once per exposure, in the given order, each time with that
 * exposure alone: x' = Den_t > 0 ? x max(N_t, 0) / Den_t : x with
 * N_t = F_t^T(u_t y_t), Den_t = F_t^T(u_t F_t x). y must be 0 where u = 0. */
void oracle_em_pass_streaming(double *x, const double *y, const double *u,
                              const double *f, int n, int H, int W, int K,
                              int r, const int *order)
{
    const long np = (long)H * W, nf = (long)r * r * H * W;
    double *Nt = (double *)malloc(sizeof(double) * nf);
    double *Dt = (double *)malloc(sizeof(double) * nf);
    for (int q = 0; q < n; q++) {
        const int t = order ? order[q] : q;
        oracle_numerator(y + t * np, u + t * np, f + (long)t * K * K, 1, H, W,
                         K, r, Nt);
        oracle_denominator(x, u + t * np, f + (long)t * K * K, 1, H, W, K, r,
                           Dt);
        oracle_apply_update(x, Nt, Dt, nf);
    }
    free(Nt);
    free(Dt);
}

/* ----------------------------------------------------------------------- */
/* Heavy-tailed noise (the outlook of Sec. 3: heavier-tailed noise terms)   */
/* ----------------------------------------------------------------------- */
/*
 * Reading: y_t = D^r(f_t * x) + sqrt(v_t) e, e Student-t with nu degrees of
 * freedom, written as a Gaussian scale mixture (e | s ~ N(0, 1/s),
 * s ~ Gamma(nu/2, rate nu/2)). The E-step gives each valid pixel the
 * expected precision scale E[s | y, x] = (nu + 1) / (nu + u (y - z)^2); the
 * weighted least-squares problem with weights u' = u E[s] is then majorised
 * exactly as in Eq. (2), so one step is
 *   N' = sum_t F_t^T(u'_t y_t), Den' = sum_t F_t^T(u'_t z_t),
 *   x' = Den' > 0 ? x max(N', 0) / Den' : x,
 * a generalised EM step: it does not decrease the Student-t likelihood. As
 * nu -> infinity, u' -> u and the step becomes Eq. (2).
 */

/* u' = u (nu + 1) / (nu + u (y - z)^2) where u != 0, else 0. */
void oracle_student_weights(const double *y, const double *u, const double *z,
                            long np, double nu, double *w)
{
    for (long i = 0; i < np; i++) {
        if (u[i] != 0.0) {
            const double d = y[i] - z[i];
            w[i] = u[i] * (nu + 1.0) / (nu + u[i] * d * d);
        } else {
            w[i] = 0.0;
        }
    }
}

/* One heavy-tailed EM step in place on x; N' and Den' are returned in
 * num_out / den_out when they are not NULL. y must be finite where u != 0. */
void oracle_em_step_student(double *x, const double *y, const double *u,
                            const double *f, int n, int H, int W, int K, int r,
                            double nu, double *num_out, double *den_out)
{
    const long np = (long)H * W, nf = (long)r * r * H * W;
    double *Num = num_out ? num_out : (double *)malloc(sizeof(double) * nf);
    double *Den = den_out ? den_out : (double *)malloc(sizeof(double) * nf);
    double *z = (double *)malloc(sizeof(double) * np);
    double *w = (double *)malloc(sizeof(double) * np);
    double *b = (double *)malloc(sizeof(double) * np);
    double *a = (double *)malloc(sizeof(double) * nf);
    memset(Num, 0, sizeof(double) * nf);
    memset(Den, 0, sizeof(double) * nf);
    for (int t = 0; t < n; t++) {
        const double *ft = f + (long)t * K * K;
        const double *yt = y + t * np, *ut = u + t * np;
        oracle_forward(x, H, W, r, ft, K, z);
        oracle_student_weights(yt, ut, z, np, nu, w);
        for (long i = 0; i < np; i++) b[i] = (w[i] != 0.0) ? w[i] * yt[i] : 0.0;
        oracle_adjoint(b, H, W, r, ft, K, a);
        for (long i = 0; i < nf; i++) Num[i] += a[i];
        for (long i = 0; i < np; i++) b[i] = w[i] * z[i];
        oracle_adjoint(b, H, W, r, ft, K, a);
        for (long i = 0; i < nf; i++) Den[i] += a[i];
    }
    oracle_apply_update(x, Num, Den, nf);
    if (!num_out) free(Num);
    if (!den_out) free(Den);
    free(z);
    free(w);
    free(b);
    free(a);
}

/* Student-t log-likelihood over the valid pixels:
 *   sum [lgamma((nu+1)/2) - lgamma(nu/2) - 1/2 log(nu pi v)
 *        - (nu+1)/2 log(1 + u (y - z)^2 / nu)]. */
double oracle_student_loglik(const double *x, const double *y, const double *v,
                             const double *u, const double *f, int n, int H,
                             int W, int K, int r, double nu)
{
    const double pi = 3.14159265358979323846264338327950;
    const long np = (long)H * W;
    const double c = lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu);
    double *z = (double *)malloc(sizeof(double) * np);
    double s = 0.0;
    for (int t = 0; t < n; t++) {
        oracle_forward(x, H, W, r, f + (long)t * K * K, K, z);
        for (long i = 0; i < np; i++) {
            const double ui = u[t * np + i];
            if (ui != 0.0) {
                const double d = y[t * np + i] - z[i];
                s += c - 0.5 * log(nu * pi * v[t * np + i]) -
                     0.5 * (nu + 1.0) * log1p(ui * d * d / nu);
            }
        }
    }
    free(z);
    return s;
}

/* ----------------------------------------------------------------------- */
/* Log-likelihood of Eq. (1) and the default initial guess                  */
/* ----------------------------------------------------------------------- */

/* chi2 = sum_{t,i: u != 0} u (y - z)^2 with z = D^r(f_t * x). */
double oracle_chi2(const double *x, const double *y, const double *u,
                   const double *f, int n, int H, int W, int K, int r)
{
    const long np = (long)H * W;
    double *z = (double *)malloc(sizeof(double) * np);
    double s = 0.0;
    for (int t = 0; t < n; t++) {
        oracle_forward(x, H, W, r, f + (long)t * K * K, K, z);
        for (long i = 0; i < np; i++) {
            double ui = u[t * np + i];
            if (ui != 0.0) {
                double d = y[t * np + i] - z[i];
                s += ui * d * d;
            }
        }
    }
    free(z);
    return s;
}

/* sum_{t,i: u != 0} log(2 pi v). */
double oracle_logdet(const double *v, const double *u, long total)
{
    const double two_pi = 6.283185307179586476925286766559;
    double s = 0.0;
    for (long i = 0; i < total; i++)
        if (u[i] != 0.0) s += log(two_pi * v[i]);
    return s;
}

/* Default strictly positive start (Sec. 2 only asks x^(0) > 0):
 * c = (sum u y / sum u) / r^2 when positive, else 1. */
double oracle_default_x0(const double *y, const double *u, long total, int r)
{
    double suy = 0.0, su = 0.0;
    for (long i = 0; i < total; i++)
        if (u[i] != 0.0) {
            suy += u[i] * y[i];
            su += u[i];
        }
    if (su > 0.0) {
        double c = suy / su / ((double)r * r);
        if (c > 0.0) return c;
    }
    return 1.0;
}

/* ----------------------------------------------------------------------- */
/* One EM iteration evaluated at selected latent pixels only                */
/* ----------------------------------------------------------------------- */

/* Coarse-grid model value z_t at (i, j): sum over the r x r fine block of
 * (f * x). */
static double model_at(const double *x, int H, int W, int r, const double *f,
                       int K, int i, int j)
{
    const int h = (K - 1) / 2;
    const int Hf = r * H, Wf = r * W;
    double s = 0.0;
    for (int da = 0; da < r; da++)
        for (int db = 0; db < r; db++) {
            int P = r * i + da, Q = r * j + db;
            for (int a = 0; a < K; a++) {
                int ii = P + h - a;
                if (ii < 0 || ii >= Hf) continue;
                for (int b = 0; b < K; b++) {
                    int jj = Q + h - b;
                    if (jj < 0 || jj >= Wf) continue;
                    s += f[a * K + b] * x[(long)ii * Wf + jj];
                }
            }
        }
    return s;
}

/* For each latent index idx[m] (into the (rH) x (rW) grid) compute, from the
 * current x, N[p], Den[p] and the updated x'[p] of one iteration of Eq. (2).
 * Only the footprint of each pixel is evaluated, so this runs at any image
 * size. y may hold NaN where u == 0 (never read there). */
void oracle_em_step_at(const double *x, const double *y, const double *u,
                       const double *f, int n, int H, int W, int K, int r,
                       const long *idx, int m, double *x_out, double *N_out,
                       double *den_out)
{
    const int h = (K - 1) / 2;
    const int Hf = r * H, Wf = r * W;
    const long np = (long)H * W;
    /* the coarse pixels reachable from one fine pixel through K taps */
    const int span = (K + r - 1) / r + 2;
    double *memo = (double *)malloc(sizeof(double) * span * span);
    char *have = (char *)malloc(span * span);
    for (int mm = 0; mm < m; mm++) {
        const int P = (int)(idx[mm] / Wf), Q = (int)(idx[mm] % Wf);
        /* coarse rows/cols touched by fine rows P-h .. P+h */
        const int ci0 = (P - h < 0 ? -1 : (P - h) / r) , cj0 = (Q - h < 0 ? -1 : (Q - h) / r);
        double Nsum = 0.0, Dsum = 0.0;
        for (int t = 0; t < n; t++) {
            const double *ft = f + (long)t * K * K;
            const double *ut = u + t * np, *yt = y + t * np;
            memset(have, 0, span * span);
            for (int a = 0; a < K; a++) {
                int PP = P - h + a;
                if (PP < 0 || PP >= Hf) continue;
                for (int b = 0; b < K; b++) {
                    int QQ = Q - h + b;
                    if (QQ < 0 || QQ >= Wf) continue;
                    int i = PP / r, j = QQ / r;
                    double uij = ut[(long)i * W + j];
                    if (uij == 0.0) continue;
                    int key = (i - ci0) * span + (j - cj0);
                    if (!have[key]) {
                        memo[key] = model_at(x, H, W, r, ft, K, i, j);
                        have[key] = 1;
                    }
                    Dsum += ft[a * K + b] * uij * memo[key];
                    Nsum += ft[a * K + b] * uij * yt[(long)i * W + j];
                }
            }
        }
        const double xp = x[idx[mm]];
        if (N_out) N_out[mm] = Nsum;
        if (den_out) den_out[mm] = Dsum;
        if (x_out) x_out[mm] = Dsum > 0.0 ? xp * fmax(Nsum, 0.0) / Dsum : xp;
    }
    free(memo);
    free(have);
}

/* ----------------------------------------------------------------------- */
/* PSF super-resolution fit, Eq. (4)                                        */
/* ----------------------------------------------------------------------- */
/*
 * h = argmin_{h >= 0}  sum_ij ([D^r(h * g)]_ij - f_ij)^2 + lambda sum_ij (grad h)_ij^2
 * Readings (Sec. 2 gives only the objective and "Adam"):
 *   - f is K x K (coarse); h lives on the fine grid of Kh = r (K-1) + 1
 *     pixels per side (odd, centre fine pixel r (K-1)/2 inside the centre
 *     coarse pixel's block, fine pixel P belonging to coarse pixel P div r);
 *   - h * g is the zero-padded 'same' convolution on the Kh x Kh grid,
 *     zero-extended to rK x rK before the r x r block sum D^r;
 *   - (grad h)^2 = (h[i+1][j]-h[i][j])^2 + (h[i][j+1]-h[i][j])^2 for the
 *     differences inside the grid;
 *   - g is a normalised Gaussian given by the caller;
 *   - Adam (Kingma & Ba) with bias correction; h >= 0 by projection after
 *     each step.
 */

/* m = D^r(pad(h * g)), m is K x K. */
void oracle_psf_model(const double *h, int Kh, const double *g, int Kg, int r,
                      int K, double *m)
{
    double *q = (double *)malloc(sizeof(double) * Kh * Kh);
    oracle_conv_same(h, Kh, Kh, g, Kg, q);
    for (int i = 0; i < K; i++)
        for (int j = 0; j < K; j++) {
            double s = 0.0;
            for (int a = 0; a < r; a++)
                for (int b = 0; b < r; b++) {
                    int P = r * i + a, Q = r * j + b;
                    if (P < Kh && Q < Kh) s += q[P * Kh + Q];
                }
            m[i * K + j] = s;
        }
    free(q);
}

/* transpose of oracle_psf_model: out (Kh x Kh) = g-correlation of the
 * replicated K x K array w, cropped to Kh x Kh. */
void oracle_psf_model_adjoint(const double *w, int K, const double *g, int Kg,
                              int r, int Kh, double *out)
{
    double *q = (double *)malloc(sizeof(double) * Kh * Kh);
    for (int P = 0; P < Kh; P++)
        for (int Q = 0; Q < Kh; Q++) q[P * Kh + Q] = w[(P / r) * K + Q / r];
    oracle_corr_same(q, Kh, Kh, g, Kg, out);
    free(q);
}

/* loss of Eq. (4) at h; the gradient goes to grad when it is not NULL */
double oracle_psf_loss(const double *h, int Kh, const double *f, int K,
                       const double *g, int Kg, int r, double lambda,
                       double *grad)
{
    double *m = (double *)malloc(sizeof(double) * K * K);
    oracle_psf_model(h, Kh, g, Kg, r, K, m);
    double loss = 0.0;
    for (int e = 0; e < K * K; e++) {
        m[e] -= f[e];
        loss += m[e] * m[e];
    }
    if (grad) {
        oracle_psf_model_adjoint(m, K, g, Kg, r, Kh, grad);
        for (int e = 0; e < Kh * Kh; e++) grad[e] *= 2.0;
    }
    for (int i = 0; i < Kh; i++)
        for (int j = 0; j < Kh; j++) {
            const double c = h[i * Kh + j];
            if (i + 1 < Kh) {
                const double d = h[(i + 1) * Kh + j] - c;
                loss += lambda * d * d;
                if (grad) {
                    grad[(i + 1) * Kh + j] += 2.0 * lambda * d;
                    grad[i * Kh + j] -= 2.0 * lambda * d;
                }
            }
            if (j + 1 < Kh) {
                const double d = h[i * Kh + j + 1] - c;
                loss += lambda * d * d;
                if (grad) {
                    grad[i * Kh + j + 1] += 2.0 * lambda * d;
                    grad[i * Kh + j] -= 2.0 * lambda * d;
                }
            }
        }
    free(m);
    return loss;
}

/* iters Adam steps from h, projected onto h >= 0 after each. Adam at a
 * fixed step does not descend monotonically (once its second moments have
 * decayed it makes intermittent excursions), so the estimate of the argmin
 * of Eq. (4) is the iterate of lowest loss among h_0 .. h_iters (the first
 * such on ties); it is written back to h and its loss returned. */
double oracle_psf_fit(double *h, int Kh, const double *f, int K, const double *g,
                      int Kg, int r, double lambda, double lr, double b1,
                      double b2, double eps, int iters)
{
    const int nh = Kh * Kh;
    double *mo = (double *)calloc(nh, sizeof(double));
    double *vo = (double *)calloc(nh, sizeof(double));
    double *gr = (double *)malloc(sizeof(double) * nh);
    double *best = (double *)malloc(sizeof(double) * nh);
    double p1 = 1.0, p2 = 1.0, lbest = 0.0;
    for (int k = 1; k <= iters; k++) {
        const double L = oracle_psf_loss(h, Kh, f, K, g, Kg, r, lambda, gr);
        if (k == 1 || L < lbest) {
            lbest = L;
            memcpy(best, h, sizeof(double) * nh);
        }
        p1 *= b1;
        p2 *= b2;
        for (int e = 0; e < nh; e++) {
            mo[e] = b1 * mo[e] + (1.0 - b1) * gr[e];
            vo[e] = b2 * vo[e] + (1.0 - b2) * gr[e] * gr[e];
            const double mh = mo[e] / (1.0 - p1), vh = vo[e] / (1.0 - p2);
            h[e] = fmax(h[e] - lr * mh / (sqrt(vh) + eps), 0.0);
        }
    }
    const double L = oracle_psf_loss(h, Kh, f, K, g, Kg, r, lambda, NULL);
    if (iters >= 1 && !(L < lbest)) {
        memcpy(h, best, sizeof(double) * nh);
    } else {
        lbest = L;
    }
    free(mo);
    free(vo);
    free(gr);
    free(best);
    return lbest;
}
