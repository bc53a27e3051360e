"""Seeded synthetic inputs for the EM multi-frame deconvolution workloads.

This module is shared by the tests, the benchmark and the smoke check. It
draws scenes, PSFs, variance maps, masks and noise; it contains none of the
EM method's arithmetic (no update, no adjoint, no likelihood). Observed
exposures are synthesised from the image model of Eq. (1) (and Eq. (3) for
super-resolution) with a library FFT convolution (scipy.signal.fftconvolve)
and a numpy block sum, which are independent of both the FP64 oracle and the
CUDA kernels.

Workload recipes follow the data described in Sec. 2 (Fig. 1: n = 33
exposures of 4K x 4K pixels with 43 x 43 PSFs) and the synthetic
stand-ins used for them:

  * ``parity``   256^2, n=4, 15x15 Moffat (beta=3, FWHM 2-4 px), sky 100.
  * ``hsc``      4096^2, n=33, 43x43 elliptical Moffat, sky 50-400, 5% masked.
  * ``sr2``      33 exposures of 2048^2 observed from a 4096^2 latent through
                 85x85 fine-grid Moffat PSFs and a 2x2 sum-downsample.
  * any of these at a reduced size through ``make_problem(...)`` arguments.

Seeds: recipe index i draws the sky from PCG64(1000+i), the PSFs from
PCG64(2000+i) and noise/masks from PCG64(3000+i).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "moffat_psf", "sersic_bn", "render_sky", "draw_masks", "Problem",
    "make_problem", "RECIPES", "fft_convolve_same", "block_sum",
]


# ---------------------------------------------------------------------------
# PSFs and sources
# ---------------------------------------------------------------------------

def gaussian_kernel(fwhm: float) -> np.ndarray:
    """Normalised circular Gaussian with the given FWHM in pixels, sampled at
    pixel centres out to 3 sigma (odd side): the broadening kernel g of the
    Eq. (4) PSF fit, whose FWHM is one coarse pixel (r fine pixels)."""
    sig = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    k = int(np.ceil(3 * sig))
    yy, xx = np.mgrid[-k:k + 1, -k:k + 1]
    g = np.exp(-(xx ** 2 + yy ** 2) / (2 * sig * sig))
    return g / g.sum()


def moffat_psf(K: int, fwhm: float, beta: float, ellip: float = 0.0,
               angle: float = 0.0) -> np.ndarray:
    """K x K Moffat profile (1 + R^2/alpha^2)^-beta sampled at pixel centres.

    alpha = FWHM / (2 sqrt(2^(1/beta) - 1)); an ellipticity e squeezes the
    minor axis by (1 - e) after a rotation by ``angle``. Normalised in FP64
    to unit sum (the PSFs of Sec. 2 conserve flux).
    """
    if K % 2 != 1:
        raise ValueError("PSF side must be odd")
    h = K // 2
    alpha = fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))
    yy, xx = np.mgrid[-h:h + 1, -h:h + 1].astype(np.float64)
    c, s = math.cos(angle), math.sin(angle)
    u = c * xx + s * yy
    v = (-s * xx + c * yy) / (1.0 - ellip)
    r2 = u * u + v * v
    p = (1.0 + r2 / (alpha * alpha)) ** (-beta)
    return p / p.sum()


def sersic_bn(n: float) -> float:
    """Ciotti & Bertin (1999) asymptotic expansion of the Sersic b_n."""
    return 2.0 * n - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n)


def _add_sersic(img: np.ndarray, cy: float, cx: float, n: float, re: float,
                q: float, ang: float, flux: float) -> None:
    H, W = img.shape
    R = int(math.ceil(8.0 * re))
    y0, y1 = max(0, int(cy) - R), min(H, int(cy) + R + 1)
    x0, x1 = max(0, int(cx) - R), min(W, int(cx) + R + 1)
    if y0 >= y1 or x0 >= x1:
        return
    yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    dy, dx = yy - cy, xx - cx
    c, s = math.cos(ang), math.sin(ang)
    u = c * dx + s * dy
    v = (-s * dx + c * dy) / q
    r = np.sqrt(u * u + v * v)
    prof = np.exp(-sersic_bn(n) * ((r / re) ** (1.0 / n) - 1.0))
    prof[r > 8.0 * re] = 0.0
    tot = prof.sum()
    if tot > 0:
        img[y0:y1, x0:x1] += flux * prof / tot


def render_sky(H: int, W: int, n_points: int, n_gal: int,
               rng: np.random.Generator, mu: float = 6.0, sigma: float = 1.5,
               re_range=(3.0, 10.0), margin: int = 0) -> np.ndarray:
    """Zero-background sky: point sources at integer pixels plus Sersic
    galaxies, all with lognormal(mu, sigma) flux. FP64."""
    img = np.zeros((H, W), np.float64)
    if n_points:
        ys = rng.integers(margin, H - margin, n_points)
        xs = rng.integers(margin, W - margin, n_points)
        fl = rng.lognormal(mu, sigma, n_points)
        np.add.at(img, (ys, xs), fl)
    for _ in range(n_gal):
        cy = rng.uniform(margin, H - margin)
        cx = rng.uniform(margin, W - margin)
        n = rng.uniform(0.5, 4.0)
        re = rng.uniform(*re_range)
        q = rng.uniform(0.5, 1.0)
        ang = rng.uniform(0.0, math.pi)
        fl = rng.lognormal(mu, sigma)
        _add_sersic(img, cy, cx, n, re, q, ang, fl)
    return img


def draw_masks(n: int, H: int, W: int, frac: float,
               rng: np.random.Generator) -> np.ndarray:
    """Per-exposure uint8 validity masks (0 = masked): bad columns of full or
    partial height plus cosmic-ray discs of radius 1-3 px, drawn until about
    ``frac`` of the pixels of each exposure are masked."""
    m = np.ones((n, H, W), np.uint8)
    if frac <= 0:
        return m
    target = frac * H * W
    offs = {rr: [(dy, dx) for dy in range(-rr, rr + 1) for dx in range(-rr, rr + 1)
                 if dy * dy + dx * dx <= rr * rr] for rr in (1, 2, 3)}
    for t in range(n):
        mt = m[t]
        # about a third of the budget in columns, the rest in cosmic rays
        while H * W - int(mt.sum()) < target / 3.0:
            c = int(rng.integers(0, W))
            if rng.uniform() < 0.5:
                r0, r1 = 0, H
            else:
                r0 = int(rng.integers(0, H))
                r1 = min(H, r0 + int(rng.integers(H // 8 + 1, H // 2 + 2)))
            mt[r0:r1, c] = 0
        while True:
            bad = H * W - int(mt.sum())
            if bad >= target:
                break
            k = max(1, int(target - bad) // 12)
            cy = rng.integers(0, H, k)
            cx = rng.integers(0, W, k)
            rad = rng.integers(1, 4, k)
            for rr, oo in offs.items():
                sel = rad == rr
                yy0, xx0 = cy[sel], cx[sel]
                for dy, dx in oo:
                    yy = np.clip(yy0 + dy, 0, H - 1)
                    xx = np.clip(xx0 + dx, 0, W - 1)
                    mt[yy, xx] = 0
    return m


# ---------------------------------------------------------------------------
# Observation synthesis (library FFT convolution, numpy block sum)
# ---------------------------------------------------------------------------

def fft_convolve_same(x: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Zero-padded 'same' convolution by scipy's FFT convolution (FP64)."""
    from scipy import fft as sfft
    from scipy.signal import fftconvolve
    with sfft.set_workers(os.cpu_count() or 1):
        return fftconvolve(x, f, mode="same")


def block_sum(z: np.ndarray, r: int) -> np.ndarray:
    """Sum over r x r blocks (fine pixel (r*i+s, r*j+t) -> coarse (i, j))."""
    if r == 1:
        return z
    H, W = z.shape[0] // r, z.shape[1] // r
    return z.reshape(H, r, W, r).sum(axis=(1, 3))


@dataclass
class Problem:
    """One deconvolution job: exposures (n x H x W), fine-grid PSFs
    (n x K x K), variances, masks, and the truth on the (rH x rW) latent grid."""
    y: np.ndarray          # float32, NaN where masked
    v: np.ndarray          # float32
    f: np.ndarray          # float32, each PSF sums to 1 in FP64 before the cast
    mask: np.ndarray       # uint8, 0 = masked
    x_true: np.ndarray     # float64
    r: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def n(self): return self.y.shape[0]
    @property
    def H(self): return self.y.shape[1]
    @property
    def W(self): return self.y.shape[2]
    @property
    def K(self): return self.f.shape[1]


RECIPES = {
    # name: (index for seeds, defaults)
    "parity": (0, dict(H=256, W=256, n=4, K=15, r=1, n_points=50, n_gal=5,
                       beta=(3.0, 3.0), fwhm=(2.0, 4.0), ellip=0.0,
                       sky=(100.0, 100.0), mask_frac=0.0, iters=50)),
    "hsc": (1, dict(H=4096, W=4096, n=33, K=43, r=1, n_points=20000,
                    n_gal=2000, beta=(2.5, 4.5), fwhm=(3.0, 7.0), ellip=0.15,
                    sky=(50.0, 400.0), mask_frac=0.05, iters=100)),
    "sr2": (2, dict(H=2048, W=2048, n=33, K=85, r=2, n_points=20000,
                    n_gal=2000, beta=(2.5, 4.5), fwhm=(6.0, 14.0), ellip=0.15,
                    sky=(50.0, 400.0), mask_frac=0.05, iters=100)),
}


def make_problem(recipe: str = "parity", *, seed_offset: int = 0,
                 noise_free: bool = False, dtype=np.float32, cache: bool = True,
                 **over) -> Problem:
    """Cached front of ``_make_problem``: when the environment variable
    EMD_SYNTH_CACHE names a directory, problems are stored there as .npz and
    reloaded on the next call with the same arguments."""
    cdir = os.environ.get("EMD_SYNTH_CACHE")
    if not (cache and cdir):
        return _make_problem(recipe, seed_offset=seed_offset, noise_free=noise_free,
                             dtype=dtype, **over)
    key = "_".join([recipe, str(seed_offset), str(int(noise_free)), np.dtype(dtype).name]
                   + [f"{k}{over[k]}" for k in sorted(over)])
    path = os.path.join(cdir, key + ".npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=True)
        return Problem(y=z["y"], v=z["v"], f=z["f"], mask=z["mask"], x_true=z["x_true"],
                       r=int(z["r"]), meta=z["meta"].item())
    p = _make_problem(recipe, seed_offset=seed_offset, noise_free=noise_free,
                      dtype=dtype, **over)
    os.makedirs(cdir, exist_ok=True)
    np.savez(path + ".tmp.npz", y=p.y, v=p.v, f=p.f, mask=p.mask, x_true=p.x_true, r=p.r,
             meta=np.array(p.meta, dtype=object))
    os.replace(path + ".tmp.npz", path)
    return p


def _make_problem(recipe: str = "parity", *, seed_offset: int = 0,
                  noise_free: bool = False, dtype=np.float32, **over) -> Problem:
    """Draw a seeded problem following ``RECIPES[recipe]``; keyword overrides
    rescale it (e.g. ``H=512, W=384, n=5``). Source counts scale with the
    latent area when H or W are overridden and counts are not given."""
    idx, d = RECIPES[recipe]
    p = dict(d)
    scale_counts = ("H" in over or "W" in over) and "n_points" not in over
    p.update(over)
    H, W, n, K, r = p["H"], p["W"], p["n"], p["K"], p["r"]
    if scale_counts:
        a = (H * W) / (d["H"] * d["W"])
        p["n_points"] = max(1, int(round(d["n_points"] * a)))
        p["n_gal"] = max(1, int(round(d["n_gal"] * a)))
    s = 1000 + idx + seed_offset
    rng_sky = np.random.Generator(np.random.PCG64(s))
    rng_psf = np.random.Generator(np.random.PCG64(s + 1000))
    rng_obs = np.random.Generator(np.random.PCG64(s + 2000))

    Hf, Wf = r * H, r * W
    re_range = (3.0 * r, 10.0 * r)
    x_true = render_sky(Hf, Wf, p["n_points"], p["n_gal"], rng_sky,
                        re_range=re_range)

    f = np.empty((n, K, K), np.float64)
    for t in range(n):
        beta = rng_psf.uniform(*p["beta"])
        fwhm = rng_psf.uniform(*p["fwhm"])
        e = rng_psf.uniform(0.0, p["ellip"]) if p["ellip"] > 0 else 0.0
        ang = rng_psf.uniform(0.0, math.pi)
        f[t] = moffat_psf(K, fwhm, beta, e, ang)
    f32 = f.astype(np.float32)

    mask = draw_masks(n, H, W, p["mask_frac"], rng_obs)
    y = np.empty((n, H, W), dtype)
    v = np.empty((n, H, W), dtype)
    for t in range(n):
        # the model uses the stored (fp32) PSF so noise-free data is exact
        z = block_sum(fft_convolve_same(x_true, f32[t].astype(np.float64)), r)
        sky = rng_obs.uniform(*p["sky"])
        vt = sky + np.maximum(z, 0.0)
        if noise_free:
            yt = z
        else:
            yt = z + np.sqrt(vt) * rng_obs.standard_normal((H, W))
        v[t] = vt
        y[t] = yt
    y[mask == 0] = np.nan
    return Problem(y=y, v=v, f=f32, mask=mask, x_true=x_true, r=r,
                   meta=dict(recipe=recipe, seed=s, **p))
