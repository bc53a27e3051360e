"""Eq. (4) PSF fit on the GPU (emd_fit_psf) against the FP64 oracle.

Tolerances. The kernel runs the oracle's projected Adam in FP32. Adam's
normalised step m / sqrt(v) has size lr whatever the gradient's size, so a
pixel whose gradient is at the level of FP32 rounding (the far wings of a
PSF, pixels on the h >= 0 bound) can take a different step than in FP64;
everywhere else the two trajectories stay within rounding of each other.
An FP32 restatement of the same steps, against the oracle, after 100 steps:
K = 15, r = 2: 3e-7 of max|h| everywhere; K = 43, r = 2: 3e-7 of max|h| on
the core (start value >= 1e-3 of its maximum), 1e-4 in the wings, 1.3e-4
relative L2, 3e-5 relative loss. The bars: core elements 1e-5 of max|h|,
relative L2 1e-3, achieved loss 1e-3 relative. Near convergence the
trajectories part further while both approach the same constrained
minimiser, so converged runs are checked against that minimiser (L-BFGS-B
in FP64) and its loss. The loss the kernel reports is checked against the
oracle's loss at the kernel's own h with the Cauchy-Schwarz bound
|dL| <= 2 sqrt(L) |d| + |d|^2 for a model error |d| <= 4e-6 |f| (60 FP32
operations per model pixel at unit roundoff 6e-8).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emd():
    from paper_2302_05804_gb300 import emd as m
    m.load()
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def default_h0(f, r):
    K = f.shape[0]
    Kh = r * (K - 1) + 1
    return np.kron(f.astype(np.float64), np.ones((r, r)))[:Kh, :Kh] / r ** 2


def coarse_psfs(n, K, seed):
    g = np.random.default_rng(seed)
    return np.stack([synth.moffat_psf(K, g.uniform(2.0, 3.5), g.uniform(2.5, 4.5),
                                      ellip=g.uniform(0, 0.15), angle=g.uniform(0, np.pi))
                     for _ in range(n)]).astype(np.float32)


def check_against_oracle(h, ho, h0, f, g, r, lam):
    core = h0 >= 1e-3 * h0.max()
    assert np.abs(h - ho)[core].max() <= 1e-5 * np.abs(ho).max()
    assert rel_l2(h, ho) <= 1e-3
    Lg = oracle.psf_loss(h.astype(np.float64), f, g, r, lam)
    Lo = oracle.psf_loss(ho, f, g, r, lam)
    assert abs(Lg - Lo) <= 1e-3 * Lo


def check_reported_loss(loss, h, f, g, r, lam):
    L = oracle.psf_loss(h.astype(np.float64), f, g, r, lam)
    d = 4e-6 * np.linalg.norm(np.asarray(f, np.float64))
    assert abs(float(loss) - L) <= 2 * np.sqrt(L) * d + d * d


@pytest.mark.parametrize("K,r,lam", [(15, 2, 1e-3), (11, 3, 1e-2), (9, 1, 0.1), (13, 2, 0.0)])
def test_fit_matches_oracle_short(emd, K, r, lam):
    f = coarse_psfs(3, K, K * 10 + r)
    g = synth.gaussian_kernel(r).astype(np.float32)
    h, loss = emd.emd_fit_psf(f, g, r, lam, 1e-4, 100)
    assert h.shape == (3, r * (K - 1) + 1, r * (K - 1) + 1)
    for t in range(3):
        h0 = default_h0(f[t], r)
        ho = oracle.psf_fit(f[t], g, r, lam, 100, 1e-4, h0)
        check_against_oracle(h[t], ho, h0, f[t], g, r, lam)
        check_reported_loss(loss[t], h[t], f[t], g, r, lam)
    assert (h >= 0).all()


def test_zero_iterations_return_the_start_and_its_loss(emd):
    K, r, lam = 11, 2, 1e-2
    f = coarse_psfs(2, K, 7)
    g = synth.gaussian_kernel(r).astype(np.float32)
    h, loss = emd.emd_fit_psf(f, g, r, lam, 1e-4, 0)
    for t in range(2):
        h0 = default_h0(f[t], r)
        np.testing.assert_allclose(h[t], h0, rtol=1e-6, atol=0)
        check_reported_loss(loss[t], h[t], f[t], g, r, lam)


def test_explicit_start_and_device_buffers(emd):
    torch = pytest.importorskip("torch")
    K, r, lam = 9, 2, 1e-3
    Kh = r * (K - 1) + 1
    f = coarse_psfs(4, K, 11)
    g = synth.gaussian_kernel(r).astype(np.float32)
    h0 = np.random.default_rng(5).uniform(0, 0.01, (4, Kh, Kh)).astype(np.float32)
    dev = torch.device("cuda:0")
    fd, gd, h0d = (torch.from_numpy(a).to(dev) for a in (f, g, h0))
    hd = torch.empty((4, Kh, Kh), dtype=torch.float32, device=dev)
    ld = torch.empty(4, dtype=torch.float32, device=dev)
    emd.emd_fit_psf(fd, gd, r, lam, 1e-4, 150, h0=h0d, h_out=hd, loss_out=ld)
    h = hd.cpu().numpy()
    loss = ld.cpu().numpy()
    for t in range(4):
        ho = oracle.psf_fit(f[t], g, r, lam, 150, 1e-4, h0[t])
        check_against_oracle(h[t], ho, np.ones_like(ho), f[t], g, r, lam)
        check_reported_loss(loss[t], h[t], f[t], g, r, lam)


def test_converged_fit_reaches_the_constrained_minimiser(emd):
    from scipy.optimize import minimize
    K, r, lam = 9, 2, 1e-3
    Kh = r * (K - 1) + 1
    g = synth.gaussian_kernel(r)
    f = synth.moffat_psf(K, 2.2, 3.0, ellip=0.1, angle=0.4)
    h, loss = emd.emd_fit_psf(f.astype(np.float32), g.astype(np.float32), r, lam, 1e-4, 20000)
    h0 = default_h0(f, r)
    ho = oracle.psf_fit(f, g, r, lam, 20000, 1e-4, h0)
    res = minimize(lambda z: oracle.psf_loss(z.reshape(Kh, Kh), f, g, r, lam), h0.ravel(),
                   method="L-BFGS-B", bounds=[(0, None)] * (Kh * Kh),
                   jac=lambda z: oracle.psf_loss(z.reshape(Kh, Kh), f, g, r, lam, grad=True)[1].ravel(),
                   options=dict(maxiter=20000, ftol=1e-16, gtol=1e-12))
    hs = res.x.reshape(Kh, Kh)
    Ls = oracle.psf_loss(hs, f, g, r, lam)
    Lg = oracle.psf_loss(h.astype(np.float64), f, g, r, lam)
    assert Lg <= Ls * (1 + 1e-4)
    assert rel_l2(h, hs) <= 1e-3
    assert rel_l2(h, ho) <= 1e-3
    assert (h >= 0).all()


def test_full_size_exposure_set_sampled(emd):
    """33 coarse 43 x 43 PSFs to 85 x 85 fine PSFs (the PSF size of the r = 2
    super-resolution workload): every fit lowers the loss and stays >= 0;
    two sampled exposures match the oracle's run."""
    K, r, lam, iters = 43, 2, 1e-3, 100
    f = coarse_psfs(33, K, 43)
    g = synth.gaussian_kernel(r).astype(np.float32)
    h, loss = emd.emd_fit_psf(f, g, r, lam, 1e-4, iters)
    _, loss0 = emd.emd_fit_psf(f, g, r, lam, 1e-4, 0)
    assert h.shape == (33, 85, 85)
    assert (h >= 0).all() and np.isfinite(h).all()
    assert (loss < loss0).all()
    for t in (0, 32):
        h0 = default_h0(f[t], r)
        ho = oracle.psf_fit(f[t], g, r, lam, iters, 1e-4, h0)
        check_against_oracle(h[t], ho, h0, f[t], g, r, lam)
        check_reported_loss(loss[t], h[t], f[t], g, r, lam)


def test_bad_arguments_raise(emd):
    f = coarse_psfs(1, 9, 1)
    g = synth.gaussian_kernel(2).astype(np.float32)
    with pytest.raises(emd.EMDError):
        emd.emd_fit_psf(f, g, 2, -1.0, 1e-4, 10)
    with pytest.raises(emd.EMDError):   # fine side 2 (128 - 1) + 1 = 255: too large
        emd.emd_fit_psf(np.ones((1, 127, 127), np.float32), g, 2, 0.0, 1e-4, 1)


@pytest.mark.parametrize("n", [1, 19, 80, 160])
def test_cluster_split_matches_oracle(emd, n):
    """The library splits each PSF over a cluster of up to 8 CTAs, fewer as
    the number of PSFs grows (one CTA each from 76 PSFs on); every split
    must give the oracle's fit."""
    K, r, lam = 11, 3, 1e-2
    f = coarse_psfs(n, K, 100 + n)
    g = synth.gaussian_kernel(r).astype(np.float32)
    h, loss = emd.emd_fit_psf(f, g, r, lam, 1e-4, 60)
    for t in sorted({0, n // 2, n - 1}):
        h0 = default_h0(f[t], r)
        ho = oracle.psf_fit(f[t], g, r, lam, 60, 1e-4, h0)
        check_against_oracle(h[t], ho, h0, f[t], g, r, lam)
        check_reported_loss(loss[t], h[t], f[t], g, r, lam)
