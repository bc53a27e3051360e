"""The FFT form of the forward model and adjoint (EMD_PREC_FFT_FP32) against
the FP64 oracle: the same bars as the direct FP32 kernel (relative L2 1e-5
after one iteration, 1e-4 after 50), on ragged shapes, masks, a delta PSF,
the largest PSF footprint, super-resolution (r = 2, 3), and the full-size
workloads on sampled pixels."""
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def start(p, seed=0):
    g = np.random.default_rng(seed)
    return (g.uniform(0.5, 1.5, (p.H, p.W)) * max(np.nanmean(p.y), 1.0)).astype(np.float32)


def gpu_run(emd, p, x0, k, prec):
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    try:
        d.set_frames(p.y, p.v, p.f, p.mask)
        d.set_precision(prec)
        d.set_x(x0)
        d.iterate(k)
        return d.x()
    finally:
        d.close()


def oracle_run(p, x0, k):
    u, y, N, _ = oracle.prepare(p)
    return oracle.em_run(x0.astype(np.float64), N, u, p.f, k, p.r)


def test_fft_parity_one_and_fifty_iterations(emd):
    p = synth.make_problem("parity")
    x0 = start(p)
    x1 = gpu_run(emd, p, x0, 1, emd.EMD_PREC_FFT_FP32)
    assert rel_l2(x1, oracle_run(p, x0, 1)) <= 1e-5
    x50 = gpu_run(emd, p, x0, 50, emd.EMD_PREC_FFT_FP32)
    assert rel_l2(x50, oracle_run(p, x0, 50)) <= 1e-4
    assert (x50 >= 0).all()


@pytest.mark.parametrize("H,W,n,K,mf", [(200, 150, 3, 15, 0.05), (130, 257, 2, 43, 0.05),
                                        (5, 7, 2, 9, 0.0), (64, 64, 1, 1, 0.1),
                                        (129, 128, 2, 3, 0.0), (70, 90, 2, 47, 0.02),
                                        (300, 87, 3, 29, 0.05)])
def test_fft_parity_shapes(emd, H, W, n, K, mf):
    p = synth.make_problem("hsc", H=H, W=W, n=n, K=K, r=1, mask_frac=mf, fwhm=(1.5, 3.0),
                           n_points=max(3, H * W // 400), n_gal=2)
    x0 = start(p, H + W)
    x1 = gpu_run(emd, p, x0, 1, emd.EMD_PREC_FFT_FP32)
    assert rel_l2(x1, oracle_run(p, x0, 1)) <= 1e-5
    x5 = gpu_run(emd, p, x0, 5, emd.EMD_PREC_FFT_FP32)
    assert rel_l2(x5, oracle_run(p, x0, 5)) <= 2e-5
    assert (x5 >= 0).all()


@pytest.mark.parametrize("H,W,n,K,r,mf", [(96, 80, 2, 15, 2, 0.05), (33, 47, 3, 21, 2, 0.0),
                                          (40, 36, 2, 7, 3, 0.05), (130, 110, 2, 85, 2, 0.02)])
def test_fft_parity_super_resolution(emd, H, W, n, K, r, mf):
    """Eq. (3): the phases' spectra and the adjoint's accumulators go
    through a per-tile scratch buffer."""
    p = synth.make_problem("hsc", H=H, W=W, n=n, K=K, r=r, mask_frac=mf,
                           fwhm=(1.5 * r, 3.0 * r), n_points=max(3, H * W // 400), n_gal=2)
    g = np.random.default_rng(H + W)
    x0 = (g.uniform(0.5, 1.5, (r * H, r * W)) * max(np.nanmean(p.y), 1.0) / r ** 2).astype(np.float32)
    x1 = gpu_run(emd, p, x0, 1, emd.EMD_PREC_FFT_FP32)
    assert rel_l2(x1, oracle_run(p, x0, 1)) <= 1e-5
    x5 = gpu_run(emd, p, x0, 5, emd.EMD_PREC_FFT_FP32)
    assert rel_l2(x5, oracle_run(p, x0, 5)) <= 2e-5
    assert (x5 >= 0).all()


@pytest.mark.parametrize("recipe", ["hsc", "sr2"])
def test_fft_full_size_sampled(emd, recipe):
    """4096^2 x 33, 43 x 43 PSFs (and 33 x 2048^2 exposures, 85 x 85 fine
    PSFs, r = 2): one FFT iteration against the oracle's single-pixel
    evaluation of Eq. (2) at sampled pixels (corners, tile seams of the
    86-pixel FFT tiles, random points), plus properties of the whole image."""
    p = synth.make_problem(recipe)
    Hf, Wf = p.r * p.H, p.r * p.W
    x0 = (np.random.default_rng(5).uniform(0.5, 1.5, (Hf, Wf)) * 10.0).astype(np.float32)
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    d.set_precision(emd.EMD_PREC_FFT_FP32)
    d.set_x(x0)
    ll0 = d.loglik()[0]
    d.iterate(1)
    x1 = d.x()
    ll1 = d.loglik()[0]
    d.close()
    assert np.isfinite(x1).all() and (x1 >= 0).all()
    assert ll1 >= ll0 - 1e-7 * abs(ll0)
    g = np.random.default_rng(17)
    hc = ((p.K - 1) // 2 + p.r - 1) // p.r
    Bt = p.r * (128 - 2 * hc)  # FFT tile seams on the latent grid
    pts = [(0, 0), (0, Wf - 1), (Hf - 1, 0), (Hf - 1, Wf - 1), (Bt - 1, Bt), (Bt, Bt - 1),
           (2 * Bt, 3 * Bt - 1), (Hf - 2, Wf // 2)]
    pts += [(int(a), int(b)) for a, b in zip(g.integers(0, Hf, 24), g.integers(0, Wf, 24))]
    idx = np.array([a * Wf + b for a, b in pts], np.int64)
    u, _ = oracle.weights(p.v, p.mask, p.y)
    xo, _, _ = oracle.em_step_at(x0, p.y, u, p.f, idx, p.r)
    got = x1.ravel()[idx].astype(np.float64)
    assert np.linalg.norm(got - xo) / np.linalg.norm(xo) <= 1e-5


def test_fft_split_launch_matches_whole_tile_kernels_bitwise(emd):
    """With at least as many tiles as SMs (here 18 x 18 tiles of 114 pixels,
    K = 15) a solo FFT iteration runs the split launch: persistent CTAs take
    equal ranges of (tile, exposure) units, and a tile cut between two CTAs
    passes the head's accumulator to the tail, which continues the sum in
    exposure order. The batch path runs whole tiles (one CTA per tile), and
    its iterates match the oracle (test_gpu_batch); the two must give the
    same bits."""
    p = synth.make_problem("hsc", H=2048, W=2048, n=3, K=15, r=1, mask_frac=0.05,
                           n_points=400, n_gal=8)
    x0 = np.full((p.H, p.W), 5.0, np.float32)

    def ctx():
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        d.set_frames(p.y, p.v, p.f, p.mask)
        d.set_precision(emd.EMD_PREC_FFT_FP32)
        d.set_x(x0)
        return d

    d = ctx()
    d.iterate(3)
    solo = d.x()
    d.close()
    b = emd.emd_batch_create(2)
    d = ctx()
    slot = emd.emd_batch_add(b, d.ctx, 3)
    steps = 0
    while emd.emd_batch_step(b) == 0:
        steps += 1
        assert steps < 10
    emd.emd_batch_sync(b)
    assert emd.emd_batch_remaining(b, slot) == 0
    batched = d.x()
    emd.emd_batch_remove(b, slot)
    emd.emd_batch_destroy(b)
    d.close()
    np.testing.assert_array_equal(solo, batched)
    assert np.isfinite(solo).all() and (solo >= 0).all()
