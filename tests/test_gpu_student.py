"""Heavy-tailed (Student-t) noise EM on the GPU against the FP64 oracle.

Same bars as the Gaussian path: relative L2 1e-5 after one iteration and
1e-4 after 30; the log-likelihood to 1e-6 relative. The data carry planted
outliers (satellite trails the mask missed) so that the weights u' really
differ from u.
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(H, W, n, K, r, seed=0, trails=True):
    p = synth.make_problem("hsc", H=H, W=W, n=n, K=K, r=r, mask_frac=0.03, seed_offset=seed,
                           fwhm=(1.5 * r, 3.0 * r), n_points=max(3, H * W // 400), n_gal=2)
    if trails:
        y = p.y.copy()
        y[0, H // 3, :] += 3000.0
        y[n - 1, :, W // 2] += 3000.0
        y[p.mask == 0] = np.nan
        p = synth.Problem(y=y, v=p.v, f=p.f, mask=p.mask, x_true=p.x_true, r=p.r, meta=p.meta)
    return p


def start(p, seed=0):
    g = np.random.default_rng(seed)
    return (g.uniform(0.5, 1.5, (p.r * p.H, p.r * p.W)) * 20.0).astype(np.float32)


def gpu_run(emd, p, x0, k, nu, prec=0):
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    try:
        d.set_frames(p.y, p.v, p.f, p.mask)
        if prec:
            d.set_precision(prec)
        d.set_noise(emd.EMD_NOISE_STUDENT_T, nu)
        d.set_x(x0)
        d.iterate(k)
        return d.x(), d.loglik()
    finally:
        d.close()


def oracle_run(p, x0, k, nu):
    u, y, _, _ = oracle.prepare(p)
    x = x0.astype(np.float64)
    for _ in range(k):
        x = oracle.em_step_student(x, y, u, p.f, nu, p.r)[0]
    return x


@pytest.mark.parametrize("H,W,n,K,r,nu", [(200, 150, 3, 15, 1, 3.0), (130, 257, 2, 43, 1, 1.0),
                                          (96, 80, 2, 15, 2, 5.0), (40, 36, 2, 7, 3, 2.0)])
def test_student_parity(emd, H, W, n, K, r, nu):
    p = problem(H, W, n, K, r, seed=H)
    x0 = start(p, H + W)
    x1, _ = gpu_run(emd, p, x0, 1, nu)
    assert rel_l2(x1, oracle_run(p, x0, 1, nu)) <= 1e-5
    x30, (ll, chi) = gpu_run(emd, p, x0, 30, nu)
    xo = oracle_run(p, x0, 30, nu)
    assert rel_l2(x30, xo) <= 1e-4
    assert (x30 >= 0).all()
    u, y, _, _ = oracle.prepare(p)
    ll_o = oracle.student_loglik(x30, y, p.v, u, p.f, nu, p.r)
    assert abs(ll - ll_o) <= 1e-6 * abs(ll_o)


def test_student_likelihood_is_monotone_on_gpu(emd):
    p = problem(128, 120, 3, 15, 1, seed=5)
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    d.set_noise(emd.EMD_NOISE_STUDENT_T, 3.0)
    prev = d.loglik()[0]
    for _ in range(25):
        d.iterate(1)
        ll = d.loglik()[0]
        assert ll >= prev - 1e-7 * abs(prev)
        prev = ll
    d.close()


def test_switching_back_to_gaussian_is_bitexact(emd):
    p = problem(96, 100, 3, 15, 1, seed=9, trails=False)
    x0 = start(p, 1)

    def run(detour):
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        d.set_frames(p.y, p.v, p.f, p.mask)
        if detour:
            d.set_noise(emd.EMD_NOISE_STUDENT_T, 2.0)
            d.iterate(2)
            d.set_noise(emd.EMD_NOISE_GAUSSIAN)
        d.set_x(x0)
        d.iterate(3)
        x = d.x()
        d.close()
        return x

    assert np.array_equal(run(False), run(True))


def test_large_nu_approaches_eq2(emd):
    p = problem(100, 90, 3, 15, 1, seed=13, trails=False)
    x0 = start(p, 2)
    xs, _ = gpu_run(emd, p, x0, 3, 1e12)
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    d.set_x(x0)
    d.iterate(3)
    xg = d.x()
    d.close()
    assert rel_l2(xs, xg) <= 1e-5


def test_student_guards(emd):
    p = problem(64, 64, 2, 9, 1, seed=3, trails=False)
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(emd.EMDError) as e:
            d.set_noise(emd.EMD_NOISE_STUDENT_T, bad)
        assert e.value.code == emd.EMD_EINVAL
    with pytest.raises(emd.EMDError):
        d.set_noise(7, 1.0)
    d.set_noise(emd.EMD_NOISE_STUDENT_T, 4.0)
    with pytest.raises(emd.EMDError) as e:
        d.set_precision(emd.EMD_PREC_SPLIT_BF16)
    assert e.value.code == emd.EMD_EUNSUPPORTED
    d.set_precision(emd.EMD_PREC_FFT_FP32)   # the FFT form takes heavy tails
    d.set_precision(emd.EMD_PREC_FP32)
    with pytest.raises(emd.EMDError) as e:
        d.iterate_streaming(1)
    assert e.value.code == emd.EMD_EUNSUPPORTED
    b = emd.emd_batch_create(2)
    with pytest.raises(emd.EMDError) as e:
        emd.emd_batch_add(b, d.ctx, 3)
    assert e.value.code == emd.EMD_EUNSUPPORTED
    emd.emd_batch_destroy(b)
    d.close()


@pytest.mark.parametrize("H,W,n,K,r,nu", [(200, 150, 3, 15, 1, 3.0), (130, 257, 2, 43, 1, 1.0),
                                          (96, 80, 2, 15, 2, 5.0)])
def test_student_parity_fft_form(emd, H, W, n, K, r, nu):
    """The heavy-tailed update in the FFT form: the forward pass writes u'z
    and u'y, the adjoint transforms both; same bars as the direct form."""
    p = problem(H, W, n, K, r, seed=H + 1)
    x0 = start(p, H + W + 1)
    x1, _ = gpu_run(emd, p, x0, 1, nu, emd.EMD_PREC_FFT_FP32)
    assert rel_l2(x1, oracle_run(p, x0, 1, nu)) <= 1e-5
    x30, (ll, _) = gpu_run(emd, p, x0, 30, nu, emd.EMD_PREC_FFT_FP32)
    xo = oracle_run(p, x0, 30, nu)
    assert rel_l2(x30, xo) <= 1e-4
    assert (x30 >= 0).all()


def test_student_noise_set_after_the_fft_form(emd):
    """Selecting the heavy-tailed model after the FFT form grows its buffers;
    switching back to Gaussian gives the Gaussian FFT iterate bit for bit."""
    p = problem(96, 100, 3, 15, 1, seed=21)
    x0 = start(p, 4)

    def run(order):
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        d.set_frames(p.y, p.v, p.f, p.mask)
        d.set_precision(emd.EMD_PREC_FFT_FP32)
        d.set_x(x0)
        for model in order:
            d.set_noise(model, 3.0)
            d.iterate(2)
        x = d.x()
        d.close()
        return x

    g = run([emd.EMD_NOISE_GAUSSIAN, emd.EMD_NOISE_GAUSSIAN])
    assert np.array_equal(g, run([emd.EMD_NOISE_GAUSSIAN, emd.EMD_NOISE_GAUSSIAN]))
    xs = run([emd.EMD_NOISE_STUDENT_T, emd.EMD_NOISE_STUDENT_T])
    xd, _ = gpu_run(emd, p, x0, 4, 3.0)
    assert rel_l2(xs, xd) <= 2e-5
