"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one part of the oracle to something fixed outside it: a
library routine (scipy.signal.convolve2d / correlate2d, torch conv2d,
scipy.optimize.nnls), a dense matrix built from library convolutions of unit
vectors, the adjoint identity, closed forms (delta-PSF coadd), fixed points
(noise-free truth), and the invariants of Sec. 2 (non-negativity,
order-independence, the monotone likelihood of EM). A dropped term, a wrong
sign or index or a transposed operand in the oracle fails at least one.
"""
import numpy as np
import pytest
import scipy.signal as ss
from scipy.optimize import nnls

import oracle
import synth


def rng(s=0):
    return np.random.default_rng(s)


def rand_psf(K, g, positive=True):
    f = g.uniform(0.0, 1.0, (K, K)) if positive else g.standard_normal((K, K))
    return f / np.abs(f).sum()


# -- convolution conventions (Eq. (1)) ----------------------------------------

@pytest.mark.parametrize("H,W,K", [(9, 7, 1), (9, 7, 3), (12, 17, 5),
                                   (16, 11, 15), (5, 6, 9), (3, 4, 7)])
def test_conv_matches_scipy_convolve2d(H, W, K):
    g = rng(H * 100 + K)
    x = g.standard_normal((H, W))
    f = g.standard_normal((K, K))
    ref = ss.convolve2d(x, f, mode="same", boundary="fill")
    np.testing.assert_allclose(oracle.conv_same(x, f), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("H,W,K", [(9, 7, 3), (12, 17, 5), (16, 11, 15), (3, 4, 7)])
def test_corr_matches_scipy_correlate2d(H, W, K):
    g = rng(H * 10 + K)
    w = g.standard_normal((H, W))
    f = g.standard_normal((K, K))
    ref = ss.correlate2d(w, f, mode="same", boundary="fill")
    np.testing.assert_allclose(oracle.corr_same(w, f), ref, rtol=1e-13, atol=1e-13)


def test_conv_matches_torch_conv2d_flipped():
    torch = pytest.importorskip("torch")
    g = rng(5)
    x = g.standard_normal((20, 13))
    f = g.standard_normal((7, 7))
    # torch conv2d is a cross-correlation; a true convolution flips the kernel
    ref = torch.nn.functional.conv2d(
        torch.from_numpy(x)[None, None], torch.from_numpy(f[::-1, ::-1].copy())[None, None],
        padding=3)[0, 0].numpy()
    np.testing.assert_allclose(oracle.conv_same(x, f), ref, rtol=1e-13, atol=1e-13)
    ref2 = torch.nn.functional.conv2d(
        torch.from_numpy(x)[None, None], torch.from_numpy(f)[None, None],
        padding=3)[0, 0].numpy()
    np.testing.assert_allclose(oracle.corr_same(x, f), ref2, rtol=1e-13, atol=1e-13)


def test_convolution_orientation_elliptical():
    # an off-centre single tap moves flux in the direction of the tap offset
    f = np.zeros((5, 5))
    f[3, 4] = 1.0                      # tap at (+1, +2) from the centre
    x = np.zeros((9, 9))
    x[4, 4] = 1.0
    z = oracle.conv_same(x, f)
    assert z[5, 6] == 1.0 and z.sum() == 1.0


# -- D^r of Eq. (3) -------------------------------------------------------------

@pytest.mark.parametrize("r", [1, 2, 3])
def test_downsample_is_block_sum_and_upsample_replicates(r):
    g = rng(r)
    zf = g.standard_normal((4 * r, 5 * r))
    np.testing.assert_allclose(oracle.downsample(zf, r),
                               zf.reshape(4, r, 5, r).sum(axis=(1, 3)), rtol=1e-14)
    w = g.standard_normal((4, 5))
    np.testing.assert_array_equal(oracle.upsample(w, r),
                                  np.kron(w, np.ones((r, r))))


# -- adjoint pair ----------------------------------------------------------------

@pytest.mark.parametrize("K", [1, 3, 15, 43])
@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("H,W", [(13, 9), (6, 20)])
def test_adjoint_identity(K, r, H, W):
    g = rng(K * 7 + r + H)
    x = g.standard_normal((r * H, r * W))
    w = g.standard_normal((H, W))
    f = g.standard_normal((K, K))
    lhs = float(np.vdot(oracle.forward(x, f, r), w))
    rhs = float(np.vdot(x, oracle.adjoint(w, f, r)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs), np.abs(x).sum())


# -- dense brute force on 8x8 -----------------------------------------------------

def dense_operator(H, W, f, r):
    """A = D^r F as a dense (H W) x (rH rW) matrix from library convolutions of
    unit vectors."""
    Hf, Wf = r * H, r * W
    A = np.zeros((H * W, Hf * Wf))
    for k in range(Hf * Wf):
        e = np.zeros(Hf * Wf)
        e[k] = 1.0
        z = ss.convolve2d(e.reshape(Hf, Wf), f, mode="same")
        A[:, k] = synth.block_sum(z, r).ravel()
    return A


@pytest.mark.parametrize("K,r", [(3, 1), (5, 1), (3, 2), (5, 2)])
def test_em_step_matches_dense_brute_force(K, r):
    g = rng(K + 10 * r)
    H = W = 8 // r
    n = 3
    f = np.stack([rand_psf(K, g) for _ in range(n)])
    x = g.uniform(0.5, 2.0, (r * H, r * W))
    y = g.normal(2.0, 1.0, (n, H, W))
    v = g.uniform(0.5, 2.0, (n, H, W))
    mask = (g.uniform(size=(n, H, W)) > 0.2).astype(np.uint8)
    u, bad = oracle.weights(v, mask)
    assert bad == 0
    N = np.zeros(r * r * H * W)
    Den = np.zeros(r * r * H * W)
    for t in range(n):
        A = dense_operator(H, W, f[t], r)
        U = np.diag(u[t].ravel())
        N += A.T @ U @ y[t].ravel()
        Den += A.T @ U @ A @ x.ravel()
    x_ref = np.where(Den > 0, x.ravel() * np.maximum(N, 0) / np.where(Den > 0, Den, 1), x.ravel())
    yy = np.where(mask != 0, y, 0.0)
    N_or = oracle.numerator(yy, u, f, r)
    np.testing.assert_allclose(N_or.ravel(), N, rtol=1e-13, atol=1e-14)
    x1, den = oracle.em_step(x, N_or, u, f, r, return_den=True)
    np.testing.assert_allclose(den.ravel(), Den, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(x1.ravel(), x_ref, rtol=1e-13, atol=1e-14)


# -- closed forms and fixed points --------------------------------------------------

@pytest.mark.parametrize("K", [1, 5])
def test_delta_psf_gives_weighted_coadd(K):
    g = rng(K)
    n, H, W = 4, 10, 12
    f = np.zeros((n, K, K))
    f[:, K // 2, K // 2] = 1.0
    y = g.normal(1.0, 2.0, (n, H, W))          # includes negative data
    v = g.uniform(0.5, 3.0, (n, H, W))
    mask = (g.uniform(size=(n, H, W)) > 0.3).astype(np.uint8)
    mask[:, 0, 0] = 0                           # pixel masked in every frame
    y[mask == 0] = np.nan
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    N = oracle.numerator(yy, u, f)
    x0 = g.uniform(0.1, 5.0, (H, W))
    x1 = oracle.em_step(x0, N, u, f)
    su = u.sum(0)
    coadd = np.where(su > 0, np.maximum((u * yy).sum(0), 0) / np.where(su > 0, su, 1), x0)
    np.testing.assert_allclose(x1, coadd, rtol=1e-15, atol=0)
    assert x1[0, 0] == x0[0, 0]
    # a fixed point afterwards (zeros absorbed)
    np.testing.assert_allclose(oracle.em_step(x1, N, u, f), x1, rtol=1e-15, atol=0)


@pytest.mark.parametrize("r,K", [(1, 7), (2, 9)])
def test_noise_free_truth_is_fixed_point(r, K):
    g = rng(3 + r)
    n, H, W = 3, 12, 10
    x_true = g.uniform(0.2, 3.0, (r * H, r * W))
    f = np.stack([rand_psf(K, g) for _ in range(n)])
    y = np.stack([synth.block_sum(ss.convolve2d(x_true, f[t], mode="same"), r)
                  for t in range(n)])
    v = g.uniform(1.0, 4.0, (n, H, W))
    mask = (g.uniform(size=(n, H, W)) > 0.1).astype(np.uint8)
    u, _ = oracle.weights(v, mask)
    yy = np.where(mask != 0, y, 0.0)
    N = oracle.numerator(yy, u, f, r)
    x1 = oracle.em_step(x_true, N, u, f, r)
    np.testing.assert_allclose(x1, x_true, rtol=1e-12)


def small_problem(seed=0, H=40, W=36, n=3, K=7, r=1, mask_frac=0.1):
    g = rng(seed)
    x_true = synth.render_sky(r * H, r * W, 12, 2, g, mu=5.0, sigma=1.0,
                              re_range=(1.5, 3.0))
    f = np.stack([synth.moffat_psf(K, g.uniform(2, 3), 3.0) for _ in range(n)])
    v = np.empty((n, H, W))
    y = np.empty((n, H, W))
    for t in range(n):
        z = synth.block_sum(ss.convolve2d(x_true, f[t], mode="same"), r)
        v[t] = 50.0 + np.maximum(z, 0)
        y[t] = z + np.sqrt(v[t]) * g.standard_normal((H, W))
    mask = (g.uniform(size=(n, H, W)) > mask_frac).astype(np.uint8)
    y[mask == 0] = np.nan
    return x_true, y, v, f, mask


@pytest.mark.parametrize("r", [1, 2])
def test_monotone_likelihood_and_nonnegativity(r):
    x_true, y, v, f, mask = small_problem(seed=11 + r, r=r, H=32 // r * 2 // 2, W=28)
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    assert (yy < 0).any()
    N = oracle.numerator(yy, u, f, r)
    x = np.full((r * y.shape[1], r * y.shape[2]), oracle.default_x0(yy, u, r))
    ll_prev = oracle.loglik(x, yy, v, u, f, r)
    iters = 200 if r == 1 else 80
    for _ in range(iters):
        x = oracle.em_step(x, N, u, f, r)
        assert (x >= 0).all()
        ll = oracle.loglik(x, yy, v, u, f, r)
        assert ll >= ll_prev - 1e-12 * abs(ll_prev)
        ll_prev = ll


def test_scaling_and_permutation_equivariance():
    x_true, y, v, f, mask = small_problem(seed=21)
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    x0 = np.full(yy.shape[1:], 3.0)
    N = oracle.numerator(yy, u, f)
    xa = oracle.em_run(x0, N, u, f, 5)
    # y, x0 -> 2^s (y, x0) scales every iterate by 2^s exactly
    s = 2.0 ** 7
    xb = oracle.em_run(x0 * s, oracle.numerator(yy * s, u, f), u, f, 5)
    np.testing.assert_array_equal(xb, xa * s)
    # v -> 2^s v leaves the iterates unchanged exactly
    u2, _ = oracle.weights(v * 4.0, mask, y)
    xc = oracle.em_run(x0, oracle.numerator(yy, u2, f), u2, f, 5)
    np.testing.assert_array_equal(xc, xa)
    # exposure order does not matter (Sec. 2: all frames at once)
    p = [2, 0, 1]
    xd = oracle.em_run(x0, oracle.numerator(yy[p], u[p], f[p]), u[p], f[p], 5)
    np.testing.assert_allclose(xd, xa, rtol=1e-13)


def test_shift_equivariance_interior():
    g = rng(4)
    n, K, H, W = 2, 5, 40, 40
    f = np.stack([rand_psf(K, g) for _ in range(n)])
    base = np.zeros((H, W))
    base[15:22, 14:20] = g.uniform(1, 5, (7, 6))
    res = []
    for dy, dx in [(0, 0), (3, 2)]:
        xt = np.roll(np.roll(base, dy, 0), dx, 1)
        y = np.stack([ss.convolve2d(xt, f[t], mode="same") for t in range(n)])
        u = np.full((n, H, W), 0.5)
        N = oracle.numerator(y, u, f)
        res.append(oracle.em_run(np.ones((H, W)), N, u, f, 2))
    a = res[0][12:26, 12:26]
    b = res[1][15:29, 14:28]
    np.testing.assert_allclose(b, a, rtol=1e-14)


def test_literal_weights_equal_inside_weights_for_constant_u():
    g = rng(9)
    n, H, W, K = 3, 14, 11, 5
    f = np.stack([rand_psf(K, g) for _ in range(n)])
    y = g.normal(3.0, 1.0, (n, H, W))
    v = np.stack([np.full((H, W), g.uniform(0.5, 2.0)) for _ in range(n)])
    u, _ = oracle.weights(v)
    x0 = g.uniform(0.5, 1.5, (H, W))
    a = oracle.em_step(x0, oracle.numerator(y, u, f), u, f)
    b = oracle.em_step_literal(x0, y, u, f)
    np.testing.assert_allclose(a, b, rtol=1e-13)


def test_flux_of_forward_and_adjoint():
    g = rng(12)
    for r in (1, 2):
        K = 7
        f = rand_psf(K, g)
        x = np.zeros((r * 20, r * 20))
        x[r * 8:r * 12, r * 8:r * 12] = g.uniform(1, 2, (4 * r, 4 * r))
        # D^r is a block SUM: flux is conserved by the forward model
        assert abs(oracle.forward(x, f, r).sum() - x.sum()) < 1e-12 * x.sum()
        w = np.zeros((20, 20))
        w[8:12, 8:12] = g.uniform(1, 2, (4, 4))
        assert abs(oracle.adjoint(w, f, r).sum() - r * r * w.sum()) < 1e-12 * w.sum()


def test_flux_conservation_at_the_fixed_point():
    """Sec. 2: with normalised PSFs the weighted flux is fixed at convergence.

    At a fixed point of Eq. (2) where every x_j > 0, N_j = Den_j for all j.
    Summing over j, with u_t a constant c_t on exposure t and every source at
    least 2K pixels from the edges (so that neither F_t nor F_t^T loses flux
    over the border): sum_t c_t sum_i y_t,i = sum_t c_t sum_j x_j, i.e.
        sum x = sum_t c_t sum y_t / sum_t c_t.
    The exposures are scaled by different transparencies s_t, so the data are
    inconsistent and the identity depends on the weights: weighting by v_t
    instead of 1/v_t would move the target by 10%. The sky is smooth Gaussian
    blobs on a tiny positive pedestal, so the fixed point is the unconstrained
    minimiser (s-bar times the truth, strictly positive) and EM reaches it
    linearly instead of creeping towards zeros. Data come from scipy's direct
    convolution, not from the oracle."""
    g = rng(5)
    H = W = 32
    n, K = 3, 5
    f = np.stack([synth.moffat_psf(K, 1.6, 3.0)] * n)
    x_true = np.full((H, W), 1e-5)
    yy, xx = np.mgrid[:H, :W]
    for _ in range(4):   # centres in [13, 19): >= 2K = 10 pixels from every edge
        ci, cj = g.uniform(13, 19, 2)
        x_true += g.lognormal(5, 0.5) * np.exp(-((yy - ci) ** 2 + (xx - cj) ** 2) / 4.5)
    s = np.array([1.0, 1.3, 0.8])
    vt = np.array([50.0, 120.0, 300.0])
    y = np.stack([s[t] * ss.convolve2d(x_true, f[t], mode="same") for t in range(n)])
    v = np.stack([np.full((H, W), vt[t]) for t in range(n)])
    u, bad = oracle.weights(v)
    assert bad == 0
    c = 1.0 / vt
    target = (c * y.sum(axis=(1, 2))).sum() / c.sum()
    wrong = (vt * y.sum(axis=(1, 2))).sum() / vt.sum()
    assert abs(wrong - target) > 0.05 * target
    N = oracle.numerator(y, u, f)
    x = oracle.em_run(np.full((H, W), oracle.default_x0(y, u)), N, u, f, 5000)
    x_next = oracle.em_step(x, N, u, f)
    assert np.abs(x_next - x).max() <= 1e-9 * x.max()   # converged
    assert (x > 0).all()
    assert abs(x.sum() - target) <= 1e-6 * target


def test_em_converges_to_nnls_solution():
    g = rng(17)
    n, H, W = 2, 6, 6
    f = np.zeros((n, 3, 3))
    f[:, 1, 1] = 0.6
    f[:, 0, 1] = f[:, 2, 1] = f[:, 1, 0] = f[:, 1, 2] = 0.1
    x_true = g.uniform(0.0, 3.0, (H, W))
    x_true[g.uniform(size=(H, W)) < 0.3] = 0.0
    v = g.uniform(0.5, 2.0, (n, H, W))
    y = np.stack([ss.convolve2d(x_true, f[t], mode="same") for t in range(n)])
    y += 0.8 * g.standard_normal(y.shape)
    u, _ = oracle.weights(v)
    A = np.vstack([np.sqrt(u[t].ravel())[:, None] * dense_operator(H, W, f[t], 1)
                   for t in range(n)])
    b = np.concatenate([np.sqrt(u[t].ravel()) * y[t].ravel() for t in range(n)])
    x_nnls, _ = nnls(A, b, maxiter=10000)
    assert (x_nnls == 0).any()                  # the constraint is active
    N = oracle.numerator(y, u, f)
    x = oracle.em_run(np.ones((H, W)), N, u, f, 100000)
    np.testing.assert_allclose(x.ravel(), x_nnls, rtol=1e-6, atol=1e-6)


# -- likelihood, weights, initial guess ----------------------------------------------

def test_loglik_matches_library_formula():
    x_true, y, v, f, mask = small_problem(seed=5, r=1)
    u, bad = oracle.weights(v, mask, y)
    assert bad == 0
    yy = np.where(mask != 0, y, 0.0)
    x = np.abs(x_true) + 1.0
    ref = 0.0
    for t in range(y.shape[0]):
        z = ss.convolve2d(x, f[t], mode="same")
        m = mask[t] != 0
        ref += ((y[t][m] - z[m]) ** 2 / v[t][m]).sum() + np.log(2 * np.pi * v[t][m]).sum()
    np.testing.assert_allclose(oracle.loglik(x, yy, v, u, f), -0.5 * ref, rtol=1e-12)


def test_weights_mask_and_validation():
    v = np.array([[1.0, 2.0], [0.0, -1.0]])[None]
    y = np.array([[1.0, np.nan], [3.0, 4.0]])[None]
    m = np.array([[1, 0], [0, 1]], np.uint8)[None]
    u, bad = oracle.weights(v, m, y)
    np.testing.assert_array_equal(u[0], [[1.0, 0.0], [0.0, 0.0]])
    assert bad == 1                             # v = -1 at a valid pixel
    u2, bad2 = oracle.weights(np.abs(v) + 1, m, y)
    assert bad2 == 0 and u2[0, 1, 0] == 0.0


def test_default_x0_closed_form():
    y = np.full((3, 4, 5), 6.0)
    u = np.full((3, 4, 5), 0.25)
    assert oracle.default_x0(y, u, 1) == 6.0
    assert oracle.default_x0(y, u, 2) == 1.5
    assert oracle.default_x0(-y, u, 1) == 1.0


@pytest.mark.parametrize("r,K", [(1, 5), (2, 7)])
def test_em_step_at_matches_full_step(r, K):
    x_true, y, v, f, mask = small_problem(seed=30 + r, r=r, H=16, W=14, K=K)
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    N = oracle.numerator(yy, u, f, r)
    x0 = np.abs(x_true) + 0.5
    x1, den = oracle.em_step(x0, N, u, f, r, return_den=True)
    idx = np.array([0, 5, x0.size // 2 + 3, x0.size - 1, x0.shape[1] * 3 + 1])
    xo, No, Do = oracle.em_step_at(x0, y, u, f, idx, r)   # NaN y where masked
    np.testing.assert_allclose(Do, den.ravel()[idx], rtol=1e-12)
    np.testing.assert_allclose(No, N.ravel()[idx], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(xo, x1.ravel()[idx], rtol=1e-12)


# -- streaming (frame-by-frame) EM, the order-dependent contrast of Sec. 2 --------

def _stream_problem(seed=41, n=3, r=1):
    x_true, y, v, f, mask = small_problem(seed=seed, H=24, W=20, n=n, K=5, r=r)
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    return x_true, yy, v, f, mask, u


def test_streaming_with_one_exposure_is_the_batch_update():
    x_true, y, v, f, mask, u = _stream_problem(n=1)
    x0 = np.abs(x_true) + 1.0
    a = oracle.em_streaming(x0, y, u, f, 3)
    b = oracle.em_run(x0, oracle.numerator(y, u, f), u, f, 3)
    np.testing.assert_allclose(a, b, rtol=1e-14)


def test_streaming_pass_is_a_sequence_of_single_frame_updates():
    x_true, y, v, f, mask, u = _stream_problem(n=3)
    x0 = np.abs(x_true) + 1.0
    order = [2, 0, 1]
    x = x0.copy()
    for t in order:
        x = oracle.em_step(x, oracle.numerator(y[t:t + 1], u[t:t + 1], f[t:t + 1]),
                           u[t:t + 1], f[t:t + 1])
    np.testing.assert_allclose(oracle.em_streaming(x0, y, u, f, 1, order=order), x, rtol=1e-14)


def test_streaming_depends_on_frame_order_unlike_eq2():
    x_true, y, v, f, mask, u = _stream_problem(n=3)
    x0 = np.abs(x_true) + 1.0
    a = oracle.em_streaming(x0, y, u, f, 2, order=[0, 1, 2])
    b = oracle.em_streaming(x0, y, u, f, 2, order=[2, 1, 0])
    assert np.linalg.norm(a - b) > 1e-6 * np.linalg.norm(a)


@pytest.mark.parametrize("r", [1, 2])
def test_streaming_keeps_the_noise_free_truth(r):
    g = rng(8)
    n, H, W, K = 3, 10, 12, 5
    x_true = g.uniform(0.2, 3.0, (r * H, r * W))
    f = np.stack([rand_psf(K, g) for _ in range(n)])
    y = np.stack([synth.block_sum(ss.convolve2d(x_true, f[t], mode="same"), r) for t in range(n)])
    u = g.uniform(0.3, 1.0, (n, H, W))
    np.testing.assert_allclose(oracle.em_streaming(x_true, y, u, f, 2, r=r), x_true, rtol=1e-12)


# -- PSF super-resolution fit, Eq. (4) ------------------------------------------------

def gauss_kernel(r):
    """Normalised Gaussian with FWHM r fine pixels (the width of Eq. (4)'s g)."""
    return synth.gaussian_kernel(r)


def psf_model_numpy(h, g, r, K):
    q = ss.convolve2d(h, g, mode="same")
    Kh = h.shape[0]
    full = np.zeros((r * K, r * K))
    full[:Kh, :Kh] = q
    return full.reshape(K, r, K, r).sum(axis=(1, 3))


def psf_loss_numpy(h, f, g, r, lam):
    K = f.shape[0]
    res = psf_model_numpy(h, g, r, K) - f
    return (res ** 2).sum() + lam * ((np.diff(h, axis=0) ** 2).sum() + (np.diff(h, axis=1) ** 2).sum())


@pytest.mark.parametrize("K,r", [(7, 2), (9, 3), (5, 1)])
def test_psf_model_library_and_adjoint(K, r):
    g_ = rng(K + r)
    Kh = oracle.psf_fine_side(K, r)
    h = g_.uniform(0, 1, (Kh, Kh))
    g = gauss_kernel(r)
    np.testing.assert_allclose(oracle.psf_model(h, g, r, K), psf_model_numpy(h, g, r, K),
                               rtol=1e-13, atol=1e-14)
    w = g_.standard_normal((K, K))
    lhs = float(np.vdot(oracle.psf_model(h, g, r, K), w))
    rhs = float(np.vdot(h, oracle.psf_model_adjoint(w, g, r, Kh)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_psf_loss_and_gradient():
    g_ = rng(3)
    K, r, lam = 9, 2, 0.3
    Kh = oracle.psf_fine_side(K, r)
    g = gauss_kernel(r)
    f = synth.moffat_psf(K, 2.5, 3.0)
    h = g_.uniform(0, 0.02, (Kh, Kh))
    L, gr = oracle.psf_loss(h, f, g, r, lam, grad=True)
    assert abs(L - psf_loss_numpy(h, f, g, r, lam)) <= 1e-12 * L
    for idx in [(0, 0), (Kh // 2, Kh // 2), (3, Kh - 1), (Kh - 1, 5)]:
        e = np.zeros_like(h)
        e[idx] = 1e-6
        fd = (psf_loss_numpy(h + e, f, g, r, lam) - psf_loss_numpy(h - e, f, g, r, lam)) / 2e-6
        assert abs(fd - gr[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_psf_fit_reaches_the_constrained_minimiser():
    from scipy.optimize import minimize
    K, r, lam = 9, 2, 1e-3
    Kh = oracle.psf_fine_side(K, r)
    g = gauss_kernel(r)
    f = synth.moffat_psf(K, 2.2, 3.0, ellip=0.1, angle=0.4)
    h0 = np.kron(f, np.ones((r, r)))[:Kh, :Kh] / r ** 2
    h = oracle.psf_fit(f, g, r, lam, 20000, 1e-4, h0)
    res = minimize(lambda z: psf_loss_numpy(z.reshape(Kh, Kh), f, g, r, lam),
                   h0.ravel(), method="L-BFGS-B", bounds=[(0, None)] * (Kh * Kh),
                   jac=lambda z: oracle.psf_loss(z.reshape(Kh, Kh), f, g, r, lam, grad=True)[1].ravel(),
                   options=dict(maxiter=20000, ftol=1e-16, gtol=1e-12))
    hs = res.x.reshape(Kh, Kh)
    Lh, Ls = psf_loss_numpy(h, f, g, r, lam), psf_loss_numpy(hs, f, g, r, lam)
    assert Lh <= Ls * (1 + 1e-6)
    assert np.linalg.norm(h - hs) <= 1e-4 * np.linalg.norm(hs)
    assert (h >= 0).all()


def adam_iterates_numpy(f, g, r, lam, lr, iters, h0):
    """Every iterate h_0 .. h_iters of projected Adam on Eq. (4) (Kingma & Ba
    with bias correction), gradients by the chain rule through the library
    model psf_model_numpy."""
    K = f.shape[0]
    Kh = h0.shape[0]
    h, m, v = h0.copy(), np.zeros_like(h0), np.zeros_like(h0)
    out = [h.copy()]
    for k in range(1, iters + 1):
        res = psf_model_numpy(h, g, r, K) - f
        rep = np.kron(res, np.ones((r, r)))[:Kh, :Kh]
        gr = 2 * ss.correlate2d(rep, g, mode="same")
        gr[1:] += 2 * lam * np.diff(h, axis=0)
        gr[:-1] -= 2 * lam * np.diff(h, axis=0)
        gr[:, 1:] += 2 * lam * np.diff(h, axis=1)
        gr[:, :-1] -= 2 * lam * np.diff(h, axis=1)
        m = 0.9 * m + 0.1 * gr
        v = 0.999 * v + 0.001 * gr * gr
        h = np.maximum(h - lr * (m / (1 - 0.9 ** k)) / (np.sqrt(v / (1 - 0.999 ** k)) + 1e-8), 0)
        out.append(h.copy())
    return out


@pytest.mark.parametrize("iters,lr", [(0, 1e-3), (1, 1e-3), (40, 1e-3), (300, 1e-2)])
def test_psf_fit_returns_the_lowest_loss_iterate(iters, lr):
    """Adam at a fixed step is not monotone: with a large step the loss
    rises again late in the run, and the fit must return the best iterate
    (the first on ties) with its loss."""
    K, r, lam = 5, 2, 1e-2
    g = gauss_kernel(r)
    f = synth.moffat_psf(K, 1.6, 3.0)
    Kh = oracle.psf_fine_side(K, r)
    h0 = np.kron(f, np.ones((r, r)))[:Kh, :Kh] / r ** 2
    hs = adam_iterates_numpy(f, g, r, lam, lr, iters, h0)
    Ls = [psf_loss_numpy(h, f, g, r, lam) for h in hs]
    kbest = int(np.argmin(Ls))
    h, L = oracle.psf_fit(f, g, r, lam, iters, lr, h0, with_loss=True)
    np.testing.assert_allclose(h, hs[kbest], rtol=1e-9, atol=1e-15)
    assert abs(L - Ls[kbest]) <= 1e-12 * Ls[kbest]
    if iters == 300:
        assert 0 < kbest < iters   # the case exercises a late rise


# -- heavy-tailed (Student-t) noise ------------------------------------------------

def forward_numpy(x, f, r):
    return np.stack([synth.block_sum(ss.convolve2d(x, f[t], mode="same"), r)
                     for t in range(f.shape[0])])


@pytest.mark.parametrize("K,r", [(3, 1), (5, 1), (3, 2)])
def test_student_step_matches_dense_brute_force(K, r):
    g = rng(70 + K + 10 * r)
    H = W = 8 // r
    n, nu = 3, 3.0
    f = np.stack([rand_psf(K, g) for _ in range(n)])
    x = g.uniform(0.5, 2.0, (r * H, r * W))
    y = g.normal(2.0, 1.5, (n, H, W))
    v = g.uniform(0.5, 2.0, (n, H, W))
    mask = (g.uniform(size=(n, H, W)) > 0.2).astype(np.uint8)
    u, _ = oracle.weights(v, mask)
    yy = np.where(mask != 0, y, 0.0)
    N = np.zeros(r * r * H * W)
    Den = np.zeros(r * r * H * W)
    for t in range(n):
        A = dense_operator(H, W, f[t], r)
        z = A @ x.ravel()
        ut = u[t].ravel()
        s = np.where(ut > 0, (nu + 1) / (nu + ut * (yy[t].ravel() - z) ** 2), 0.0)
        N += A.T @ (ut * s * yy[t].ravel())
        Den += A.T @ (ut * s * z)
    x_ref = np.where(Den > 0, x.ravel() * np.maximum(N, 0) / np.where(Den > 0, Den, 1), x.ravel())
    x1, num, den = oracle.em_step_student(x, yy, u, f, nu, r)
    np.testing.assert_allclose(num.ravel(), N, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(den.ravel(), Den, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(x1.ravel(), x_ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("r", [1, 2])
def test_student_reduces_to_eq2_as_nu_grows(r):
    x_true, y, v, f, mask = small_problem(seed=80 + r, r=r, H=24, W=20, K=5)
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    N = oracle.numerator(yy, u, f, r)
    x0 = np.full((r * 24, r * 20), 2.0)
    xg = oracle.em_step(x0, N, u, f, r)
    xs, num, _ = oracle.em_step_student(x0, yy, u, f, 1e13, r)
    np.testing.assert_allclose(num, N, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(xs, xg, rtol=1e-9, atol=1e-12)


def test_student_loglik_matches_scipy_t_logpdf():
    from scipy.stats import t as student_t
    for r, nu in [(1, 2.5), (2, 7.0)]:
        x_true, y, v, f, mask = small_problem(seed=90 + r, r=r, H=16, W=14, K=5)
        u, _ = oracle.weights(v, mask, y)
        yy = np.where(mask != 0, y, 0.0)
        x = x_true * 0.9 + 0.5
        z = forward_numpy(x, f, r)
        ok = mask != 0
        ref = student_t.logpdf(yy[ok], df=nu, loc=z[ok], scale=np.sqrt(v[ok])).sum()
        got = oracle.student_loglik(x, yy, v, u, f, nu, r)
        assert abs(got - ref) <= 1e-10 * abs(ref)


def test_student_weights_closed_form():
    g = rng(95)
    y, z = g.normal(0, 3, 50), g.normal(0, 3, 50)
    u = g.uniform(0.1, 2, 50)
    u[::7] = 0.0
    w = oracle.student_weights(y, u, z, 4.0)
    np.testing.assert_allclose(w[u > 0], (u * 5.0 / (4.0 + u * (y - z) ** 2))[u > 0], rtol=1e-15)
    assert (w[u == 0] == 0).all()


@pytest.mark.parametrize("r", [1, 2])
def test_student_em_is_monotone_and_keeps_the_truth(r):
    """A generalised EM step never lowers the Student-t likelihood (with
    outliers, masks and negative data), and noise-free data leave the truth
    fixed."""
    x_true, y, v, f, mask = small_problem(seed=100 + r, r=r, H=24, W=22, K=5)
    g = rng(7)
    y[0, 5, :] += 400.0                      # a satellite trail in one exposure
    y[1, g.integers(0, 24, 12), g.integers(0, 22, 12)] += 300.0
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    nu = 3.0
    x = np.full((r * 24, r * 22), oracle.default_x0(yy, u, r))
    ll = oracle.student_loglik(x, yy, v, u, f, nu, r)
    for _ in range(60 if r == 1 else 30):
        x = oracle.em_step_student(x, yy, u, f, nu, r)[0]
        assert (x >= 0).all()
        ll1 = oracle.student_loglik(x, yy, v, u, f, nu, r)
        assert ll1 >= ll - 1e-12 * abs(ll)
        ll = ll1
    y0 = forward_numpy(x_true, f, r)
    x1 = oracle.em_step_student(x_true, y0, u, f, nu, r)[0]
    np.testing.assert_allclose(x1, x_true, rtol=1e-12)


def test_student_em_resists_outliers_better_than_eq2():
    x_true, y, v, f, mask = small_problem(seed=120, H=32, W=30, n=4, K=5, mask_frac=0.0)
    y[0, 10, :] += 2000.0                    # satellite trails the mask missed
    y[2, :, 7] += 2000.0
    u, _ = oracle.weights(v, mask, y)
    yy = np.where(mask != 0, y, 0.0)
    x0 = np.full((32, 30), oracle.default_x0(yy, u))
    N = oracle.numerator(yy, u, f)
    xg, xs = x0.copy(), x0.copy()
    for _ in range(150):
        xg = oracle.em_step(xg, N, u, f)
        xs = oracle.em_step_student(xs, yy, u, f, 3.0)[0]
    eg = np.linalg.norm(forward_numpy(xg, f, 1) - forward_numpy(x_true, f, 1))
    es = np.linalg.norm(forward_numpy(xs, f, 1) - forward_numpy(x_true, f, 1))
    assert es < 0.5 * eg
