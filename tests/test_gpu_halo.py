"""The halo-exchange FP32 kernel (EMD_PREC_FP32, csrc/emd_halo.cu) against
the CTA-pair kernel (EMD_PREC_FP32_PAIR) and against the FP64 oracle.

Both kernels evaluate every output with the same FP32 operations in the same
order (the tap order of each forward and adjoint sum, w = u z, Den + sum,
the guarded ratio of Eq. (2)), so their iterates must agree bit for bit.
Shapes cover one tile, ragged edges, one row and one column of tiles, K = 1,
r = 2, and grids large enough that the w ring's slots are reused within a
launch; several iterations in a row also check that the kernel's flags and
counters are reset for the next launch."""
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


def run(emd, p, x0, k, prec):
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    try:
        d.set_frames(p.y, p.v, p.f, p.mask)
        d.set_precision(prec)
        d.set_x(x0)
        out = []
        for _ in range(k):
            d.iterate(1)
            out.append(d.x())
        return out
    finally:
        d.close()


def start(p, seed=0):
    g = np.random.default_rng(seed)
    return (g.uniform(0.5, 1.5, (p.r * p.H, p.r * p.W)) * 10.0).astype(np.float32)


# (H, W, n, K, r) with 64 x 128 tiles: two tiles; ragged 5 x 3 tiles; two
# rows of tiles; one column; K = 1; r = 2 with a ragged grid; 16 x 8 tiles x 12
# exposures (1536 forward items > 979 ring slots: slots reused in the launch)
CASES = [(96, 80, 3, 15, 1), (300, 257, 5, 43, 1), (100, 1500, 3, 21, 1),
         (1400, 90, 3, 21, 1), (260, 300, 4, 1, 1), (200, 330, 4, 9, 2),
         (1024, 1024, 12, 43, 1)]


@pytest.mark.parametrize("H,W,n,K,r", CASES)
def test_bit_identical_to_cta_pair_kernel(emd, H, W, n, K, r):
    p = synth.make_problem("hsc", H=H, W=W, n=n, K=K, r=r, mask_frac=0.05,
                           fwhm=(2.0 * r, 5.0 * r), n_points=60, n_gal=4, seed_offset=H + W + K)
    x0 = start(p, seed=n)
    a = run(emd, p, x0, 3, emd.EMD_PREC_FP32)
    b = run(emd, p, x0, 3, emd.EMD_PREC_FP32_PAIR)
    for it in range(3):
        assert np.array_equal(a[it], b[it]), (it, np.abs(a[it] - b[it]).max())


def test_oracle_parity_with_ring_reuse(emd):
    """A ragged 11 x 6 grid of 64 x 128 tiles with 40 exposures: 2640 forward
    items through a ring of 975 slots, so slots are rewritten within every
    launch; one and five iterations against the oracle at the FP32 path's
    tolerances."""
    p = synth.make_problem("hsc", H=700, W=650, n=40, K=15, r=1, mask_frac=0.05,
                           fwhm=(2.0, 4.0), n_points=80, n_gal=5, seed_offset=3)
    x0 = start(p, seed=1)
    xs = run(emd, p, x0, 5, emd.EMD_PREC_FP32)
    u, y, N, _ = oracle.prepare(p)
    x1 = oracle.em_run(x0.astype(np.float64), N, u, p.f, 1, p.r)
    e1 = np.linalg.norm(xs[0] - x1) / np.linalg.norm(x1)
    assert e1 <= 1e-5, e1
    x5 = oracle.em_run(x1, N, u, p.f, 4, p.r)
    e5 = np.linalg.norm(xs[4] - x5) / np.linalg.norm(x5)
    assert e5 <= 1e-4, e5


def test_alternating_with_the_pair_kernel_and_streaming(emd):
    """The ring kernel and the CTA-pair kernel share the context's Den plane:
    alternate them (and the streaming pass) and compare with running the
    CTA-pair kernel throughout."""
    p = synth.make_problem("hsc", H=260, W=270, n=4, K=15, r=1, mask_frac=0.05,
                           fwhm=(2.0, 4.0), n_points=40, n_gal=3, seed_offset=9)
    x0 = start(p, seed=2)

    def seq(first):
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        try:
            d.set_frames(p.y, p.v, p.f, p.mask)
            d.set_x(x0)
            d.set_precision(first)
            d.iterate(2)
            d.iterate_streaming(1)
            d.iterate(2)
            return d.x()
        finally:
            d.close()

    assert np.array_equal(seq(emd.EMD_PREC_FP32), seq(emd.EMD_PREC_FP32_PAIR))


STUDENT_CASES = [(300, 257, 5, 43, 1), (200, 330, 4, 9, 2), (700, 650, 40, 15, 1)]


@pytest.mark.parametrize("H,W,n,K,r", STUDENT_CASES)
def test_heavy_tailed_bit_identical_to_cta_pair_kernel(emd, H, W, n, K, r):
    """Student-t noise (nu = 3): the halo kernel's one-launch step (forward
    once, adjoints of u'z and u'y) against the CTA-pair kernel's two launches
    (N' with its own forward pass, then Den' and the update)."""
    p = synth.make_problem("hsc", H=H, W=W, n=n, K=K, r=r, mask_frac=0.05,
                           fwhm=(2.0 * r, 5.0 * r), n_points=60, n_gal=4, seed_offset=7 * H + K)
    x0 = start(p, seed=n + 1)

    def go(prec):
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        try:
            d.set_frames(p.y, p.v, p.f, p.mask)
            d.set_noise(emd.EMD_NOISE_STUDENT_T, 3.0)
            d.set_precision(prec)
            d.set_x(x0)
            out = []
            for _ in range(3):
                d.iterate(1)
                out.append(d.x())
            return out
        finally:
            d.close()

    a, b = go(emd.EMD_PREC_FP32), go(emd.EMD_PREC_FP32_PAIR)
    for it in range(3):
        assert np.array_equal(a[it], b[it]), (it, np.abs(a[it] - b[it]).max())


def test_switching_noise_models_in_one_context(emd):
    """Gaussian, then Student-t, then Gaussian again in one context: the ring
    is re-laid out (two tiles per slot and back) and its counters restart
    from zero; the iterates equal the CTA-pair kernel's."""
    p = synth.make_problem("hsc", H=520, W=400, n=6, K=15, r=1, mask_frac=0.05,
                           fwhm=(2.0, 4.0), n_points=40, n_gal=3, seed_offset=21)
    x0 = start(p, seed=3)

    def go(prec):
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        try:
            d.set_frames(p.y, p.v, p.f, p.mask)
            d.set_precision(prec)
            d.set_x(x0)
            d.iterate(2)
            d.set_noise(emd.EMD_NOISE_STUDENT_T, 4.0)
            d.iterate(2)
            d.set_noise(emd.EMD_NOISE_GAUSSIAN)
            d.iterate(2)
            return d.x()
        finally:
            d.close()

    assert np.array_equal(go(emd.EMD_PREC_FP32), go(emd.EMD_PREC_FP32_PAIR))


@pytest.mark.parametrize("H,W,n,K,r,nu", [(300, 257, 5, 43, 1, 0.0), (200, 330, 4, 9, 2, 0.0),
                                          (520, 400, 6, 15, 1, 3.0), (1024, 1024, 12, 43, 1, 0.0)])
def test_loglik_against_cta_pair_kernel(emd, H, W, n, K, r, nu):
    """emd_loglik's data term from the forward-only halo kernel (each pixel
    once, FP64 partial sums per (tile, exposure group) added in a fixed
    order) against the CTA-pair kernel's: the same FP32 model values summed
    in another order, so equal to FP64 rounding; and repeatable bit for bit."""
    p = synth.make_problem("hsc", H=H, W=W, n=n, K=K, r=r, mask_frac=0.05,
                           fwhm=(2.0 * r, 5.0 * r), n_points=60, n_gal=4, seed_offset=H + n)
    x0 = start(p, seed=5)
    out = {}
    for prec in (emd.EMD_PREC_FP32, emd.EMD_PREC_FP32_PAIR):
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        try:
            d.set_frames(p.y, p.v, p.f, p.mask)
            if nu > 0:
                d.set_noise(emd.EMD_NOISE_STUDENT_T, nu)
            d.set_precision(prec)
            d.set_x(x0)
            out[prec] = [d.loglik(), d.loglik()]
        finally:
            d.close()
    (ll_a, chi_a), (ll_a2, chi_a2) = out[emd.EMD_PREC_FP32]
    (ll_b, chi_b), _ = out[emd.EMD_PREC_FP32_PAIR]
    assert ll_a == ll_a2 and chi_a == chi_a2
    assert abs(chi_a - chi_b) <= 1e-12 * abs(chi_b)
    assert abs(ll_a - ll_b) <= 1e-12 * abs(ll_b)


# tile shapes of the halo-exchange kernel: 64, 48 and 32 rows of 128 columns
TILE_CASES = [(300, 257, 5, 43, 1, 0.0), (1024, 1024, 12, 43, 1, 0.0), (200, 330, 4, 9, 2, 0.0),
              (96, 80, 3, 15, 1, 0.0), (260, 300, 4, 21, 1, 3.0)]


@pytest.mark.parametrize("H,W,n,K,r,nu", TILE_CASES)
def test_tile_shapes_give_bit_identical_iterates(emd, H, W, n, K, r, nu):
    """Every output's taps are summed in the same order whatever block of
    the tile it falls in, so all tile shapes give the same iterates bit for bit (ragged
    last rows of tiles, ring reuse at 1024^2 x 12, r = 2, heavy-tailed
    noise), and they match the oracle."""
    p = synth.make_problem("hsc", H=H, W=W, n=n, K=K, r=r, mask_frac=0.05,
                           fwhm=(2.0 * r, 5.0 * r), n_points=60, n_gal=4, seed_offset=H + K)
    x0 = start(p, seed=n)
    out = {}
    shapes = (emd.EMD_TILE_64, emd.EMD_TILE_48, emd.EMD_TILE_32)
    for shape in shapes:
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        try:
            d.set_frames(p.y, p.v, p.f, p.mask)
            if nu > 0:
                d.set_noise(emd.EMD_NOISE_STUDENT_T, nu)
            d.set_tile_shape(shape)
            assert d.tile_shape() == (shape, True)
            d.set_x(x0)
            d.iterate(3)
            out[shape] = d.x()
        finally:
            d.close()
    for shape in shapes[1:]:
        np.testing.assert_array_equal(out[shape], out[emd.EMD_TILE_64])
    if nu == 0:
        u, y, N, _ = oracle.prepare(p)
        xo = oracle.em_run(x0, N, u, p.f, 3, p.r)
        assert np.linalg.norm(out[emd.EMD_TILE_64] - xo) / np.linalg.norm(xo) <= 2e-5


def test_autotuner_decides_a_tile_shape(emd):
    """With EMD_TILE_AUTO (the default) the first iterations of a new problem
    shape time the candidate tile shapes; the decision is kept for the
    problem shape and the iterates equal those of a fixed shape."""
    p = synth.make_problem("hsc", H=640, W=512, n=6, K=43, mask_frac=0.05, n_points=80,
                           n_gal=4, seed_offset=5)
    x0 = start(p, seed=2)
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    d.set_x(x0)
    done = 0
    while done < 16:
        d.iterate(1)
        done += 1
        emd.emd_get_x(d.ctx, np.empty((p.H, p.W), np.float32))   # synchronises
        if d.tile_shape()[1]:
            break
    shape, decided = d.tile_shape()
    assert decided and shape in (1, 2, 3)
    d.iterate(1)   # one iteration on the decided shape
    done += 1
    xt = d.x()
    d.close()
    # the same number of iterations on a fixed shape
    e = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    e.set_frames(p.y, p.v, p.f, p.mask)
    e.set_tile_shape(emd.EMD_TILE_64)
    e.set_x(x0)
    e.iterate(done)
    np.testing.assert_array_equal(xt, e.x())
    e.close()
    # a second context of the same shape starts with the decision
    f = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    f.set_frames(p.y, p.v, p.f, p.mask)
    assert f.tile_shape() == (shape, True)
    f.close()
    g = emd.Deconvolver(8, 8, 1, 3, 1)
    try:
        with pytest.raises(emd.EMDError):
            g.set_tile_shape(9)
    finally:
        g.close()
