"""Host-side pin of the polyphase form of Eq. (3) that the GPU kernels use for
r > 1, in FP64 against the oracle's forward model D^r(f * x) and its
adjoint.

With h = (K - 1) / 2, hc = ceil(h / r) and Kc = 2 hc + 1, the phase
(py, px) of the fine latent, x_p(i, j) = x(r i + py, r j + px), meets the
phase kernel
    k_p[sy][sx] = sum_{dy, dx in [0, r)} f(dy + h - r sy - py, dx + h - r sx - px)
for sy, sx in [-hc, hc] (zero where the index leaves f), and
    D^r(f * x)(i, j) = sum_p sum_{sy, sx} k_p[sy][sx] x_p(i + sy, j + sx),
    (F^T D^rT w)(r i + py, r j + px) = sum_{sy, sx} k_p[sy][sx] w(i - sy, j - sx),
with x_p and w zero outside the image: r^2 Kc x Kc kernels on the coarse
grid, (K + r - 1)^2 multiply-adds per coarse pixel instead of r^2 K^2."""
import numpy as np
import pytest

import oracle


def phase_kernels(f, r):
    K = f.shape[0]
    h = (K - 1) // 2
    hc = (h + r - 1) // r
    Kc = 2 * hc + 1
    k = np.zeros((r, r, Kc, Kc))
    for py in range(r):
        for px in range(r):
            for sy in range(-hc, hc + 1):
                for sx in range(-hc, hc + 1):
                    acc = 0.0
                    for dy in range(r):
                        for dx in range(r):
                            a, b = dy + h - r * sy - py, dx + h - r * sx - px
                            if 0 <= a < K and 0 <= b < K:
                                acc += f[a, b]
                    k[py, px, sy + hc, sx + hc] = acc
    return k, hc


def shifted(img, sy, sx):
    """img(i + sy, j + sx), zero outside"""
    H, W = img.shape
    out = np.zeros_like(img)
    ys, ye = max(0, -sy), min(H, H - sy)
    xs, xe = max(0, -sx), min(W, W - sx)
    out[ys:ye, xs:xe] = img[ys + sy:ye + sy, xs + sx:xe + sx]
    return out


@pytest.mark.parametrize("H,W,K,r", [(40, 37, 15, 2), (30, 33, 9, 3), (24, 20, 21, 2), (17, 19, 1, 2)])
def test_forward_and_adjoint_in_polyphase_form(H, W, K, r):
    rng = np.random.default_rng(K * 10 + r)
    x = rng.uniform(0.0, 2.0, (r * H, r * W))
    w = rng.normal(size=(H, W))
    f = rng.uniform(0.0, 1.0, (K, K))
    f /= f.sum()
    k, hc = phase_kernels(f, r)
    assert k.shape[2] == 2 * (((K - 1) // 2 + r - 1) // r) + 1
    z = np.zeros((H, W))
    den = np.zeros((r * H, r * W))
    for py in range(r):
        for px in range(r):
            xp = x[py::r, px::r]
            dp = np.zeros((H, W))
            for sy in range(-hc, hc + 1):
                for sx in range(-hc, hc + 1):
                    c = k[py, px, sy + hc, sx + hc]
                    z += c * shifted(xp, sy, sx)
                    dp += c * shifted(w, -sy, -sx)
            den[py::r, px::r] = dp
    z_ref = oracle.forward(x, f, r)
    den_ref = oracle.adjoint(w, f, r)
    assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()
    assert np.abs(den - den_ref).max() <= 1e-12 * np.abs(den_ref).max()


@pytest.mark.parametrize("K,r", [(85, 2), (43, 2), (15, 3), (9, 2)])
def test_phase_kernels_carry_every_tap_once_per_fine_offset(K, r):
    """sum over phases of a phase kernel's taps = r^2 sum(f) (each fine pixel
    of a coarse pixel meets every tap once), and the polyphase window has
    (K + r - 1)^2 distinct input offsets per coarse pixel."""
    f = np.random.default_rng(K).uniform(0.1, 1.0, (K, K))
    k, hc = phase_kernels(f, r)
    assert k.sum() == pytest.approx(r * r * f.sum(), rel=1e-12)
    nonzero = sum(int((k[py, px] != 0).sum()) for py in range(r) for px in range(r))
    assert nonzero <= (K + r - 1) ** 2 <= r * r * (2 * hc + 1) ** 2
