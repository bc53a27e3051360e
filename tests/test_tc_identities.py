"""Host-side pins of the tensor-core form (csrc/emd_tc.cu), in FP64 with
numpy against the oracle's convolution of Eq. (1).

* The forward model on a 128 x 128 tile as a sum of GEMMs, one per filter
  row a: Z = sum_a X_a T_a, X_a the band of x rows shifted by a (128 rows x
  Kd columns, the band starting hc + dlt columns left of the tile, dlt =
  hc mod 8, Kd = rup(128 + 2 hc + dlt, 16)) and T_a[k][n] = kf[a][k - n -
  dlt] (kf the PSF rotated by 180 degrees, zero outside the band).
* T_a transposed with its columns reversed is a Hankel matrix: its 8 x 8
  core matrices depend only on the sum of their block indices, so
  Kd / 8 + 15 distinct core matrices describe it.
* The precision of the operand splits: x = x_hi + x_lo with both parts in
  bf16 (8 significant bits, round to nearest even: each rounding within
  2^-8 of the value) or fp16 (11 bits, 2^-11, with power-of-two scaling)
  leaves at most 2^-16 (bf16) or 2^-22 (fp16) of |x|; the split
  product x_hi f_hi + x_hi f_lo + x_lo f_hi, and the single bf16 / fp16
  product, stay within the bars the GPU precision tests use (relative L2
  1e-4 for the split forms, 5e-3 for bf16, 2e-3 for fp16) on a tile of the
  HSC-shaped problem (43 x 43 PSF)."""
import numpy as np
import pytest

import oracle

M = 128


def rup(v, m):
    return (v + m - 1) // m * m


def band_geometry(K):
    hc = (K - 1) // 2
    dlt = hc % 8
    Kd = rup(M + 2 * hc + dlt, 16)
    return hc, dlt, Kd


def band(x, i0, j0, hc, dlt, Kd):
    """rows [i0 - hc, i0 + 128 + hc), columns [j0 - hc - dlt, ... + Kd), zero
    outside the image"""
    H, W = x.shape
    out = np.zeros((M + 2 * hc, Kd))
    r0, c0 = i0 - hc, j0 - hc - dlt
    rs, re = max(r0, 0), min(r0 + M + 2 * hc, H)
    cs, ce = max(c0, 0), min(c0 + Kd, W)
    out[rs - r0:re - r0, cs - c0:ce - c0] = x[rs:re, cs:ce]
    return out


def toeplitz_rows(f, dlt, Kd):
    """T[a] (Kd x 128): T[a][k][n] = kf[a][k - n - dlt]"""
    K = f.shape[0]
    kf = f[::-1, ::-1]
    T = np.zeros((K, Kd, M))
    k = np.arange(Kd)[:, None]
    n = np.arange(M)[None, :]
    m = k - n - dlt
    ok = (m >= 0) & (m < K)
    for a in range(K):
        T[a][ok] = kf[a][m[ok]]
    return T


def tile_gemm(bnd, T):
    """sum_a X_a T_a, X_a = rows [a, a + 128) of the band"""
    Z = np.zeros((M, M))
    for a in range(T.shape[0]):
        Z += bnd[a:a + M] @ T[a]
    return Z


@pytest.mark.parametrize("K", [43, 15, 9, 1])
def test_tile_convolution_is_a_sum_of_band_gemms(K):
    rng = np.random.default_rng(K)
    H, W = 300, 280
    x = rng.uniform(0.0, 3.0, (H, W))
    f = rng.uniform(0.0, 1.0, (K, K))
    f /= f.sum()
    hc, dlt, Kd = band_geometry(K)
    assert Kd % 16 == 0 and (M + 2 * hc + dlt) <= Kd
    T = toeplitz_rows(f, dlt, Kd)
    z_ref = oracle.conv_same(x, f)
    for i0, j0 in [(0, 0), (128, 128), (172, 152)]:   # corner, interior, ragged edge
        Z = tile_gemm(band(x, i0, j0, hc, dlt, Kd), T)
        ph, pw = min(M, H - i0), min(M, W - j0)
        np.testing.assert_allclose(Z[:ph, :pw], z_ref[i0:i0 + ph, j0:j0 + pw],
                                   rtol=0, atol=1e-12 * z_ref.max())


@pytest.mark.parametrize("K", [43, 15, 85])
def test_band_operand_is_hankel_in_8x8_core_matrices(K):
    rng = np.random.default_rng(5)
    f = rng.uniform(0.1, 1.0, (K, K))
    hc, dlt, Kd = band_geometry(K)
    T = toeplitz_rows(f, dlt, Kd)
    for a in (0, K // 2, K - 1):
        Hk = T[a].T[::-1]                       # 128 x Kd, Hk[n'][k] = T[k][127 - n']
        blocks = {}
        for nb in range(M // 8):
            for kb in range(Kd // 8):
                blk = Hk[8 * nb:8 * nb + 8, 8 * kb:8 * kb + 8]
                key = nb + kb
                if key in blocks:
                    np.testing.assert_array_equal(blk, blocks[key])
                else:
                    blocks[key] = blk
                # inside a core matrix the entries depend on r + c only
                r, c = np.indices((8, 8))
                for s in range(15):
                    vals = blk[(r + c) == s]
                    assert (vals == vals[0]).all()
        assert len(blocks) == Kd // 8 + 15


def bf16(x):
    """float32 -> bf16 (round to nearest, ties to even), returned as float32"""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def split(x, rnd):
    x = np.asarray(x, np.float32)
    hi = rnd(x)
    lo = rnd(x - hi)          # x - hi is exact in float32
    return hi, lo


def test_bf16_rounding_and_split_representation():
    rng = np.random.default_rng(1)
    x = (rng.uniform(0.5, 2.0, 100000) * 2.0 ** rng.integers(-20, 20, 100000)).astype(np.float32)
    hi, lo = split(x, bf16)
    assert (np.abs(hi.astype(np.float64) - x) <= 2.0 ** -8 * np.abs(x)).all()
    # 8 significant bits: the low 16 bits of the float32 pattern are zero
    assert (hi.view(np.uint32) & 0xFFFF == 0).all() and (lo.view(np.uint32) & 0xFFFF == 0).all()
    rest = np.abs(x.astype(np.float64) - hi - lo)
    assert (rest <= 2.0 ** -16 * np.abs(x)).all()
    # ties go to even
    t = np.array([np.float32(1.0) + np.float32(2.0 ** -8), np.float32(1.0) + np.float32(3 * 2.0 ** -8)],
                 np.float32)
    np.testing.assert_array_equal(bf16(t), np.array([1.0, 1.0 + 2.0 ** -6], np.float32))


def test_fp16_split_with_power_of_two_scaling():
    rng = np.random.default_rng(2)
    x = rng.uniform(0.0, 1.0, 50000).astype(np.float32) * np.float32(37.5)
    s = np.float32(2.0 ** np.floor(np.log2(2.0 ** 14 / x.max())))   # max -> <= 2^14
    xs = x * s                                                      # exact (power of two)
    assert xs.max() <= 2.0 ** 14
    hi, lo = split(xs, fp16)
    big = xs >= 2.0 ** -14                                          # fp16 normal range
    rest = np.abs(xs.astype(np.float64) - hi - lo)
    assert (rest[big] <= 2.0 ** -22 * xs[big] + 2.0 ** -25).all()
    np.testing.assert_array_equal((hi / s) * s, hi)                 # unscaling is exact


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mode,bar", [("split_bf16", 1e-4), ("split_fp16", 1e-4),
                                      ("bf16", 5e-3), ("fp16", 2e-3)])
def test_tile_product_precision_within_the_bars(mode, bar):
    rng = np.random.default_rng(9)
    K = 43
    H = W = 256
    x = rng.uniform(0.0, 50.0, (H, W)).astype(np.float32)
    yy, xx = np.mgrid[-21:22, -21:22]
    f = np.exp(-(xx ** 2 + yy ** 2) / (2 * 3.0 ** 2)).astype(np.float32)
    f /= f.sum()
    hc, dlt, Kd = band_geometry(K)
    bnd = band(x.astype(np.float64), 64, 64, hc, dlt, Kd).astype(np.float32)
    T = toeplitz_rows(f.astype(np.float64), dlt, Kd).astype(np.float32)
    exact = tile_gemm(bnd.astype(np.float64), T.astype(np.float64))
    if mode.endswith("fp16"):
        gs = np.float32(2.0 ** np.floor(np.log2(2.0 ** 14 / f.max())))
        xs = np.float32(2.0 ** np.floor(np.log2(2.0 ** 14 / x.max())))
        bnd_s, T_s, rnd, unscale = bnd * xs, T * gs, fp16, 1.0 / (float(xs) * float(gs))
    else:
        bnd_s, T_s, rnd, unscale = bnd, T, bf16, 1.0
    Xh, Xl = split(bnd_s, rnd)
    Th, Tl = split(T_s, rnd)
    Xh, Xl, Th, Tl = (a.astype(np.float64) for a in (Xh, Xl, Th, Tl))
    if mode.startswith("split"):
        Z = np.zeros((M, M))
        for a in range(K):
            Z += Xh[a:a + M] @ Th[a] + Xh[a:a + M] @ Tl[a] + Xl[a:a + M] @ Th[a]
    else:
        Z = np.zeros((M, M))
        for a in range(K):
            Z += Xh[a:a + M] @ Th[a]
    err = rel_l2(Z * unscale, exact)
    assert err <= bar
    if mode.startswith("split"):
        assert err <= 1e-5      # the split's residual is the dropped lo x lo product
