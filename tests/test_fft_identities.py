"""Host-side pins of the identities the FFT form (csrc/emd_fft.cu) rests on,
checked in FP64 with numpy's FFT against the oracle's direct operators of
Eq. (1)-(2), and of the work split of its persistent launch.

* Overlap-save: for an output tile with origin (i0, j0) and side
  B = 128 - 2 hc, the circular convolution of the 128 x 128 input region
  with rows/cols [i0 - hc, i0 - hc + 128) (zero outside the image) and the
  K x K PSF at the top-left of a zero 128 x 128 array holds the "same"
  convolution z(i0 + p, j0 + q) at (p + 2 hc, q + 2 hc), and the circular
  correlation of the w region holds F^T w at (p, q), for p, q < B.
* Two real rows as one complex row: C = FFT(a + i b) gives
  FFT(a) = (C(k) + conj C(-k)) / 2 and FFT(b) = (C(k) - conj C(-k)) / (2i);
  the inverse packs two half spectra as E + i O.
* Bins 0 and 64 of a real row's spectrum are real, so columns 0 and 64 of
  the half spectra travel as one complex column c0 + i c64 (forward: split
  by the same symmetry; inverse: real and imaginary parts).
* The split launch: whole waves grid-stride, the last wave's (tile,
  exposure) units spread over all CTAs (forward), its tiles cut into
  exposure ranges chained across CTAs (adjoint); every unit once, and each
  chained part after its predecessor in the CTA sequences."""
import numpy as np
import pytest

import oracle

N = 128


def tiles_of(H, W, B):
    for i0 in range(0, H, B):
        for j0 in range(0, W, B):
            yield i0, j0


def region(img, i0, j0, hc):
    """the 128 x 128 region with origin (i0 - hc, j0 - hc), zero outside"""
    H, W = img.shape
    out = np.zeros((N, N))
    r0, c0 = i0 - hc, j0 - hc
    rs, re = max(r0, 0), min(r0 + N, H)
    cs, ce = max(c0, 0), min(c0 + N, W)
    out[rs - r0:re - r0, cs - c0:ce - c0] = img[rs:re, cs:ce]
    return out


def psf_array(f):
    k = np.zeros((N, N))
    k[:f.shape[0], :f.shape[1]] = f
    return k


@pytest.mark.parametrize("H,W,K", [(300, 257, 43), (200, 131, 15), (128, 90, 1)])
def test_overlap_save_forward_and_adjoint(H, W, K):
    rng = np.random.default_rng(H + K)
    x = rng.uniform(0.0, 2.0, (H, W))
    w = rng.normal(size=(H, W))
    f = rng.uniform(0.0, 1.0, (K, K))
    f /= f.sum()
    hc = (K - 1) // 2
    B = N - 2 * hc
    kh = np.fft.fft2(psf_array(f))
    z = np.zeros((H, W))
    den = np.zeros((H, W))
    for i0, j0 in tiles_of(H, W, B):
        ph, pw = min(B, H - i0), min(B, W - j0)
        c = np.real(np.fft.ifft2(np.fft.fft2(region(x, i0, j0, hc)) * kh))
        z[i0:i0 + ph, j0:j0 + pw] = c[2 * hc:2 * hc + ph, 2 * hc:2 * hc + pw]
        d = np.real(np.fft.ifft2(np.fft.fft2(region(w, i0, j0, hc)) * np.conj(kh)))
        den[i0:i0 + ph, j0:j0 + pw] = d[:ph, :pw]
    z_ref = oracle.conv_same(x, f)
    den_ref = oracle.corr_same(w, f)
    assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()
    assert np.abs(den - den_ref).max() <= 1e-12 * np.abs(den_ref).max()


def test_a_window_one_row_or_column_wider_would_wrap():
    """The kept window is exactly B = 128 - 2 hc: one more row reads a
    wrapped (circular) term."""
    rng = np.random.default_rng(3)
    K, hc = 43, 21
    B = N - 2 * hc
    x = rng.uniform(0.5, 1.5, (400, 400))
    f = rng.uniform(0.0, 1.0, (K, K))
    c = np.real(np.fft.ifft2(np.fft.fft2(region(x, 100, 100, hc)) * np.fft.fft2(psf_array(f))))
    z_ref = oracle.conv_same(x, f)
    assert abs(c[2 * hc + B - 1, 2 * hc] - z_ref[100 + B - 1, 100]) <= 1e-12 * z_ref.max()
    # index 2 hc + B wraps to row 0 of the circular result
    assert abs(c[(2 * hc + B) % N, 2 * hc] - z_ref[100 + B, 100]) > 1e-6 * z_ref.max()


def test_two_real_rows_as_one_complex_row():
    rng = np.random.default_rng(7)
    a, b = rng.normal(size=N), rng.normal(size=N)
    C = np.fft.fft(a + 1j * b)
    Cm = np.conj(C[(-np.arange(N)) % N])
    np.testing.assert_allclose((C + Cm) / 2, np.fft.fft(a), atol=1e-12)
    np.testing.assert_allclose((C - Cm) / 2j, np.fft.fft(b), atol=1e-12)
    # the inverse: half spectra (bins 0..64) of the two rows -> e + i o
    E, O = np.fft.fft(a), np.fft.fft(b)
    m = np.arange(N)
    Ef = np.where(m <= 64, E[np.minimum(m, 64)], np.conj(E[(N - m) % N]))
    Of = np.where(m <= 64, O[np.minimum(m, 64)], np.conj(O[(N - m) % N]))
    back = np.fft.ifft(Ef + 1j * Of)
    np.testing.assert_allclose(back.real, a, atol=1e-12)
    np.testing.assert_allclose(back.imag, b, atol=1e-12)


def test_columns_zero_and_nyquist_travel_as_one_complex_column():
    rng = np.random.default_rng(11)
    X = rng.normal(size=(N, N))
    Hr = np.fft.fft(X, axis=1)[:, :65]          # row half spectra
    assert np.abs(Hr[:, 0].imag).max() <= 1e-12 * np.abs(Hr).max()
    assert np.abs(Hr[:, 64].imag).max() <= 1e-12 * np.abs(Hr).max()
    # forward: one column FFT of c0 + i c64, split by Hermitian symmetry
    C = np.fft.fft(Hr[:, 0].real + 1j * Hr[:, 64].real)
    Cm = np.conj(C[(-np.arange(N)) % N])
    X2 = np.fft.fft2(X)
    np.testing.assert_allclose((C + Cm) / 2, X2[:, 0], atol=1e-9)
    np.testing.assert_allclose((C - Cm) / 2j, X2[:, 64], atol=1e-9)
    # inverse: the two Hermitian column spectra as S0 + i S64, real and
    # imaginary parts of one inverse FFT
    s = np.fft.ifft(X2[:, 0] + 1j * X2[:, 64])
    np.testing.assert_allclose(s.real, Hr[:, 0].real, atol=1e-9)
    np.testing.assert_allclose(s.imag, Hr[:, 64].real, atol=1e-9)


# -- the split launch's work split (fft_forward_split_kernel,
#    fft_adjoint_split_kernel), restated ---------------------------------------

def forward_units(tiles, P, n):
    Wf, R = tiles // P, tiles % P
    per_cta = []
    for b in range(P):
        units = [(b + P * i, e) for i in range(Wf) for e in range(n)]
        U, base = R * n, Wf * P * n
        u, ue = b * U // P, (b + 1) * U // P
        while u < ue:
            tile, t0 = (base + u) // n, (base + u) % n
            t1 = min(n, t0 + (ue - u))
            units += [(tile, e) for e in range(t0, t1)]
            u += t1 - t0
        per_cta.append(units)
    return per_cta


def adjoint_items(tiles, P, n):
    """per CTA, in order: (tile, k0, k1, part q, predecessor CTA or -1, last)"""
    Wf, R = tiles // P, tiles % P
    k = max(1, min(n, P // R)) if R > 0 else 0
    per_cta = []
    for b in range(P):
        has = b < k * R
        q, j = (b // R, b % R) if has else (0, 0)
        pos = -1 if not has else (Wf if k == 1 else q * Wf // (k - 1))
        items = []
        for it in range(Wf + has):
            if has and it == pos:
                items.append((Wf * P + j, q * n // k, (q + 1) * n // k, q,
                              (q - 1) * R + j if q > 0 else -1, q == k - 1))
            else:
                items.append((b + P * (it - (1 if has and it > pos else 0)), 0, n, 0, -1, True))
        per_cta.append(items)
    return per_cta


@pytest.mark.parametrize("tiles,P,n", [(2304, 152, 33), (324, 152, 3), (576, 152, 33),
                                       (153, 152, 2), (2305, 148, 1), (1000, 152, 4)])
def test_split_launch_covers_every_unit_once_in_exposure_order(tiles, P, n):
    fw = [u for units in forward_units(tiles, P, n) for u in units]
    assert sorted(fw) == [(t, e) for t in range(tiles) for e in range(n)]
    adj = adjoint_items(tiles, P, n)
    seen = {}
    where = {}
    for b, items in enumerate(adj):
        for pos, (tile, k0, k1, q, prev, last) in enumerate(items):
            assert k1 > k0
            for e in range(k0, k1):
                assert (tile, e) not in seen
                seen[(tile, e)] = (b, pos)
            where[(tile, q)] = (b, pos, k0, k1, prev, last)
    assert len(seen) == tiles * n
    for (tile, q), (b, pos, k0, k1, prev, last) in where.items():
        if q > 0:
            pb, ppos, _, pk1, _, _ = where[(tile, q - 1)]
            assert prev == pb != b and pk1 == k0 and ppos <= pos
        assert last == ((tile, q + 1) not in where)
        assert (k1 == n) == last
    # each CTA publishes at most one partial accumulator (its slot)
    for items in adj:
        assert sum(1 for it in items if not it[5]) <= 1
