"""The C-ABI library loads and exports every entry point include/*.h declares
(no GPU needed: only host-side calls are made)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(emd_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2302_05804_gb300 import build, emd
    build.build()
    return emd.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "emd_iterate" in names and "emd_set_frames" in names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_names_match_header():
    from paper_2302_05804_gb300 import emd
    for n in declared_symbols():
        assert hasattr(emd, n), f"python binding lacks {n}"


def test_ctx_bytes_host_only(lib):
    from paper_2302_05804_gb300 import emd
    b = emd.emd_ctx_bytes(256, 256, 4, 15, 1)
    assert b > 2 * 4 * 256 * 256 * 4      # u and y planes at least
    big = emd.emd_ctx_bytes(4096, 4096, 33, 43, 1)
    assert 4.4e9 < big < 6e9
    # invalid shapes: even PSF, r = 0, empty image, oversized footprint
    assert emd.emd_ctx_bytes(256, 256, 4, 14, 1) == 0
    assert emd.emd_ctx_bytes(256, 256, 4, 15, 0) == 0
    assert emd.emd_ctx_bytes(0, 256, 4, 15, 1) == 0
    assert emd.emd_ctx_bytes(256, 256, 0, 15, 1) == 0
    assert emd.emd_ctx_bytes(256, 256, 4, 101, 1) == 0
    assert emd.emd_ctx_bytes(256, 256, 4, 85, 2) > 0   # hc = 21 on the coarse grid


def test_create_rejects_bad_shapes_before_touching_the_gpu(lib):
    from paper_2302_05804_gb300 import emd
    for args in [(64, 64, 2, 4, 1), (64, 64, 2, 5, 0), (-1, 64, 2, 5, 1)]:
        with pytest.raises(emd.EMDError) as ei:
            emd.emd_create(*args)
        assert ei.value.code == emd.EMD_EINVAL
        assert emd.emd_last_error()


def test_null_context_is_an_error(lib):
    from paper_2302_05804_gb300 import emd
    with pytest.raises(emd.EMDError) as ei:
        emd.emd_iterate(None, 1)
    assert ei.value.code == emd.EMD_EINVAL


def test_fit_psf_rejects_bad_arguments_before_touching_the_gpu(lib):
    import numpy as np
    from paper_2302_05804_gb300 import emd
    g = np.ones((3, 3), np.float32) / 9
    for f, r, lam, lr, it in [(np.ones((1, 8, 8), np.float32), 2, 0.0, 1e-4, 1),   # even K
                              (np.ones((1, 9, 9), np.float32), 0, 0.0, 1e-4, 1),   # r = 0
                              (np.ones((1, 9, 9), np.float32), 2, -1.0, 1e-4, 1),  # lambda < 0
                              (np.ones((1, 9, 9), np.float32), 2, 0.0, 0.0, 1),    # lr = 0
                              (np.ones((1, 9, 9), np.float32), 2, 0.0, 1e-4, -1)]:  # iters < 0
        with pytest.raises(emd.EMDError) as e:
            emd.emd_fit_psf(f, g, r, lam, lr, it)
        assert e.value.code == emd.EMD_EINVAL


def test_ctx_bytes_precision_host_only(lib):
    from paper_2302_05804_gb300 import emd
    base = emd.emd_ctx_bytes(4096, 4096, 33, 43, 1)
    # FP32: the halo-exchange kernel's buffer serves its three tile shapes
    # (TH = 64, 48, 32 rows of 128 columns; grid caps 320, 480, 640 CTAs):
    # R = L + dmax + 1 + cap slots, L = dmax + 2 cap (adjoint lag), dmax = 32 + 1
    # tile ids. Control words (256 B), slot flags for the most slots (TH = 32:
    # 1987), tile counters for the most tiles (32 x 128 = 4096), then the
    # largest ring (TH = 48: 1507 slots of 48 x 128 floats).
    ring = 256 + 8192 + 16384 + 1507 * 48 * 128 * 4
    assert emd.emd_ctx_bytes_precision(4096, 4096, 33, 43, 1, emd.EMD_PREC_FP32) == base + ring
    assert emd.emd_ctx_bytes_precision(4096, 4096, 33, 43, 1, emd.EMD_PREC_FP32_PAIR) == base
    # small problems: the ring holds all n * T tiles (4 exposures x 12 tiles
    # of 48 rows is the largest)
    small = emd.emd_ctx_bytes(256, 256, 4, 15, 1)
    assert (emd.emd_ctx_bytes_precision(256, 256, 4, 15, 1, emd.EMD_PREC_FP32)
            == small + 256 + 256 + 256 + 48 * 48 * 128 * 4)
    fft = emd.emd_ctx_bytes_precision(4096, 4096, 33, 43, 1, emd.EMD_PREC_FFT_FP32)
    assert base + 33 * 4096 * 4096 * 4 < fft < base + 33 * 4300 * 4300 * 4 + 10e6
    assert emd.emd_ctx_bytes_precision(4096, 4096, 33, 43, 1, emd.EMD_PREC_SPLIT_BF16) > base
    assert emd.emd_ctx_bytes_precision(256, 256, 4, 14, 1, emd.EMD_PREC_FFT_FP32) == 0
    assert emd.emd_ctx_bytes_precision(256, 256, 4, 15, 1, 99) == 0


def test_frame_stats_noalloc_binding_checks_before_the_call(lib):
    """The C side of emd_frame_stats_noalloc cannot see buffer sizes; the
    binding refuses host tensors, wrong dtypes and short buffers before the
    library is called."""
    import torch
    from paper_2302_05804_gb300 import emd
    y = torch.ones((2, 4, 4), dtype=torch.float32)
    out = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(TypeError):                    # host (CPU) tensors
        emd.emd_frame_stats_noalloc(y, y, None, 4, 4, 2, out)
    with pytest.raises(TypeError):                    # numpy arrays
        emd.emd_frame_stats_noalloc(y.numpy(), y.numpy(), None, 4, 4, 2, out)
    if torch.cuda.is_available():
        yd = y.cuda()
        with pytest.raises(TypeError):                # float32 out
            emd.emd_frame_stats_noalloc(yd, yd, None, 4, 4, 2, torch.zeros(8, device="cuda"))
        with pytest.raises(ValueError):               # out shorter than 4 n
            emd.emd_frame_stats_noalloc(yd, yd, None, 4, 4, 2,
                                        torch.zeros(7, dtype=torch.float64, device="cuda"))
        with pytest.raises(ValueError):               # y shorter than n H W
            emd.emd_frame_stats_noalloc(yd, yd, None, 4, 4, 3,
                                        torch.zeros(12, dtype=torch.float64, device="cuda"))


def test_loglik_has_the_two_argument_form(lib):
    """emd_loglik(ctx, out) as the boundary declares it; the data term comes
    from emd_loglik_chi2."""
    import ctypes
    assert lib.emd_loglik.argtypes == [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    assert len(lib.emd_loglik_chi2.argtypes) == 3
    assert lib.emd_loglik(None, None) == -1           # EMD_EINVAL: no context
