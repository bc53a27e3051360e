"""Host-side pins of the benchmark's roofline numerators and bookkeeping
(bench.py): the algorithmic flop count of Eq. (2) against a direct count of
the operators' multiply-adds, the tensor-core form's executed flops and the
FFT form's transform flops against their per-tile counts, the kernel names
the FFT roofline record carries, and the rule that a committed DRAM traffic
figure is used only while its kernel's source is unchanged."""
import json

import numpy as np
import pytest

import bench


def direct_macs(H, W, n, K, r):
    """multiply-adds of one iteration of Eq. (2) counted operator by operator:
    per exposure the forward model D^r(f * x) and its adjoint, each a sum over
    the taps that reach one coarse pixel. With r > 1 a coarse pixel sums r^2
    fine pixels, each K^2 taps, but the fine pixels of one coarse pixel share
    taps: the distinct (fine pixel of x, tap) pairs reaching it form the
    (K + r - 1) x (K + r - 1) window of the polyphase kernels."""
    if r == 1:
        per_pixel = K * K
    else:
        # distinct input offsets reaching one coarse pixel: fine offsets
        # d = p - a for p in [0, r), a in [0, K) (per axis)
        offs = {p - a for p in range(r) for a in range(K)}
        per_pixel = len(offs) ** 2
    return 2 * n * H * W * per_pixel   # forward and adjoint


@pytest.mark.parametrize("H,W,n,K,r", [(4096, 4096, 33, 43, 1), (2048, 2048, 33, 85, 2),
                                       (256, 256, 4, 15, 1), (96, 80, 2, 15, 3)])
def test_algorithmic_flops_is_two_flops_per_operator_multiply_add(H, W, n, K, r):
    assert bench.algorithmic_flops(H, W, n, K, r) == 2 * direct_macs(H, W, n, K, r)


def test_headline_flops_per_iteration():
    # 4 n H W K^2 at 4096^2 x 33, K = 43
    assert bench.algorithmic_flops(4096, 4096, 33, 43, 1) == pytest.approx(4.095e12, rel=1e-3)


def test_tensor_core_executed_flops_count():
    H = W = 4096
    n, K = 33, 43
    hc = 21
    Kd = -(-(128 + 2 * hc + (hc % 8)) // 16) * 16
    assert Kd == 176
    tiles = 32 * 32
    per_gemm = 2 * 128 * 128 * Kd
    # per tile, exposure and filter row: a forward and an adjoint GEMM per product
    for nprod in (1, 3):
        assert bench.tc_executed_flops(H, W, n, K, 1, nprod) == tiles * n * (2 * hc + 1) * nprod * 2 * per_gemm
    assert bench.tc_executed_flops(H, W, n, K, 1, 3) == pytest.approx(50.3e12, rel=2e-3)


def test_fft_transform_flops_count():
    # 2304 tiles of 86 outputs; per tile x^ once + one inverse per exposure
    # (forward), one transform per exposure + one inverse (adjoint)
    fl = bench.fft_flops(4096, 4096, 33, 43, 1, 0.0)
    tiles = 48 * 48
    transforms = tiles * 2 * (33 + 1)
    assert transforms == 156672
    per = 2.5 * 128 * 128 * np.log2(128 * 128)
    products = tiles * 2 * 33 * 6 * 128 * 65
    assert fl == pytest.approx(transforms * per + products, rel=1e-12)
    # the heavy-tailed model transforms the numerator planes too
    assert bench.fft_flops(4096, 4096, 33, 43, 1, 3.0) > 1.4 * fl


def test_fft_kernel_names():
    split = "fft_forward_split_kernel + fft_adjoint_split_kernel"
    whole = "fft_forward_kernel + fft_adjoint_kernel"
    assert bench.fft_kernels(4096, 4096, 33, 43, 1, 0.0, 152) == split    # 2304 tiles
    assert bench.fft_kernels(1024, 1024, 33, 43, 1, 0.0, 152) == whole    # 144 tiles < 152
    assert bench.fft_kernels(4096, 4096, 33, 43, 1, 3.0, 152) == whole    # heavy-tailed
    assert bench.fft_kernels(2048, 2048, 33, 85, 2, 0.0, 152) == whole    # r = 2


def test_committed_traffic_only_for_the_measured_source(monkeypatch):
    rec = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "halo_hsc_traffic.json")))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: rec["source_hash"])
    assert bench.committed_traffic("halo", "hsc") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "0" * 16)
    assert bench.committed_traffic("halo", "hsc") is None
    assert bench.committed_traffic("halo", "no_such_workload") is None
