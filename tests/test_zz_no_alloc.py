"""emd_frame_stats_noalloc, the entry point that allocates no device memory.

It serves callers that cannot call cudaMalloc (work issued during CUDA-graph
stream capture, pipelines that reserve device memory up front, frameworks
that own all device memory). Its output must agree with what the context
path computes in emd_set_frames: the log-likelihood constant (recovered from
emd_loglik_chi2 as -2 l - chi2) and the default start c = sum u y / sum u
(emd_get_x right after emd_set_frames), and both with the FP64 oracle's
sum log(2 pi v) and default start (Sec. 2, Eq. (2)). Two calls in a row on
different frame sets check that the shared scratch array carries nothing
over; the device's free memory is the same before and after the second.

This file sorts last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_frame_stats_noalloc_matches_context_path():
    torch = pytest.importorskip("torch")
    from paper_2302_05804_gb300 import emd
    emd.load()
    for call, (seed, mask_frac) in enumerate(((0, 0.05), (1, 0.1))):   # two calls in a row
        p = synth.make_problem("parity", seed_offset=seed, mask_frac=mask_frac)
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
        d.set_frames(p.y, p.v, p.f, p.mask)
        x0 = d.x()
        ll, chi2 = d.loglik()
        d.close()
        logdet_ctx = -2.0 * ll - chi2

        y = torch.from_numpy(p.y).cuda()
        v = torch.from_numpy(p.v).cuda()
        m = torch.from_numpy(p.mask).cuda()
        out = torch.full((p.n * 4,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        emd.emd_frame_stats_noalloc(y, v, m, p.H, p.W, p.n, out)
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the kernels; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        o = out.cpu().numpy().reshape(p.n, 4)
        assert np.isfinite(o).all()
        assert (o[:, 3] == 0).all()
        logdet = o[:, 0].sum()
        assert abs(logdet - logdet_ctx) <= 1e-9 * abs(logdet_ctx)
        c = o[:, 1].sum() / o[:, 2].sum() / p.r ** 2
        assert abs(np.float32(c) - x0[0, 0]) <= 1e-6 * abs(c)
        assert (x0 == x0[0, 0]).all()

        # against the FP64 oracle: sum over valid pixels of log(2 pi v), and
        # the default start (u = 1/v in FP64 there, in FP32 here)
        u_o, y_o, _, c_o = oracle.prepare(p)
        logdet_o = oracle.logdet(np.where(p.mask != 0, p.v.astype(np.float64), 1.0), u_o)
        assert abs(logdet - logdet_o) <= 1e-9 * abs(logdet_o)
        assert abs(c - c_o) <= 1e-6 * abs(c_o)


def test_frame_stats_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    from paper_2302_05804_gb300 import emd
    n_max = 64
    y = torch.ones((n_max + 1, 4, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros(((n_max + 1) * 4,), dtype=torch.float64, device="cuda")
    with pytest.raises(emd.EMDError) as ei:
        emd.emd_frame_stats_noalloc(y, y, None, 4, 4, n_max + 1, out)
    assert ei.value.code == emd.EMD_EINVAL and "maximum" in str(ei.value)
    # host pointers are refused by the library itself (the binding would
    # refuse them before the call, so call the C entry point directly)
    host = np.ones((1, 4, 4), np.float32)
    host_out = np.zeros(4, np.float64)
    rc = emd.load().emd_frame_stats_noalloc(host.ctypes.data, host.ctypes.data, None, 4, 4, 1,
                                            host_out.ctypes.data, None)
    assert rc == emd.EMD_EINVAL
    rc = emd.load().emd_frame_stats_noalloc(y.data_ptr(), y.data_ptr(), None, 4, 4, 1,
                                            host_out.ctypes.data, None)
    assert rc == emd.EMD_EINVAL
    with pytest.raises(TypeError):
        emd.emd_frame_stats_noalloc(host, host, None, 4, 4, 1, out)
    # an invalid valid pixel is counted and left out of the sums
    v = torch.ones((2, 4, 4), dtype=torch.float32, device="cuda")
    v[1, 2, 3] = -1.0
    yy = torch.full((2, 4, 4), 3.0, dtype=torch.float32, device="cuda")
    o = torch.zeros((8,), dtype=torch.float64, device="cuda")
    emd.emd_frame_stats_noalloc(yy, v, None, 4, 4, 2, o)
    torch.cuda.synchronize()
    o = o.cpu().numpy().reshape(2, 4)
    assert o[0, 3] == 0 and o[1, 3] == 1
    assert o[0, 2] == 16.0 and o[1, 2] == 15.0 and o[1, 1] == 45.0
