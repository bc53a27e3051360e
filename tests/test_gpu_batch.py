"""Batching: jobs of different shapes advancing together in one persistent
kernel per step give bit-for-bit the iterates they give alone, including a
job that joins while others are running (continuous batching), and each
job's iterate matches the FP64 oracle's Eq. (2) iterate from the same start
(1e-5 after one iteration, 1e-4 after several)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

JOBS = [
    dict(H=200, W=150, n=3, K=15, r=1, mask_frac=0.05, n_points=60, n_gal=2),
    dict(H=130, W=257, n=2, K=43, r=1, mask_frac=0.05, n_points=60, n_gal=2),
    dict(H=96, W=80, n=2, K=15, r=2, fwhm=(3.0, 6.0), mask_frac=0.05, n_points=30, n_gal=2),
    dict(H=64, W=64, n=4, K=7, r=1, mask_frac=0.0, n_points=20, n_gal=1),
    dict(H=300, W=310, n=5, K=21, r=1, mask_frac=0.05, n_points=150, n_gal=3),
]


def make(i):
    return synth.make_problem("hsc", seed_offset=i, **JOBS[i])


def oracle_x(p, k):
    u, y, N, _ = oracle.prepare(p)
    return oracle.em_run(np.full((p.r * p.H, p.r * p.W), 5.0), N, u, p.f, k, p.r)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ctx_for(emd, p):
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    d.set_x(np.full((p.r * p.H, p.r * p.W), 5.0, np.float32))
    return d


def test_batch_matches_solo_runs_bitwise():
    from paper_2302_05804_gb300 import emd
    iters = [6, 4, 7, 3, 5]
    probs = [make(i) for i in range(len(JOBS))]
    solo = []
    for p, k in zip(probs, iters):
        d = ctx_for(emd, p)
        d.iterate(k)
        solo.append(d.x())
        d.close()
    b = emd.emd_batch_create(8)
    ds = [ctx_for(emd, p) for p in probs]
    slots = {}
    # four jobs start together; the fifth joins after two steps
    for i in range(4):
        slots[i] = emd.emd_batch_add(b, ds[i].ctx, iters[i])
    done, step = 0, 0
    while done < len(probs):
        if step == 2:
            slots[4] = emd.emd_batch_add(b, ds[4].ctx, iters[4])
        done += emd.emd_batch_step(b)
        step += 1
        assert step < 50
    emd.emd_batch_sync(b)
    for i in range(len(probs)):
        assert emd.emd_batch_remaining(b, slots[i]) == 0
        np.testing.assert_array_equal(ds[i].x(), solo[i])
    cfg = emd.emd_batch_config(b)
    assert 1 <= cfg["clusters"] <= cfg["max_clusters"] and cfg["order"] in (0, 1)
    assert cfg["form"] in (0, 1)  # halo-exchange or CTA-pair kernel (tried in turn above)
    assert cfg["tile_shape"] in (1, 2)  # the halo-exchange kernel's tile shapes tried
    for i in range(len(probs)):
        emd.emd_batch_remove(b, slots[i])
        ds[i].close()
    emd.emd_batch_destroy(b)


def test_batch_remove_midway_keeps_reached_iterate():
    from paper_2302_05804_gb300 import emd
    p = make(0)
    d = ctx_for(emd, p)
    b = emd.emd_batch_create(2)
    s = emd.emd_batch_add(b, d.ctx, 10)
    for _ in range(3):
        emd.emd_batch_step(b)
    emd.emd_batch_sync(b)
    assert emd.emd_batch_remaining(b, s) == 7
    emd.emd_batch_remove(b, s)
    x3 = d.x()
    e = ctx_for(emd, p)
    e.iterate(3)
    np.testing.assert_array_equal(x3, e.x())
    d.close(); e.close()
    emd.emd_batch_destroy(b)


def test_mixed_direct_and_fft_batch_matches_solo_runs_bitwise():
    """FFT-form jobs run in the persistent FFT kernels of the same step (one
    forward launch and one adjoint launch over all their tiles), FP32 jobs in
    the halo-exchange kernel's merged work list (or, while the tuner tries
    it, the CTA-pair kernel), an EMD_PREC_FP32_PAIR job always in the
    CTA-pair kernel; each job's iterate equals its solo run bit for bit,
    including r = 2 and a job that joins mid-run."""
    from paper_2302_05804_gb300 import emd
    iters = [5, 4, 6, 3, 4]
    forms = [emd.EMD_PREC_FFT_FP32, emd.EMD_PREC_FP32, emd.EMD_PREC_FFT_FP32,
             emd.EMD_PREC_FP32_PAIR, emd.EMD_PREC_FP32]
    probs = [make(i) for i in range(len(JOBS))]

    def ctx(i):
        d = ctx_for(emd, probs[i])
        d.set_precision(forms[i])
        return d

    solo = []
    for i in range(len(probs)):
        d = ctx(i)
        d.iterate(iters[i])
        solo.append(d.x())
        d.close()
    b = emd.emd_batch_create(8)
    ds = [ctx(i) for i in range(len(probs))]
    slots = {}
    for i in range(4):
        slots[i] = emd.emd_batch_add(b, ds[i].ctx, iters[i])
    done, step = 0, 0
    while done < len(probs):
        if step == 1:
            slots[4] = emd.emd_batch_add(b, ds[4].ctx, iters[4])
        done += emd.emd_batch_step(b)
        step += 1
        assert step < 50
    emd.emd_batch_sync(b)
    for i in range(len(probs)):
        assert emd.emd_batch_remaining(b, slots[i]) == 0
        xb = ds[i].x()
        np.testing.assert_array_equal(xb, solo[i])
        err = rel_l2(xb, oracle_x(probs[i], iters[i]))
        print(f"job {i} (mode {forms[i]}, r = {probs[i].r}): rel L2 vs oracle after "
              f"{iters[i]} iterations = {err:.2e}")
        assert err <= 1e-4
        emd.emd_batch_remove(b, slots[i])
        ds[i].close()
    emd.emd_batch_destroy(b)


def test_mixed_batch_one_iteration_against_the_oracle():
    """One iteration of every job in a mixed batch (FFT, halo-exchange and
    CTA-pair forms, r = 1 and 2, PSFs 7 to 43) against the oracle at the
    one-iteration bar; one job joins after the others' step."""
    from paper_2302_05804_gb300 import emd
    forms = [emd.EMD_PREC_FFT_FP32, emd.EMD_PREC_FP32, emd.EMD_PREC_FP32,
             emd.EMD_PREC_FP32_PAIR, emd.EMD_PREC_FFT_FP32]
    probs = [make(i) for i in range(len(JOBS))]
    ds = []
    for i, p in enumerate(probs):
        d = ctx_for(emd, p)
        d.set_precision(forms[i])
        ds.append(d)
    b = emd.emd_batch_create(8)
    slots = [emd.emd_batch_add(b, ds[i].ctx, 1) for i in range(4)]
    assert emd.emd_batch_step(b) == 4
    slots.append(emd.emd_batch_add(b, ds[4].ctx, 1))
    assert emd.emd_batch_step(b) == 1
    emd.emd_batch_sync(b)
    for i, p in enumerate(probs):
        err = rel_l2(ds[i].x(), oracle_x(p, 1))
        print(f"job {i} (mode {forms[i]}, r = {p.r}): rel L2 vs oracle after 1 iteration = {err:.2e}")
        assert err <= 1e-5
        emd.emd_batch_remove(b, slots[i])
        ds[i].close()
    emd.emd_batch_destroy(b)


def test_fft_only_batch():
    from paper_2302_05804_gb300 import emd
    probs = [make(i) for i in (0, 3)]
    solo = []
    for p in probs:
        d = ctx_for(emd, p)
        d.set_precision(emd.EMD_PREC_FFT_FP32)
        d.iterate(3)
        solo.append(d.x())
        d.close()
    b = emd.emd_batch_create(4)
    ds = []
    for p in probs:
        d = ctx_for(emd, p)
        d.set_precision(emd.EMD_PREC_FFT_FP32)
        ds.append(d)
    sl = [emd.emd_batch_add(b, d.ctx, 3) for d in ds]
    for _ in range(3):
        emd.emd_batch_step(b)
    emd.emd_batch_sync(b)
    for d, s_, x in zip(ds, sl, solo):
        np.testing.assert_array_equal(d.x(), x)
        emd.emd_batch_remove(b, s_)
        d.close()
    emd.emd_batch_destroy(b)
