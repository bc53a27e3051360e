"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle) against the closed form they must equal, and the CUDA path against
the stored values."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    with open(os.path.join(HERE, "golden", name)) as fh:
        return json.load(fh)


def test_delta_psf_fixture_is_the_weighted_coadd():
    """Sec. 2, Eq. (2) with f_t = delta: x1 = max(sum u y / sum u, 0) where a
    valid exposure exists, x0 elsewhere (u = 1/v on valid pixels)."""
    d = load("delta_psf_coadd.json")
    y, v, m = np.array(d["y"]), np.array(d["v"]), np.array(d["mask"])
    x0, x1 = np.array(d["x0"]), np.array(d["x1"])
    u = np.where(m != 0, 1.0 / v, 0.0)
    su = u.sum(0)
    coadd = np.where(su > 0, np.maximum((u * np.where(m != 0, y, 0)).sum(0), 0)
                     / np.where(su > 0, su, 1), x0)
    np.testing.assert_allclose(x1, coadd, rtol=1e-15, atol=0)
    assert x1[3, 0] == x0[3, 0] and x1[0, 2] == 0.0   # all masked; negative mean clipped


def test_oracle_reproduces_the_stored_values():
    d = load("delta_psf_coadd.json")
    y, v, m = np.array(d["y"]), np.array(d["v"]), np.array(d["mask"], np.uint8)
    yy = np.where(m != 0, y, 0.0)
    u, _ = oracle.weights(v, m, yy)
    f = np.ones((d["n"], 1, 1))
    x1 = oracle.em_run(np.array(d["x0"]), oracle.numerator(yy, u, f), u, f, 1)
    np.testing.assert_array_equal(x1, np.array(d["x1"]))


@pytest.mark.gpu
def test_cuda_path_matches_the_stored_values():
    from paper_2302_05804_gb300 import emd
    d = load("delta_psf_coadd.json")
    y = np.array(d["y"], np.float32)
    v = np.array(d["v"], np.float32)
    m = np.array(d["mask"], np.uint8)
    y[m == 0] = np.nan
    c = emd.Deconvolver(d["H"], d["W"], d["n"], 1, 1)
    try:
        c.set_frames(y, v, np.ones((d["n"], 1, 1), np.float32), m)
        c.set_x(np.array(d["x0"], np.float32))
        c.iterate(1)
        x1 = c.x()
    finally:
        c.close()
    np.testing.assert_allclose(x1, np.array(d["x1"]), rtol=1e-6, atol=1e-7)
