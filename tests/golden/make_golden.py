"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Run from the repository root: ``python tests/golden/make_golden.py``. Every
value it stores comes from ``oracle/`` (never from the CUDA library); the
tests check the stored values against closed forms of the paper's update
(Sec. 2, Eq. (2)) and the CUDA path against the stored values.

delta_psf_coadd.json -- Eq. (2) with delta PSFs (f_t = [[1]]): one iteration
from any positive start gives the weighted coadd x = max(sum_t u_t y_t /
sum_t u_t, 0) at every pixel with a valid exposure, and leaves x unchanged
where every exposure is masked. Inputs are small exact binary fractions, so
the expected values are exact in FP64.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def delta_psf_case():
    H, W, n = 4, 5, 3
    y = np.array([[[3, 1, -2, 4, 0], [1, 2, 3, 4, 5], [6, -1, 2, 0, 1], [2, 2, 2, 2, 2]],
                  [[1, 3, 2, -4, 0], [5, 4, 3, 2, 1], [2, 1, 0, 8, 3], [4, 4, 4, 4, 4]],
                  [[0, 2, -6, 4, 8], [1, 1, 1, 1, 1], [2, 5, 2, 0, 3], [1, 2, 3, 4, 5]]], float)
    v = np.array([1.0, 2.0, 4.0])[:, None, None] * np.ones((n, H, W))
    mask = np.ones((n, H, W), np.uint8)
    mask[0, 1, 2] = 0
    mask[1, 2, 4] = 0
    mask[:, 3, 0] = 0          # every exposure masked at (3, 0): x keeps its start
    f = np.ones((n, 1, 1))
    x0 = np.full((H, W), 0.75)
    u, bad = oracle.weights(v, mask, np.where(mask != 0, y, 0.0))
    assert bad == 0
    yy = np.where(mask != 0, y, 0.0)
    N = oracle.numerator(yy, u, f)
    x1 = oracle.em_run(x0, N, u, f, 1)
    return {"citation": "Sec. 2, Eq. (2) with delta PSFs: the weighted coadd",
            "H": H, "W": W, "n": n, "K": 1, "r": 1,
            "y": y.tolist(), "v": v.tolist(), "mask": mask.tolist(), "x0": x0.tolist(),
            "x1": x1.tolist()}


if __name__ == "__main__":
    out = os.path.join(HERE, "delta_psf_coadd.json")
    with open(out, "w") as fh:
        json.dump(delta_psf_case(), fh, indent=1)
    print("wrote", out)
