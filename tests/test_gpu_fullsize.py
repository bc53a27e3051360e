"""Full-size workloads through the C ABI, checked on sampled outputs.

At 4096^2 x 33 exposures with 43 x 43 PSFs (and 33 x 2048^2 exposures with
85 x 85 fine PSFs at r = 2) the oracle cannot run whole iterations, so one
GPU iteration from a known start is compared pixel by pixel with the
oracle's single-pixel evaluation of Eq. (2) at sampled latent pixels
(corners, edges, masked columns and random interior points). Properties
that hold at any size (non-negativity, finite values, monotone likelihood)
are checked on the full image.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def sample_idx(Hf, Wf, k, seed):
    g = np.random.default_rng(seed)
    pts = [(0, 0), (0, Wf - 1), (Hf - 1, 0), (Hf - 1, Wf - 1), (Hf // 2, 0), (1, Wf // 3),
           (127, 128), (128, 127), (Hf - 2, Wf - 129)]
    pts += [(int(a), int(b)) for a, b in zip(g.integers(0, Hf, k), g.integers(0, Wf, k))]
    return np.array([a * Wf + b for a, b in pts], np.int64)


@pytest.mark.parametrize("recipe,k", [("hsc", 24), ("sr2", 4)])
def test_full_size_one_iteration_sampled(recipe, k, request):
    from paper_2302_05804_gb300 import emd
    p = request.getfixturevalue("hsc_problem") if recipe == "hsc" else synth.make_problem(recipe)
    Hf, Wf = p.r * p.H, p.r * p.W
    x0 = (np.random.default_rng(5).uniform(0.5, 1.5, (Hf, Wf)) * 10.0).astype(np.float32)
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    d.set_x(x0)
    ll0 = d.loglik()[0]
    d.iterate(1)
    x1 = d.x()
    ll1 = d.loglik()[0]
    d.iterate(2)
    x3 = d.x()
    ll3 = d.loglik()[0]
    u_g = d.weights()
    d.close()
    assert np.array_equal(u_g == 0, p.mask == 0)
    assert np.isfinite(x3).all() and (x3 >= 0).all()
    assert ll1 >= ll0 - 1e-7 * abs(ll0) and ll3 >= ll1 - 1e-7 * abs(ll1)
    idx = sample_idx(Hf, Wf, k, seed=11)
    u, _ = oracle.weights(p.v, p.mask, p.y)
    xo, No, Do = oracle.em_step_at(x0, p.y, u, p.f, idx, p.r)
    got = x1.ravel()[idx].astype(np.float64)
    err = np.abs(got - xo) / np.maximum(np.abs(xo), 1e-30)
    # per-pixel relative error; the L2 criterion of the iteration is 1e-5
    assert np.linalg.norm(got - xo) / np.linalg.norm(xo) <= 1e-5, err.max()


@pytest.mark.parametrize("mode,tol", [(1, 5e-3), (2, 2e-3), (3, 1e-4), (4, 1e-4)])
def test_full_size_tensor_core_forms_sampled(mode, tol, hsc_problem):
    """The tensor-core forms (BF16, FP16, split BF16, split FP16) at the size
    the bench times them (4096^2 x 33, 43 x 43 PSFs): one iteration against
    the oracle's single-pixel evaluation at sampled pixels, with the bars of
    the smaller tensor-core parity cases (the operand rounding of each form)."""
    from paper_2302_05804_gb300 import emd
    p = hsc_problem
    x0 = (np.random.default_rng(5).uniform(0.5, 1.5, (p.H, p.W)) * 10.0).astype(np.float32)
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r)
    d.set_frames(p.y, p.v, p.f, p.mask)
    d.set_precision(mode)
    d.set_x(x0)
    d.iterate(1)
    x1 = d.x()
    d.close()
    assert np.isfinite(x1).all() and (x1 >= 0).all()
    idx = sample_idx(p.H, p.W, 24, seed=13)
    u, _ = oracle.weights(p.v, p.mask, p.y)
    xo, _, _ = oracle.em_step_at(x0, p.y, u, p.f, idx, p.r)
    got = x1.ravel()[idx].astype(np.float64)
    assert np.linalg.norm(got - xo) / np.linalg.norm(xo) <= tol
