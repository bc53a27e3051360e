"""FP64 CPU oracle of the EM multi-frame deconvolution update (Sec. 2).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the product path. The arithmetic
lives in ``emd_oracle.c`` (plain C, FP64); this module compiles it with gcc
and marshals numpy arrays. It shares no code with the CUDA library.

Every function takes and returns float64 numpy arrays (inputs of other
dtypes are converted), C order:
    x      (rH, rW) latent image
    y, v   (n, H, W) exposures and variances (y may hold NaN where masked)
    u      (n, H, W) weights, 1/v where valid and 0 where masked
    f      (n, K, K) PSFs (fine grid when r > 1)
    mask   (n, H, W) uint8, 0 = masked
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile emd_oracle.c into liboracle.so next to it (gcc -O2)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", _LIB_PATH,
            _SRC, "-lm"]
    cmds = [base[:1] + ["-fopenmp"] + base[1:]] if openmp else []
    cmds.append(base)
    err = None
    for cmd in cmds:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            return _LIB_PATH
        err = r.stderr
    raise RuntimeError(f"oracle build failed:\n{err}")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            dp = C.POINTER(C.c_double)
            i = C.c_int
            lib.oracle_num_threads.restype = i
            lib.oracle_conv_same.argtypes = [dp, i, i, dp, i, dp]
            lib.oracle_corr_same.argtypes = [dp, i, i, dp, i, dp]
            lib.oracle_downsample.argtypes = [dp, i, i, i, dp]
            lib.oracle_upsample.argtypes = [dp, i, i, i, dp]
            lib.oracle_forward.argtypes = [dp, i, i, i, dp, i, dp]
            lib.oracle_adjoint.argtypes = [dp, i, i, i, dp, i, dp]
            lib.oracle_weights.argtypes = [dp, dp, C.c_void_p, C.c_long, dp]
            lib.oracle_weights.restype = C.c_long
            lib.oracle_numerator.argtypes = [dp, dp, dp, i, i, i, i, i, dp]
            lib.oracle_denominator.argtypes = [dp, dp, dp, i, i, i, i, i, dp]
            lib.oracle_apply_update.argtypes = [dp, dp, dp, C.c_long]
            lib.oracle_em_step.argtypes = [dp, dp, dp, dp, i, i, i, i, i, C.c_void_p]
            lib.oracle_em_run.argtypes = [dp, dp, dp, dp, i, i, i, i, i, i]
            lib.oracle_em_step_literal.argtypes = [dp, dp, dp, C.c_void_p, dp,
                                                   i, i, i, i]
            lib.oracle_em_pass_streaming.argtypes = [dp, dp, dp, dp, i, i, i, i, i,
                                                     C.c_void_p]
            lib.oracle_psf_model.argtypes = [dp, i, dp, i, i, i, dp]
            lib.oracle_psf_model_adjoint.argtypes = [dp, i, dp, i, i, i, dp]
            lib.oracle_psf_loss.argtypes = [dp, i, dp, i, dp, i, i, C.c_double, C.c_void_p]
            lib.oracle_psf_loss.restype = C.c_double
            d_ = C.c_double
            lib.oracle_psf_fit.argtypes = [dp, i, dp, i, dp, i, i, d_, d_, d_, d_, d_, i]
            lib.oracle_psf_fit.restype = d_
            lib.oracle_student_weights.argtypes = [dp, dp, dp, C.c_long, d_, dp]
            lib.oracle_em_step_student.argtypes = [dp, dp, dp, dp, i, i, i, i, i, d_,
                                                   C.c_void_p, C.c_void_p]
            lib.oracle_student_loglik.argtypes = [dp, dp, dp, dp, dp, i, i, i, i, i, d_]
            lib.oracle_student_loglik.restype = d_
            lib.oracle_chi2.argtypes = [dp, dp, dp, dp, i, i, i, i, i]
            lib.oracle_chi2.restype = C.c_double
            lib.oracle_logdet.argtypes = [dp, dp, C.c_long]
            lib.oracle_logdet.restype = C.c_double
            lib.oracle_default_x0.argtypes = [dp, dp, C.c_long, i]
            lib.oracle_default_x0.restype = C.c_double
            lib.oracle_em_step_at.argtypes = [dp, dp, dp, dp, i, i, i, i, i,
                                              C.POINTER(C.c_long), i,
                                              C.c_void_p, C.c_void_p, C.c_void_p]
            _lib = lib
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def num_threads() -> int:
    return _load().oracle_num_threads()


# -- operators --------------------------------------------------------------

def conv_same(x, f):
    """(f*x) zero-padded 'same' convolution, Eq. (1)."""
    x, f = _d(x), _d(f)
    out = np.empty_like(x)
    _load().oracle_conv_same(_p(x), x.shape[0], x.shape[1], _p(f), f.shape[0], _p(out))
    return out


def corr_same(w, f):
    """F^T w: correlation with f, the transpose of conv_same."""
    w, f = _d(w), _d(f)
    out = np.empty_like(w)
    _load().oracle_corr_same(_p(w), w.shape[0], w.shape[1], _p(f), f.shape[0], _p(out))
    return out


def downsample(zf, r):
    zf = _d(zf)
    H, W = zf.shape[0] // r, zf.shape[1] // r
    out = np.empty((H, W))
    _load().oracle_downsample(_p(zf), H, W, r, _p(out))
    return out


def upsample(w, r):
    w = _d(w)
    out = np.empty((w.shape[0] * r, w.shape[1] * r))
    _load().oracle_upsample(_p(w), w.shape[0], w.shape[1], r, _p(out))
    return out


def forward(x, f, r=1):
    """z = D^r(f * x) (Eq. (1), Eq. (3))."""
    x, f = _d(x), _d(f)
    H, W = x.shape[0] // r, x.shape[1] // r
    z = np.empty((H, W))
    _load().oracle_forward(_p(x), H, W, r, _p(f), f.shape[0], _p(z))
    return z


def adjoint(w, f, r=1):
    """F^T (D^r)^T w."""
    w, f = _d(w), _d(f)
    out = np.empty((w.shape[0] * r, w.shape[1] * r))
    _load().oracle_adjoint(_p(w), w.shape[0], w.shape[1], r, _p(f), f.shape[0], _p(out))
    return out


# -- EM ---------------------------------------------------------------------

def weights(v, mask=None, y=None):
    """u = 1/v where valid, 0 where masked. Returns (u, number_of_bad)."""
    v = _d(v)
    y = None if y is None else _d(y)
    u = np.empty_like(v)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    bad = _load().oracle_weights(_p(v), None if y is None else _p(y),
                                 None if m is None else m.ctypes.data,
                                 v.size, _p(u))
    return u, int(bad)


def _dims(u, f, r):
    n, H, W = u.shape
    return n, H, W, f.shape[1], r


def numerator(y, u, f, r=1):
    y, u, f = _d(y), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    N = np.empty((r * H, r * W))
    _load().oracle_numerator(_p(y), _p(u), _p(f), n, H, W, K, r, _p(N))
    return N


def denominator(x, u, f, r=1):
    x, u, f = _d(x), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    D = np.empty((r * H, r * W))
    _load().oracle_denominator(_p(x), _p(u), _p(f), n, H, W, K, r, _p(D))
    return D


def em_step(x, N, u, f, r=1, return_den=False):
    """One iteration of Eq. (2); returns the new x (and Den)."""
    x, N, u, f = _d(x).copy(), _d(N), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    den = np.empty_like(x) if return_den else None
    _load().oracle_em_step(_p(x), _p(N), _p(u), _p(f), n, H, W, K, r,
                           None if den is None else den.ctypes.data)
    return (x, den) if return_den else x


def em_run(x, N, u, f, k, r=1):
    x, N, u, f = _d(x).copy(), _d(N), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    _load().oracle_em_run(_p(x), _p(N), _p(u), _p(f), n, H, W, K, r, int(k))
    return x


def em_step_literal(x, y, u, f, mask=None):
    """Eq. (2) with u_t applied after F_t^T (r = 1)."""
    x, y, u, f = _d(x).copy(), _d(y), _d(u), _d(f)
    n, H, W = u.shape
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    _load().oracle_em_step_literal(_p(x), _p(y), _p(u),
                                   None if m is None else m.ctypes.data,
                                   _p(f), n, H, W, f.shape[1])
    return x


def em_streaming(x, y, u, f, k, r=1, order=None):
    """k passes of the frame-by-frame (streaming) EM; y zero where u = 0."""
    x, y, u, f = _d(x).copy(), _d(y), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    o = None
    if order is not None:
        o = np.ascontiguousarray(order, dtype=np.int32)
    for _ in range(int(k)):
        _load().oracle_em_pass_streaming(_p(x), _p(y), _p(u), _p(f), n, H, W, K, r,
                                         None if o is None else o.ctypes.data)
    return x


# -- PSF super-resolution fit, Eq. (4) ------------------------------------------

def psf_fine_side(K, r):
    return r * (K - 1) + 1


def psf_model(h, g, r, K):
    """D^r(h * g) on the K x K coarse grid."""
    h, g = _d(h), _d(g)
    m = np.empty((K, K))
    _load().oracle_psf_model(_p(h), h.shape[0], _p(g), g.shape[0], r, K, _p(m))
    return m


def psf_model_adjoint(w, g, r, Kh):
    w, g = _d(w), _d(g)
    out = np.empty((Kh, Kh))
    _load().oracle_psf_model_adjoint(_p(w), w.shape[0], _p(g), g.shape[0], r, Kh, _p(out))
    return out


def psf_loss(h, f, g, r, lam, grad=False):
    h, f, g = _d(h), _d(f), _d(g)
    gr = np.empty_like(h) if grad else None
    L = _load().oracle_psf_loss(_p(h), h.shape[0], _p(f), f.shape[0], _p(g), g.shape[0], r,
                                float(lam), None if gr is None else gr.ctypes.data)
    return (L, gr) if grad else L


def psf_fit(f, g, r, lam, iters, lr, h0, b1=0.9, b2=0.999, eps=1e-8, with_loss=False):
    """iters projected Adam steps on Eq. (4) from h0; the iterate of lowest
    loss among h0 .. h_iters (and that loss when with_loss)."""
    h, f, g = _d(h0).copy(), _d(f), _d(g)
    L = _load().oracle_psf_fit(_p(h), h.shape[0], _p(f), f.shape[0], _p(g), g.shape[0], r,
                               float(lam), float(lr), float(b1), float(b2), float(eps), int(iters))
    return (h, L) if with_loss else h


def student_weights(y, u, z, nu):
    """u' = u (nu+1) / (nu + u (y-z)^2) where u != 0 (heavy-tailed E-step)."""
    y, u, z = _d(y), _d(u), _d(z)
    w = np.empty_like(u)
    _load().oracle_student_weights(_p(y), _p(u), _p(z), u.size, float(nu), _p(w))
    return w


def em_step_student(x, y, u, f, nu, r=1):
    """One heavy-tailed (Student-t, nu degrees of freedom) EM step.
    Returns (x', N', Den')."""
    x, y, u, f = _d(x).copy(), _d(y), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    num = np.empty_like(x)
    den = np.empty_like(x)
    _load().oracle_em_step_student(_p(x), _p(y), _p(u), _p(f), n, H, W, K, r, float(nu),
                                   num.ctypes.data, den.ctypes.data)
    return x, num, den


def student_loglik(x, y, v, u, f, nu, r=1):
    """Student-t log-likelihood of x over the valid pixels."""
    x, y, v, u, f = _d(x), _d(y), _d(v), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    return _load().oracle_student_loglik(_p(x), _p(y), _p(v), _p(u), _p(f), n, H, W, K, r,
                                         float(nu))


def chi2(x, y, u, f, r=1):
    x, y, u, f = _d(x), _d(y), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    return _load().oracle_chi2(_p(x), _p(y), _p(u), _p(f), n, H, W, K, r)


def logdet(v, u):
    v, u = _d(v), _d(u)
    return _load().oracle_logdet(_p(v), _p(u), v.size)


def loglik(x, y, v, u, f, r=1):
    """l(x) = -1/2 [chi2 + sum log(2 pi v)] over valid pixels."""
    return -0.5 * (chi2(x, y, u, f, r) + logdet(v, u))


def default_x0(y, u, r=1):
    y, u = _d(y), _d(u)
    return _load().oracle_default_x0(_p(y), _p(u), y.size, r)


def em_step_at(x, y, u, f, idx, r=1):
    """x', N and Den of one Eq. (2) iteration at latent flat indices idx."""
    x, y, u, f = _d(x), _d(y), _d(u), _d(f)
    n, H, W, K, r = _dims(u, f, r)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = idx.size
    xo, No, Do = np.empty(m), np.empty(m), np.empty(m)
    _load().oracle_em_step_at(_p(x), _p(y), _p(u), _p(f), n, H, W, K, r,
                              idx.ctypes.data_as(C.POINTER(C.c_long)), m,
                              xo.ctypes.data, No.ctypes.data, Do.ctypes.data)
    return xo, No, Do


def prepare(problem):
    """u, numerator N and default x0 of a synth.Problem (FP64)."""
    u, bad = weights(problem.v, problem.mask, problem.y)
    if bad:
        raise ValueError(f"{bad} valid pixels with invalid data")
    y = np.where(problem.mask != 0, problem.y.astype(np.float64), 0.0)
    N = numerator(y, u, problem.f, problem.r)
    c = default_x0(y, u, problem.r)
    return u, y, N, c
