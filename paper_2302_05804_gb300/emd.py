"""Thin Python binding of the C ABI in include/emd.h (argument marshalling
only; every step of the EM iteration runs in the CUDA library).

Functions carry the C names. Array arguments may be numpy arrays (host) or
torch tensors (host or CUDA); they must be C-contiguous with the dtype the
ABI states (float32, or uint8 for masks). The library refuses to run
without its compiled extension: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

EMD_OK = 0
EMD_EINVAL = -1
EMD_ENOMEM = -2
EMD_ECUDA = -3
EMD_ESTATE = -4
EMD_EDATA = -5
EMD_ETIMEOUT = -6
EMD_EUNSUPPORTED = -7

EMD_PREC_FP32 = 0
EMD_PREC_BF16 = 1
EMD_PREC_FP16 = 2
EMD_PREC_SPLIT_BF16 = 3
EMD_PREC_SPLIT_FP16 = 4
EMD_PREC_FFT_FP32 = 5
EMD_PREC_FP32_PAIR = 6
EMD_NOISE_GAUSSIAN = 0
EMD_NOISE_STUDENT_T = 1
EMD_TILE_AUTO = 0
EMD_TILE_64 = 1
EMD_TILE_48 = 2
EMD_TILE_32 = 3

EXPORTS = [
    "emd_create", "emd_ctx_bytes", "emd_destroy", "emd_last_error", "emd_set_stream",
    "emd_set_frames", "emd_set_x", "emd_iterate", "emd_get_x", "emd_loglik", "emd_loglik_chi2",
    "emd_set_precision", "emd_get_numerator", "emd_get_weights", "emd_frame_stats_noalloc",
    "emd_batch_create", "emd_batch_destroy", "emd_batch_add", "emd_batch_remove",
    "emd_batch_step", "emd_batch_remaining", "emd_batch_sync", "emd_batch_config",
    "emd_selftest_wait_timeout", "emd_iterate_streaming", "emd_fit_psf", "emd_set_noise",
    "emd_measure_fma_rate", "emd_ctx_bytes_precision", "emd_set_tile_shape", "emd_get_tile_shape",
]


class EMDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libemd.so; raise if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(
                    f"{path} is missing: build the CUDA extension first "
                    "(python -m paper_2302_05804_gb300.build)")
            _build.build()
        lib = C.CDLL(path)
        vp, i, dp = C.c_void_p, C.c_int, C.POINTER(C.c_double)
        lib.emd_create.argtypes = [i, i, i, i, i]
        lib.emd_create.restype = vp
        lib.emd_ctx_bytes.argtypes = [i, i, i, i, i]
        lib.emd_ctx_bytes_precision.argtypes = [i, i, i, i, i, i]
        lib.emd_ctx_bytes_precision.restype = C.c_size_t
        lib.emd_ctx_bytes.restype = C.c_size_t
        lib.emd_destroy.argtypes = [vp]
        lib.emd_destroy.restype = None
        lib.emd_last_error.argtypes = []
        lib.emd_last_error.restype = C.c_char_p
        lib.emd_set_stream.argtypes = [vp, vp]
        lib.emd_set_frames.argtypes = [vp, vp, vp, vp, vp]
        lib.emd_set_x.argtypes = [vp, vp]
        lib.emd_iterate.argtypes = [vp, i]
        lib.emd_get_x.argtypes = [vp, vp]
        lib.emd_loglik.argtypes = [vp, dp]
        lib.emd_loglik_chi2.argtypes = [vp, dp, dp]
        lib.emd_set_precision.argtypes = [vp, i]
        lib.emd_get_numerator.argtypes = [vp, vp]
        lib.emd_get_weights.argtypes = [vp, vp]
        lib.emd_frame_stats_noalloc.argtypes = [vp, vp, vp, i, i, i, vp, vp]
        lib.emd_frame_stats_noalloc.restype = i
        lib.emd_iterate_streaming.argtypes = [vp, i, vp]
        lib.emd_iterate_streaming.restype = i
        lib.emd_selftest_wait_timeout.argtypes = [vp, i]
        lib.emd_selftest_wait_timeout.restype = i
        ip = C.POINTER(C.c_int)
        lib.emd_batch_create.argtypes = [i]
        lib.emd_batch_create.restype = vp
        lib.emd_batch_destroy.argtypes = [vp]
        lib.emd_batch_destroy.restype = None
        lib.emd_batch_add.argtypes = [vp, vp, i]
        lib.emd_batch_remove.argtypes = [vp, i]
        lib.emd_batch_step.argtypes = [vp, ip]
        lib.emd_batch_remaining.argtypes = [vp, i]
        lib.emd_batch_sync.argtypes = [vp]
        lib.emd_batch_config.argtypes = [vp, ip, ip, ip, ip, ip]
        lib.emd_set_tile_shape.argtypes = [vp, i]
        lib.emd_set_tile_shape.restype = i
        lib.emd_get_tile_shape.argtypes = [vp, ip, ip]
        lib.emd_get_tile_shape.restype = i
        lib.emd_fit_psf.argtypes = [vp, i, i, i, vp, i, vp, C.c_float, C.c_float, i, vp, vp]
        lib.emd_fit_psf.restype = i
        lib.emd_set_noise.argtypes = [vp, i, C.c_double]
        lib.emd_set_noise.restype = i
        lib.emd_measure_fma_rate.argtypes = [i, dp]
        lib.emd_measure_fma_rate.restype = i
        for name in ("emd_batch_add", "emd_batch_remove", "emd_batch_step",
                     "emd_batch_remaining", "emd_batch_sync", "emd_batch_config"):
            getattr(lib, name).restype = i
        for name in ("emd_set_stream", "emd_set_frames", "emd_set_x", "emd_iterate",
                     "emd_get_x", "emd_loglik", "emd_loglik_chi2", "emd_set_precision",
                     "emd_get_numerator",
                     "emd_get_weights"):
            getattr(lib, name).restype = i
        _lib = lib
        return lib


def _check(rc: int):
    if rc != EMD_OK:
        raise EMDError(rc, load().emd_last_error().decode())


def _ptr(a, dtype, name: str):
    """Data pointer of a contiguous numpy array or torch tensor of dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{name}: need a C-contiguous {np.dtype(dtype)} array")
        return a.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        tdt = {np.float32: torch.float32, np.uint8: torch.uint8}[np.dtype(dtype).type]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"{name}: need a contiguous {tdt} tensor")
        return a.data_ptr()
    raise TypeError(f"{name}: unsupported array type {type(a)}")


# -- C-ABI wrappers (same names) ---------------------------------------------

def emd_create(H: int, W: int, n: int, psf_k: int, r: int = 1) -> int:
    h = load().emd_create(H, W, n, psf_k, r)
    if not h:
        raise EMDError(EMD_EINVAL, load().emd_last_error().decode())
    return h


def emd_ctx_bytes(H: int, W: int, n: int, psf_k: int, r: int = 1) -> int:
    return int(load().emd_ctx_bytes(H, W, n, psf_k, r))


def emd_ctx_bytes_precision(H: int, W: int, n: int, psf_k: int, r: int, mode: int) -> int:
    return int(load().emd_ctx_bytes_precision(H, W, n, psf_k, r, int(mode)))


def emd_destroy(ctx) -> None:
    if ctx:
        load().emd_destroy(ctx)


def emd_last_error() -> str:
    return load().emd_last_error().decode()


def emd_set_stream(ctx, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(load().emd_set_stream(ctx, stream))


def emd_set_frames(ctx, y, v, f, mask=None) -> None:
    _check(load().emd_set_frames(ctx, _ptr(y, np.float32, "y"), _ptr(v, np.float32, "v"),
                                 _ptr(f, np.float32, "f"), _ptr(mask, np.uint8, "mask")))


def emd_set_x(ctx, x0) -> None:
    _check(load().emd_set_x(ctx, _ptr(x0, np.float32, "x0")))


def emd_iterate(ctx, k: int) -> None:
    _check(load().emd_iterate(ctx, int(k)))


def emd_iterate_streaming(ctx, k: int, order=None) -> None:
    """k streaming passes (one update per exposure, in `order`)."""
    arr = None
    if order is not None:
        arr = (C.c_int * len(order))(*[int(t) for t in order])
    _check(load().emd_iterate_streaming(ctx, int(k), arr))


def emd_get_x(ctx, out) -> None:
    _check(load().emd_get_x(ctx, _ptr(out, np.float32, "out")))


def emd_get_numerator(ctx, out) -> None:
    _check(load().emd_get_numerator(ctx, _ptr(out, np.float32, "out")))


def emd_get_weights(ctx, out) -> None:
    _check(load().emd_get_weights(ctx, _ptr(out, np.float32, "out")))


def emd_loglik(ctx) -> float:
    """The log-likelihood of the current iterate (FP64)."""
    ll = C.c_double()
    _check(load().emd_loglik(ctx, C.byref(ll)))
    return ll.value


def emd_loglik_chi2(ctx):
    """Returns (loglik, chi2), both FP64."""
    ll, chi = C.c_double(), C.c_double()
    _check(load().emd_loglik_chi2(ctx, C.byref(ll), C.byref(chi)))
    return ll.value, chi.value


def emd_frame_stats_noalloc(y, v, mask, H: int, W: int, n: int, out, stream=None) -> None:
    """Per-exposure FP64 statistics (n x 4 doubles into the device tensor
    ``out``) from device tensors y, v, mask; allocates no device memory.

    The C side cannot see buffer sizes, so they are checked here: y and v
    must be float32 CUDA tensors of at least n*H*W elements, mask (optional)
    a uint8 CUDA tensor of at least n*H*W, out a contiguous float64 CUDA
    tensor of at least 4*n, all on the current device."""
    import torch
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    H, W, n = int(H), int(W), int(n)
    need = max(n, 0) * max(H, 0) * max(W, 0)
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t, dt, cnt in (("y", y, torch.float32, need), ("v", v, torch.float32, need),
                             ("mask", mask, torch.uint8, need),
                             ("out", out, torch.float64, 4 * max(n, 0))):
        if t is None and name == "mask":
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name}: need a CUDA tensor")
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"{name}: need a contiguous {dt} tensor")
        if t.device.index != dev:
            raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is cuda:{dev}")
        if t.numel() < cnt:
            raise ValueError(f"{name}: {t.numel()} elements, need at least {cnt}")
    _check(load().emd_frame_stats_noalloc(y.data_ptr(), v.data_ptr(),
                                          None if mask is None else mask.data_ptr(), H, W, n,
                                          out.data_ptr(), stream))


def emd_fit_psf(f, g, r: int, lam: float, lr: float, iters: int, h0=None, h_out=None,
                loss_out=None):
    """Eq. (4) fit of n super-resolved PSFs: f is n x K x K (or K x K), g is
    Kg x Kg, both float32 (numpy or torch, host or device). Returns (h, loss):
    h is n x Kh x Kh with Kh = r (K-1) + 1 (h_out when given), loss the n
    final Eq. (4) losses (loss_out when given; host array otherwise)."""
    single = len(f.shape) == 2
    n = 1 if single else int(f.shape[0])
    K, Kg = int(f.shape[-1]), int(g.shape[-1])
    Kh = r * (K - 1) + 1
    own_h, own_l = h_out is None, loss_out is None
    if own_h:
        h_out = np.empty((n, Kh, Kh), np.float32)
    if own_l:
        loss_out = np.empty(n, np.float32)
    _check(load().emd_fit_psf(_ptr(f, np.float32, "f"), n, K, int(r), _ptr(g, np.float32, "g"), Kg,
                              _ptr(h0, np.float32, "h0"), float(lam), float(lr), int(iters),
                              _ptr(h_out, np.float32, "h_out"),
                              _ptr(loss_out, np.float32, "loss_out")))
    if single:
        return (h_out[0] if own_h else h_out), (float(loss_out[0]) if own_l else loss_out)
    return h_out, loss_out


def emd_selftest_wait_timeout(ctx, spins: int = 1000) -> int:
    """Returns the raw status (EMD_ETIMEOUT expected)."""
    return int(load().emd_selftest_wait_timeout(ctx, int(spins)))


def emd_measure_fma_rate(iters: int = 20000) -> float:
    """Measured FP32 FMA rate of the current GPU, TFLOP/s."""
    out = C.c_double()
    _check(load().emd_measure_fma_rate(int(iters), C.byref(out)))
    return out.value


def emd_set_noise(ctx, model: int, nu: float = 0.0) -> None:
    """EMD_NOISE_GAUSSIAN or EMD_NOISE_STUDENT_T with nu degrees of freedom."""
    _check(load().emd_set_noise(ctx, int(model), float(nu)))


def emd_set_precision(ctx, mode: int) -> None:
    _check(load().emd_set_precision(ctx, int(mode)))


def emd_batch_create(max_jobs: int):
    h = load().emd_batch_create(int(max_jobs))
    if not h:
        raise EMDError(EMD_EINVAL, load().emd_last_error().decode())
    return h


def emd_batch_destroy(b) -> None:
    if b:
        load().emd_batch_destroy(b)


def emd_batch_add(b, ctx, iterations: int) -> int:
    rc = load().emd_batch_add(b, ctx, int(iterations))
    if rc < 0:
        _check(rc)
    return rc


def emd_batch_remove(b, slot: int) -> None:
    _check(load().emd_batch_remove(b, int(slot)))


def emd_batch_step(b) -> int:
    """One iteration for every active job; returns how many finished."""
    fin = C.c_int(0)
    _check(load().emd_batch_step(b, C.byref(fin)))
    return fin.value


def emd_batch_remaining(b, slot: int) -> int:
    rc = load().emd_batch_remaining(b, int(slot))
    if rc < 0:
        _check(rc)
    return rc


def emd_batch_sync(b) -> None:
    _check(load().emd_batch_sync(b))


def emd_batch_config(b):
    c, o, m, f, t = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(load().emd_batch_config(b, C.byref(c), C.byref(o), C.byref(m), C.byref(f),
                                   C.byref(t)))
    return {"clusters": c.value, "order": o.value, "max_clusters": m.value, "form": f.value,
            "tile_shape": t.value}


def emd_set_tile_shape(ctx, shape: int) -> None:
    """Tile shape of the FP32 halo-exchange iteration: an EMD_TILE_* value
    (EMD_TILE_AUTO: the autotuner's choice)."""
    _check(load().emd_set_tile_shape(ctx, int(shape)))


def emd_get_tile_shape(ctx):
    """(shape, decided): the tile shape the next FP32 iteration uses."""
    sh, d = C.c_int(), C.c_int()
    _check(load().emd_get_tile_shape(ctx, C.byref(sh), C.byref(d)))
    return sh.value, bool(d.value)


# -- convenience wrapper --------------------------------------------------------

class Deconvolver:
    """Owns one context: ``Deconvolver(H, W, n, K, r)``, then
    ``set_frames``, ``iterate``, ``x()``, ``loglik()``."""

    def __init__(self, H, W, n, K, r=1, stream=None):
        self.H, self.W, self.n, self.K, self.r = H, W, n, K, r
        self.ctx = emd_create(H, W, n, K, r)
        if stream is not None:
            emd_set_stream(self.ctx, stream)

    def close(self):
        if self.ctx:
            emd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_frames(self, y, v, f, mask=None):
        emd_set_frames(self.ctx, y, v, f, mask)

    def set_x(self, x0):
        emd_set_x(self.ctx, x0)

    def iterate(self, k):
        emd_iterate(self.ctx, k)

    def iterate_streaming(self, k, order=None):
        emd_iterate_streaming(self.ctx, k, order)

    def set_precision(self, mode):
        emd_set_precision(self.ctx, mode)

    def set_noise(self, model, nu=0.0):
        emd_set_noise(self.ctx, model, nu)

    def set_tile_shape(self, shape):
        emd_set_tile_shape(self.ctx, shape)

    def tile_shape(self):
        return emd_get_tile_shape(self.ctx)

    def x(self, out=None):
        if out is None:
            out = np.empty((self.r * self.H, self.r * self.W), np.float32)
        emd_get_x(self.ctx, out)
        return out

    def numerator(self):
        out = np.empty((self.r * self.H, self.r * self.W), np.float32)
        emd_get_numerator(self.ctx, out)
        return out

    def weights(self):
        out = np.empty((self.n, self.H, self.W), np.float32)
        emd_get_weights(self.ctx, out)
        return out

    def loglik(self):
        """(loglik, chi2) of the current iterate."""
        return emd_loglik_chi2(self.ctx)
