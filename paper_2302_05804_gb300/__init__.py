"""GB300-native EM multi-frame deconvolution (arXiv:2302.05804, Sec. 2).

The compute path is the C-ABI CUDA library libemd.so (include/emd.h); this
package holds its build script and a thin ctypes binding with the same
function names.
"""
from .emd import *  # noqa: F401,F403
from .emd import Deconvolver, EMDError, load  # noqa: F401

__all__ = [n for n in dir() if n.startswith(("emd_", "EMD_"))] + ["Deconvolver", "EMDError", "load"]
