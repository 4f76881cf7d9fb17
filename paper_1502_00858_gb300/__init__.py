"""GB300 consensus-ADMM calibration across frequency (Yatawatta 2015, arXiv:1502.00858).

The computation lives in libcalib.so (CUDA, sm_103a); `capi` is its Python binding and
`Calibrator` a small convenience wrapper around a context.
"""
from . import capi
from .calibrator import Calibrator

__all__ = ["capi", "Calibrator"]
