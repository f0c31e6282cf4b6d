"""GB300-native photometric bundle adjustment: inverse compositional with
proxy templates (IC) and forwards compositional (FC), after Ham, Lucey and
Singh (ICCV 2017, arXiv 1704.06967).

The compute path is libpba.so (hand-written CUDA for sm_103a, C ABI in
include/pba.h); `pba` is its thin ctypes binding.
"""
from .pba import Batch, Bundle, PbaError, declared_symbols, load

__all__ = ["Batch", "Bundle", "PbaError", "declared_symbols", "load"]
