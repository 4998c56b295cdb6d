"""GB300-native batched matrix functions by parallel shifted solves.

Method: S. Blanes, "Parallel computation of functions of matrices and their
action on vectors", arXiv:2210.03714.  The compute path is the CUDA library
lib/libfm.so (C ABI in include/fm.h); this package is its Python binding.
"""
from ._ffi import lib, FmError, BUILTIN, default_opts, exported_symbols, last_stats  # noqa: F401
from .api import (Coeffs, Packed, expm, phi1, expmv, phi1mv, expm_batched,  # noqa: F401
                  phi1_batched, expmv_batched, phi1mv_batched, expmv_adjoint_batched,
                  select_batched, ExpmvFn, trid_expmv_batched, cossin, cossin_batched, rfun,
                  rfun_batched, band_expmv_batched,
                  autotune)

__all__ = ["lib", "FmError", "Coeffs", "Packed", "expm", "phi1", "expmv", "phi1mv",
           "expm_batched", "phi1_batched", "expmv_batched", "phi1mv_batched",
           "expmv_adjoint_batched", "select_batched", "ExpmvFn", "trid_expmv_batched", "cossin",
           "cossin_batched", "rfun", "rfun_batched", "band_expmv_batched",
           "autotune"]
