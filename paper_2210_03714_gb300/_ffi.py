"""ctypes view of the C ABI in include/fm.h (argument marshalling only).

Every function here has the name of its C counterpart and forwards plain
pointers and sizes.  Loading fails loudly when lib/libfm.so is missing: there
is no fallback implementation.
"""
import ctypes as C
import os

from . import _build

c_dp = C.POINTER(C.c_double)
c_ip = C.POINTER(C.c_int)
c_lp = C.POINTER(C.c_long)
c_i64p = C.POINTER(C.c_int64)

FM_OK, FM_EINVAL, FM_ESHAPE, FM_ENOMEM, FM_ECUDA, FM_ESINGULAR, FM_ENOCONV, FM_ETIMEOUT = range(8)
FM_FP64, FM_FP32_IR, FM_BF16_IR, FM_MIXED = 0, 1, 2, 3
PRECISION = {"fp64": FM_FP64, "fp32_ir": FM_FP32_IR, "bf16_ir": FM_BF16_IR, "mixed": FM_MIXED}
FM_ROUNDOFF, FM_PLAIN = 0, 1
BUILTIN = {"R4": 0, "R4_phi1": 1, "R4_phi1_a5": 2, "R8": 3, "R8_phi1": 4, "R5": 5, "R10": 6,
           "R10star": 7, "pade22": 8, "pade22_phi1": 9, "R8_cos": 10, "R8_sin": 11,
           "R8_phi2": 12, "frac4_exp": 13, "frac4_phi1": 14, "frac4_log1m": 15}
JOB = {"expm": 0, "phi1": 1, "expmv": 2, "phi1mv": 3, "zexpm": 4, "zexpmv": 5, "expmv_adj": 6,
       "cossin": 7, "rfun": 8}
FUNC = {"exp": 0, "phi1": 1, "phi2": 2, "cos": 3, "sin": 4, "log1m": 5}
MAX_TERMS = 16


class fm_coeffs(C.Structure):
    _fields_ = [("k", C.c_int), ("c_re", c_dp), ("c_im", c_dp), ("b_re", c_dp), ("b_im", c_dp),
                ("conj_pair", C.c_int), ("a0", C.c_double), ("d1", C.c_double),
                ("d2", C.c_double), ("order", C.c_int), ("theta", C.c_double)]


class fm_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("form", C.c_int), ("max_ir_iters", C.c_int),
                ("ir_tol", C.c_double), ("anorm", C.c_double), ("s_fixed", C.c_int),
                ("nsteps", C.c_long), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
                ("path", C.c_int)]


class fm_stats(C.Structure):
    _fields_ = [("products", C.c_longlong), ("product_flops", C.c_double),
                ("digit_flops", C.c_double), ("corrections", C.c_int),
                ("launches", C.c_longlong), ("tile_ms", C.c_double)]


def last_stats():
    """fm_last_stats of the calling thread as a dict."""
    s = fm_stats()
    lib().fm_last_stats(C.byref(s))
    return {k: getattr(s, k) for k, _ in fm_stats._fields_}


class FmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("fm status %d: %s" % (status, msg))
        self.status = status


_lib = None

# name -> (restype, argtypes)
_P = C.c_void_p
_SIGS = {
    "fm_coeffs_builtin": (C.c_int, [C.c_int, C.POINTER(fm_coeffs)]),
    "fm_theta": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_double, c_dp]),
    "fm_opts_default": (None, [C.POINTER(fm_opts)]),
    "fm_workspace_size": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.POINTER(fm_opts)]),
    "fm_max_dim": (C.c_int, []),
    "fm_expm": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, _P, C.c_int, C.c_double, _P, C.c_int,
                          C.POINTER(fm_opts), _P, c_ip, c_ip]),
    "fm_zexpm": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, _P, C.c_int, C.c_double, _P, C.c_int,
                           C.POINTER(fm_opts), _P, c_ip, c_ip]),
    "fm_phi1": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, _P, C.c_int,
                          C.c_double, _P, C.c_int, _P, C.c_int, C.POINTER(fm_opts), _P, c_ip, c_ip]),
    "fm_expmv": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, _P, C.c_int, C.c_double, C.c_int, _P,
                           C.c_int, _P, C.c_int, C.POINTER(fm_opts), _P, c_ip, c_lp]),
    "fm_zexpmv": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, _P, C.c_int, C.c_double, C.c_int, _P,
                            C.c_int, _P, C.c_int, C.POINTER(fm_opts), _P, c_ip, c_lp]),
    "fm_phi1mv": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, _P, C.c_int,
                            C.c_double, C.c_int, _P, C.c_int, _P, C.c_int, C.POINTER(fm_opts), _P,
                            c_ip, c_ip]),
    "fm_expm_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, _P, _P, _P, _P, _P, _P,
                                  _P, C.POINTER(fm_opts), _P]),
    "fm_zexpm_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, _P, _P, _P, _P, _P, _P,
                                   _P, C.POINTER(fm_opts), _P]),
    "fm_phi1_batched": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, C.c_int, _P,
                                  _P, _P, _P, _P, _P, _P, _P, C.POINTER(fm_opts), _P]),
    "fm_expmv_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, _P, _P, _P, _P, C.c_int,
                                   _P, _P, _P, _P, _P, C.POINTER(fm_opts), _P]),
    "fm_zexpmv_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, _P, _P, _P, _P,
                                    C.c_int, _P, _P, _P, _P, _P, C.POINTER(fm_opts), _P]),
    "fm_phi1mv_batched": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, C.c_int,
                                    _P, _P, _P, _P, C.c_int, _P, _P, _P, _P, _P,
                                    C.POINTER(fm_opts), _P]),
    "fm_expmv_adjoint_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, _P, _P, _P, _P,
                                           _P, _P, _P, _P, _P, _P, _P, _P, C.POINTER(fm_opts),
                                           _P]),
    "fm_trid_expmv_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, _P, _P, _P, _P,
                                        _P, _P, _P, _P, C.POINTER(fm_opts), _P]),
    "fm_trid_workspace_size": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    "fm_band_expmv_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, C.c_int, _P, _P,
                                        _P, _P, _P, _P, C.POINTER(fm_opts), _P]),
    "fm_band_workspace_size": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int]),
    "fm_cossin": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, _P, C.c_int,
                            C.c_double, _P, C.c_int, _P, C.c_int, C.POINTER(fm_opts), _P, c_ip,
                            c_ip]),
    "fm_cossin_batched": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, C.c_int,
                                    _P, _P, _P, _P, _P, _P, _P, _P, C.POINTER(fm_opts), _P]),
    "fm_rfun": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, _P, C.c_int, C.c_double, _P, C.c_int,
                          C.POINTER(fm_opts), _P, c_ip]),
    "fm_rfun_batched": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, C.c_int, _P, _P, _P, _P, _P, _P,
                                  C.POINTER(fm_opts), _P]),
    "fm_autotune": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, C.c_int,
                              C.POINTER(fm_opts), _P, c_ip, c_dp, c_ip]),
    "fm_autotune_reset": (None, []),
    "fm_select_batched": (C.c_int, [C.POINTER(fm_coeffs), C.POINTER(fm_coeffs), C.c_int, C.c_int,
                                    C.c_int, _P, _P, _P, _P, _P, _P, C.POINTER(fm_opts), _P]),
    "fm_expm_noalloc": (C.c_int, [C.POINTER(fm_coeffs), C.c_int, _P, C.c_int, C.c_double, _P,
                                  C.c_int, C.POINTER(fm_opts), _P, c_ip, c_ip]),
    "fm_last_error": (C.c_char_p, []),
    "fm_last_stats": (None, [C.c_void_p]),
    "fm_version": (C.c_char_p, []),
}


def lib():
    """Load lib/libfm.so (building it in-tree first if the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libfm.so is missing and could not be built")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names declared in include/fm.h that the binding knows about."""
    return sorted(_SIGS)


def check(status):
    if status != FM_OK:
        raise FmError(status, lib().fm_last_error().decode(errors="replace"))
    return status


def default_opts(**kw):
    o = fm_opts()
    lib().fm_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "form" and isinstance(v, str):
            v = {"roundoff": FM_ROUNDOFF, "plain": FM_PLAIN}[v]
        if k == "path" and isinstance(v, str):
            v = {"auto": 0, "cta": 1, "grid": 2, "team": 3}[v]
        setattr(o, k, v)
    return o
