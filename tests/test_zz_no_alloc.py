"""fm_expm_noalloc: exp(tA) for callers that cannot allocate device memory.

Its scratch is a fixed array inside the library image, shared by every call.
These checks call it through the C ABI twice in a row (different orders and
precisions, so the second call runs over whatever the first left in the
array) and compare each result with fm_expm on the same input and with the
oracle, within the parity tolerance of the other GPU tests.  The file is collected last so that a
failure here does not stop the rest of a -x run.
"""
import ctypes as C

import numpy as np
import pytest

import oracle

from _common import TOL_FP64, need_gpu

pytestmark = pytest.mark.gpu


def _call(L, fn, cs, A, F, opts, torch):
    info, s = C.c_int(-99), C.c_int(-99)
    d = A.shape[0]
    st = fn(C.byref(cs), d, C.c_void_p(A.data_ptr()), d, 1.0, C.c_void_p(F.data_ptr()), d,
            C.byref(opts), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(info),
            C.byref(s))
    return st, info.value, s.value


def test_noalloc_matches_expm_twice():
    torch = need_gpu()
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import _ffi, workloads as wl
    L = fm.lib()
    cs = _ffi.fm_coeffs()
    assert L.fm_coeffs_builtin(3, C.byref(cs)) == 0  # R8
    cases = [(128, "mixed", 8.0, 1), (37, "fp64", 2.5, 2), (96, "mixed", 0.7, 3)]
    for d, prec, nrm, seed in cases:
        An = wl.dense_scaled(d, nrm, seed, scale_sqrt=True)
        F_or, s_or, _ = oracle.expm(An, 1.0, "R8")
        A = torch.tensor(An, device="cuda")
        o = _ffi.default_opts(precision=prec)
        F_ref = torch.empty_like(A)
        st, info_ref, s_ref = _call(L, L.fm_expm, cs, A, F_ref, o, torch)
        assert st == 0 and info_ref == 0
        for _ in range(2):  # two calls in a row on the shared array
            F = torch.full_like(A, float("nan"))
            st, info, s = _call(L, L.fm_expm_noalloc, cs, A, F, o, torch)
            assert st == 0, L.fm_last_error()
            assert info == 0 and s == s_ref == s_or
            err = float((F - F_ref).norm() / F_ref.norm())
            assert err <= TOL_FP64, (d, prec, err)
            Fh = F.cpu().numpy()
            err = float(np.linalg.norm(Fh - F_or) / np.linalg.norm(F_or))
            assert err <= TOL_FP64, (d, prec, err)


def test_noalloc_rejects_too_large():
    torch = need_gpu()
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import _ffi
    L = fm.lib()
    cs = _ffi.fm_coeffs()
    L.fm_coeffs_builtin(3, C.byref(cs))
    A = torch.eye(129, dtype=torch.float64, device="cuda")
    F = torch.empty_like(A)
    st, _, _ = _call(L, L.fm_expm_noalloc, cs, A, F, _ffi.default_opts(), torch)
    assert st == _ffi.FM_ESHAPE
    assert b"FM_NOALLOC_MAX_DIM" in L.fm_last_error()
