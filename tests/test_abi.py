"""CPU checks of the C ABI: the library builds, loads, and exports every
entry point that include/fm.h declares; no compute call is made."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "fm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fm_[a-z0-9_]+)\s*\(", src)))


def test_header_parses():
    names = header_functions()
    assert "fm_expm" in names and "fm_expm_batched" in names and len(names) >= 20


def test_library_exports_every_declared_symbol():
    import paper_2210_03714_gb300 as fm
    L = fm.lib()
    missing = [n for n in header_functions() if not hasattr(L, n)]
    assert not missing, missing
    # the Python binding covers the same names
    assert set(header_functions()) <= set(fm.exported_symbols())


def test_host_only_calls():
    """Calls that need no GPU: builtins, theta, defaults, argument errors."""
    import ctypes as C
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import _ffi
    L = fm.lib()
    assert L.fm_version().startswith(b"fm")
    assert L.fm_max_dim() >= 512
    cs = _ffi.fm_coeffs()
    assert L.fm_coeffs_builtin(3, C.byref(cs)) == 0 and cs.k == 9
    assert L.fm_coeffs_builtin(99, C.byref(cs)) == _ffi.FM_EINVAL
    o = _ffi.fm_opts()
    L.fm_opts_default(C.byref(o))
    assert o.precision == _ffi.FM_MIXED and o.max_ir_iters == 2 and o.s_fixed == -1
    # argument validation happens before any device work
    st = L.fm_expm(C.byref(cs), 0, None, 0, 1.0, None, 0, None, None, None, None)
    assert st == _ffi.FM_ESHAPE
    st = L.fm_expm(C.byref(cs), 4, None, 4, 1.0, None, 4, None, None, None, None)
    assert st == _ffi.FM_EINVAL
    assert b"NULL" in L.fm_last_error()


def test_builtin_sets_match_oracle_exact_values():
    """The library's own coefficient tables (printed rationals, and the phi_1
    sets it derives by exact Lagrange interpolation) equal the oracle's exact
    rationals to the last bit, and its theta agrees with the oracle's."""
    import paper_2210_03714_gb300 as fm
    from oracle import coeffs as oc
    for name in ["R4", "R4_phi1", "R4_phi1_a5", "R8", "R8_phi1", "R5", "R10", "R10star",
                 "R8_cos", "R8_sin", "R8_phi2", "frac4_exp", "frac4_phi1", "frac4_log1m"]:
        lib = fm.Coeffs(name).as_dict()
        ex = oc.SETS[name]
        assert lib["c_re"] == [float(c) for c in ex.c], name
        assert lib["b_re"] == [float(b) for b in ex.b], name
        assert lib["a0"] == float(ex.a0()), name
        if name.startswith("R10"):
            assert lib["d1"] == float(ex.d[1]) and lib["d2"] == float(ex.d[2])
        th = oc.theta(ex, oc.U_FP64)
        assert abs(lib["theta"] / th - 1) < 1e-10, name
    for name in ["pade22", "pade22_phi1"]:
        lib = fm.Coeffs(name).as_dict()
        ref = oc.oracle_coeffs(name)
        assert abs(lib["c_re"][0] - ref["c_re"][0]) < 1e-16
        assert abs(lib["c_im"][0] - ref["c_im"][0]) < 1e-16
        assert abs(lib["b_im"][0] - ref["b_im"][0]) < 1e-15
        assert abs(lib["theta"] / ref["theta"] - 1) < 1e-8


def test_workspace_size_monotone():
    import paper_2210_03714_gb300 as fm
    L = fm.lib()
    a = L.fm_workspace_size(0, 16, 64, 0, 9, None)
    b = L.fm_workspace_size(0, 16, 256, 0, 9, None)
    assert 0 < a < b
    assert L.fm_workspace_size(0, 16, 100000, 0, 9, None) == 0


def test_trid_host_validation():
    """fm_trid_expmv_batched rejects bad shapes, NULL pointers and complex
    node sets before any device work; its scratch size grows with the batch
    and the order and is 0 for bad arguments."""
    import ctypes as C
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import _ffi
    L = fm.lib()
    cs = _ffi.fm_coeffs()
    assert L.fm_coeffs_builtin(_ffi.BUILTIN["R10"], C.byref(cs)) == 0
    args = [None] * 8
    assert L.fm_trid_expmv_batched(C.byref(cs), 0, 10, *args, None, None) == _ffi.FM_ESHAPE
    assert L.fm_trid_expmv_batched(C.byref(cs), 4, 10, *args, None, None) == _ffi.FM_EINVAL
    assert b"NULL" in L.fm_last_error()
    fake = [C.c_void_p(256)] * 7 + [None]   # never dereferenced: rejected first
    cp = _ffi.fm_coeffs()
    assert L.fm_coeffs_builtin(_ffi.BUILTIN["pade22"], C.byref(cp)) == 0
    assert L.fm_trid_expmv_batched(C.byref(cp), 4, 10, *fake, None, None) == _ffi.FM_EINVAL
    a = L.fm_trid_workspace_size(10, 100, 10)
    assert 0 < a < L.fm_trid_workspace_size(20, 100, 10)
    assert a < L.fm_trid_workspace_size(10, 200, 10)
    assert L.fm_trid_workspace_size(0, 100, 10) == 0
    assert L.fm_trid_workspace_size(10, 100, 17) == 0


def test_precision_and_path_routing():
    """Each precision value runs where its arithmetic exists: FM_FP32_IR on the
    one-CTA kernels, FM_BF16_IR on the grid paths; a combination that does not
    exist is rejected before any device work (the pointers are never used)."""
    import ctypes as C
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import _ffi
    L = fm.lib()
    cs = _ffi.fm_coeffs()
    assert L.fm_coeffs_builtin(_ffi.BUILTIN["R8"], C.byref(cs)) == 0
    fake = C.c_void_p(256)
    for prec, path in ((_ffi.FM_FP32_IR, 2), (_ffi.FM_BF16_IR, 1)):
        o = _ffi.default_opts(precision=prec, path=path)
        st = L.fm_expm(C.byref(cs), 64, fake, 64, 1.0, fake, 64, C.byref(o), None, None, None)
        assert st == _ffi.FM_EINVAL, (prec, path)
        assert b"FM_" in L.fm_last_error()
    o = _ffi.default_opts(precision=9)
    st = L.fm_expm(C.byref(cs), 64, fake, 64, 1.0, fake, 64, C.byref(o), None, None, None)
    assert st == _ffi.FM_EINVAL
    # FM_FP32_IR beyond the one-CTA kernels' order
    o = _ffi.default_opts(precision="fp32_ir")
    st = L.fm_expm(C.byref(cs), 2048, fake, 2048, 1.0, fake, 2048, C.byref(o), None, None, None)
    assert st == _ffi.FM_EINVAL
    # batched actions have no grid form
    o = _ffi.default_opts(precision="bf16_ir")
    st = L.fm_expmv_batched(C.byref(cs), 4, 16, fake, fake, fake, fake, 1, fake, fake, fake, fake,
                            None, C.byref(o), None)
    assert st == _ffi.FM_EINVAL
    # the team path: single-matrix exp in double, d <= 512
    for prec, d in ((_ffi.FM_FP32_IR, 64), (_ffi.FM_BF16_IR, 64), (_ffi.FM_FP64, 513)):
        o = _ffi.default_opts(precision=prec, path="team")
        st = L.fm_expm(C.byref(cs), d, fake, d, 1.0, fake, d, C.byref(o), None, None, None)
        assert st == _ffi.FM_EINVAL, (prec, d)
    o = _ffi.default_opts(path="team")
    st = L.fm_phi1(C.byref(cs), C.byref(cs), 64, fake, 64, 1.0, fake, 64, None, 64, C.byref(o),
                   None, None, None)
    assert st == _ffi.FM_EINVAL
    st = L.fm_expm_batched(C.byref(cs), 4, 16, fake, fake, fake, fake, fake, fake, None,
                           C.byref(o), None)
    assert st == _ffi.FM_EINVAL
    o = _ffi.default_opts()
    o.path = 4
    st = L.fm_expm(C.byref(cs), 64, fake, 64, 1.0, fake, 64, C.byref(o), None, None, None)
    assert st == _ffi.FM_EINVAL
    assert L.fm_workspace_size(0, 1, 512, 0, 9, C.byref(_ffi.default_opts(path="team"))) > 0
    assert L.fm_workspace_size(0, 1, 513, 0, 9, C.byref(_ffi.default_opts(path="team"))) == 0
    # workspace sizes follow the same routes
    assert L.fm_workspace_size(0, 1, 64, 0, 9, C.byref(_ffi.default_opts(precision="bf16_ir"))) > 0
    assert L.fm_workspace_size(2, 8, 64, 1, 9, C.byref(_ffi.default_opts(precision="bf16_ir"))) == 0
    assert L.fm_workspace_size(0, 1, 4096, 0, 9, C.byref(_ffi.default_opts(precision="fp32_ir"))) == 0


def test_conjugate_pair_host_rules():
    """Conjugate-pair sets reach the dense kernels; the adjoint and the
    tridiagonal action reject them before any device work."""
    import ctypes as C
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import _ffi
    L = fm.lib()
    cp = _ffi.fm_coeffs()
    assert L.fm_coeffs_builtin(_ffi.BUILTIN["pade22"], C.byref(cp)) == 0 and cp.conj_pair == 1
    fake = C.c_void_p(256)
    o = _ffi.default_opts(nsteps=4)
    st = L.fm_expmv_adjoint_batched(C.byref(cp), 2, 8, fake, fake, fake, fake, fake, fake, fake,
                                    fake, fake, fake, fake, fake, C.byref(o), None)
    assert st == _ffi.FM_EINVAL and b"conj" in L.fm_last_error()
    bad = _ffi.fm_coeffs()
    C.memmove(C.byref(bad), C.byref(cp), C.sizeof(cp))
    bad.conj_pair = 2
    st = L.fm_expm(C.byref(bad), 8, fake, 8, 1.0, fake, 8, None, None, None, None)
    assert st == _ffi.FM_EINVAL


def test_select_host_validation():
    """fm_select_batched (step a1 alone) checks its job and pointers first."""
    import ctypes as C
    import paper_2210_03714_gb300 as fm
    from paper_2210_03714_gb300 import _ffi
    L = fm.lib()
    cs = _ffi.fm_coeffs()
    assert L.fm_coeffs_builtin(_ffi.BUILTIN["R8"], C.byref(cs)) == 0
    fake = C.c_void_p(256)
    args = [fake] * 6
    assert L.fm_select_batched(C.byref(cs), None, 99, 4, 16, *args, None, None) == _ffi.FM_EINVAL
    assert L.fm_select_batched(C.byref(cs), None, 1, 4, 16, *args, None, None) == _ffi.FM_EINVAL
    assert L.fm_select_batched(C.byref(cs), None, 0, 0, 16, *args, None, None) == _ffi.FM_ESHAPE
    assert L.fm_select_batched(C.byref(cs), None, 0, 4, 16, None, *args[1:], None,
                               None) == _ffi.FM_EINVAL
