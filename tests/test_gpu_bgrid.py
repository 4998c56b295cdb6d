"""Parity of the batched grid path (one launch per step over the whole batch,
tensor-core products per 128 x 64 tile of every matrix) with the FP64 oracle.

Same bar as the one-CTA kernels: relative Frobenius error <= 1e-12 per result;
ragged orders spanning several tiles and ragged edges; the 4096-matrix batch
of the benchmark sampled one result at a time; masked matrices (non-finite
input) leave the others untouched.
"""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu

RAGGED = [1, 2, 5, 16, 17, 31, 48, 63, 64, 65, 100, 129, 200, 256]


@pytest.fixture(scope="module")
def fm():
    need_gpu()
    import paper_2210_03714_gb300 as fm_
    fm_.lib()
    return fm_


def T(x):
    import torch
    x = np.ascontiguousarray(x)
    dt = torch.complex128 if np.iscomplexobj(x) else torch.float64
    return torch.tensor(x, dtype=dt, device="cuda")


def test_bgrid_ragged(fm):
    rng = np.random.default_rng(7)
    norms = rng.uniform(0.5, 8.0, len(RAGGED))
    mats = [wl.dense_scaled(d, n, 100 + i, scale_sqrt=True)
            for i, (d, n) in enumerate(zip(RAGGED, norms))]
    ts = rng.uniform(0.5, 1.5, len(RAGGED))
    cs = oracle_set("R8")
    P = fm.Packed([T(m) for m in mats])
    F, info, s = fm.expm_batched(P, T(ts), fm.Coeffs(cs), path="grid")
    F = F.cpu().numpy()
    info, s = info.cpu().numpy(), s.cpu().numpy()
    for b, (M, t) in enumerate(zip(mats, ts)):
        ref, s_ref, _ = oracle.expm(M, t, cs)
        assert info[b] == 0 and s[b] == s_ref
        assert relerr(P.get(F, b), ref) <= TOL_FP64, (b, RAGGED[b])


def test_bgrid_complex_and_sets(fm):
    """Complex matrices (two product parts), and R4 (a zero node) on real ones."""
    import torch
    rng = np.random.default_rng(8)
    dims = [3, 40, 130]
    mats = []
    for i, d in enumerate(dims):
        G = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        mats.append(G * (2.0 + i) / np.abs(G).sum(0).max())
    cs = oracle_set("R8")
    P = fm.Packed([T(m) for m in mats], dtype=torch.complex128)
    F, info, s = fm.expm_batched(P, 1.0, fm.Coeffs(cs), path="grid")
    F, info, s = F.cpu().numpy(), info.cpu().numpy(), s.cpu().numpy()
    for b, M in enumerate(mats):
        ref, s_ref, _ = oracle.zexpm(M, 1.0, cs)
        assert info[b] == 0 and s[b] == s_ref
        assert relerr(P.get(F, b), ref) <= TOL_FP64
    cs4 = oracle_set("R4")
    real = [wl.dense_scaled(d, 1.0, 300 + d) for d in (20, 70)]
    P = fm.Packed([T(m) for m in real])
    F, info, s = fm.expm_batched(P, 1.0, fm.Coeffs(cs4), path="grid")
    F, info, s = F.cpu().numpy(), info.cpu().numpy(), s.cpu().numpy()
    for b, M in enumerate(real):
        ref, s_ref, _ = oracle.expm(M, 1.0, cs4)
        assert info[b] == 0 and s[b] == s_ref
        assert relerr(P.get(F, b), ref) <= TOL_FP64


def test_bgrid_masked_matrices(fm):
    """A non-finite matrix gets info -2; a zero matrix gives I exactly; the
    others are unaffected."""
    A0 = wl.dense_scaled(50, 3.0, 1)
    A1 = wl.dense_scaled(60, 3.0, 2)
    A1[5, 7] = np.inf
    A2 = np.zeros((33, 33))
    A3 = wl.dense_scaled(140, 6.0, 3)
    mats = [A0, A1, A2, A3]
    P = fm.Packed([T(m) for m in mats])
    F, info, s = fm.expm_batched(P, 1.0, "R8", path="grid")
    F, info, s = F.cpu().numpy(), info.cpu().numpy(), s.cpu().numpy()
    assert list(info) == [0, -2, 0, 0]
    assert np.array_equal(P.get(F, 2), np.eye(33)) and s[2] == 0
    for b in (0, 3):
        ref, s_ref, _ = oracle.expm(mats[b], 1.0, "R8")
        assert s[b] == s_ref and relerr(P.get(F, b), ref) <= TOL_FP64


def test_bgrid_matches_cta_path(fm):
    import torch
    dims, mats, norms = wl.batch_mixed_d(300, seed=77)
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    F1, i1, s1 = fm.expm_batched(P, 1.0, "R8", path="cta")
    F2, i2, s2 = fm.expm_batched(P, 1.0, "R8", path="grid")
    assert int((i1 != 0).sum()) == 0 and int((i2 != 0).sum()) == 0
    assert torch.equal(s1, s2)
    worst = max(relerr(P.get(F2, b).cpu().numpy(), P.get(F1, b).cpu().numpy())
                for b in range(len(dims)))
    assert worst <= TOL_FP64


def test_bgrid_full_size_sampled(fm):
    """The 4096-matrix batch in the configuration the benchmark times."""
    import torch
    dims, mats, norms = wl.batch_mixed_d(4096)
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    F, info, s = fm.expm_batched(P, 1.0, "R8", path="grid")
    torch.cuda.synchronize()
    assert int((info != 0).sum().item()) == 0
    s = s.cpu().numpy()
    rng = np.random.default_rng(12)
    pick = list(rng.choice(4096, 14, replace=False)) + [int(np.argmax(dims)), int(np.argmin(dims))]
    for b in pick:
        ref, s_ref, _ = oracle.expm(mats[b], 1.0, "R8")
        assert s[b] == s_ref
        assert relerr(P.get(F, b).cpu().numpy(), ref) <= TOL_FP64, (b, dims[b])


def test_bgrid_phi1_and_action(fm):
    """phi_1 and exp from one set of corrections (two weight vectors), the
    doublings as paired products, and W = phi_1(tA) V, on a ragged batch."""
    import torch
    dims = [3, 40, 100, 130, 200]
    rng = np.random.default_rng(9)
    mats = [wl.dense_scaled(d, 3.0, 900 + d) for d in dims]
    ts = rng.uniform(0.5, 1.0, len(dims))
    ce, cp = oracle_set("R8"), oracle_set("R8_phi1")
    P = fm.Packed([T(m) for m in mats])
    Phi, E, info, s = fm.phi1_batched(P, T(ts), fm.Coeffs(ce), fm.Coeffs(cp), path="grid")
    Phi, E, info, s = Phi.cpu().numpy(), E.cpu().numpy(), info.cpu().numpy(), s.cpu().numpy()
    m = 3
    V = rng.standard_normal(sum(dims) * m)
    W, info2, s2 = fm.phi1mv_batched(P, T(V), m, T(ts), fm.Coeffs(ce), fm.Coeffs(cp), path="grid")
    W, info2 = W.cpu().numpy(), info2.cpu().numpy()
    o = 0
    for b, (M, t) in enumerate(zip(mats, ts)):
        Phi_ref, E_ref, s_ref, _ = oracle.phi1(M, t, ce, cp)
        assert info[b] == 0 and s[b] == s_ref and info2[b] == 0
        assert relerr(P.get(Phi, b), Phi_ref) <= TOL_FP64
        assert relerr(P.get(E, b), E_ref) <= TOL_FP64
        d = dims[b]
        Vb = V[o:o + d * m].reshape(d, m)
        W_ref, _, _ = oracle.phi1mv(M, Vb, t, ce, cp)
        assert relerr(W[o:o + d * m].reshape(d, m), W_ref) <= TOL_FP64
        o += d * m


def spread(A, cs, form, F_ref):
    """Relative difference of two correct double evaluations (the oracle on
    P A P^T mapped back against the oracle on A): sets whose weights cancel
    (R10*: sum |b_i c_i| = 1.3e6) and the plain form of Eq. rat1 amplify the
    rounding of each system by their weights (Sec. 4.3)."""
    d = A.shape[0]
    p = np.random.default_rng(5).permutation(d)
    F2, _, _ = oracle.expm(A[np.ix_(p, p)], 1.0, cs, form)
    q = np.argsort(p)
    return relerr(F2[np.ix_(q, q)], F_ref)


@pytest.mark.parametrize("name,form", [("R10", "roundoff"), ("R10star", "roundoff"),
                                       ("R8", "plain"), ("R4", "plain")])
def test_bgrid_hybrid_and_plain(fm, name, form):
    """Sets with the hybrid terms d1 B + d2 B^2 (F starts from the multiple of
    I and those terms before the shifted systems add to it) and the plain
    form (no pair fusion: one system per node, b (I + Y) added), on ragged
    orders; the combination ends in the deviation F - I that the squarings
    take.  Bar: max(1e-12, twice the spread of two correct double
    evaluations)."""
    cs = oracle_set(name)
    fo = oracle.ROUNDOFF if form == "roundoff" else oracle.PLAIN
    mats = [wl.dense_scaled(d, 2.0 + 0.5 * i, 700 + d) for i, d in enumerate((17, 64, 130))]
    P = fm.Packed([T(m) for m in mats])
    F, info, s = fm.expm_batched(P, 1.0, fm.Coeffs(cs), path="grid", form=form)
    F, info, s = F.cpu().numpy(), info.cpu().numpy(), s.cpu().numpy()
    for b, M in enumerate(mats):
        ref, s_ref, _ = oracle.expm(M, 1.0, cs, fo)
        assert info[b] == 0 and s[b] == s_ref
        bar = max(TOL_FP64, 2.0 * spread(M, cs, fo, ref))
        assert relerr(P.get(F, b), ref) <= bar, (b, relerr(P.get(F, b), ref), bar)
