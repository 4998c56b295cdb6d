"""The C ABI's own guarantees on the GPU: step a1 alone (fm_select_batched)
against the oracle's choice of s and N; per-matrix status -4 for an order
outside [1, dmax] on every batched path; the precision values; and calls on
two streams at once with the library-managed scratch (one buffer per stream)."""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu


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


def test_select_matches_oracle_and_calls(fm):
    """s and N for a ragged batch equal the oracle's (Sec. 1: smallest s with
    ||tA||_1 / 2^s <= theta; N = ceil(||tA||_1 / theta)) and what the calls
    themselves report; a non-finite matrix gets -2."""
    import torch
    dims = [1, 5, 16, 33, 64, 100]
    mats = [wl.dense_scaled(d, 0.3 + 1.7 * i, 200 + i) for i, d in enumerate(dims)]
    mats[2] = mats[2].copy()
    mats[2][1, 1] = np.inf
    ts = np.linspace(0.5, 2.0, len(dims))
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    th = oracle.CS("R8").theta
    s, info = fm.select_batched(P, T(ts), "R8", "expm")
    N, info2 = fm.select_batched(P, T(ts), "R8", "expmv")
    s, N, info, info2 = (x.cpu().numpy() for x in (s, N, info, info2))
    for b, (M, t) in enumerate(zip(mats, ts)):
        if b == 2:
            assert info[b] == -2 and info2[b] == -2
            continue
        eta = oracle.norm1(t * M)
        assert info[b] == 0 and s[b] == oracle.select_s(eta, th)
        assert N[b] == oracle.select_nsteps(eta, th)
    # phi_1 takes the smaller theta of its two sets
    sp, _ = fm.select_batched(P, T(ts), "R8", "phi1", cphi="R8_phi1")
    thp = min(th, oracle.CS("R8_phi1").theta)
    assert int(sp[0]) == oracle.select_s(oracle.norm1(ts[0] * mats[0]), thp)
    # the same s as the batched call reports
    good = [m for b, m in enumerate(mats) if b != 2]
    Q = fm.Packed([torch.from_numpy(m) for m in good], device="cuda")
    tq = T(np.delete(ts, 2))
    _, _, s_call = fm.expm_batched(Q, tq, "R8", precision="fp64")
    s_sel, _ = fm.select_batched(Q, tq, "R8", "expm")
    assert np.array_equal(s_call.cpu().numpy(), s_sel.cpu().numpy())


def test_select_feeds_the_adjoint(fm):
    """ExpmvFn without nsteps takes N from fm_select_batched (the action's own N)."""
    import torch
    A, v, y = wl.grad_batch(batch=3, d=12, seed=41)
    At = T(A).requires_grad_(True)
    vt = T(v).requires_grad_(True)
    w = fm.ExpmvFn.apply(At, vt)
    for b in range(3):
        w_ref, N, _ = oracle.expmv(A[b], v[b], 1.0, "R8")
        assert relerr(w[b].detach().cpu().numpy(), w_ref) <= TOL_FP64
    ((w - T(y)) ** 2).sum().backward()
    assert torch.isfinite(At.grad).all() and torch.isfinite(vt.grad).all()


@pytest.mark.parametrize("prec,path", [("fp64", "cta"), ("mixed", "cta"), ("mixed", "grid")])
def test_bad_order_is_reported_per_matrix(fm, prec, path):
    """d_dev[b] outside [1, dmax]: info -4 for that matrix only, the others
    exact as usual, its output untouched."""
    import torch
    dims = [64, 70, 80]
    mats = [wl.dense_scaled(d, 2.0, 300 + i, scale_sqrt=True) for i, d in enumerate(dims)]
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    P.d_dev[1] = 5000  # beyond dmax: left out
    F = torch.full_like(P.flat, 7.0)
    F, info, s = fm.expm_batched(P, 1.0, "R8", precision=prec, path=path, out=F)
    info = info.cpu().numpy()
    assert info[1] == -4 and info[0] == 0 and info[2] == 0
    assert bool((P.get(F, 1) == 7.0).all())
    for b in (0, 2):
        ref, _, _ = oracle.expm(mats[b], 1.0, "R8")
        assert relerr(P.get(F, b).cpu().numpy(), ref) <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp32_ir", "bf16_ir"])
def test_explicit_precision_values(fm, prec):
    """FM_FP32_IR runs the one-CTA kernels, FM_BF16_IR the grid path; both
    reach the oracle at 1e-12."""
    A = wl.dense_scaled(96, 4.0, 51)
    F_ref, s_ref, _ = oracle.expm(A, 1.0, "R8")
    F, info, s = fm.expm(T(A), 1.0, "R8", precision=prec)
    assert info == 0 and s == s_ref
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64
    st = fm.last_stats()
    assert (st["products"] > 0) == (prec == "bf16_ir")  # the grid path counts its products


def test_two_streams_library_scratch(fm):
    """Two batched calls queued on two streams at once, each with the library's
    own scratch (one buffer per stream), give the results of the same calls
    made one at a time."""
    import torch
    dims = [40, 64, 96]
    sets = []
    for k in range(2):
        mats = [wl.dense_scaled(d, 1.0 + 2 * k + i, 500 + 10 * k + i, scale_sqrt=True)
                for i, d in enumerate(dims)]
        sets.append(fm.Packed([torch.from_numpy(m) for m in mats], device="cuda"))
    ref = []
    for P in sets:
        F, info, _ = fm.expm_batched(P, 1.0, "R8", precision="fp64")
        torch.cuda.synchronize()
        ref.append(F.clone())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for rep in range(3):
        outs = []
        for P, st in zip(sets, streams):
            with torch.cuda.stream(st):
                F, info, _ = fm.expm_batched(P, 1.0, "R8", precision="fp64")
                outs.append((F, info))
        torch.cuda.synchronize()
        for (F, info), R in zip(outs, ref):
            assert int((info != 0).sum()) == 0
            assert torch.equal(F, R)
