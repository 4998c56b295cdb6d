"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Both sides get the same seeded inputs (paper_2210_03714_gb300.workloads) and
the same coefficient values (the oracle's exact sets rounded to double).  The
bar: relative Frobenius error <= 1e-12 per result for both precision modes
(the mixed mode refines to double accuracy).
"""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, diffusion_bar, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module")
def fm():
    torch = need_gpu()
    import paper_2210_03714_gb300 as fm_
    fm_.lib()
    return fm_


def T(x, dtype=None):
    import torch
    x = np.ascontiguousarray(x)
    if dtype is None:
        dtype = torch.complex128 if np.iscomplexobj(x) else torch.float64
    return torch.tensor(x, dtype=dtype, device="cuda")


# ---------------------------------------------------------------------------
# the single d = 64 problem (R4, k = 4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_single_d64_expm_r4(fm, prec):
    A, v = wl.single_d64()
    cs = oracle_set("R4")
    F_ref, s_ref, info_ref = oracle.expm(A, 1.0, cs)
    F, info, s = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision=prec)
    assert info == 0 and s == s_ref == 10
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


@pytest.mark.parametrize("prec", PRECS)
def test_single_d64_expmv_r4(fm, prec):
    A, v = wl.single_d64()
    cs = oracle_set("R4")
    W_ref, N_ref, _ = oracle.expmv(A, v, 1.0, cs)
    W, info, N = fm.expmv(T(A), T(v), 1.0, fm.Coeffs(cs), precision=prec)
    assert info == 0 and N == N_ref
    assert relerr(W.cpu().numpy(), W_ref) <= TOL_FP64


def test_builtin_coeffs_match(fm):
    """The library's built-in R8 against the oracle's own exact set."""
    A, _ = wl.single_d64(5)
    F_ref, _, _ = oracle.expm(A, 1.0, "R8")
    F, info, _ = fm.expm(T(A), 1.0, "R8")
    assert info == 0 and relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


# ---------------------------------------------------------------------------
# batches: ragged orders spanning several tiles, and edge sizes
# ---------------------------------------------------------------------------

RAGGED = [1, 2, 5, 16, 17, 31, 48, 63, 64, 65, 100, 129, 200, 256]


# the double form runs one CTA per matrix; the mixed form on both paths
# (automatic selection takes the grid path for these batches)
PREC_PATH = [("fp64", "auto"), ("mixed", "cta"), ("mixed", "auto")]


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_batched_expm_ragged(fm, prec, path):
    rng = np.random.default_rng(7)
    norms = rng.uniform(0.5, 8.0, len(RAGGED))
    mats = [wl.dense_scaled(d, n, 100 + i, scale_sqrt=True) for i, (d, n) in enumerate(zip(RAGGED, norms))]
    ts = rng.uniform(0.5, 1.5, len(RAGGED))
    cs = oracle_set("R8")
    P = fm.Packed([T(m) for m in mats])
    F, info, s = fm.expm_batched(P, T(ts), fm.Coeffs(cs), precision=prec, path=path)
    F = F.cpu().numpy()
    info, s = info.cpu().numpy(), s.cpu().numpy()
    for b, (M, t) in enumerate(zip(mats, ts)):
        ref, s_ref, _ = oracle.expm(M, t, cs)
        assert info[b] == 0 and s[b] == s_ref
        assert relerr(P.get(F, b), ref) <= TOL_FP64, (b, RAGGED[b])


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_batched_expm_mixed_d_full_size_sampled(fm, prec, path):
    """The 4096-matrix batch (d uniform over {16..256}, ||A||_1 in [0.5, 8], R8)
    in the launch configuration the benchmark times; 16 sampled results are
    recomputed by the oracle one by one; every status must be 0."""
    import torch
    dims, mats, norms = wl.batch_mixed_d(4096)
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    F, info, s = fm.expm_batched(P, 1.0, "R8", precision=prec, path=path)
    torch.cuda.synchronize()
    assert int((info != 0).sum().item()) == 0
    s = s.cpu().numpy()
    rng = np.random.default_rng(11)
    pick = list(rng.choice(4096, 14, replace=False)) + [int(np.argmax(dims)), int(np.argmin(dims))]
    for b in pick:
        ref, s_ref, _ = oracle.expm(mats[b], 1.0, "R8")
        got = P.get(F, b).cpu().numpy()
        assert s[b] == s_ref
        assert relerr(got, ref) <= TOL_FP64, (b, dims[b])


@pytest.mark.parametrize("prec", PRECS)
def test_phi1_small(fm, prec):
    A = wl.dense_scaled(40, 3.0, 21)
    ce, cp = oracle_set("R8"), oracle_set("R8_phi1")
    Phi_ref, E_ref, s_ref, _ = oracle.phi1(A, 0.7, ce, cp)
    Phi, E, info, s = fm.phi1(T(A), 0.7, fm.Coeffs(ce), fm.Coeffs(cp), precision=prec)
    assert info == 0 and s == s_ref
    assert relerr(Phi.cpu().numpy(), Phi_ref) <= TOL_FP64
    assert relerr(E.cpu().numpy(), E_ref) <= TOL_FP64


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_phi1_diffusion_sampled(fm, prec, path):
    """A = -L + 0.1 N (d = 512, stiff; s = 11..17 doublings): phi1(tA) and
    exp(tA) for a batch of 16 of the 512-matrix workload, two results against
    the oracle.  The s doublings amplify rounding in any double evaluation:
    two correct double evaluations by the oracle itself (the matrix and its
    permuted copy) differ by 7e-13 .. 2.9e-11 for s = 11 .. 17.  The bar is
    twice that measured spread at the result's s (diffusion_bar)."""
    import torch
    mats, ts, u0, bb = wl.diffusion_batch(batch=16)
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    Phi, E, info, s = fm.phi1_batched(P, T(ts), "R8", "R8_phi1", precision=prec, path=path)
    assert int((info != 0).sum().item()) == 0
    s = s.cpu().numpy()
    for b in (0, 7):
        Phi_ref, E_ref, s_ref, _ = oracle.phi1(mats[b], ts[b], "R8", "R8_phi1")
        assert s[b] == s_ref
        assert relerr(P.get(Phi, b).cpu().numpy(), Phi_ref) <= diffusion_bar(s_ref, "phi1")
        assert relerr(P.get(E, b).cpu().numpy(), E_ref) <= diffusion_bar(s_ref, "exp")


@pytest.mark.parametrize("prec", PRECS)
def test_phi1_diffusion_full_batch(fm, prec):
    """The full diffusion workload: 512 matrices of order 512 in one call;
    every status 0, three results (first, middle, last) against the oracle
    (same s, the bar of the sampled test: twice the measured spread of two
    correct double evaluations at that s)."""
    import torch
    mats, ts, u0, bb = wl.diffusion_batch(batch=512)
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    Phi, E, info, s = fm.phi1_batched(P, T(ts), "R8", "R8_phi1", precision=prec)
    torch.cuda.synchronize()
    assert int((info != 0).sum().item()) == 0
    s = s.cpu().numpy()
    assert 11 <= s.min() and s.max() <= 17  # the doublings this workload needs
    for b in (0, 255, 511):
        Phi_ref, E_ref, s_ref, _ = oracle.phi1(mats[b], ts[b], "R8", "R8_phi1")
        assert s[b] == s_ref
        assert relerr(P.get(Phi, b).cpu().numpy(), Phi_ref) <= diffusion_bar(s_ref, "phi1")
        assert relerr(P.get(E, b).cpu().numpy(), E_ref) <= diffusion_bar(s_ref, "exp")


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_phi1mv_diffusion_sampled(fm, prec, path):
    """u(t) = u0 + t phi1(tA)(A u0 + b) for the same workload.  The product
    phi1(tA) w with w = A u0 + b (dominated by the stiff modes that phi1
    damps) has condition kappa = ||phi1|| ||w|| / ||phi1 w||; errors are
    reported on w and u, with the bar of the matrix test times kappa, and for
    u also times ||t phi1 w|| / ||u|| (the sum u0 + t phi1 w cancels)."""
    import torch
    mats, ts, u0, bb = wl.diffusion_batch(batch=16)
    rhs = np.stack([M @ u + b for M, u, b in zip(mats, u0, bb)])
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    W, info, s = fm.phi1mv_batched(P, T(rhs.ravel()), 1, T(ts), "R8", "R8_phi1", precision=prec,
                                   path=path)
    assert int((info != 0).sum().item()) == 0
    W = W.cpu().numpy().reshape(16, 512)
    s = s.cpu().numpy()
    for b in (0, 7):
        Phi_ref, _, s_ref, _ = oracle.phi1(mats[b], ts[b], "R8", "R8_phi1")
        w_ref = Phi_ref @ rhs[b]
        assert s[b] == s_ref
        kappa = np.linalg.norm(Phi_ref, 2) * np.linalg.norm(rhs[b]) / np.linalg.norm(w_ref)
        tol = diffusion_bar(s_ref, "phi1") * kappa
        assert relerr(W[b], w_ref) <= tol
        u = u0[b] + ts[b] * W[b]
        u_ref = u0[b] + ts[b] * w_ref
        amp = ts[b] * np.linalg.norm(w_ref) / np.linalg.norm(u_ref)
        assert relerr(u, u_ref) <= tol * max(1.0, amp)


@pytest.mark.parametrize("prec", PRECS)
def test_expmv_block_and_batched(fm, prec):
    cs = oracle_set("R8")
    A = wl.dense_scaled(48, 4.0, 31)
    V = np.random.default_rng(32).standard_normal((48, 8))
    W_ref, N_ref, _ = oracle.expmv(A, V, 1.0, cs)
    W, info, N = fm.expmv(T(A), T(V), 1.0, fm.Coeffs(cs), precision=prec)
    assert info == 0 and N == N_ref and relerr(W.cpu().numpy(), W_ref) <= TOL_FP64
    dims = [7, 33, 64, 90]
    mats = [wl.dense_scaled(d, 2.0, 40 + d, scale_sqrt=True) for d in dims]
    m = 3
    Vs = [np.random.default_rng(50 + d).standard_normal((d, m)) for d in dims]
    P = fm.Packed([T(x) for x in mats])
    Wb, info, Ns = fm.expmv_batched(P, T(np.concatenate([v.ravel() for v in Vs])), m, 0.8,
                                    fm.Coeffs(cs), precision=prec)
    Wb = Wb.cpu().numpy()
    o = 0
    for b, d in enumerate(dims):
        ref, N_ref, _ = oracle.expmv(mats[b], Vs[b], 0.8, cs)
        assert int(Ns[b]) == N_ref
        assert relerr(Wb[o:o + d * m].reshape(d, m), ref) <= TOL_FP64
        o += d * m


@pytest.mark.parametrize("prec", PRECS)
def test_zexpm_hermitian(fm, prec):
    d = 48
    g = np.random.default_rng(60)
    G = (g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))) / np.sqrt(d)
    H = (G + G.conj().T) / 2
    A = -1j * H * (6.0 / np.abs(np.linalg.eigvalsh(H)).max())
    cs = oracle_set("R8")
    F_ref, s_ref, _ = oracle.zexpm(A, 1.0, cs)
    F, info, s = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision=prec)
    assert info == 0 and s == s_ref
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


@pytest.mark.parametrize("prec", PRECS)
def test_zexpmv_hermitian_block(fm, prec):
    A, V, rho = wl.hermitian_action(d=64, m=6, rho=20.0, seed=61)
    cs = oracle_set("R8")
    W_ref, N_ref, _ = oracle.zexpmv(A, V, 1.0, cs, anorm=rho)
    W, info, N = fm.expmv(T(A), T(V), 1.0, fm.Coeffs(cs), precision=prec, anorm=rho)
    assert info == 0 and N == N_ref
    assert relerr(W.cpu().numpy(), W_ref) <= TOL_FP64


def test_adjoint_vs_oracle(fm):
    """Gradient of L = ||exp(A)v - y||^2 (N fixed) against the oracle's
    gradient at 1e-8 relative, for a d = 128 batch of 3."""
    import torch
    A, v, y = wl.grad_batch(batch=3)
    Ns = [oracle.select_nsteps(np.abs(a).sum(0).max(), oracle.CS("R8").theta) for a in A]
    cs = oracle_set("R8")
    P = fm.Packed([T(a) for a in A])
    w_fwd = []
    for b in range(3):
        w, N, _ = oracle.expmv(A[b], v[b], 1.0, cs, nsteps=Ns[b])
        w_fwd.append(w)
    wbar = np.concatenate([2 * (w - yy) for w, yy in zip(w_fwd, y)])
    W, Abar, vbar, info = fm.expmv_adjoint_batched(P, T(v.ravel()), T(wbar), Ns, 1.0,
                                                   fm.Coeffs(cs))
    assert int((info != 0).sum().item()) == 0
    W, Abar, vbar = W.cpu().numpy(), Abar.cpu().numpy(), vbar.cpu().numpy()
    for b in range(3):
        Ab_ref, vb_ref, _ = oracle.expmv_adjoint(A[b], v[b], wbar[b * 128:(b + 1) * 128], Ns[b],
                                                  1.0, cs)
        assert relerr(W[b * 128:(b + 1) * 128], w_fwd[b]) <= TOL_FP64
        assert relerr(Abar[b * 128 * 128:(b + 1) * 128 * 128].reshape(128, 128), Ab_ref) <= 1e-8
        assert relerr(vbar[b * 128:(b + 1) * 128], vb_ref) <= 1e-8


def test_adjoint_full_batch(fm):
    """The full gradient workload: 256 matrices of order 128 (N from each
    matrix's norm), forward action and adjoint in one call each; three
    results against the oracle (forward at 1e-12, gradients at 1e-8)."""
    import torch
    A, v, y = wl.grad_batch(batch=256)
    theta = oracle.CS("R8").theta
    Ns = [oracle.select_nsteps(np.abs(a).sum(0).max(), theta) for a in A]
    cs = oracle_set("R8")
    P = fm.Packed([T(a) for a in A])
    W0, info0, N0 = fm.expmv_batched(P, T(v.ravel()), 1, 1.0, fm.Coeffs(cs), precision="fp64")
    assert int((info0 != 0).sum().item()) == 0
    assert [int(x) for x in N0.cpu().numpy()] == Ns
    W0 = W0.cpu().numpy()
    wbar = 2 * (W0 - y.ravel())
    W, Abar, vbar, info = fm.expmv_adjoint_batched(P, T(v.ravel()), T(wbar), Ns, 1.0,
                                                   fm.Coeffs(cs))
    torch.cuda.synchronize()
    assert int((info != 0).sum().item()) == 0
    W, Abar, vbar = W.cpu().numpy(), Abar.cpu().numpy(), vbar.cpu().numpy()
    d = 128
    for b in (0, 128, 255):
        w_ref, N_ref, _ = oracle.expmv(A[b], v[b], 1.0, cs, nsteps=Ns[b])
        assert relerr(W[b * d:(b + 1) * d], w_ref) <= TOL_FP64
        Ab_ref, vb_ref, _ = oracle.expmv_adjoint(A[b], v[b], wbar[b * d:(b + 1) * d], Ns[b], 1.0, cs)
        assert relerr(Abar[b * d * d:(b + 1) * d * d].reshape(d, d), Ab_ref) <= 1e-8
        assert relerr(vbar[b * d:(b + 1) * d], vb_ref) <= 1e-8


def test_autograd_function_fd(fm):
    """ExpmvFn backward against central differences of its own forward."""
    import torch
    A, v, y = wl.grad_batch(batch=2, d=16, seed=4100)
    Ns = [oracle.select_nsteps(np.abs(a).sum(0).max(), oracle.CS("R8").theta) for a in A]
    At = T(A).requires_grad_(True)
    vt = T(v).requires_grad_(True)
    yt = T(y)
    w = fm.ExpmvFn.apply(At, vt, Ns)
    L = ((w - yt) ** 2).sum()
    L.backward()
    dA = torch.tensor(np.random.default_rng(5).standard_normal(A.shape), device="cuda")
    dv = torch.tensor(np.random.default_rng(6).standard_normal(v.shape), device="cuda")
    h = 1e-5
    with torch.no_grad():
        Lp = ((fm.ExpmvFn.apply(At + h * dA, vt + h * dv, Ns) - yt) ** 2).sum()
        Lm = ((fm.ExpmvFn.apply(At - h * dA, vt - h * dv, Ns) - yt) ** 2).sum()
    fd = float((Lp - Lm) / (2 * h))
    an = float((At.grad * dA).sum() + (vt.grad * dv).sum())
    assert abs(fd - an) <= 2e-7 * max(1.0, abs(an))


def test_autograd_function_fd_d128(fm):
    """The same central-difference check on the gradient workload's own order
    (d = 128, N from the norm, two matrices), in two random directions."""
    import torch
    A, v, y = wl.grad_batch(batch=2, d=128, seed=4200)
    Ns = [oracle.select_nsteps(np.abs(a).sum(0).max(), oracle.CS("R8").theta) for a in A]
    At = T(A).requires_grad_(True)
    vt = T(v).requires_grad_(True)
    yt = T(y)
    L = ((fm.ExpmvFn.apply(At, vt, Ns) - yt) ** 2).sum()
    L.backward()
    h = 1e-5
    for seed in (7, 8):
        g = np.random.default_rng(seed)
        dA = torch.tensor(g.standard_normal(A.shape), device="cuda")
        dv = torch.tensor(g.standard_normal(v.shape), device="cuda")
        with torch.no_grad():
            Lp = ((fm.ExpmvFn.apply(At + h * dA, vt + h * dv, Ns) - yt) ** 2).sum()
            Lm = ((fm.ExpmvFn.apply(At - h * dA, vt - h * dv, Ns) - yt) ** 2).sum()
        fd = float((Lp - Lm) / (2 * h))
        an = float((At.grad * dA).sum() + (vt.grad * dv).sum())
        assert abs(fd - an) <= 2e-7 * max(1.0, abs(an)), (seed, fd, an)


def test_autograd_fp32_forward(fm):
    """The gradient workload with the forward action in single-precision
    factors plus refinement: the forward result against the oracle at 1e-12,
    the gradients (the double adjoint with the forward's N) equal to those of
    the double forward, and against the oracle's at 1e-8."""
    import torch
    A, v, y = wl.grad_batch(batch=4, d=128, seed=4300)
    Ns = [oracle.select_nsteps(np.abs(a).sum(0).max(), oracle.CS("R8").theta) for a in A]
    grads = []
    for prec in ("fp32_ir", "fp64"):
        At = T(A).requires_grad_(True)
        vt = T(v).requires_grad_(True)
        w = fm.ExpmvFn.apply(At, vt, None, 1.0, "R8", prec)
        for b in range(len(A)):
            W_ref, N_ref, _ = oracle.expmv(A[b], v[b], 1.0, "R8")
            assert N_ref == Ns[b]
            assert relerr(w[b].detach().cpu().numpy(), W_ref) <= TOL_FP64
        ((w - T(y)) ** 2).sum().backward()
        grads.append((At.grad.cpu().numpy(), vt.grad.cpu().numpy()))
    for g1, g2 in zip(grads[0], grads[1]):
        assert relerr(g1, g2) <= 1e-10
    for b in range(len(A)):
        W_ref, _, _ = oracle.expmv(A[b], v[b], 1.0, "R8")
        wbar = 2 * (W_ref - y[b])
        Ab_ref, vb_ref, _ = oracle.expmv_adjoint(A[b], v[b], wbar, Ns[b], 1.0, "R8")
        assert relerr(grads[0][0][b], Ab_ref) <= 1e-8
        assert relerr(grads[0][1][b], vb_ref) <= 1e-8


# ---------------------------------------------------------------------------
# status codes and degenerate cases
# ---------------------------------------------------------------------------

def test_status_codes(fm):
    import torch
    # non-finite input
    A = np.eye(5)
    A[2, 3] = np.nan
    _, info, _ = fm.expm(T(A), 1.0, "R8")
    assert info == -2
    # zero pivot: a caller bound that understates ||A|| (s = 0) puts an
    # eigenvalue of B at 1/c for the pair c = +-2/15 (terms 3 and 4), solved
    # as one system I - c^2 B^2: fl(c^2) * 7.5^2 rounds to exactly 1
    c = 0.13333333333333333
    assert (c * c) * (7.5 * 7.5) == 1.0
    A = np.diag([7.5, 0.1, 0.2])
    _, info, _ = fm.expm(T(A), 1.0, "R8", anorm=1e-3, precision="fp64")
    assert info == 3 * 3 + 1
    # single-precision factors with refinement switched off and a tolerance
    # set: flagged as not converged
    A = wl.dense_scaled(20, 2.0, 3)
    _, info, _ = fm.expm(T(A), 1.0, "R8", precision="fp32_ir", max_ir_iters=0, ir_tol=1e-12)
    assert info == -1
    # d = 1: the scalar approximant, against the oracle and exp within the
    # round-off bound of the roundoff form: 2^s times (sum_i |b_i c_i| theta + 1) u
    # per evaluation (Sec. 4.3), with a factor 2 of slack.  The kernels solve
    # each +-c pair as one system (Sec. 1), a different rounding order than the
    # oracle's per-node terms, so the two agree to that bound, not to 1 ulp.
    F, info, s = fm.expm(T(np.array([[0.3]])), 1.0, "R8")
    ref, s_ref, _ = oracle.expm(np.array([[0.3]]), 1.0, "R8")
    cancel = sum(abs(b * c) for b, c in zip(oracle_set("R8")["b_re"], oracle_set("R8")["c_re"]))
    bound = 2 ** s * (cancel * oracle_set("R8")["theta"] + 1) * 2 * 2.0 ** -53
    assert info == 0 and s == s_ref and abs(F.item() - ref[0, 0]) <= bound
    assert abs(F.item() - np.exp(0.3)) < bound
    # the zero matrix
    F, info, s = fm.expm(T(np.zeros((9, 9))), 1.0, "R8")
    assert info == 0 and s == 0 and float((F - torch.eye(9, dtype=torch.float64, device="cuda")).abs().max()) == 0
    # a bad order inside a batch is reported per matrix and skipped
    P = fm.Packed([T(np.eye(3)), T(np.eye(4))])
    P.d_dev[1] = 5000
    P.dmax = 4
    F, info, s = fm.expm_batched(P, 1.0, "R8")
    assert info.cpu().tolist() == [0, -4]
    # argument errors raise
    with pytest.raises(fm.FmError):
        fm.expm(T(np.eye(3)), 1.0, {"c_re": [0.1], "b_re": [1.0], "a0": 1.0, "theta": -1.0,
                                    "conj_pair": 2})


def test_invariant_full_size(fm):
    """e^{A} e^{-A} = I for the largest orders of the batch workload."""
    import torch
    for d in (256, 512):
        A = wl.dense_scaled(d, 8.0, 70 + d, scale_sqrt=True)
        E1, i1, _ = fm.expm(T(A), 1.0, "R8")
        E2, i2, _ = fm.expm(T(A), -1.0, "R8")
        assert i1 == 0 and i2 == 0
        err = float((E1 @ E2 - torch.eye(d, dtype=torch.float64, device="cuda")).abs().max())
        assert err < 1e-11
