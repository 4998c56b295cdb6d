"""Writes tests/golden/hermitian_d4096.npz: the CPU oracle's action
exp(tA) V on a few columns of the complex Hermitian workload at full size.

A = -iH, H = (G + G^H)/2 with G complex N(0,1)/sqrt(d), d = 4096, scaled to
spectral radius 20; V complex N(0,1), 4096 x 256 (workloads.hermitian_action,
seed 2000); t = 1; coefficient set R8 (Eq. Frac8ci/Frac8bi); roundoff form
(Eq. ParallRoundOff).  The action of Sec. 1 acts on each column of V on its
own, so the oracle runs on the stored columns only.  Three runs:
  - anorm = 20 (N = ceil(20 / theta) = 206, the full workload);
  - N = 16 forced (a short chain; spectral radius 20/16 of B keeps the shifted
    systems well inside the region where the grid path's correction
    iteration converges);
  - both again on the permuted copy P A P^T (and P V): r(P B P^T)^N P V =
    P r(B)^N V, so mapping it back gives a second correct double evaluation
    that rounds in another order; the largest relative distance per column
    between the two is stored as the spread of two correct double
    evaluations (spread_full, spread_n16).  At N = 16 the step matrix B has
    spectral radius 1.25, far outside the set's theta, so r(B) is not close
    to exp(B) and its shifted systems are less well conditioned: its spread
    is larger than at N = 206.

Only oracle/ and the seeded input generator are called.  The result also
records the scale that gives H spectral radius 20 (so a test rebuilds A bit
for bit without an eigenvalue routine, whose last bits differ between
machines) and checks of the inputs (Frobenius norm of A, the selected columns
of V).  Run from the repository root: python tests/golden/make_hermitian_golden.py
(about fifteen minutes of CPU per run; the four run in parallel processes)."""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

D, M, RHO, SEED = 4096, 256, 20.0, 2000
COLS = [0, 128, 255]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hermitian_d4096.npz")


PERM_SEED = 5


def _run(args):
    nsteps, scale, permute = args
    import oracle
    from paper_2210_03714_gb300 import workloads as wl
    A, V, rho = wl.hermitian_action(d=D, m=M, rho=RHO, seed=SEED, scale=scale)
    Vc = V[:, COLS].copy()
    anorm_f = float(np.linalg.norm(A))
    if permute:
        p = np.random.default_rng(PERM_SEED).permutation(D)
        A = A[np.ix_(p, p)]
        Vc = Vc[p]
    W, N, info = oracle.zexpmv(A, Vc, 1.0, "R8", oracle.ROUNDOFF, anorm=rho, nsteps=nsteps)
    assert info == 0, info
    if permute:
        W = W[np.argsort(p)]
        Vc = Vc[np.argsort(p)]
    return nsteps, permute, W, N, anorm_f, Vc


def main():
    from paper_2210_03714_gb300 import workloads as wl
    H, _ = wl.hermitian_parts(D, M, SEED)
    scale = wl.hermitian_scale(H, RHO)
    del H
    ctx = mp.get_context("spawn")
    with ctx.Pool(4) as pool:
        res = pool.map(_run, [(0, scale, False), (16, scale, False), (0, scale, True),
                              (16, scale, True)])
    out = {"cols": np.array(COLS), "seed": SEED, "d": D, "m": M, "rho": RHO, "scale": scale}
    perm = {}
    for nsteps, permute, W, N, anorm_f, Vc in res:
        key = "full" if nsteps == 0 else "n16"
        if permute:
            perm[key] = W
            continue
        out["W_" + key] = W
        out["N_" + key] = N
        out["A_fro"] = anorm_f
        out["V_cols"] = Vc
    for key in ("full", "n16"):
        W, Wp = out["W_" + key], perm[key]
        out["spread_" + key] = max(float(np.linalg.norm(W[:, j] - Wp[:, j]) / np.linalg.norm(W[:, j]))
                                   for j in range(len(COLS)))
    np.savez(OUT, **out)
    print("wrote", OUT, {k: np.shape(v) for k, v in out.items()})


if __name__ == "__main__":
    main()
