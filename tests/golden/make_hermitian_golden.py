"""Writes tests/golden/hermitian_d4096.npz: the CPU oracle's action
exp(tA) V on a few columns of the complex Hermitian workload at full size.

A = -iH, H = (G + G^H)/2 with G complex N(0,1)/sqrt(d), d = 4096, scaled to
spectral radius 20; V complex N(0,1), 4096 x 256 (workloads.hermitian_action,
seed 2000); t = 1; coefficient set R8 (Eq. Frac8ci/Frac8bi); roundoff form
(Eq. ParallRoundOff).  The action of Sec. 1 acts on each column of V on its
own, so the oracle runs on the stored columns only.  Two step counts:
anorm = 20 (N = ceil(20 / theta) = 206, the full workload) and N = 4.

Only oracle/ and the seeded input generator are called.  The result also
records the scale that gives H spectral radius 20 (so a test rebuilds A bit
for bit without an eigenvalue routine, whose last bits differ between
machines) and checks of the inputs (Frobenius norm of A, the selected columns
of V).  Run from the
repository root: python tests/golden/make_hermitian_golden.py  (about ten
minutes of CPU per step count; both run in parallel processes)."""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

D, M, RHO, SEED = 4096, 256, 20.0, 2000
COLS = [0, 128, 255]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hermitian_d4096.npz")


def _run(args):
    nsteps, scale = args
    import oracle
    from paper_2210_03714_gb300 import workloads as wl
    A, V, rho = wl.hermitian_action(d=D, m=M, rho=RHO, seed=SEED, scale=scale)
    W, N, info = oracle.zexpmv(A, V[:, COLS], 1.0, "R8", oracle.ROUNDOFF, anorm=rho,
                               nsteps=nsteps)
    assert info == 0, info
    return nsteps, W, N, float(np.linalg.norm(A)), V[:, COLS].copy()


def main():
    from paper_2210_03714_gb300 import workloads as wl
    H, _ = wl.hermitian_parts(D, M, SEED)
    scale = wl.hermitian_scale(H, RHO)
    del H
    ctx = mp.get_context("spawn")
    with ctx.Pool(2) as pool:
        res = pool.map(_run, [(0, scale), (4, scale)])
    out = {"cols": np.array(COLS), "seed": SEED, "d": D, "m": M, "rho": RHO, "scale": scale}
    for nsteps, W, N, anorm_f, Vc in res:
        key = "full" if nsteps == 0 else "n4"
        out["W_" + key] = W
        out["N_" + key] = N
        out["A_fro"] = anorm_f
        out["V_cols"] = Vc
    np.savez(OUT, **out)
    print("wrote", OUT, {k: np.shape(v) for k, v in out.items()})


if __name__ == "__main__":
    main()
