"""Writes tests/golden/diffusion_spread.txt: how far two correct double
evaluations of phi_1(tA) and exp(tA) differ on the stiff diffusion workload.

Workload: A = -L + 0.1 N, L = trid{-1, 2, -1} / h^2, d = 512
(workloads.diffusion_batch, seed 3000), t log-uniform in [1e-4, 1e-2], sets
R8 and R8_phi1, s = 11..17 doublings of Sec. 1 (phi1(2X) = (e^X + I) phi1(X) / 2).
For each s, the first matrix of the 512-matrix batch with that s is evaluated
by the oracle as given, and again as the permuted copy P A P^T for two seeded
random permutations P; f(P A P^T) = P f(A) P^T, so mapping the second result
back gives a second correct double evaluation that rounds in another order.
The file lists, per s, the largest relative Frobenius distance between the
two evaluations over the two permutations, for phi_1 and for exp.

Only oracle/ and the seeded input generator are called.  Run from the
repository root: python tests/golden/make_diffusion_spread.py  (a few minutes)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "diffusion_spread.txt")
PERM_SEEDS = (1, 2)


def relerr(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def spread(A, t, seed):
    """(s, phi_1 distance, exp distance) between the oracle on A and on P A P^T."""
    import oracle
    Phi, E, s, info = oracle.phi1(A, t, "R8", "R8_phi1")
    assert info == 0
    p = np.random.default_rng(seed).permutation(A.shape[0])
    Phip, Ep, sp, info = oracle.phi1(A[np.ix_(p, p)], t, "R8", "R8_phi1")
    assert info == 0 and sp == s
    q = np.argsort(p)
    return s, relerr(Phip[np.ix_(q, q)], Phi), relerr(Ep[np.ix_(q, q)], E)


def pick(mats, ts):
    """First matrix index for each s the batch reaches."""
    import oracle
    th = min(oracle.CS("R8").theta, oracle.CS("R8_phi1").theta)
    first = {}
    for b, (A, t) in enumerate(zip(mats, ts)):
        s = oracle.select_s(oracle.norm1(t * A), th)
        first.setdefault(s, b)
    return first


def main():
    from paper_2210_03714_gb300 import workloads as wl
    mats, ts, _, _ = wl.diffusion_batch(batch=512)
    rows = []
    for s, b in sorted(pick(mats, ts).items()):
        res = [spread(mats[b], ts[b], seed) for seed in PERM_SEEDS]
        assert all(r[0] == s for r in res)
        rows.append((s, b, max(r[1] for r in res), max(r[2] for r in res)))
        print(rows[-1], flush=True)
    with open(OUT, "w") as f:
        f.write("# s  matrix  phi1_spread  exp_spread   (written by make_diffusion_spread.py)\n")
        for s, b, sp, se in rows:
            f.write("%d %d %.6e %.6e\n" % (s, b, sp, se))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
