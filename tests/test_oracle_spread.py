"""How far two correct double evaluations of the stiff phi_1 workload differ
(no GPU).  The GPU bar for that workload rests on tests/golden/diffusion_spread.txt,
written by make_diffusion_spread.py from the oracle alone; this test
re-measures one entry and checks the table's shape.

f(P A P^T) = P f(A) P^T for a permutation P, so the oracle on the permuted copy
is a second correct double evaluation whose every dot product and elimination
step rounds in another order (Sec. 1's doublings phi1(2X) = (e^X + I) phi1(X)/2
then amplify the difference)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_diffusion_spread as mds  # noqa: E402
from _common import _spread_table, diffusion_bar, TOL_FP64  # noqa: E402

U = 2.0 ** -53


def test_table_covers_the_workload():
    rows = _spread_table()
    assert sorted(rows) == list(range(11, 18))  # the s this workload reaches
    for s, (b, sp, se) in rows.items():
        # a double evaluation after s doublings carries about 2^s u of rounding:
        # the measured spread sits between 2^(s-1) u and 2^(s+3) u
        assert 2.0 ** (s - 1) * U <= sp <= 2.0 ** (s + 3) * U, s
        assert 2.0 ** (s - 1) * U <= se <= 2.0 ** (s + 3) * U, s
    # at s = 17 two correct double evaluations already differ by more than 1e-12
    assert rows[17][2] > 10 * TOL_FP64
    assert diffusion_bar(17, "exp") == 2.0 * rows[17][2]


def test_remeasure_one_entry():
    """s = 11 (the cheapest), the first of the two permutations: the same
    distances as the stored table's (which keeps the larger of the two)."""
    from paper_2210_03714_gb300 import workloads as wl
    rows = _spread_table()
    b = rows[11][0]
    mats, ts, _, _ = wl.diffusion_batch(batch=512)
    s, sp, se = mds.spread(mats[b], ts[b], mds.PERM_SEEDS[0])
    assert s == 11
    assert sp <= rows[11][1] * 1.05 and se <= rows[11][2] * 1.05
    assert max(sp, se) >= 0.5 * max(rows[11][1], rows[11][2])


def test_hermitian_action_spread():
    """The full-size Hermitian action (N = 206 steps): the spread of two correct
    double evaluations stored with the oracle's result (the oracle on A and on
    P A P^T, d = 4096) against one re-measured here at d = 256.  Rounding of the
    roundoff form accumulates over the N steps (about N u (sum_i |b_i c_i| theta
    + 1) at most) and grows with the length d of the dot products; the stored
    spread must lie between the d = 256 one and 8 times it (at most the sqrt(d)
    growth of random rounding, times 2), and above 1e-12: two correct double
    evaluations at this size do not agree to 1e-12."""
    import numpy as np
    import oracle
    from oracle import coeffs as oc
    from paper_2210_03714_gb300 import workloads as wl
    g = np.load(os.path.join(HERE, "golden", "hermitian_d4096.npz"))
    stored = float(g["spread_full"])
    A, V, rho = wl.hermitian_action(d=256, m=3, rho=20.0, seed=2000)
    W, N, _ = oracle.zexpmv(A, V, 1.0, "R8", anorm=rho)
    p = np.random.default_rng(5).permutation(256)
    W2, N2, _ = oracle.zexpmv(A[np.ix_(p, p)], V[p], 1.0, "R8", anorm=rho)
    W2 = W2[np.argsort(p)]
    assert N == N2 == int(g["N_full"]) == 206
    s256 = max(float(np.linalg.norm(W[:, j] - W2[:, j]) / np.linalg.norm(W[:, j])) for j in range(3))
    cs = oc.oracle_coeffs("R8")
    per_step = sum(abs(b * c) for b, c in zip(cs["b_re"], cs["c_re"])) * cs["theta"] + 1
    assert s256 <= 4 * N * U * per_step
    assert s256 <= stored <= 8 * s256
    assert stored > TOL_FP64
