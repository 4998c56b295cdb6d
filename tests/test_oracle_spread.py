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
