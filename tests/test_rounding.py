"""The one rounding of each exact product sum (hi 2^24 + lo) 2^e2 to double,
as the tile kernels' epilogues do it with 64-bit integer operations
(round_hl), checked on the host against exact rational arithmetic: Python's
float(Fraction) rounds to nearest, ties to even.  Cases: random sums of
either sign over the whole range the exact sums take (|hi|, |lo| < 2^62),
exact ties, values just above and below a tie, lo carrying into hi and
borrowing from it, and the 63-bit boundary where the routine switches to a
sticky bit.  Results stay in the normal range (the routine truncates
subnormal results, which no product here reaches)."""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def exact(hi, lo, e2):
    v = Fraction(hi * (1 << 24) + lo) * (Fraction(2) ** e2)
    return struct.unpack("<Q", struct.pack("<d", float(v)))[0]


def cases():
    rng = random.Random(20261204)
    out = []
    for _ in range(20000):
        hi = rng.randrange(-(1 << 62) + 1, 1 << 62)
        lo = rng.randrange(-(1 << 62) + 1, 1 << 62)
        out.append((hi, lo, rng.randrange(-160, -40)))
    for _ in range(5000):  # small sums: no sticky bit, fewer than 53 bits
        out.append((rng.randrange(-(1 << 20), 1 << 20), rng.randrange(-(1 << 40), 1 << 40),
                    rng.randrange(-120, -20)))
    for _ in range(5000):  # exact ties and their neighbours at random bit lengths
        nb = rng.randrange(55, 86)
        m = rng.randrange(1 << 52, 1 << 53)
        sh = nb - 53
        base = m << sh
        for dv in (-1, 0, 1):
            v = base + (1 << (sh - 1)) + dv
            v = -v if rng.random() < 0.5 else v
            hi, lo = divmod(v, 1 << 24)
            if rng.random() < 0.5:  # the same value with lo carrying into hi
                hi, lo = hi - 1, lo + (1 << 24)
            out.append((hi, lo, rng.randrange(-150, -60)))
    for k in range(-3, 4):  # around the 63-bit switch to a sticky bit
        for s in (1, -1):
            v = s * ((1 << 63) + k)
            hi, lo = divmod(v, 1 << 24)
            out.append((hi, lo, -70))
    return out


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("round") / "rounding_harness")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                           os.path.join(HERE, "rounding_harness.cu"), "-o", exe])
    return exe


def test_round_hl_matches_exact_rounding(harness):
    cs = cases()
    inp = "".join("%d %d %d\n" % c for c in cs)
    res = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True)
    got = [int(x, 16) for x in res.stdout.split()]
    assert len(got) == len(cs)
    bad = [(c, hex(g), hex(exact(*c))) for c, g in zip(cs, got) if g != exact(*c)]
    assert not bad, bad[:5]
