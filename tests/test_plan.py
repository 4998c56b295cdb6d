"""The planner of the shifted systems (plan_systems, the host and device
code every dense path runs) built for the host with g++, checked against the
paper's forms with the oracle's exact coefficient sets: the +-c node pairs of
R8 fused into one system I - c^2 B^2 with weights (b+ + b-) and (b+ - b-) c
(Sec. 1: one product x^2 and one inverse per pair of roots), lone nodes
kept, the conjugate-pair term of Eq. (Pade4) as the real system
I - 2 Re(c) B + |c|^2 B^2 with 2 Re(b c) and -2 Re(b) |c|^2 (roundoff form) or
2 Re(b) and -2 Re(b conj(c)) (plain form), the one-product form y, x of every
quadratic system consistent with its right-hand side, and the plain form's
base a0 minus the weights its nodes carry."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import coeffs as oc

HERE = os.path.dirname(os.path.abspath(__file__))
U = 2.0 ** -53
FIELDS = "node quad cr ci u1r u1i u2r u2i wr wi gr gi ar ai br bi yr yi xr xi".split()


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_harness")
    subprocess.check_call([gxx, "-O2", "-std=c++17", os.path.join(HERE, "plan_harness.cpp"),
                           "-o", exe])
    return exe


def plan(exe, name, form, fuse):
    d = oc.oracle_coeffs(name)
    k = len(d["c_re"])
    lines = ["%d %d %d %d" % (form, int(fuse), d["conj_pair"], k)]
    for i in range(k):
        lines.append("%r %r %r %r" % (d["c_re"][i], d["c_im"][i], d["b_re"][i], d["b_im"][i]))
    lines.append("%r" % d["a0"])
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    ns, base = out[0].split()
    systems = []
    for row in out[1:1 + int(ns)]:
        v = row.split()
        systems.append({f: (int(x) if f in ("node", "quad") else float(x)) for f, x in zip(FIELDS, v)})
    return d, float(base), systems


def close(x, ref, scale):
    return abs(x - ref) <= 8 * U * max(abs(scale), abs(ref), 1e-300)


def test_r8_pairs_fused(harness):
    d, base, S = plan(harness, "R8", 0, True)
    cs = oc.SETS["R8"]
    assert len(S) == 4 and all(s["quad"] == 1 for s in S) and base == d["a0"]
    for s in S:
        i = s["node"]
        c = cs.c[i]
        j = cs.c.index(-c)
        bp, bm = float(cs.b[i]), float(cs.b[j])
        cf = float(c)
        assert s["u1r"] == 0.0 and s["u2i"] == 0.0 and close(s["u2r"], cf * cf, cf * cf)
        assert close(s["yr"], bp + bm, abs(bp) + abs(bm))
        assert close(s["xr"], (bp - bm) * cf, (abs(bp) + abs(bm)) * abs(cf))
        assert close(s["ar"], (bp - bm) * cf, (abs(bp) + abs(bm)) * abs(cf))
        assert close(s["br"], (bp + bm) * cf * cf, (abs(bp) + abs(bm)) * cf * cf)


def test_r8_unfused_and_plain(harness):
    cs = oc.SETS["R8"]
    _, base, S = plan(harness, "R8", 0, False)  # one system per nonzero node
    assert len(S) == 8 and all(s["quad"] == 0 for s in S)
    for s in S:
        assert s["cr"] == float(cs.c[s["node"]]) and s["wr"] == float(cs.b[s["node"]])
    d, base, S = plan(harness, "R8", 1, True)  # plain form: no fusion, base = a0 - sum b_i
    assert len(S) == 8 and all(s["quad"] == 0 for s in S)
    ref = float(sum(cs.b)) + float(cs.d[0]) - sum(float(b) for b, c in zip(cs.b, cs.c) if c != 0)
    assert close(base, ref, sum(abs(float(b)) for b in cs.b))


@pytest.mark.parametrize("form", [0, 1])
def test_conjugate_pair_system(harness, form):
    d, base, S = plan(harness, "pade22", form, True)
    assert len(S) == 1 and S[0]["quad"] == 1
    s = S[0]
    c = complex(d["c_re"][0], d["c_im"][0])
    b = complex(d["b_re"][0], d["b_im"][0])
    c2 = abs(c) ** 2
    sc = 4 * (abs(b) * (1 + abs(c)) ** 2)
    assert close(s["u1r"], 2 * c.real, 2 * abs(c)) and close(s["u2r"], -c2, c2)
    if form == 0:
        assert s["gr"] == 0.0
        assert close(s["ar"], 2 * (b * c).real, sc) and close(s["br"], -2 * b.real * c2, sc)
        assert base == d["a0"]
    else:
        assert close(s["gr"], 2 * b.real, sc) and close(s["ar"], -2 * (b * c.conjugate()).real, sc)
        assert s["br"] == 0.0
        assert close(base, d["a0"] - 2 * b.real, sc)
    # the grid paths' form (I + Y)(g I + a B + b B^2) = g I + y Y + x (I + Y) B
    assert close(s["yr"], s["gr"] + s["br"] / s["u2r"], sc / c2)
    assert close(s["xr"], s["ar"] - s["br"] * s["u1r"] / s["u2r"], sc / c2)


def test_quadratic_systems_reproduce_the_set_on_scalars(harness):
    """On scalars x the planned systems give back r(x) - r(0) of Eq.
    (ParallRoundOff) (R8) and 2 Re(b c x / (1 - c x)) (Pade22)."""
    for name in ("R8", "pade22"):
        d, base, S = plan(harness, name, 0, True)
        for x in (0.01, -0.03, 0.05):
            got = 0.0
            for s in S:
                m = 1 - s["u1r"] * x - s["u2r"] * x * x
                got += (s["gr"] + s["ar"] * x + s["br"] * x * x) / m
            if name == "R8":
                ref = sum(b * c * x / (1 - c * x) for b, c in zip(d["b_re"], d["c_re"]) if c != 0)
            else:
                c = complex(d["c_re"][0], d["c_im"][0])
                b = complex(d["b_re"][0], d["b_im"][0])
                ref = 2 * (b * c * x / (1 - c * x)).real
            assert abs(got - ref) <= 1e-12 * (1 + abs(ref)), (name, x, got, ref)
