"""CPU replay of the table-driven exp/expm1 steps of csrc/exp_table.cuh (Tang's method, used by the
FP64 face potentials and the FP64 z sweep's nonlinear stage), with the reduction constants read from
that header: exp within 2 ulp of the host's exp on [-60, 0], expm1 within 2e-14 relative of the
host's expm1 (tiny arguments and the m = -1 band included).  Fused multiply-adds are replayed
exactly with rationals, as the device rounds them once."""
import math
import os
import random
import re
import struct
from fractions import Fraction

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1410_2788_gb300", "csrc", "exp_table.cuh")


def _constants():
    txt = open(HDR).read()
    out = {}
    for name in ("kInvL", "kL1", "kL2", "kShift"):
        m = re.search(r"constexpr double %s = ([0-9.eE+-]+);" % name, txt)
        assert m, name
        out[name] = float(m.group(1))
    return out


C = _constants()
T = [2.0 ** (j / 32) for j in range(32)]


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _reduce(x):
    t = _fma(x, C["kInvL"], C["kShift"])
    n = struct.unpack("<q", struct.pack("<d", t))[0] & 0xFFFFFFFF
    if n >= 2 ** 31:
        n -= 2 ** 32
    nd = t - C["kShift"]
    r = _fma(-nd, C["kL1"], x)
    r = _fma(-nd, C["kL2"], r)
    q = _fma(r, 1 / 720, 1 / 120)
    for c in (1 / 24, 1 / 6, 0.5, 1.0):
        q = _fma(q, r, c)
    return n, r * q


def exp_nonpos(x):
    if x < -700.0:
        return 0.0
    n, p = _reduce(x)
    tj = T[n & 31]
    return math.ldexp(_fma(tj, p, tj), n >> 5)


def expm1_nonpos(x):
    if x < -700.0:
        return -1.0
    n, p = _reduce(x)
    m, tj = n >> 5, T[n & 31]
    if m == 0:
        return p
    if m == -1:
        return 0.5 * _fma(tj, p, tj - 2.0)
    return math.ldexp(_fma(tj, p, tj), m) - 1.0


def test_constants_split_ln2_over_32():
    assert abs(C["kL1"] - math.log(2) / 32) == 0.0
    # the low part carries what the double ln2/32 drops: |kL2| below half an ulp of kL1
    assert 0 < abs(C["kL2"]) < math.ulp(C["kL1"])
    assert abs(C["kInvL"] - 32 / math.log(2)) <= math.ulp(32 / math.log(2))
    assert C["kShift"] == 1.5 * 2 ** 52


def test_exp_within_two_ulp():
    rng = random.Random(11)
    xs = [-rng.random() * 60 for _ in range(3000)] + [0.0, -1e-300, -700.0, -699.5]
    for x in xs:
        a, b = exp_nonpos(x), math.exp(x)
        assert abs(a - b) <= 2 * math.ulp(b), (x, a, b)


def test_expm1_relative_error():
    rng = random.Random(12)
    xs = [-rng.random() * 40 for _ in range(2000)] + [-10 ** rng.uniform(-14, 0.3) for _ in range(2000)]
    xs += [-math.log(2) / 64 * k for k in (0.5, 1.0, 1.01, 63.9, 64.1)] + [-1e-300]
    for x in xs:
        a, b = expm1_nonpos(x), math.expm1(x)
        assert abs(a - b) <= 2e-14 * abs(b) + 1e-320, (x, a, b)
    assert expm1_nonpos(0.0) == 0.0 and expm1_nonpos(-800.0) == -1.0
