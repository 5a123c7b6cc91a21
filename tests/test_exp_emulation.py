"""The library's table-driven exponential (Tang 1989), replayed on the CPU.

The constants are read from the device header and the operation sequence is replayed
with correctly rounded fused multiply-adds (exact rational arithmetic, rounded once),
so the test pins the constants and the accuracy claim (<= 1.3 ulp against a 120-bit
exponential) without a GPU; the GPU test compares the device routine with CUDA's exp
and the host libm.
"""
import math
import os
import re
import struct
from fractions import Fraction

import pytest

mp = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_2504_04941_gb300", "csrc", "kt_exp.cuh")
INTERNAL = os.path.join(os.path.dirname(HERE), "paper_2504_04941_gb300", "csrc", "kt_internal.h")


def _const(src: str, name: str) -> float:
    m = re.search(r"const double " + name + r"\s*=\s*([0-9a-fA-Fx.p+\-]+);", src)
    assert m, name
    tok = m.group(1)
    return float.fromhex(tok) if "x" in tok else float(tok)


def _fma(a: float, b: float, c: float) -> float:
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _from_bits(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


@pytest.fixture(scope="module")
def tang():
    src = open(HDR).read()
    ntab = int(re.search(r"kExpTable\s*=\s*(\d+);", open(INTERNAL).read()).group(1))
    inv_l, shift = _const(src, "inv_l"), _const(src, "shift")
    l_head, l_tail = _const(src, "l_head"), _const(src, "l_tail")
    mp.mp.prec = 200
    # the constants are what their comments say
    assert ntab == 256
    assert abs(Fraction(inv_l) - Fraction(str(mp.mpf(ntab) / mp.log(2)))) <= Fraction(math.ulp(inv_l))
    assert shift == 1.5 * 2.0 ** 52
    l_exact = mp.log(2) / ntab
    assert abs(mp.mpf(l_head) + mp.mpf(l_tail) - l_exact) <= mp.mpf(math.ulp(l_tail)) / 2   # tail rounded once
    assert Fraction(l_head).denominator <= 2 ** (32 - 1 - math.floor(math.log2(l_head)))   # 32 bits
    tab = [float(mp.power(2, mp.mpf(j) / ntab)) for j in range(ntab)]
    shift_bits = ntab.bit_length() - 1

    def f(x: float) -> float:
        t = _fma(x, inv_l, shift)
        n = _bits(t) & 0xFFFFFFFF
        n = n - (1 << 32) if n >= (1 << 31) else n
        nd = t - shift
        j = n & (ntab - 1)
        m = (n - j) >> shift_bits
        r = _fma(-nd, l_tail, _fma(-nd, l_head, x))
        q = _fma(r, 1.0 / 24.0, 1.0 / 6.0)
        q = _fma(r, q, 0.5)
        p = _fma(r * r, q, r)
        s = tab[j]
        v = _fma(s, p, s)
        return _from_bits(_bits(v) + (m << 52))
    return f


def test_table_exp_within_1_3_ulp(tang):
    import random
    rng = random.Random(5)
    xs = [rng.uniform(-708.0, 709.0) for _ in range(3000)] + [rng.uniform(-1.0, 1.0) for _ in range(1000)]
    xs += [k * math.log(2) / 256 for k in range(-2000, 2000, 37)] + [0.0, -708.0, 709.0, 1e-300, -1e-300]
    worst = 0.0
    for x in xs:
        e = mp.exp(mp.mpf(x))
        worst = max(worst, float(abs(mp.mpf(tang(x)) - e) / math.ulp(float(e))))
    assert worst <= 1.3, worst
