"""The constants and truncation claims of the double-float sine / cosine
(csrc/df_trig.cuh), checked against the mathematics on the CPU."""
import math
import os
import re
from fractions import Fraction

import pytest

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_1609_04493_gb300", "csrc",
                      "df_trig.cuh")


def _const(name):
    text = open(HEADER).read()
    m = re.search(r"constexpr double %s = ([0-9.e+-]+);" % name, text)
    assert m, name
    return float(m.group(1))


def test_pi_over_two_split():
    """Head: the double nearest pi/2; tail: the double nearest pi/2 - head;
    together pi/2 to 1.5e-33."""
    sympy = pytest.importorskip("sympy")
    head, tail = _const("kDfPio2Head"), _const("kDfPio2Tail")
    half_pi = sympy.pi / 2
    assert head == float(sympy.N(half_pi, 40))
    rest = half_pi - sympy.Rational(Fraction(head))
    assert tail == float(sympy.N(rest, 40))
    assert abs(float(sympy.N(rest - sympy.Rational(Fraction(tail)), 40))) < 1.6e-33


def test_two_over_pi():
    assert abs(_const("kDfTwoOverPi") - 2 / math.pi) <= 2 ** -53


def test_taylor_truncation_and_fp32_tail():
    """For |r| <= 0.8 the first omitted terms are below 1e-16, and the terms
    summed in FP32 are below 3e-9 of the result."""
    r = 0.8
    assert r ** 17 / math.factorial(17) < 1e-16 * math.sin(r)
    assert r ** 18 / math.factorial(18) < 1e-16 * math.cos(r)
    assert r ** 11 / math.factorial(11) < 3e-9 * math.sin(r)
    assert r ** 12 / math.factorial(12) < 3e-9 * math.cos(r)
    # and the reduction keeps |r| within pi/4 (plus rounding) < 0.8
    assert math.pi / 4 * (1 + 2 ** -50) < r
