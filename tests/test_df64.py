"""Pins the double-float arithmetic used by the small eigen-solvers
(paper_1612_07875_gb300/csrc/df64.cuh): the header is compiled for the host
with g++ and every result is compared with exact rational arithmetic.
A df64 value hi + lo carries about 48 bits; the bounds below allow a few
units of 2^-46 relative error (2^-44 for division and square root)."""
import os
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "df64_check.cpp")
INC = os.path.join(ROOT, "paper_1612_07875_gb300", "csrc")


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("df64") / "df64_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + INC, SRC, "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return [ln.split() for ln in out.splitlines()]


def F(h):
    return Fraction(float.fromhex(h))


def _rel(got, exact, scale=None):
    den = abs(exact) if scale is None else scale
    if den == 0:
        return abs(got)
    return abs(got - exact) / den


def test_conversion_from_double_is_48_bit(lines):
    n = 0
    for ln in lines:
        if ln[0] != "from":
            continue
        x, hi, lo = F(ln[1]), F(ln[2]), F(ln[3])
        assert _rel(hi + lo, x) <= Fraction(1, 2 ** 47)
        n += 1
    assert n > 1000


def test_conversion_from_int64_exact_below_2_48(lines):
    for ln in lines:
        if ln[0] == "ll":
            v = int(ln[1])
            got = F(ln[2]) + F(ln[3])
            assert got == v


@pytest.mark.parametrize("op,bound", [("add", 2 ** -46), ("sub", 2 ** -46), ("mul", 2 ** -45),
                                      ("div", 2 ** -44), ("sqrt", 2 ** -44), ("fma", 2 ** -45),
                                      ("recip", 2 ** -45)])
def test_operations_against_exact_rationals(lines, op, bound):
    worst = Fraction(0)
    cnt = 0
    for ln in lines:
        if ln[0] != op:
            continue
        vals = [F(h) for h in ln[1:]]
        if op == "fma":
            a, b, c, r = vals[0] + vals[1], vals[2] + vals[3], vals[4] + vals[5], vals[6] + vals[7]
            exact = a * b + c
            # error relative to the terms (a*b and c may cancel)
            e = _rel(r, exact, abs(a * b) + abs(c))
        else:
            a, b, r = vals[0] + vals[1], vals[2] + vals[3], vals[4] + vals[5]
            if op == "add":
                exact = a + b
            elif op == "sub":
                exact = a - b
            elif op == "mul":
                exact = a * b
            elif op == "div":
                exact = a / b
            elif op == "recip":
                exact = 1 / b
            else:
                # compare r^2 with a: relative error of sqrt is half that of r^2
                e = _rel(r * r, a) / 2
                worst = max(worst, e)
                cnt += 1
                continue
            e = _rel(r, exact)
        worst = max(worst, e)
        cnt += 1
    assert cnt > 1000
    assert worst <= Fraction(bound), float(worst)
