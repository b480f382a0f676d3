"""The integer evaluation of sum_j x_j - M x_0 that the FP64 residual kernel
uses for constant-coefficient cubic cells (mg_exact.h), compiled for the
host with g++ and checked against exact rational arithmetic: the error is
at most half an ulp of the result plus M/32 ulp of the largest input (the
alignment grid), equal to the correctly rounded value when every input lies
on that grid, never worse than the FP64 evaluation by more than that grid
bound, and it declines (FP64 fallback) for infinities and NaN."""
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("exact") / "exact_lap_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "native", "exact_lap_check.cpp")])
    return exe


def run(prog, rows):
    text = "".join("%d %s\n" % (len(r) - 1, " ".join(float(x).hex() for x in r)) for r in rows)
    out = subprocess.run([prog], input=text.encode(), stdout=subprocess.PIPE, check=True).stdout.decode().split()
    return [None if o == "fallback" else float.fromhex(o) for o in out]


def exact(r):
    M = len(r) - 1
    return sum(Fraction(x) for x in r[1:]) - M * Fraction(r[0])


def ulp(x):
    return math.ulp(x) if x != 0 else math.ulp(0.0)


def random_rows(rng, n, M):
    rows = []
    for _ in range(n):
        kind = rng.integers(0, 4)
        if kind == 0:  # smooth field: nearby values, heavy cancellation
            c = rng.normal() * 10.0 ** rng.integers(-8, 8)
            rows.append([c] + list(c * (1 + 1e-4 * rng.normal(size=M))))
        elif kind == 1:  # mixed magnitudes and signs
            rows.append(list(rng.normal(size=M + 1) * 10.0 ** rng.integers(-30, 30, size=M + 1)))
        elif kind == 2:  # zeros and a lone value
            r = [0.0] * (M + 1)
            r[rng.integers(0, M + 1)] = rng.normal() * 10.0 ** rng.integers(-300, 300)
            rows.append(r)
        else:  # denormals and tiny values
            rows.append(list(rng.normal(size=M + 1) * 5e-320))
    return rows


@pytest.mark.parametrize("M", [4, 6])
def test_error_bound_against_exact_arithmetic(prog, M):
    rng = np.random.default_rng(M)
    rows = random_rows(rng, 4000, M)
    got = run(prog, rows)
    for r, g in zip(rows, got):
        ex = exact(r)
        if g is None:  # only outside the normal range
            assert abs(float(ex)) < 1e-300 or abs(float(ex)) > 1e300, r
            continue
        big = max(abs(x) for x in r)
        bound = Fraction(ulp(g)) / 2 + Fraction(M) * Fraction(ulp(big)) / 32
        assert abs(Fraction(g) - ex) <= bound, (r, g, float(ex))
        # never worse than FP64 arithmetic by more than the alignment grid
        naive = sum(r[1:]) - M * r[0]
        assert abs(Fraction(g) - ex) <= abs(Fraction(naive) - ex) + Fraction(M) * Fraction(ulp(big)) / 32 + Fraction(ulp(g))


@pytest.mark.parametrize("M", [4, 6])
def test_correctly_rounded_on_the_grid(prog, M):
    """Values sharing one exponent (and integers) lie on the alignment grid:
    the result is the correctly rounded exact sum."""
    rng = np.random.default_rng(10 + M)
    rows = [list(1.0 + rng.random(M + 1)) for _ in range(2000)]
    rows += [list(rng.integers(-2 ** 40, 2 ** 40, size=M + 1).astype(float)) for _ in range(1000)]
    for r, g in zip(rows, run(prog, rows)):
        assert g == float(exact(r)), (r, g)


def test_non_finite_inputs_fall_back(prog):
    rows = [[1.0, math.inf, 0, 0, 0], [math.nan, 1, 2, 3, 4], [1.0, 2, 3, 4, -math.inf, 0, 0]]
    assert run(prog, rows) == [None, None, None]


@pytest.fixture(scope="module")
def prog2(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("exactf") / "exact_float_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "native", "exact_float_check.cpp")])
    return exe


def test_integer_float_conversion_is_round_to_nearest_even(prog2):
    """mg_to_float (the FP32 defect without the FP64 conversion instruction)
    equals the IEEE conversion bit for bit: normal, denormal, overflow,
    halfway cases, zeros, infinities."""
    rng = np.random.default_rng(7)
    xs = list(rng.normal(size=3000) * 10.0 ** rng.integers(-50, 50, size=3000))
    xs += list(rng.normal(size=500) * 1e-40) + list(rng.normal(size=200) * 1e-45)
    xs += [0.0, -0.0, math.inf, -math.inf, 3.5e38, -3.5e38, 3.4028235677973366e38, 1.401298464324817e-45 / 2,
           1.401298464324817e-45 * 1.5, 1.1754943508222875e-38, 1.1754942106924411e-38]
    # exact halfway points between FP32 neighbours
    for _ in range(500):
        f = np.float32(rng.normal() * 10.0 ** rng.integers(-30, 30))
        up = np.nextafter(f, np.float32(np.inf))
        xs.append((float(f) + float(up)) / 2)
    text = "".join("C %s\n" % float(x).hex() for x in xs)
    out = subprocess.run([prog2], input=text.encode(), stdout=subprocess.PIPE, check=True).stdout.decode().split()
    with np.errstate(over="ignore"):
        ref = [int(np.array([x], np.float64).astype(np.float32).view(np.uint32)[0]) for x in xs]
    assert [int(o, 16) for o in out] == ref


def test_block_alignment_round_trip(prog2):
    """mg_fix / mg_unfix: a value at the alignment exponent or up to 5 below
    it comes back exactly; smaller values come back within the grid step."""
    rng = np.random.default_rng(8)
    rows = []
    for _ in range(3000):
        x = rng.normal() * 10.0 ** rng.integers(-20, 20)
        e = int(np.frexp(abs(x))[1]) + 1022 if x != 0 else 1
        rows.append((min(2046, e + int(rng.integers(0, 20))), x))
    text = "".join("F %d %s\n" % (em, float(x).hex()) for em, x in rows)
    out = subprocess.run([prog2], input=text.encode(), stdout=subprocess.PIPE, check=True).stdout.decode().split()
    for (em, x), o in zip(rows, out):
        got = float.fromhex(o)
        step = 2.0 ** (em - 1080)
        e = int(np.frexp(abs(x))[1]) + 1022 if x != 0 else 1
        if em - e <= 5:
            assert got == x, (em, x, got)
        else:
            assert abs(got - x) <= step / 2 + math.ulp(got) / 2, (em, x, got)


def test_integer_widening_is_exact(prog2):
    """mg_from_float (FP32 to FP64 for the update phi += e without the
    conversion instruction) equals the exact widening: normals, denormals,
    zeros, infinities."""
    rng = np.random.default_rng(9)
    bits = list(rng.integers(0, 2 ** 32, size=5000, dtype=np.uint64))
    bits += [0, 0x80000000, 1, 0x807FFFFF, 0x00400000, 0x7F7FFFFF, 0xFF7FFFFF, 0x7F800000, 0xFF800000, 0x00800000]
    bits = [int(b) for b in bits if (int(b) >> 23) & 0xFF != 0xFF or (int(b) & 0x7FFFFF) == 0]  # NaN payloads aside
    text = "".join("W %x\n" % b for b in bits)
    out = subprocess.run([prog2], input=text.encode(), stdout=subprocess.PIPE, check=True).stdout.decode().split()
    ref = [float(np.array([b], np.uint32).view(np.float32)[0]) for b in bits]
    assert [float.fromhex(o) for o in out] == ref
