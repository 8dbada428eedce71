"""The exact fixed-point sums behind the persistent solvers' reductions.

Every CTA adds its double-float partial of a CG inner product (the r.z,
p.Ap and scale-step sums of Section II-C's solve) as eight 36-bit digits of
an integer in units of 2^-149; the total is read back as a double-float.
These CPU tests build the same header with the host compiler and check it
against exact rational arithmetic (fractions.Fraction): the digits of one
float are its exact value, the total of many partials is their exact sum
truncated to 48 significant bits, the order of the partials does not change
a bit, and the edge cases (cancellation to zero, subnormals, sums beyond the
float range, non-finite partials) come out as stated.
"""
import ctypes as C
import os
import random
import shutil
import struct
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2207_12244_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp(prefix="df_exact_")
    so = os.path.join(d, "libexact.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "exact_sum_harness.cpp"), "-o", so], check=True)
    L = C.CDLL(so)
    L.exact_total.argtypes = [C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_float)]
    L.float_digit_of.argtypes = [C.c_float, C.c_int]
    L.float_digit_of.restype = C.c_longlong
    yield L
    shutil.rmtree(d, ignore_errors=True)


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def total(L, pairs):
    a = np.ascontiguousarray(np.asarray(pairs, dtype=np.float32).reshape(-1))
    out = (C.c_float * 2)()
    L.exact_total(a.ctypes.data_as(C.POINTER(C.c_float)), len(a) // 2, out)
    return np.float32(out[0]), np.float32(out[1])


def exact(pairs):
    s = Fraction(0)
    for hi, lo in pairs:
        s += Fraction(float(np.float32(hi))) + Fraction(float(np.float32(lo)))
    return s


def rand_pairs(rng, n, emin, emax):
    """Double-float partials (hi, lo with |lo| <= ulp(hi) / 2) of random sign
    and exponent."""
    out = []
    for _ in range(n):
        hi = np.float32(rng.choice([-1, 1]) * rng.uniform(1, 2) * 2.0 ** rng.integers(emin, emax))
        lo = np.float32(float(hi) * rng.uniform(-2 ** -24, 2 ** -24))
        out.append((hi, lo))
    return out


def test_digits_of_one_float_are_its_exact_value(lib):
    rng = np.random.default_rng(0)
    vals = [0.0, -0.0, 1.0, -1.5, f32(3.4028235e38), f32(-3.4028235e38), f32(1.17549435e-38),
            f32(1.4e-45), f32(-2.8e-45), f32(5.877472e-39)]
    vals += [float(np.float32(rng.standard_normal() * 2.0 ** rng.integers(-140, 120)))
             for _ in range(300)]
    for v in vals:
        digits = [lib.float_digit_of(v, k) for k in range(8)]
        assert sum(1 for d in digits if d) <= 2
        assert all(abs(d) < 2 ** 36 for d in digits)
        got = sum(Fraction(d) * Fraction(2) ** (36 * k) for k, d in enumerate(digits))
        assert got * Fraction(2) ** -149 == Fraction(v)


def test_total_is_the_exact_sum_truncated_to_48_bits(lib):
    rng = np.random.default_rng(1)
    for trial in range(60):
        n = int(rng.integers(1, 256))
        lo_e = int(rng.integers(-140, 60))
        pairs = rand_pairs(rng, n, lo_e, lo_e + int(rng.integers(1, 40)))
        hi, lo = total(lib, pairs)
        s = exact(pairs)
        got = Fraction(float(hi)) + Fraction(float(lo))
        if s == 0:
            assert got == 0
            continue
        # truncation toward zero after 48 bits, then two exact float parts
        assert abs(got) <= abs(s) and (got == 0 or (got > 0) == (s > 0))
        assert abs(s - got) <= abs(s) * Fraction(2) ** -47 + Fraction(2) ** -149
        # hi is the leading 24 bits, lo the next 24
        assert abs(float(lo)) <= abs(float(hi)) * 2.0 ** -23


def test_order_of_the_partials_does_not_change_a_bit(lib):
    rng = np.random.default_rng(2)
    pairs = rand_pairs(rng, 152, -30, 30) + rand_pairs(rng, 40, -120, -80)
    ref = total(lib, pairs)
    for _ in range(20):
        random.Random(int(rng.integers(1 << 30))).shuffle(pairs)
        got = total(lib, pairs)
        assert got[0].tobytes() == ref[0].tobytes() and got[1].tobytes() == ref[1].tobytes()


def test_cancellation_subnormals_and_range(lib):
    rng = np.random.default_rng(3)
    pairs = rand_pairs(rng, 100, -20, 20)
    both = pairs + [(-h, -l) for h, l in pairs]
    assert total(lib, both) == (0.0, 0.0)
    # a sum of subnormals is exact
    sub = [(np.float32(2.0 ** -149 * k), np.float32(0.0)) for k in range(1, 30)]
    hi, lo = total(lib, sub)
    assert Fraction(float(hi)) + Fraction(float(lo)) == exact(sub)
    # a negative total keeps its sign and magnitude
    neg = [(np.float32(-3.0), np.float32(0.0)), (np.float32(1.0), np.float32(2.0 ** -30))]
    hi, lo = total(lib, neg)
    assert Fraction(float(hi)) + Fraction(float(lo)) == exact(neg)
    # beyond the float range the total overflows to infinity, as a float sum would
    big = [(np.float32(3.0e38), np.float32(0.0))] * 4
    assert np.isinf(total(lib, big)[0]) and total(lib, big)[0] > 0
    assert np.isinf(total(lib, [(-a, -b) for a, b in big])[0])
    # 255 partials at the float maximum still carry exactly (no digit overflow)
    mx = [(np.float32(3.4028235e38), np.float32(0.0)), (np.float32(-3.4028235e38), np.float32(0.0))]
    assert total(lib, mx * 127) == (0.0, 0.0)


def test_non_finite_partial_makes_the_total_nan(lib):
    rng = np.random.default_rng(4)
    pairs = rand_pairs(rng, 50, -10, 10)
    for bad in (np.inf, -np.inf, np.nan):
        for where in (0, 25, 49):
            p = list(pairs)
            p[where] = (np.float32(bad), np.float32(0.0))
            hi, lo = total(lib, p)
            assert np.isnan(hi) and np.isnan(lo)
    # a non-finite low part too, and with many large finite partials beside it
    p = [(np.float32(3.0e38), np.float32(0.0))] * 254 + [(np.float32(1.0), np.float32(np.nan))]
    assert np.isnan(total(lib, p)[0])
    p = [(np.float32(-3.4e38), np.float32(0.0))] * 1022 + [(np.float32(np.inf), np.float32(0.0))]
    assert np.isnan(total(lib, p)[0])


def test_up_to_1023_partials(lib):
    """Plans with two CTAs per SM give a keyframe up to 304 CTAs; the digits
    hold 1023 partials exactly."""
    rng = np.random.default_rng(5)
    pairs = rand_pairs(rng, 1023, 100, 127)
    hi, lo = total(lib, pairs)
    s = exact(pairs)
    if abs(s) < 2 ** 128:
        got = Fraction(float(hi)) + Fraction(float(lo))
        assert abs(s - got) <= abs(s) * Fraction(2) ** -47
    else:
        assert np.isinf(hi)
    # 1023 partials at the float maximum: the total overflows to infinity
    mx = [(np.float32(3.4028235e38), np.float32(2.0 ** 103))] * 1023
    assert np.isinf(total(lib, mx)[0]) and total(lib, mx)[0] > 0
    assert np.isinf(total(lib, [(-a, -b) for a, b in mx])[0])


def test_carry_rounds_equal_the_sequential_carries(lib):
    """The solvers resolve the digit sums' carries across the lanes of a
    group in rounds; on every kind of digit-sum vector (random, every digit at
    its extremes, carries rippling through full digits, negative totals,
    zero, non-finite marks, overflow) the result is the sequential one."""
    L = lib
    for f in (L.total_by_rounds, L.total_sequential):
        f.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_float)]

    def both(raw):
        a = np.ascontiguousarray(np.asarray(raw, dtype=np.int64))
        o1, o2 = (C.c_float * 2)(), (C.c_float * 2)()
        L.total_by_rounds(a.ctypes.data_as(C.POINTER(C.c_longlong)), o1)
        L.total_sequential(a.ctypes.data_as(C.POINTER(C.c_longlong)), o2)
        return (np.float32(o1[0]).tobytes() + np.float32(o1[1]).tobytes(),
                np.float32(o2[0]).tobytes() + np.float32(o2[1]).tobytes())

    rng = np.random.default_rng(7)
    mask = (1 << 36) - 1
    cases = [[0] * 8, [mask] * 7 + [0], [mask] * 7 + [-1], [1] + [0] * 7, [-1] + [0] * 7,
             [0] * 7 + [1 << 36], [0] * 7 + [(1 << 35) - 1], [0] * 7 + [-(1 << 35)],
             [mask + 1] + [mask] * 6 + [0], [-(1 << 46)] * 8, [(1 << 46) - 1] * 7 + [0]]
    for _ in range(3000):
        kind = rng.integers(0, 4)
        if kind == 0:
            raw = rng.integers(-(1 << 46), 1 << 46, 8)
            raw[7] = rng.integers(-(1 << 34), 1 << 34)
        elif kind == 1:
            raw = rng.choice([0, 1, -1, mask, mask + 1, -mask], 8)
        elif kind == 2:
            raw = rng.integers(0, 1 << 37, 8) * rng.choice([1, -1], 8)
            raw[5:] = 0
        else:
            raw = np.zeros(8, dtype=np.int64)
            raw[rng.integers(0, 8)] = rng.integers(-(1 << 46), 1 << 46)
        cases.append([int(v) for v in raw])
    for raw in cases:
        a, b = both(raw)
        assert a == b, raw
