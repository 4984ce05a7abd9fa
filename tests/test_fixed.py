"""The fixed-point conversions of the split-precision GEMM (csrc/fixed.cuh),
compiled as host C++ and checked on the CPU against exact integer and rational
arithmetic: integer accumulators times 2^e2 rounded once to FP64 (ties to
even, including ties decided only by bits below the leading 64 of a 128-bit
sum), the 48-bit fixed-point value of an element under its row scale (nearest,
ties away from zero, |F| <= 2^48), and the row scale itself.  The same source
compiles into the device kernels (slicers, GEMM epilogue, split-K reduction)."""
import math
import os
import random
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("fixed") / "check_fixed"
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-o", str(out),
                    os.path.join(HERE, "digits", "check_fixed.cpp")], check=True)
    return str(out)


def _run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split()


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _f64(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _scaled(v, e2):
    """v * 2^e2 rounded once, ties to even: CPython's int -> float conversion
    is correctly rounded and the power-of-two scaling of a normal result is
    exact."""
    return math.ldexp(float(v), e2)


def _e2_for(v, rng):
    # keep |v| * 2^e2 well inside the normal range
    return rng.randint(-900, 900 - abs(v).bit_length())


def _ints(rng, maxbits, count):
    vals = []
    for _ in range(count):
        b = rng.randint(1, maxbits)
        v = rng.getrandbits(b) | (1 << (b - 1))
        vals.append(-v if rng.random() < 0.5 else v)
    # ties at every position of the rounding bit, with and without bits below it
    for s in range(1, maxbits - 53 + 1):
        for mant in (1 << 52, (1 << 52) | 1, (1 << 53) - 1, (1 << 53) - 2):
            base = (mant << s) | (1 << (s - 1))
            if base.bit_length() > maxbits:
                continue
            vals += [base, -base]
            if s >= 2:
                vals += [base + 1, -(base + 1), base - 1]
            if s > 64:
                vals += [base | (1 << (s - 60)), base | 1]     # the deciding bit only in the low word
    vals += [1, -1, 2, (1 << 53) + 1, (1 << maxbits) - 1, -((1 << maxbits) - 1), 1 << (maxbits - 1)]
    return vals


def test_i64_to_f64_scaled_is_correctly_rounded(exe):
    rng = random.Random(11)
    vals = _ints(rng, 63, 40000) + [-(1 << 63)]
    cases = [(v, _e2_for(v, rng)) for v in vals] + [(v, 0) for v in vals[:2000]]
    got = _run(exe, [f"i64 {v & M64:016x} {e2}" for v, e2 in cases])
    assert len(got) == len(cases)
    for (v, e2), g in zip(cases, got):
        assert _f64(int(g, 16)) == _scaled(v, e2), (v, e2, g)


def test_i128_to_f64_scaled_is_correctly_rounded(exe):
    rng = random.Random(12)
    vals = _ints(rng, 126, 60000) + [-(1 << 127), (1 << 127) - 1, -((1 << 127) - 1), (1 << 64), (1 << 64) - 1]
    cases = [(v, _e2_for(v, rng)) for v in vals]
    M128 = (1 << 128) - 1
    got = _run(exe, [f"i128 {((v & M128) >> 64):016x} {(v & M64):016x} {e2}" for v, e2 in cases])
    assert len(got) == len(cases)
    bad = [(v, e2, g) for (v, e2), g in zip(cases, got) if _f64(int(g, 16)) != _scaled(v, e2)]
    assert not bad, bad[:5]


def test_i128_ties_below_the_high_word_round_up():
    """A planted two-step conversion (high and low parts rounded apart, then
    added) misses the ties the single rounding gets right: the expected values
    used above are sensitive to double rounding."""
    v = ((1 << 52) << 70) | (1 << 69) | 1                # even mantissa, above the tie only through bit 0
    hi, lo = v >> 62, v & ((1 << 62) - 1)
    two_step = math.ldexp(float(hi), 62) + float(lo)
    assert _scaled(v, 0) != two_step and _scaled(v, 0) == float(Fraction(v))


def _fixed48_ref(x, e):
    """x * 2^(48 - e) to the nearest integer, ties away from zero; 0 for zero
    and subnormal x."""
    if x == 0 or abs(x) < 2.0 ** -1022:
        return 0
    y = abs(Fraction(x) * Fraction(2) ** (48 - e))
    q = int(y + Fraction(1, 2))      # floor(y + 1/2)
    return -q if x < 0 else q


def test_to_fixed48_rounds_to_nearest_and_stays_within_48_bits(exe):
    rng = random.Random(13)
    cases = []
    for _ in range(40000):
        e = rng.randint(-300, 300)
        x = math.ldexp(rng.uniform(-1.0, 1.0), e) * (1 - 2 ** -53)   # |x| < 2^e
        if rng.random() < 0.2:
            x = math.ldexp(x, -rng.randint(0, 80))                  # much smaller than the scale
        cases.append((x, e))
    for e in (0, 5, -7):
        for b in range(0, 49):                                        # exact ties: odd halves of the unit 2^(e-48)
            m = (rng.getrandbits(b) << 1) | 1
            for x in (math.ldexp(m, e - 49), -math.ldexp(m, e - 49)):
                if abs(x) < 2.0 ** e:
                    cases.append((x, e))
        cases += [(0.0, e), (-0.0, e), (5e-324, e), (math.ldexp(1.0, e) * (1 - 2 ** -53), e)]
    got = _run(exe, [f"fx {_bits(x):016x} {e}" for x, e in cases])
    assert len(got) == len(cases)
    for (x, e), g in zip(cases, got):
        F = int(g, 16)
        F = F - (1 << 64) if F >> 63 else F
        assert F == _fixed48_ref(x, e), (x, e, F)
        assert abs(F) <= 1 << 48


def _fixed_ref(x, e, nbits):
    if x == 0 or abs(x) < 2.0 ** -1022:
        return 0
    y = abs(Fraction(x) * Fraction(2) ** (nbits - e))
    q = int(y + Fraction(1, 2))
    return -q if x < 0 else q


def test_to_fixed_56_bits(exe):
    """The 56-bit form of the seven-slice operands: more bits than a double
    carries, so values near the scale are shifted left (exactly) and small
    ones rounded; |F| <= 2^56."""
    rng = random.Random(17)
    cases = []
    for _ in range(20000):
        e = rng.randint(-300, 300)
        x = math.ldexp(rng.uniform(-1.0, 1.0), e) * (1 - 2 ** -53)
        if rng.random() < 0.3:
            x = math.ldexp(x, -rng.randint(0, 90))
        cases.append((x, e))
    for e in (0, 9):
        for b in range(0, 57):
            m = (rng.getrandbits(b) << 1) | 1
            for x in (math.ldexp(m, e - 57), -math.ldexp(m, e - 57)):
                if abs(x) < 2.0 ** e:
                    cases.append((x, e))
        cases += [(0.0, e), (5e-324, e), (math.ldexp(1.0, e) * (1 - 2 ** -53), e)]
    got = _run(exe, [f"fxn 56 {_bits(x):016x} {e}" for x, e in cases])
    for (x, e), g in zip(cases, got):
        F = int(g, 16)
        F = F - (1 << 64) if F >> 63 else F
        assert F == _fixed_ref(x, e, 56), (x, e, F)
        assert abs(F) <= 1 << 56
    # the 48-bit form is the same function at nbits = 48
    got48 = _run(exe, [f"fxn 48 {_bits(x):016x} {e}" for x, e in cases[:2000]])
    got_fx = _run(exe, [f"fx {_bits(x):016x} {e}" for x, e in cases[:2000]])
    assert got48 == got_fx


def test_exponent_of_max_bounds_the_group(exe):
    rng = random.Random(14)
    xs = [math.ldexp(rng.uniform(0.5, 1.0), rng.randint(-1020, 1020)) for _ in range(20000)]
    xs += [0.0, 5e-324, 2.0 ** -1022, 1.0, 0.5, 2.0 ** 1023, float.fromhex("0x1.fffffffffffffp+1023")]
    got = [int(g) for g in _run(exe, [f"em {_bits(x):016x}" for x in xs])]
    for x, e in zip(xs, got):
        if x < 2.0 ** -1022:
            assert e == -1000
        else:
            assert Fraction(x) < Fraction(2) ** e <= 2 * Fraction(x), (x, e)
