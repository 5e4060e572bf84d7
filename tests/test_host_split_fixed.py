"""Scalar arithmetic of the error-free splitting behind the FP64-accurate
products (Ozaki, Ogita, Oishi & Rump 2012), checked on the CPU.

The split kernels call mpl::oz_digits and mpl::oz_fixed_value
(csrc/oz_fixed.cuh).  These tests compile both for the host and compare
them, value by value, with their definitions in exact arithmetic:
  * the digits: the 64-bit fixed point U = round(x 2^(63 - ex)) (half away
    from zero), then the balanced digits taken from the top, each the
    nearest integer (half up) of what remains, and the bf16 pattern of each
    digit; the digits must also add back to U and stay within |q| <= 128;
  * the value of an accumulator pair: 2^ex (hi 2^-24 + lo 2^-56) as a
    rational number, rounded once to the nearest double (Python's
    Fraction -> float rounds correctly), which the kernel must reproduce
    bit for bit.
"""
import math
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_12528_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include "oz_fixed.cuh"
// argv[1] = d: lines "bits ex" -> the 8 digit patterns;
// argv[1] = v: lines "hi lo ex" -> the bit pattern of oz_fixed_value
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[2], "r");
  if (argv[1][0] == 'd') {
    unsigned long long b;
    int ex;
    while (std::fscanf(f, "%llx %d", &b, &ex) == 2) {
      double x;
      std::memcpy(&x, &b, 8);
      uint16_t d[8];
      mpl::oz_digits(x, ex, d);
      for (int i = 0; i < 8; ++i) std::printf("%04x%c", d[i], i == 7 ? '\n' : ' ');
    }
  } else {
    long long hi, lo;
    int ex;
    while (std::fscanf(f, "%lld %lld %d", &hi, &lo, &ex) == 3) {
      const double v = mpl::oz_fixed_value(hi, lo, ex);
      unsigned long long b;
      std::memcpy(&b, &v, 8);
      std::printf("%016llx\n", b);
    }
  }
  return 0;
}
"""


def _compiler():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def reference_digits(x, ex):
    """The splitting by its definition, in Python integers."""
    bits = struct.unpack("<Q", struct.pack("<d", x))[0]
    E = (bits >> 52) & 0x7FF
    M = (bits & ((1 << 52) - 1)) | ((1 << 52) if E else 0)
    e2 = max(E, 1) - 1075 + 63 - ex            # |x| 2^(63 - ex) = M 2^e2
    if e2 >= 0:
        U = M << e2
    else:                                      # floor(M 2^e2 + 1/2)
        U = (M + (1 << (-e2 - 1))) >> (-e2) if -e2 - 1 < 200 else 0
    if bits >> 63:
        U = -U
    q, R = [], U
    for i in range(8):
        sh = 56 - 8 * i
        d = (R + (1 << (sh - 1))) >> sh if sh else R   # floor(R / 2^sh + 1/2)
        R -= d << sh
        q.append(d)
    return U, q


def bf16_pattern(q):
    return int(np.array([q], dtype=np.float32).view(np.uint32)[0] >> 16)


def cases():
    rng = np.random.default_rng(20230224)
    out = []
    # random values over a wide range of magnitudes, row exponents at or above theirs
    for _ in range(6000):
        x = float(rng.uniform(-1, 1)) * math.ldexp(1.0, int(rng.integers(-300, 300)))
        ex = (math.frexp(x)[1] if x != 0 else 0) + int(rng.integers(0, 70))
        out.append((x, ex))
    # random finite bit patterns (subnormals included), exponent just above
    for _ in range(4000):
        b = int(rng.integers(0, 2 ** 63, dtype=np.uint64)) | (int(rng.integers(0, 2)) << 63)
        x = struct.unpack("<d", struct.pack("<Q", b))[0]
        if not math.isfinite(x):
            continue
        out.append((x, (math.frexp(x)[1] if x != 0 else 0) + int(rng.integers(0, 4))))
    # exact halves at every digit boundary: U = k 2^s + 2^(s-1) (+-1)
    for s in range(1, 57):
        for k in (-200, -129, -128, -127, -1, 0, 1, 127, 128, 129, 255):
            for d in (-1, 0, 1):
                U = k * (1 << s) + (1 << (s - 1)) + d
                if U == 0 or abs(U) >= 1 << 62:
                    continue
                x = math.ldexp(float(U), -63)      # ex = 0: U = x 2^63 exactly when U has <= 53 bits
                if int(math.ldexp(x, 63)) == U:
                    out.append((x, 0))
    # extremes
    for x, ex in ((0.0, 0), (-0.0, 0), (5e-324, -1073), (-5e-324, -1060), (1.7976931348623157e308, 1024),
                  (-1.7976931348623157e308, 1024), (1.0, 1), (-1.0, 1), (0.5, 0), (2.0 ** -1022, -1021)):
        out.append((x, ex))
    return out


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = _compiler()
    if nvcc is None:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("ozdigits")
    src = d / "harness.cu"
    src.write_text(HARNESS)
    exe = d / "harness"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_digits_match_the_definition(harness, tmp_path):
    cs = cases()
    inp = tmp_path / "in.txt"
    inp.write_text("".join(f"{struct.unpack('<Q', struct.pack('<d', x))[0]:016x} {ex}\n" for x, ex in cs))
    r = subprocess.run([str(harness), "d", str(inp)], capture_output=True, text=True, check=True)
    lines = r.stdout.strip().split("\n")
    assert len(lines) == len(cs)
    for (x, ex), line in zip(cs, lines):
        got = [int(t, 16) for t in line.split()]
        U, q = reference_digits(x, ex)
        assert all(abs(d) <= 128 for d in q), (x, ex, q)
        assert sum(d << (56 - 8 * i) for i, d in enumerate(q)) == U, (x, ex)
        assert got == [bf16_pattern(d) for d in q], (x, ex, q, got)


def test_reference_worked_example():
    """Hand-worked: U = 3 2^48 + 2^47 (ex = 0) has the digits 0, 4, -128, 0,
    0, 0, 0, 0 -- what remains above 2^48 is 3.5, rounded half up to 4,
    leaving -2^47 = -128 2^40 (half down would give 3 and +128 instead)."""
    U0 = 3 * (1 << 48) + (1 << 47)
    U, q = reference_digits(math.ldexp(float(U0), -63), 0)
    assert U == U0
    assert q == [0, 4, -128, 0, 0, 0, 0, 0]


def value_cases():
    """(hi, lo, ex) as the kernels produce them (|hi| < 2^59, |lo| < 2^62),
    with ex keeping the result normal, plus the branch boundaries of
    top = hi + floor(lo / 2^32) at +-2^53 and exact halves."""
    rng = np.random.default_rng(1202)
    out = []
    for _ in range(6000):
        hi = int(rng.integers(-(1 << 59) + 1, 1 << 59))
        lo = int(rng.integers(-(1 << 62) + 1, 1 << 62))
        out.append((hi, lo, int(rng.integers(-900, 900))))
    for _ in range(3000):   # small hi: the exact branch, low word significant
        hi = int(rng.integers(-(1 << 40), 1 << 40))
        lo = int(rng.integers(-(1 << 62) + 1, 1 << 62))
        out.append((hi, lo, int(rng.integers(-60, 60))))
    for top in (1 << 53, (1 << 53) - 1, (1 << 53) + 1, -(1 << 53), -(1 << 53) + 1, -(1 << 53) - 1,
                (1 << 54) + 1, -(1 << 54) - 1, (1 << 59) - 1, -(1 << 59) + 1, 0, 1, -1):
        for low in (0, 1, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, (1 << 32) - 1):
            for lo_top in (0, 5, -5):   # split top between hi and lo's upper bits
                hi = top - lo_top
                lo = (lo_top << 32) + low
                if abs(hi) < 1 << 59:
                    out.append((hi, lo, 0))
    return out


def test_fixed_value_is_rounded_once(harness, tmp_path):
    cs = value_cases()
    inp = tmp_path / "vin.txt"
    inp.write_text("".join(f"{hi} {lo} {ex}\n" for hi, lo, ex in cs))
    r = subprocess.run([str(harness), "v", str(inp)], capture_output=True, text=True, check=True)
    lines = r.stdout.strip().split("\n")
    assert len(lines) == len(cs)
    from fractions import Fraction
    for (hi, lo, ex), line in zip(cs, lines):
        exact = (Fraction(hi) / (1 << 24) + Fraction(lo) / (1 << 56)) * (Fraction(2) ** ex)
        want = struct.unpack("<Q", struct.pack("<d", float(exact)))[0]
        assert int(line, 16) == want, (hi, lo, ex, float(exact))


def test_fixed_value_reference_catches_double_rounding():
    """The exact reference is not the kernel's arithmetic: converting top
    first and adding the low word afterwards (two roundings) differs from it
    on a case where top is odd and above 2^53 and the low word breaks the tie."""
    from fractions import Fraction
    top, low = (1 << 53) + 1, 1            # exact value top + 2^-32: just above the midpoint
    two_roundings = float(top) + math.ldexp(float(low), -32)
    exact = float(Fraction(top) + Fraction(low, 1 << 32))
    assert exact == float((1 << 53) + 2) and two_roundings == float(1 << 53)
