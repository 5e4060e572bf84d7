"""Digits of the error-free splitting behind the FP64-accurate products
(Ozaki, Ogita, Oishi & Rump 2012), checked on the CPU.

The split kernels call mpl::oz_digits (csrc/oz_digits.cuh).  This test
compiles that function for the host and compares it, value by value, with
the splitting written out from its definition in Python integers: the
64-bit fixed point U = round(x 2^(63 - ex)) (half away from zero), then the
balanced digits taken from the top, each the nearest integer (half up) of
what remains, and the bf16 pattern of each digit.  It also checks that the
digits add back to U exactly and stay within |q| <= 128 (exact in bf16).
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
#include "oz_digits.cuh"
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "r");
  unsigned long long b;
  int ex;
  while (std::fscanf(f, "%llx %d", &b, &ex) == 2) {
    double x;
    std::memcpy(&x, &b, 8);
    uint16_t d[8];
    mpl::oz_digits(x, ex, d);
    for (int i = 0; i < 8; ++i) std::printf("%04x%c", d[i], i == 7 ? '\n' : ' ');
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
    r = subprocess.run([str(harness), str(inp)], capture_output=True, text=True, check=True)
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
