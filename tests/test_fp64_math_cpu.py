"""The FP64 helpers of the CUDA path's FP64 mode (csrc/fp64_math.cuh), built
for the host with the same IEEE and integer operations the device runs (no
contraction):

* widen_f32 returns the conversion instruction's double for every float bit
  pattern below 2^24 (zeros, all subnormals, the smallest normals), every
  subnormal with the sign set, and a stride-7 sweep of all other finite
  patterns;
* exp_neg_fx (exp(-y) in fixed-point integer arithmetic after Tang's
  table-driven method) is within 0.53 units in the last place of long
  double exp over 2e7 points of [0, 700], small arguments down to 2^-80 and
  the neighbours of multiples of ln2/256; it is exactly 1 at 0 and hands
  negative arguments, arguments above 700 and NaN to the library exp;
* the exact inner products (xd_*) equal the exact rational sums rounded to
  nearest (below)."""
import os
import struct
import subprocess
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fp64_helpers_on_the_host(tmp_path):
    exe = str(tmp_path / "fp64_math_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_1406_5161_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fp64_math_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe, "7"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout


# ---- exact inner products (xd_format / xd_add / xd_round)

def _f32(v):
    return np.float32(v)


def _bits(v):
    return int(np.array([v], dtype=np.float32).view(np.uint32)[0])


def _exact(x, z):
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, z)), Fraction(0))


def _double_bits(fr):
    # Python's int / int true division rounds correctly (nearest, ties to even)
    v = fr.numerator / fr.denominator if fr != 0 else 0.0
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def _xd_cases():
    rng = np.random.default_rng(11)
    cases = []
    for n in list(range(1, 17)) + [31, 54, 64, 200, 1000]:
        for _ in range(6):
            cases.append((rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)))
    # a wide spread of exponents inside the window (31 binades below the
    # largest value for rows up to 2^16 entries), signs mixed
    for n in (3, 12, 40):
        for _ in range(20):
            e = rng.integers(-15, 16, size=(2, n))
            s = rng.choice([-1.0, 1.0], size=(2, n))
            m = rng.uniform(1, 2, size=(2, n))
            cases.append(((s[0] * m[0] * 2.0 ** e[0]).astype(np.float32), (s[1] * m[1] * 2.0 ** e[1]).astype(np.float32)))
    # exact and near cancellation: x.z = 0, and 0 up to one tiny product
    for _ in range(20):
        a = rng.standard_normal(8).astype(np.float32)
        cases.append((np.concatenate([a, a]), np.concatenate([a, -a])))
        t = np.float32(2.0 ** -25)
        cases.append((np.concatenate([a, a, [t]]), np.concatenate([a, -a, [np.float32(1.5)]])))
    # ties: 1 + 2^-53 (to even: 1), 1 + 2^-52 + 2^-53 (up), -(1 + 3 2^-53)
    one, h = _f32(1.0), _f32(2.0 ** -27)
    cases.append((np.array([one, h], np.float32), np.array([one, _f32(2.0 ** -26)], np.float32)))
    cases.append((np.array([one, h, h], np.float32), np.array([one, _f32(2.0 ** -25), _f32(2.0 ** -26)], np.float32)))
    cases.append((np.array([-one, h, h], np.float32), np.array([one, _f32(-2.0 ** -25), _f32(-2.0 ** -26)], np.float32)))
    # zeros among the values, all-zero rows, the largest and smallest normal floats
    cases.append((np.array([0.0, 1.0, -0.0, 2.5], np.float32), np.array([3.0, 0.0, 7.0, -0.5], np.float32)))
    cases.append((np.zeros(5, np.float32), rng.standard_normal(5).astype(np.float32)))
    big = np.float32(3.0e38)
    cases.append((np.array([big, big], np.float32), np.array([big, -big / 2], np.float32)))
    # the accumulator's headroom: the largest mantissas, all at the top
    # exponent, in the longest rows of their bit length (1, 3, 1023, 1000)
    top = np.array([0x3fffffff], np.uint32).view(np.float32)[0]
    for n in (1, 3, 1000, 1023):
        cases.append((np.full(n, top, np.float32), np.full(n, top, np.float32)))
        cases.append((np.full(n, -top, np.float32), np.full(n, top, np.float32)))
    # the window's edge: values 31 binades apart on each side
    cases.append((np.array([1.0, 2.0 ** -31, -3.0 * 2.0 ** -31], np.float32),
                  np.array([2.0 ** -31, 1.0, 1.0], np.float32)))
    small = np.float32(2.0 ** -126)
    cases.append((np.array([small, small * 3], np.float32), np.array([small, small], np.float32)))
    return cases


def test_exact_inner_products_on_the_host(tmp_path):
    """xd: every inner product inside the format's window equals the exact
    rational sum rounded to the nearest double (ties to even), whatever the
    order of the terms and their split over lanes; operands outside the
    window (a spread of exponents wider than s / 2, a subnormal value) turn
    the format off; xd_round rounds 128-bit integers exactly."""
    exe = str(tmp_path / "fp64_math_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_1406_5161_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fp64_math_check.cpp"), "-o", exe], check=True)
    cases = _xd_cases()
    off_cases = [
        (np.array([1.0, 2.0 ** -60], np.float32), np.array([1.0, 1.0], np.float32)),   # spread 60 > s/2
        (np.array([1.0, 2.0 ** -32], np.float32), np.array([1.0, 1.0], np.float32)),   # just outside
        (np.array([1.0, 1e-40], np.float32), np.array([1.0, 1.0], np.float32)),         # subnormal
    ]
    rng = np.random.default_rng(5)
    rounds = []
    for _ in range(3000):
        hi = int(rng.integers(0, 2 ** 63)) >> int(rng.integers(0, 64))
        lo = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        if rng.random() < 0.3:
            lo &= ~((1 << int(rng.integers(0, 64))) - 1)   # many trailing zeros: exact ties happen
        if rng.random() < 0.5:   # negative: two's complement
            v = -((hi << 64) | lo) & ((1 << 128) - 1)
            hi, lo = v >> 64, v & ((1 << 64) - 1)
        rounds.append((hi, lo, int(rng.integers(-400, 200))))
    rounds += [(0, 1, 0), (0, (1 << 53) + 1, 0), (0, (1 << 54) + 2, -3), (1, 0, -64), ((1 << 64) - 1, (1 << 64) - 1, 0)]
    # ties and near ties at leading-bit positions in every limb: 2^P + 2^(P-53)
    # (a tie, even significand), the same with an odd significand, and one
    # unit above and below the tie (the deciding bit far below the window)
    for P in (54, 60, 63, 64, 70, 95, 96, 100, 117, 126):
        for v in (2 ** P + 2 ** (P - 53), 2 ** P + 2 ** (P - 52) + 2 ** (P - 53),
                  2 ** P + 2 ** (P - 53) + 1, 2 ** P + 2 ** (P - 53) - 1):
            for sgn in (1, -1):
                w = (sgn * v) & ((1 << 128) - 1)
                rounds.append((w >> 64, w & ((1 << 64) - 1), -7))
    lines = []
    for x, z in cases + off_cases:
        lines.append("D %d %s" % (len(x), " ".join("%08x %08x" % (_bits(a), _bits(b)) for a, b in zip(x, z))))
    for hi, lo, u in rounds:
        lines.append("R %x %x %d" % (hi, lo, u))
    r = subprocess.run([exe, "xd"], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr
    out = r.stdout.split("\n")
    assert out[len(lines)] == "xd bad 0"
    for i, (x, z) in enumerate(cases):
        assert out[i] != "off", i
        assert int(out[i], 16) == _double_bits(_exact(x, z)), (i, x, z)
    for j in range(len(off_cases)):
        assert out[len(cases) + j] == "off"
    base = len(cases) + len(off_cases)
    for j, (hi, lo, u) in enumerate(rounds):
        v = (hi << 64) | lo
        if v >> 127:
            v -= 1 << 128
        want = _double_bits(Fraction(v) * Fraction(2) ** u)
        assert int(out[base + j], 16) == want, (hi, lo, u)
