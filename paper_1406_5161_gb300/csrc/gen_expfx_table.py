"""Writes expfx_table.inc, the table and constants of exp_neg_fx in
fp64_math.cuh (exp(-y) in fixed-point integer arithmetic after the
table-driven method of P. T. P. Tang, ACM TOMS 15(2), 1989), all computed
with mpmath at 80 digits:

* kExpfxTab[j] = 2^(-j/256) in Q63 (value * 2^63, rounded to nearest),
  j = 0..255 (2^63 for j = 0);
* kExpfxInvL54 = 256 / ln 2 * 2^54, rounded to nearest;
* kExpfxLH, kExpfxLL: ln 2 / 256 * 2^64 split into its integer part and the
  next 64 bits (floor), so that n ln2/256 is known to about 2^-128 * n;
* kExpfxC2 .. kExpfxC5 = 1/k! in Q63, rounded to nearest.

Usage: python paper_1406_5161_gb300/csrc/gen_expfx_table.py
"""
import os

import mpmath as mp

mp.mp.dps = 80
HERE = os.path.dirname(os.path.abspath(__file__))


def q(x, bits):
    return int(mp.nint(x * mp.power(2, bits)))


if __name__ == "__main__":
    ln2 = mp.log(2)
    L = ln2 / 256
    lh = int(mp.floor(L * mp.power(2, 64)))
    ll = int(mp.floor((L * mp.power(2, 64) - lh) * mp.power(2, 64)))
    lines = ["// written by gen_expfx_table.py (mpmath, 80 digits)"]
    lines.append("constexpr uint64_t kExpfxInvL54 = 0x%016xull;   // 256 / ln 2 * 2^54" % q(256 / ln2, 54))
    lines.append("constexpr uint64_t kExpfxLH = 0x%016xull;       // floor(ln 2 / 256 * 2^64)" % lh)
    lines.append("constexpr uint64_t kExpfxLL = 0x%016xull;       // its next 64 bits" % ll)
    for k in (2, 3, 4, 5):
        lines.append("constexpr uint64_t kExpfxC%d = 0x%016xull;       // 1/%d! in Q63" % (k, q(1 / mp.factorial(k), 63), k))
    lines.append("// 2^(-j/256) in Q63, j = 0..255")
    lines.append("#define SVM_EXPFX_TABLE \\")
    vals = [q(mp.power(2, -mp.mpf(j) / 256), 63) for j in range(256)]
    for k in range(0, 256, 4):
        lines.append("    " + ", ".join("0x%016xull" % v for v in vals[k:k + 4]) + (", \\" if k + 4 < 256 else ""))
    with open(os.path.join(HERE, "expfx_table.inc"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
