"""Writes exp2_table.inc: 2^(j/256) for j = 0..255, each correctly rounded to
double (mpmath at 60 digits), as exact hexadecimal literals. The table of the
table-driven exponential in fp64_math.cuh (Tang, ACM TOMS 15(2), 1989).

Usage: python paper_1406_5161_gb300/csrc/gen_exp2_table.py
"""
import os

import mpmath as mp

mp.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))

if __name__ == "__main__":
    lines = ["// 2^(j/256), j = 0..255, correctly rounded (written by gen_exp2_table.py)"]
    vals = [float(mp.power(2, mp.mpf(j) / 256)) for j in range(256)]
    for k in range(0, 256, 4):
        lines.append("    " + ", ".join(v.hex() for v in vals[k:k + 4]) + ",")
    with open(os.path.join(HERE, "exp2_table.inc"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
