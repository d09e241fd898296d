"""Write two_point.tsv: the exact dual optimum of the two-point problem.

Points x1 = 0 (y = +1) and x2 = dist (y = -1) in one dimension, RBF kernel
k = exp(-gamma * dist^2). The dual (Eq. lagdual with Eq. eqconst) forces
alpha1 = alpha2 = a and reduces to max 2a - a^2 (1 - k), so
a* = min(C, 1 / (1 - k)); with a* < C, f1 = f2 = 0 and b = 0. Values are
computed with mpmath at 40 digits from that closed form (no solver code).
The paper prints no worked example, so this is the only stored fixture.
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
CASES = [(1.0, 100.0, 0.5), (0.25, 100.0, 1.0), (3.0, 0.4, 0.1), (2.0, 1.0, 0.05),
         (0.5, 5.0, 0.3), (1.5, 2.0, 0.2)]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "two_point.tsv")
    with open(out, "w") as fh:
        fh.write("# dist(float32)\tC\tgamma\tk\talpha_star\n")
        for dist, C, gamma in CASES:
            d = mp.mpf(float(np.float32(dist)))
            k = mp.exp(-mp.mpf(gamma) * d * d)
            a = min(mp.mpf(C), 1 / (1 - k))
            fh.write(f"{float(d)!r}\t{C!r}\t{gamma!r}\t{mp.nstr(k, 25)}\t{mp.nstr(a, 25)}\n")
