"""The FP64 oracle against closed forms, a brute-force QP solver, numpy
recomputations and invariants (no GPU)."""
import pytest

import os, sys
sys.path.insert(0, os.path.dirname(__file__))
import oracle_pins as P  # noqa: E402


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(orc, check):
    check()


def test_bruteforce_n12(orc):
    P.check_bruteforce(cases=((12, 7, 1.0),))


def test_two_point_golden(orc):
    """Stored closed-form optimum of the two-point dual (tests/golden)."""
    import numpy as np
    from paper_1406_5161_gb300 import synth
    path = os.path.join(os.path.dirname(__file__), "golden", "two_point.tsv")
    rows = [ln.split("\t") for ln in open(path) if not ln.startswith("#")]
    assert len(rows) >= 5
    for dist, C, gamma, k, a_star in rows:
        X = synth.csr_from_dense(np.array([[0.0], [float(dist)]], dtype=np.float32), True)
        y = np.array([1, -1], dtype=np.int8)
        r = orc.smo(X, y, float(C), float(gamma), 1e-9, max_iter=10)
        assert abs(r["alpha"][0] - float(a_star)) <= 1e-13 * float(a_star)
        assert abs(r["alpha"][1] - float(a_star)) <= 1e-13 * float(a_star)
