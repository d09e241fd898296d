"""The stored oracle answer for the full covtype-shaped workload
(tests/golden/covtype_full*, written by make_covtype_full.py from oracle/
alone: without shrinking, and with the Multi500 policy) is complete and
consistent: it belongs to the generator's current
output, its alpha is feasible (0 <= alpha <= C, sum y alpha = 0) and has the
recorded hash and support-vector counts, its gap met the stopping rule
(Eq. kktterm), and the 10,000 held-out decision values are all there."""
import hashlib
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
from make_covtype_full import input_digest  # noqa: E402
from paper_1406_5161_gb300 import synth  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


import pytest  # noqa: E402


@pytest.mark.parametrize("tag", ["covtype_full", "covtype_full_multi500"])
def test_covtype_full_answer_is_consistent(tag):
    meta = json.load(open(os.path.join(GOLDEN, tag + ".json")))
    dec = np.loadtxt(os.path.join(GOLDEN, tag + "_decision.txt"), comments="#")
    a = np.load(os.path.join(GOLDEN, tag + "_alpha.npz"))["alpha"]
    p = synth.covtype_like()
    assert input_digest(p) == meta["input_sha256"]
    assert (meta["n"], meta["d"], meta["C"], meta["gamma"], meta["tau"]) == (p.X.n, p.X.d, p.C, p.gamma, p.tau)
    assert hashlib.sha256(a.tobytes()).hexdigest() == meta["alpha_sha256"]
    assert a.shape == (p.X.n,) and (a >= 0).all() and (a <= p.C).all()
    assert abs(float((a * p.y).sum())) <= 1e-9 * len(a) * p.C
    assert int((a > 0).sum()) == meta["n_sv"] and int((a == p.C).sum()) == meta["n_bound_sv"]
    assert meta["kkt_gap"] <= 2 * p.tau
    assert abs(meta["kkt_objective"] - meta["objective"]) <= 1e-9 * abs(meta["objective"])
    assert dec.shape == (p.Z.n,) and np.isfinite(dec).all()
    assert int((dec > 0).sum()) == meta["held_out_positive"]
