"""FP64 solves on the matrices that take each arithmetic of the FP64 row pass.

The FP64 mode computes inner products exactly in 128-bit integers when the
matrix's nonzero values lie within 31 binades below the largest and none is
subnormal, else as FP64 sums in row order. The 2,000-row Gaussian-mixture
problem is solved, with rows held on chip and streamed, after three changes
to its matrix:

* one value scaled by 2^-60: outside the window, the FP64 row-sum path;
* every zero of the dense rows stored explicitly: the exact path meeting
  zero entries (m = 0);
* columns scaled by powers of two from 2^-5 to 2^5: the exact path with the
  values spread over 23 of its 31 binades (the N(0, 1) values alone span
  18).

Each must meet the acceptance bar against the FP64 oracle on the same matrix:
the first 200 (i_up, i_low) pairs equal except at the oracle's near ties,
the oracle's KKT check at exit, and the dual objective within 1e-5.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

from test_gpu_smo import check_end_state, first_mismatch, gpu_train

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


def _variant(kind):
    p = synth.gaussian_mixture()
    a = p.X.to_dense()
    if kind == "outside_window":
        X = synth.csr_from_dense(a)
        X.values[5] = np.float32(X.values[5] * 2.0 ** -60)
    elif kind == "explicit_zeros":
        a[:, ::3] = 0.0
        X = synth.csr_from_dense(a, keep_zeros=True)
    elif kind == "wide_exponents":
        scale = 2.0 ** np.linspace(-5, 5, a.shape[1]).round()
        X = synth.csr_from_dense((a * scale).astype(np.float32))
    else:
        raise ValueError(kind)
    gamma = p.gamma if kind != "wide_exponents" else p.gamma * 2.0 ** -10
    return dataclasses.replace(p, X=X, gamma=gamma)


@pytest.fixture(scope="module", params=["outside_window", "explicit_zeros", "wide_exponents"])
def problem(request):
    p = _variant(request.param)
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=400)
    assert ref["status"] == 0
    return p, ref


@pytest.mark.parametrize("flags", [0, pkg.SVM_FLAG_STREAM_ROWS], ids=["resident", "streamed"])
def test_fp64_formats_match_the_oracle(problem, flags):
    p, ref = problem
    r, _, _ = gpu_train(p, trace_len=400, flags=flags)
    assert r["status"] == pkg.SVM_OK
    t = first_mismatch(r["trace"], ref["trace"], ref["margin"], 400)
    assert t >= 200
    check_end_state(p, r, ref)
