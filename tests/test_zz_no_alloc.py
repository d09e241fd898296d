"""The allocation-free training call (svm_train_fixed_workspace) against
svm_train, through the C ABI.

The fixed-workspace call serves callers that cannot allocate device memory
during a solve; all its scratch is one array reserved when the library loads.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone."""
import numpy as np
import pytest

import oracle
import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


def _both(p, flags=0):
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    ref = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, flags=flags)
    fix = pkg.svm_train_fixed_workspace(Xd, yd, p.C, p.gamma, p.tau, flags=flags)
    return ref, fix


def _check(p, ref, fix):
    assert fix["status"] == pkg.SVM_OK and ref["status"] == pkg.SVM_OK
    a_ref = ref["alpha"].cpu().numpy()
    a_fix = fix["alpha"].cpu().numpy()
    # the same solve: objective within 1e-5 relative, multipliers and b close
    w_ref = oracle.kkt(p.X, p.y, a_ref, p.C, p.gamma)
    w_fix = oracle.kkt(p.X, p.y, a_fix, p.C, p.gamma)
    assert w_fix["gap"] <= 2 * p.tau + 1e-9
    assert abs(w_fix["objective"] - w_ref["objective"]) <= 1e-5 * abs(w_ref["objective"])
    assert np.abs(a_fix - a_ref).max() <= 1e-9
    assert abs(fix["b"] - ref["b"]) <= 1e-9


def test_two_calls_in_a_row_match_svm_train():
    # two different problems back to back: the second call must not see the
    # first call's leftovers in the shared workspace
    p1 = synth.gaussian_mixture(n=1500, n_test=0, seed=31)
    p2 = synth.onehot_sparse(n=3000, n_test=0, seed=32)
    r1, f1 = _both(p1)
    r2, f2 = _both(p2)
    _check(p1, r1, f1)
    _check(p2, r2, f2)
    # and the first problem again after the second
    r3, f3 = _both(p1)
    _check(p1, r3, f3)


def test_second_order_selection_matches_svm_train():
    for p in (synth.gaussian_mixture(n=1500, n_test=0, seed=31), synth.onehot_sparse(n=3000, n_test=0, seed=32)):
        r, f = _both(p, flags=pkg.SVM_FLAG_WSS2)
        _check(p, r, f)
        assert f["iters"] == r["iters"]


def test_limit_is_reported():
    p = synth.onehot_sparse(n=140000, n_test=0, seed=33)
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    r = pkg.svm_train_fixed_workspace(Xd, yd, p.C, p.gamma, p.tau, check=False)
    assert r["status"] == pkg.SVM_ERR_UNSUPPORTED
    assert "131072" in pkg.svm_last_error()
