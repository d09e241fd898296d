"""Warm start / resume (svm_params.alpha0, through the C ABI).

A training can resume from the multipliers of an interrupted one: alpha0
gives alpha, the index sets follow from it (Eq. setinfo) and f is recomputed
on the device from Eq. (fcache) by the reconstruction contraction. The
resumed solve must reach the uninterrupted solve's optimum (the oracle's
KKT check, objective within 1e-9 relative in FP64), and alpha0 = 0 must be
the plain start exactly.
"""
import numpy as np
import pytest

import oracle
import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


def _dev(p):
    return pkg.to_device(p.X), torch.as_tensor(p.y, device="cuda")


@pytest.mark.parametrize("name,prec,policy", [
    ("dense", pkg.SVM_FP64, None), ("binary", pkg.SVM_FP64, "Multi5pc"),
    ("dense", pkg.SVM_FP64, "Multi5pc"), ("dense", pkg.SVM_MIXED_BF16, "Multi5pc")])
def test_resume_reaches_the_same_optimum(name, prec, policy):
    p = synth.gaussian_mixture(n=2000, n_test=0, seed=91) if name == "dense" else \
        synth.onehot_sparse(n=5000, n_test=0, seed=92)
    Xd, yd = _dev(p)
    pol = pkg.POLICIES[policy] if policy else None
    full = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=prec, shrink=pol)
    assert full["status"] == pkg.SVM_OK
    half = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=prec, shrink=pol, max_iter=full["iters"] // 2)
    assert half["status"] == pkg.SVM_NOT_CONVERGED
    res = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=prec, shrink=pol, alpha0=half["alpha"])
    assert res["status"] == pkg.SVM_OK
    wf, wr = full["stats"]["objective"], res["stats"]["objective"]
    tol = 1e-9 if prec == pkg.SVM_FP64 else 1e-5
    assert abs(wr - wf) <= tol * abs(wf)
    # resuming costs roughly the steps that were left
    assert res["iters"] <= full["iters"] - half["iters"] + full["iters"] // 4
    if prec == pkg.SVM_FP64:
        kk = oracle.kkt(p.X, p.y, res["alpha"].cpu().numpy(), p.C, p.gamma)
        assert kk["gap"] <= 2 * p.tau + 1e-9


def test_zero_alpha0_is_the_plain_start_and_bad_alpha0_is_refused():
    p = synth.gaussian_mixture(n=1000, n_test=0, seed=93)
    Xd, yd = _dev(p)
    a = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, trace_len=300)
    b = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, trace_len=300,
                      alpha0=torch.zeros(p.X.n, dtype=torch.float64, device="cuda"))
    assert a["iters"] == b["iters"] and np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["alpha"].cpu().numpy(), b["alpha"].cpu().numpy())
    bad = torch.full((p.X.n,), 2 * p.C, dtype=torch.float64, device="cuda")
    r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, alpha0=bad, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG and "alpha0" in pkg.svm_last_error()
    unbalanced = torch.zeros(p.X.n, dtype=torch.float64, device="cuda")
    unbalanced[0] = 0.5
    r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, alpha0=unbalanced, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG
