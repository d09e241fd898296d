"""The resident model handle (svm_model_create / svm_model_decision /
svm_model_free, through the C ABI).

A model keeps only the support vectors of a training (the rows with
alpha > 0, Section III-A), their alpha y, b and the kernel on the device;
its decisions (Eq. classi before the sign) must equal svm_decision's on the
training inputs bit for bit (same rows in the same order, same arithmetic),
for every precision and input kind, over repeated calls, with the caller's
training buffers gone.
"""
import gc

import numpy as np
import pytest

import oracle
import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


CASES = {
    "dense-fp64": (lambda: synth.gaussian_mixture(n=1500, n_test=700, seed=81), pkg.SVM_FP64),
    "dense-mixed-tc": (lambda: synth.gaussian_mixture(n=1500, n_test=700, seed=82), pkg.SVM_MIXED_BF16),
    "dense-mixed-simt": (lambda: synth.gaussian_mixture(n=1500, n_test=700, seed=83), pkg.SVM_MIXED_BF16_SIMT),
    "binary": (lambda: synth.onehot_sparse(n=3000, n_test=900, seed=84), pkg.SVM_FP64),
    "ragged": (lambda: synth.random_sparse(2001, 150, 0.05, seed=85, C=2.0, gamma=0.2), pkg.SVM_FP64),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_model_decision_equals_svm_decision(name):
    make, prec = CASES[name]
    p = make()
    Z = p.Z if p.Z is not None and p.Z.n > 0 else p.X
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=prec)
    ref = pkg.svm_decision(Xd, yd, r["alpha"], r["b"], p.gamma, pkg.to_device(Z), precision=prec).cpu().numpy()
    model = pkg.Model(Xd, yd, r["alpha"], r["b"], p.gamma, precision=prec)
    info = model.info()
    assert info["n_sv"] == int((r["alpha"] > 0).sum().item())
    assert info["d"] == p.X.d and info["b"] == r["b"]
    del Xd, yd, r            # the model owns its rows
    gc.collect()
    torch.cuda.empty_cache()
    for _ in range(2):       # repeated decisions on device and host queries
        dz = model.decision(pkg.to_device(Z)).cpu().numpy()
        assert np.array_equal(dz, ref)
        dh = model.decision(Z)
        assert np.array_equal(dh, ref)
    model.free()
    model.free()             # idempotent


def test_model_matches_oracle_and_edge_cases():
    p = synth.gaussian_mixture(n=800, n_test=500, seed=86)
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau)
    dref = oracle.decision(p.X, p.y, ref["alpha"], ref["b"], p.gamma, p.Z)
    with pkg.Model(p.X, p.y, ref["alpha"], ref["b"], p.gamma) as m:
        assert np.abs(m.decision(p.Z) - dref).max() <= 1e-9
        # other kernels keep their own arithmetic
    with pkg.Model(p.X, p.y, ref["alpha"], ref["b"], p.gamma, kernel=pkg.SVM_KERNEL_POLY,
                   degree=2, coef0=1.0) as m:
        d1 = m.decision(p.Z)
        d2 = pkg.svm_decision(p.X, p.y, ref["alpha"], ref["b"], p.gamma, p.Z,
                              kernel=pkg.SVM_KERNEL_POLY, degree=2, coef0=1.0)
        assert np.array_equal(d1, d2)
    # no support vector: the decision is -b everywhere
    with pkg.Model(p.X, p.y, np.zeros(p.X.n), 0.25, p.gamma) as m:
        assert m.info()["n_sv"] == 0
        assert np.all(m.decision(p.Z) == -0.25)
    # wrong width of the queries
    q = synth.gaussian_mixture(n=10, n_test=0, d=7, seed=87)
    with pkg.Model(p.X, p.y, ref["alpha"], ref["b"], p.gamma) as m:
        with pytest.raises(pkg.SvmError):
            m.decision(q.X)
