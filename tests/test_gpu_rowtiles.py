"""Kernel rows on the tensor cores in the mixed-precision solve (through the
C ABI).

With SVM_MIXED_BF16 (RBF, d <= 256) the row pass forms the two kernel rows
K(x_up, .) and K(x_low, .) of Eq. (fup) from tiles of 16 active rows times
the two target rows on the tensor cores (BF16 inputs, FP32 accumulation).
Against the CSR row pass on the CUDA cores (SVM_FLAG_CUDA_CORE_ROWS: same
BF16 values, FP32 sums in another order) the solves must agree within the
mixed path's rounding; across launch shapes the tile path must give the same
solve bit for bit; and the end state must pass the FP64 oracle's checks at
the mixed path's tolerance.
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

MIXED = pkg.SVM_MIXED_BF16
TILES = pkg.SVM_FLAG_TENSOR_ROWS


def _run(p, **kw):
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=MIXED, **kw)
    assert r["status"] == pkg.SVM_OK
    return r


PROBLEMS = {
    "dense20": lambda: synth.gaussian_mixture(n=3000, n_test=0, seed=41),
    "dense64": lambda: synth.gaussian_mixture(n=4000, n_test=0, d=64, seed=47, gamma=0.01),
    "covtype54": lambda: synth.covtype_like(n=6000, n_test=0, seed=42),
    "ragged90": lambda: synth.random_sparse(4001, 90, 0.08, seed=43, C=2.0, gamma=0.1),
    "dense256": lambda: synth.gaussian_mixture(n=2500, n_test=0, d=256, seed=44),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("policy", ["Original", "Multi5pc"])
def test_tiles_agree_with_cuda_core_rows(name, policy):
    p = PROBLEMS[name]()
    pol = pkg.POLICIES[policy]
    a = _run(p, shrink=pol, flags=TILES)
    b = _run(p, shrink=pol, flags=pkg.SVM_FLAG_CUDA_CORE_ROWS)
    assert a["stats"]["row_tiles"] == 1 and b["stats"]["row_tiles"] == 0
    wa, wb = a["stats"]["objective"], b["stats"]["objective"]
    assert abs(wa - wb) <= 1e-6 * abs(wb)
    # the mixed end state against the FP64 oracle's checks
    alpha = a["alpha"].cpu().numpy()
    kk = oracle.kkt(p.X, p.y, alpha, p.C, p.gamma)
    assert abs(kk["objective"] - wb) <= 2e-4 * abs(wb)
    assert (alpha >= 0).all() and (alpha <= p.C).all() and abs((alpha * p.y).sum()) <= 1e-9 * len(alpha)


def test_tiles_give_one_solve_over_launch_shapes():
    p = PROBLEMS["covtype54"]()
    pol = pkg.POLICIES["Multi5pc"]
    runs = {
        "one-cluster": _run(p, shrink=pol, trace_len=5000, ctas=16, flags=TILES),
        "clusters8": _run(p, shrink=pol, trace_len=5000, ctas=152, flags=TILES),
        "flat": _run(p, shrink=pol, trace_len=5000, ctas=152, flags=TILES | pkg.SVM_FLAG_NO_CLUSTERS),
        "streamed": _run(p, shrink=pol, trace_len=5000, ctas=152, flags=TILES | pkg.SVM_FLAG_STREAM_ROWS),
    }
    assert runs["one-cluster"]["stats"]["cluster_size"] == 16
    assert runs["streamed"]["stats"]["resident"] == 0
    base = runs["one-cluster"]
    for name, r in runs.items():
        assert r["stats"]["row_tiles"] == 1, name
        assert r["iters"] == base["iters"], name
        assert np.array_equal(r["trace"], base["trace"]), name
        assert np.array_equal(r["alpha"].cpu().numpy(), base["alpha"].cpu().numpy()), name
        assert r["b"] == base["b"], name


def test_automatic_choice_and_range():
    # dense rows of 64 columns: tiles by default; 20 columns or sparse rows: CSR
    assert _run(synth.gaussian_mixture(n=2000, n_test=0, d=64, seed=46))["stats"]["row_tiles"] == 1
    assert _run(PROBLEMS["dense20"]())["stats"]["row_tiles"] == 0
    assert _run(PROBLEMS["covtype54"]())["stats"]["row_tiles"] == 0
    wide = synth.gaussian_mixture(n=600, n_test=0, d=300, seed=45)
    assert _run(wide, flags=TILES)["stats"]["row_tiles"] == 0
    p = PROBLEMS["dense20"]()
    assert _run(p, cache_mb=16, flags=TILES)["stats"]["row_tiles"] == 0   # the kernel-row cache keeps the CSR pass
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=pkg.SVM_MIXED_BF16_SIMT, flags=TILES)
    assert r["stats"]["row_tiles"] == 0
