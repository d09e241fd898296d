"""GPU parity of the second-order working-set selection (SVM_FLAG_WSS2)
against the oracle's second-order runs (through the C ABI).

i_up as in Eq. (bminmax); i_low the row t of I_low with f_t > f_up of largest
gain (f_t - f_up)^2 / (K_uu + K_tt - 2 K_ut), the selection the paper leaves
to future work (Section VI). Acceptance as for the first-order path: the
pairs equal the oracle's for the first 200 steps except after a near tie
(I_up margin below 1e-12, or the best gain ahead of the runner-up by less than
1e-12 relative), the oracle's KKT check and objective at exit, identical
solves over every launch shape.
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

from test_gpu_smo import check_end_state, first_mismatch, gpu_train  # noqa: E402

WSS2 = pkg.SVM_FLAG_WSS2


def _problem(name):
    if name.startswith("dense"):
        return synth.gaussian_mixture(n=2000, n_test=0, seed=71)
    if name.startswith("ragged"):
        return synth.random_sparse(3001, 300, 0.02, seed=5, binary=False, C=2.0, gamma=0.2)
    return synth.onehot_sparse(n=6000, n_test=0, seed=12)


CASES = {
    "dense-resident": 0,
    "dense-streamed": pkg.SVM_FLAG_STREAM_ROWS,
    "bits-resident": 0,
    "bits-streamed": pkg.SVM_FLAG_STREAM_ROWS,
    "csr-binary": pkg.SVM_FLAG_CSR_ROWS,
    "ragged-resident": 0,
    "ragged-streamed": pkg.SVM_FLAG_STREAM_ROWS,
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_pairs_match_oracle(name):
    p = _problem(name)
    ref = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, trace_len=400)
    assert ref["status"] == 0
    r, _, _ = gpu_train(p, trace_len=400, flags=CASES[name] | WSS2)
    assert r["status"] == pkg.SVM_OK
    if name.startswith("bits"):
        assert r["stats"]["bit_rows"] == 1
    t = first_mismatch(r["trace"], ref["trace"], ref["margin"], 400)
    assert t >= min(200, ref["iters"]), t
    alpha, _ = check_end_state(p, r, ref)
    if t == min(400, ref["iters"]) and r["iters"] == ref["iters"]:
        assert np.abs(alpha - ref["alpha"]).max() <= 1e-9
    # the second-order rule takes fewer steps than the first-order one here
    first = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau)
    assert r["iters"] < first["iters"]


@pytest.mark.parametrize("flags", [0, pkg.SVM_FLAG_CSR_ROWS], ids=["bits", "csr"])
def test_launch_shapes_give_identical_solves(flags):
    """The gain exchange inside one 16-CTA cluster, across clusters of 8 and
    without clusters: the same steps to the same alpha."""
    p = synth.onehot_sparse(n=6000, n_test=0, seed=12)
    kind, value, recon = pkg.POLICIES["Multi5pc"]
    runs = {}
    for name, kw in {"single16": dict(ctas=16), "clusters8": dict(ctas=152),
                     "flat": dict(ctas=152, flags=flags | WSS2 | pkg.SVM_FLAG_NO_CLUSTERS),
                     "auto": dict()}.items():
        kw.setdefault("flags", flags | WSS2)
        r, _, _ = gpu_train(p, shrink=(kind, value, recon), trace_len=2000, **kw)
        assert r["status"] == pkg.SVM_OK
        runs[name] = r
    assert runs["single16"]["stats"]["cluster_size"] == 16
    assert runs["clusters8"]["stats"]["cluster_size"] == 8
    assert runs["flat"]["stats"]["cluster_size"] == 1
    base = runs["single16"]
    for name, r in runs.items():
        assert r["iters"] == base["iters"], name
        assert np.array_equal(r["trace"], base["trace"]), name
        assert np.array_equal(r["alpha"].cpu().numpy(), base["alpha"].cpu().numpy()), name
        assert r["b"] == base["b"], name


@pytest.fixture(scope="module")
def shrink_problem():
    p = synth.onehot_sparse(n=6000, n_test=0, seed=12)
    plain = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, trace_len=300)
    first = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau)
    return p, plain, first


@pytest.mark.parametrize("name", ["Multi5pc", "Multi2", "Multi50pc", "Single500", "Single5pc"])
def test_shrinking_policies_match_oracle(shrink_problem, name):
    p, plain, first = shrink_problem
    kind, value, recon = pkg.POLICIES[name]
    ref = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, p.tau, kind, value, recon, trace_len=100000, wss=2)
    assert ref["status"] == 0
    flags = WSS2 | (pkg.SVM_FLAG_STREAM_ROWS if name.startswith("Single") else 0)
    r, _, _ = gpu_train(p, shrink=(kind, value, recon), trace_len=100000, flags=flags)
    assert r["status"] == pkg.SVM_OK
    m = min(len(ref["trace"]), len(r["trace"]))
    diff = np.nonzero((r["trace"][:m] != ref["trace"][:m]).any(axis=1))[0]
    if len(diff) and diff[0] < 200:
        tt = diff[0]
        assert tt < len(plain["margin"]) and plain["margin"][tt].min() < 1e-12
    if not len(diff) and r["iters"] == ref["iters"]:
        assert r["stats"]["shrink_events"] == ref["n_shrink"]
        assert r["stats"]["reconstructions"] == ref["n_recon"]
    check_end_state(p, r, first)


def test_dense_fp64_shrinking_reaches_optimum():
    p = synth.gaussian_mixture(n=3000, n_test=0, seed=21)
    first = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau)
    for name in ["Multi5pc", "Single500"]:
        kind, value, recon = pkg.POLICIES[name]
        r, _, _ = gpu_train(p, shrink=(kind, value, recon), flags=WSS2)
        check_end_state(p, r, first)


def test_mixed_precision_reaches_fp64_optimum():
    p = synth.gaussian_mixture(n=3000, n_test=0, seed=22)
    ref = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau)
    r, _, _ = gpu_train(p, precision=pkg.SVM_MIXED_BF16, flags=WSS2,
                        shrink=pkg.POLICIES["Multi5pc"])
    assert r["status"] == pkg.SVM_OK
    kk = oracle.kkt(p.X, p.y, r["alpha"].cpu().numpy(), p.C, p.gamma)
    assert abs(kk["objective"] - ref["objective"]) <= 2e-3 * abs(ref["objective"])


@pytest.mark.parametrize("kind,c0,deg", [(pkg.SVM_KERNEL_LINEAR, 0.0, 1), (pkg.SVM_KERNEL_POLY, 1.0, 3)],
                         ids=["linear", "poly3"])
def test_other_kernels_match_oracle(kind, c0, deg):
    p = synth.gaussian_mixture(n=1500, n_test=0, seed=63)
    with oracle.kernel_spec(kind, c0, deg):
        ref = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, trace_len=300, max_iter=200000)
        assert ref["status"] == 0
        r, _, _ = gpu_train(p, trace_len=300, kernel=kind, degree=deg, coef0=c0, flags=WSS2)
        assert r["status"] == pkg.SVM_OK
        t = first_mismatch(r["trace"], ref["trace"], ref["margin"], 300)
        assert t >= min(200, ref["iters"])
        check_end_state(p, r, ref)


def test_duplicate_points_and_step_limit():
    # identical rows: eta = 0 in the gain (floored at 1e-12) and in the step
    x = np.tile(np.array([[0.5, -1.0, 2.0]], dtype=np.float32), (12, 1))
    x[6:] += 1.0
    X = synth.csr_from_dense(x, keep_zeros=True)
    y = np.array([1, -1] * 6, dtype=np.int8)
    ref = oracle.smo_wss2(X, y, 1.0, 0.3, 1e-3, trace_len=1000)
    r = pkg.svm_train(X, y, 1.0, 0.3, 1e-3, trace_len=1000, flags=WSS2)
    assert r["iters"] == ref["iters"]
    assert np.array_equal(r["trace"], ref["trace"].astype(np.int32))
    assert np.abs(r["alpha"] - ref["alpha"]).max() <= 1e-12
    p = synth.small_dense(500, 6, seed=3, C=1.0, gamma=0.1)
    ref = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, max_iter=7)
    r = pkg.svm_train(p.X, p.y, p.C, p.gamma, p.tau, max_iter=7, flags=WSS2)
    assert r["status"] == pkg.SVM_NOT_CONVERGED and r["iters"] == 7
    assert np.abs(r["alpha"] - ref["alpha"]).max() <= 1e-12
