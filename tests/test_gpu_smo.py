"""GPU parity of the fused SMO path against the FP64 oracle (through the C ABI).

Acceptance (FP64 mode, lowest-index ties):
* the selected (i_up, i_low) pairs equal the oracle's for the first 200
  steps, except at a step where the oracle's best and second-best violation
  values differ by less than 1e-12 (after such a near tie the paths may
  legitimately diverge);
* at exit both runs pass the oracle's KKT check (b_low - b_up <= 2 tau with f
  recomputed from alpha in FP64), the dual objectives agree within 1e-5
  relative, decision values on held-out points within 1e-3 absolute and
  their signs on at least 99.9% of the points.
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

TIE = 1e-12


def first_mismatch(gpu_trace, ref_trace, ref_margin, n):
    """Index of the first differing pair within the first n steps (n if none);
    asserts that a difference only happens at an oracle near-tie."""
    m = min(n, len(ref_trace))
    assert len(gpu_trace) >= m, (len(gpu_trace), m)
    for t in range(m):
        if gpu_trace[t, 0] != ref_trace[t, 0] or gpu_trace[t, 1] != ref_trace[t, 1]:
            assert ref_margin is not None and ref_margin[t].min() < TIE, \
                f"step {t}: gpu {gpu_trace[t]} oracle {ref_trace[t]} margin {None if ref_margin is None else ref_margin[t]}"
            return t
    return m


def check_end_state(p, r, ref, alpha_tol=None):
    alpha = r["alpha"].cpu().numpy() if hasattr(r["alpha"], "cpu") else r["alpha"]
    kk = oracle.kkt(p.X, p.y, alpha, p.C, p.gamma)
    assert kk["gap"] <= 2 * p.tau + 1e-9, kk["gap"]
    assert abs(kk["objective"] - ref["objective"]) <= 1e-5 * abs(ref["objective"])
    assert (alpha >= 0).all() and (alpha <= p.C).all()
    assert abs((alpha * p.y).sum()) <= 1e-10 * len(alpha) * p.C
    if alpha_tol is not None:
        assert np.abs(alpha - ref["alpha"]).max() <= alpha_tol
    return alpha, kk


def gpu_train(p, **kw):
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, **kw)
    return r, Xd, yd


@pytest.fixture(scope="module")
def c1():
    p = synth.gaussian_mixture()
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=400)
    return p, ref


@pytest.mark.parametrize("flags", [0, pkg.SVM_FLAG_STREAM_ROWS], ids=["resident", "streamed"])
def test_gaussian_mixture_2000_fp64(c1, flags):
    p, ref = c1
    r, Xd, yd = gpu_train(p, trace_len=400, flags=flags)
    assert r["status"] == pkg.SVM_OK
    assert r["stats"]["binary_input"] == 0
    t = first_mismatch(r["trace"], ref["trace"], ref["margin"], 400)
    assert t >= 200
    alpha, kk = check_end_state(p, r, ref)
    if t == 400 and r["iters"] == ref["iters"]:
        assert np.abs(alpha - ref["alpha"]).max() <= 1e-9
    # held-out decision values (10,000 points)
    dz = pkg.svm_decision(Xd, yd, r["alpha"], r["b"], p.gamma, pkg.to_device(p.Z)).cpu().numpy()
    dref = oracle.decision(p.X, p.y, ref["alpha"], ref["b"], p.gamma, p.Z)
    assert np.abs(dz - dref).max() <= 1e-3
    assert (np.sign(dz) == np.sign(dref)).mean() >= 0.999


def test_decision_matches_oracle_for_same_alpha(c1):
    p, ref = c1
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    a = torch.as_tensor(ref["alpha"], device="cuda")
    dz = pkg.svm_decision(Xd, yd, a, ref["b"], p.gamma, pkg.to_device(p.Z)).cpu().numpy()
    dref = oracle.decision(p.X, p.y, ref["alpha"], ref["b"], p.gamma, p.Z)
    assert np.abs(dz - dref).max() <= 1e-10 * max(1.0, np.abs(dref).max())
    # host buffers give the same values
    dh = pkg.svm_decision(p.X, p.y, ref["alpha"], ref["b"], p.gamma, p.Z)
    assert np.array_equal(dh, dz)


@pytest.fixture(scope="module")
def c2():
    p = synth.onehot_sparse()
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=400)
    return p, ref


@pytest.mark.parametrize("flags", [0, pkg.SVM_FLAG_STREAM_ROWS, pkg.SVM_FLAG_CSR_ROWS,
                                   pkg.SVM_FLAG_CSR_ROWS | pkg.SVM_FLAG_STREAM_ROWS],
                         ids=["bits-resident", "bits-streamed", "csr-resident", "csr-streamed"])
def test_onehot_32561_binary_fp64(c2, flags):
    p, ref = c2
    r, Xd, yd = gpu_train(p, trace_len=400, flags=flags)
    assert r["status"] == pkg.SVM_OK
    assert r["stats"]["binary_input"] == 1
    assert r["stats"]["bit_rows"] == int(not flags & pkg.SVM_FLAG_CSR_ROWS)
    t = first_mismatch(r["trace"], ref["trace"], ref["margin"], 400)
    assert t >= 200
    check_end_state(p, r, ref)
    # sampled held-out decision values against the oracle's model
    Zs = p.Z.take(np.arange(0, p.Z.n, 10))
    dz = pkg.svm_decision(Xd, yd, r["alpha"], r["b"], p.gamma, pkg.to_device(Zs)).cpu().numpy()
    dref = oracle.decision(p.X, p.y, ref["alpha"], ref["b"], p.gamma, Zs)
    assert np.abs(dz - dref).max() <= 1e-3
    assert (np.sign(dz) == np.sign(dref)).mean() >= 0.999


@pytest.mark.parametrize("flags", [0, pkg.SVM_FLAG_STREAM_ROWS], ids=["resident", "streamed"])
@pytest.mark.parametrize("binary", [False, True])
def test_ragged_sparse_rows(binary, flags):
    # ragged row lengths including empty rows, several CTAs and a ragged tail
    p = synth.random_sparse(3001, 300, 0.02, seed=5, binary=binary, C=2.0, gamma=0.2)
    assert (np.diff(p.X.indptr) == 0).any()
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=100000)
    r, _, _ = gpu_train(p, trace_len=100000, flags=flags)
    assert r["stats"]["binary_input"] == int(binary)
    assert r["stats"]["resident"] == int(flags == 0)
    t = first_mismatch(r["trace"], ref["trace"], ref["margin"], 100000)
    assert t >= min(200, ref["iters"])
    alpha, _ = check_end_state(p, r, ref)
    if t == ref["iters"] and r["iters"] == ref["iters"]:
        assert np.abs(alpha - ref["alpha"]).max() <= 1e-9


@pytest.mark.parametrize("d", [1, 37, 128, 129, 256, 257])
def test_bit_mask_rows_equal_csr_rows(d):
    """Binary rows read as bit masks (4 words up to d = 128, 8 up to 256) give
    the same steps and the same alpha as the CSR gather and the oracle; d = 257
    falls back to CSR rows. Empty rows, a ragged tail and, at d = 1, many
    duplicate rows (flat curvature) are included."""
    n = 2501
    p = synth.random_sparse(n, d, min(0.5, 6.0 / d), seed=d, binary=True, C=1.5, gamma=0.15)
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=300)
    a, _, _ = gpu_train(p, trace_len=300)
    b, _, _ = gpu_train(p, trace_len=300, flags=pkg.SVM_FLAG_CSR_ROWS)
    assert a["stats"]["bit_rows"] == int(d <= 256) and b["stats"]["bit_rows"] == 0
    assert np.array_equal(a["trace"], b["trace"])
    assert a["iters"] == b["iters"]
    assert np.array_equal(a["alpha"].cpu().numpy(), b["alpha"].cpu().numpy())
    t = first_mismatch(a["trace"], ref["trace"], ref["margin"], 300)
    assert t >= min(200, ref["iters"])
    check_end_state(p, a, ref)


@pytest.mark.parametrize("flags", [0, pkg.SVM_FLAG_CSR_ROWS], ids=["bits", "csr"])
def test_launch_shapes_give_identical_solves(flags):
    """One 16-CTA cluster (no global exchange), clusters of 8 over the whole
    GPU, and no clusters: the selection is exact and each f update is per
    row, so all shapes take the same steps to the same alpha."""
    p = synth.onehot_sparse(n=6000, n_test=0, seed=12)
    kind, value, recon = pkg.POLICIES["Multi5pc"]
    runs = {}
    for name, kw in {"single16": dict(ctas=16), "clusters8": dict(ctas=152),
                     "flat": dict(ctas=152, flags=flags | pkg.SVM_FLAG_NO_CLUSTERS),
                     "auto": dict()}.items():
        kw.setdefault("flags", flags)
        r, _, _ = gpu_train(p, shrink=(kind, value, recon), trace_len=2000, **kw)
        assert r["status"] == pkg.SVM_OK
        runs[name] = r
    assert runs["single16"]["stats"]["cluster_size"] == 16 and runs["single16"]["stats"]["ctas"] == 16
    assert runs["clusters8"]["stats"]["cluster_size"] == 8
    assert runs["flat"]["stats"]["cluster_size"] == 1
    base = runs["single16"]
    for name, r in runs.items():
        assert r["iters"] == base["iters"], name
        assert np.array_equal(r["trace"], base["trace"]), name
        assert np.array_equal(r["alpha"].cpu().numpy(), base["alpha"].cpu().numpy()), name
        assert r["b"] == base["b"], name


@pytest.mark.parametrize("dist,C,gamma", [(1.0, 100.0, 0.5), (3.0, 0.4, 0.1)])
def test_two_points_closed_form(dist, C, gamma):
    X = synth.csr_from_dense(np.array([[0.0], [dist]], dtype=np.float32), keep_zeros=True)
    y = np.array([1, -1], dtype=np.int8)
    r = pkg.svm_train(X, y, C, gamma, 1e-6)
    k = np.exp(-gamma * dist * dist)
    a_star = min(C, 2.0 / (2.0 - 2.0 * k))
    assert r["iters"] == 1
    assert np.allclose(r["alpha"], a_star, rtol=1e-14, atol=0)


def test_duplicate_points_flat_curvature():
    # identical rows make eta = 0 (the end-point rule of the pair step)
    x = np.tile(np.array([[0.5, -1.0, 2.0]], dtype=np.float32), (12, 1))
    x[6:] += 1.0
    X = synth.csr_from_dense(x, keep_zeros=True)
    y = np.array([1, -1] * 6, dtype=np.int8)
    ref = oracle.smo(X, y, 1.0, 0.3, 1e-3, trace_len=1000)
    r = pkg.svm_train(X, y, 1.0, 0.3, 1e-3, trace_len=1000)
    assert r["iters"] == ref["iters"]
    assert np.array_equal(r["trace"], ref["trace"].astype(np.int32))
    assert np.abs(r["alpha"] - ref["alpha"]).max() <= 1e-12


def test_max_iter_reports_not_converged():
    p = synth.small_dense(500, 6, seed=3, C=1.0, gamma=0.1)
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=7)
    r = pkg.svm_train(p.X, p.y, p.C, p.gamma, p.tau, max_iter=7)
    assert r["status"] == pkg.SVM_NOT_CONVERGED and r["iters"] == 7
    assert np.abs(r["alpha"] - ref["alpha"]).max() <= 1e-12


def test_host_and_device_inputs_agree_and_are_deterministic():
    p = synth.random_sparse(2000, 50, 0.2, seed=9, C=1.0, gamma=0.1)
    a = pkg.svm_train(p.X, p.y, p.C, p.gamma, p.tau)
    b, _, _ = gpu_train(p)
    c, _, _ = gpu_train(p)
    assert np.array_equal(a["alpha"], b["alpha"].cpu().numpy())
    assert np.array_equal(b["alpha"].cpu().numpy(), c["alpha"].cpu().numpy())
    assert a["b"] == b["b"] == c["b"]


def test_invalid_inputs_are_rejected():
    p = synth.small_dense(20, 3, seed=1)
    y1 = np.ones(20, dtype=np.int8)
    r = pkg.svm_train(p.X, y1, 1.0, 0.1, 1e-3, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG and "both classes" in pkg.svm_last_error()
    bad = synth.CSR(p.X.n, p.X.d, p.X.indptr.copy(), p.X.indices.copy(), p.X.values.copy())
    bad.indices[0], bad.indices[1] = bad.indices[1], bad.indices[0]
    r = pkg.svm_train(bad, p.y, 1.0, 0.1, 1e-3, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG and "increasing" in pkg.svm_last_error()
    y2 = p.y.copy()
    y2[3] = 0
    r = pkg.svm_train(p.X, y2, 1.0, 0.1, 1e-3, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG and "labels" in pkg.svm_last_error()
    wide = synth.CSR(p.X.n, 2, p.X.indptr, p.X.indices, p.X.values)
    r = pkg.svm_train(wide, p.y, 1.0, 0.1, 1e-3, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG


SHRINK_CASES = ["Single2", "Single500", "Single5pc", "Single50pc", "Multi2", "Multi500",
                "Multi1000", "Multi5pc", "Multi10pc", "Multi50pc", "Single1000", "Single10pc"]


@pytest.fixture(scope="module")
def shrink_problem():
    p = synth.onehot_sparse(n=6000, n_test=0, seed=12)
    plain = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=300)
    return p, plain


@pytest.mark.parametrize("name", SHRINK_CASES)
def test_shrinking_policies_match_oracle(shrink_problem, name):
    p, plain = shrink_problem
    kind, value, recon = pkg.POLICIES[name]
    ref = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, p.tau, kind, value, recon, trace_len=100000,
                            events=100000)
    flags = pkg.SVM_FLAG_STREAM_ROWS if name.startswith("Single") else 0
    r, _, _ = gpu_train(p, shrink=(kind, value, recon), trace_len=100000, flags=flags,
                        active_trace_len=100000)
    assert r["status"] == pkg.SVM_OK
    # pairs: identical to the oracle's shrinking run (near ties excepted via
    # the plain run's margins over the common prefix)
    m = min(len(ref["trace"]), len(r["trace"]))
    diff = np.nonzero((r["trace"][:m] != ref["trace"][:m]).any(axis=1))[0]
    if len(diff) and diff[0] < 200:
        tt = diff[0]
        assert tt < len(plain["margin"]) and plain["margin"][tt].min() < TIE
    if not len(diff) and r["iters"] == ref["iters"]:
        assert r["stats"]["shrink_events"] == ref["n_shrink"]
        assert r["stats"]["reconstructions"] == ref["n_recon"]
        # the schedule itself (Algorithm 4, Table 3): the step of every shrink
        # test and the active-set size after it equal the oracle's, whose
        # schedule is pinned to the definitions on the CPU
        want = np.array([(e["step"], e["active"]) for e in ref["events"] if e["kind"] == 1],
                        dtype=np.int64).reshape(-1, 2)
        assert np.array_equal(r["active_trace"], want)
    check_end_state(p, r, plain)


def test_shrinking_dense_fp64_matches_plain_optimum():
    p = synth.gaussian_mixture(n=3000, n_test=0, seed=21)
    plain = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau)
    for name in ["Multi5pc", "Single500"]:
        kind, value, recon = pkg.POLICIES[name]
        r, _, _ = gpu_train(p, shrink=(kind, value, recon))
        check_end_state(p, r, plain)


# ---------------------------------------------------------------- kernel-row cache
def _cache_pair(p, **kw):
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    on = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, trace_len=2000, **kw)
    off = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, trace_len=2000, cache_mb=-1,
                        **{k: v for k, v in kw.items() if k != "cache_mb"})
    return on, off


def _same(on, off):
    assert on["iters"] == off["iters"]
    assert np.array_equal(on["trace"], off["trace"])
    assert np.array_equal(on["alpha"].cpu().numpy(), off["alpha"].cpu().numpy())
    assert on["b"] == off["b"]
    assert off["stats"]["cache_slots"] == 0


@pytest.mark.parametrize("flags", [0, pkg.SVM_FLAG_STREAM_ROWS], ids=["resident", "streamed"])
def test_kernel_row_cache_direct_is_exact(c1, flags):
    """All n rows cached (direct slots): the solve is bit-for-bit the one
    that recomputes every kernel row, and most rows come from the cache."""
    p, ref = c1
    on, off = _cache_pair(p, flags=flags)
    assert on["stats"]["cache_slots"] == p.X.n
    _same(on, off)
    s = on["stats"]
    assert s["cache_hits"] + s["cache_misses"] == 2 * on["iters"]
    assert s["cache_hits"] > s["cache_misses"]
    check_end_state(p, on, ref)


@pytest.mark.parametrize("precision", [pkg.SVM_FP64, pkg.SVM_MIXED_BF16_SIMT], ids=["fp64", "mixed"])
@pytest.mark.parametrize("shrink", [None, "Multi5pc"])
def test_kernel_row_cache_with_evictions_is_exact(precision, shrink):
    """A cache far smaller than n rows (4-way sets, least recently used way
    evicted), with and without shrinking, FP64 and mixed rows: identical to
    the solve without a cache."""
    p = synth.covtype_like(n=12000, n_test=0, seed=17)
    pol = pkg.POLICIES[shrink] if shrink else None
    on, off = _cache_pair(p, precision=precision, shrink=pol, cache_mb=8)
    s = on["stats"]
    assert 64 <= s["cache_slots"] < p.X.n
    assert s["cache_misses"] > s["cache_slots"]          # rows were evicted and recomputed
    assert s["cache_hits"] > 0
    _same(on, off)


# ---------------------------------------------------------------- other kernels
KERNELS = [(pkg.SVM_KERNEL_LINEAR, 0.0, 1), (pkg.SVM_KERNEL_POLY, 1.0, 3),
           (pkg.SVM_KERNEL_SIGMOID, -1.0, 0)]


@pytest.mark.parametrize("kind,c0,deg", KERNELS, ids=["linear", "poly3", "sigmoid"])
@pytest.mark.parametrize("binary", [False, True], ids=["dense", "binary"])
def test_other_kernels_match_oracle(kind, c0, deg, binary):
    """Linear, polynomial and sigmoid kernels (FP64): pairs as the oracle's,
    the oracle's KKT check and objective, decision values; binary inputs take
    the general path with explicit unit values."""
    if binary:
        p = synth.random_sparse(1500, 60, 0.1, seed=61, binary=True, C=1.0, gamma=0.05)
        Z = synth.random_sparse(500, 60, 0.1, seed=62, binary=True).X
    else:
        p = synth.gaussian_mixture(n=1500, n_test=500, seed=63)
        Z = p.Z
    with oracle.kernel_spec(kind, c0, deg):
        ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=300, max_iter=200000)
        assert ref["status"] == 0
        r, Xd, yd = gpu_train(p, trace_len=300, kernel=kind, degree=deg, coef0=c0)
        assert r["status"] == pkg.SVM_OK
        assert r["stats"]["binary_input"] == 0
        t = first_mismatch(r["trace"], ref["trace"], ref["margin"], 300)
        assert t >= min(200, ref["iters"])
        check_end_state(p, r, ref)
        dz = pkg.svm_decision(Xd, yd, r["alpha"], r["b"], p.gamma, pkg.to_device(Z), kernel=kind,
                              degree=deg, coef0=c0).cpu().numpy()
        dref = oracle.decision(p.X, p.y, ref["alpha"], ref["b"], p.gamma, Z)
    assert np.abs(dz - dref).max() <= 1e-3 * max(1.0, np.abs(dref).max())
    assert (np.sign(dz) == np.sign(dref)).mean() >= 0.999


@pytest.mark.parametrize("kind,c0,deg", KERNELS[:2], ids=["linear", "poly3"])
def test_other_kernels_mixed_precision(kind, c0, deg):
    """The mixed row pass with another kernel reaches the FP64 optimum within
    the perturbation of BF16 values."""
    p = synth.gaussian_mixture(n=1500, n_test=0, seed=64)
    with oracle.kernel_spec(kind, c0, deg):
        ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=200000)
        r, _, _ = gpu_train(p, kernel=kind, degree=deg, coef0=c0, precision=pkg.SVM_MIXED_BF16)
        assert r["status"] == pkg.SVM_OK
        kk = oracle.kkt(p.X, p.y, r["alpha"].cpu().numpy(), p.C, p.gamma)
    assert abs(kk["objective"] - ref["objective"]) <= 2e-3 * abs(ref["objective"])


def test_kernel_arguments_are_checked():
    p = synth.small_dense(20, 3, seed=1)
    r = pkg.svm_train(p.X, p.y, 1.0, 0.1, 1e-3, kernel=9, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG and "kernel" in pkg.svm_last_error()
    r = pkg.svm_train(p.X, p.y, 1.0, 0.1, 1e-3, kernel=pkg.SVM_KERNEL_POLY, degree=0, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG and "degree" in pkg.svm_last_error()


def test_active_set_trajectory():
    """svm_params.active_trace: (step, active rows) after each shrink event of
    Eq. (shrink): one row per event, steps increasing, sizes within [2, n],
    shrinking between reconstructions, and the counts the kernel reports."""
    p = synth.onehot_sparse(n=6000, n_test=0, seed=12)
    kind, value, recon = pkg.POLICIES["Multi5pc"]
    r, _, _ = gpu_train(p, shrink=(kind, value, recon), active_trace_len=1000)
    at = r["active_trace"]
    s = r["stats"]
    assert len(at) == s["shrink_events"] >= 2
    assert (np.diff(at[:, 0]) > 0).all() and at[-1, 0] <= r["iters"]
    assert (at[:, 1] >= 2).all() and (at[:, 1] <= p.X.n).all()
    # between two reconstructions the active set only shrinks
    rises = int((np.diff(at[:, 1]) > 0).sum())
    assert rises <= s["reconstructions"]
    # the same solve without a trajectory buffer
    r2, _, _ = gpu_train(p, shrink=(kind, value, recon))
    assert r2["iters"] == r["iters"]
    assert np.array_equal(r2["alpha"].cpu().numpy(), r["alpha"].cpu().numpy())
