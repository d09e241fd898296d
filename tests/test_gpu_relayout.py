"""GPU tests of the active-set re-layout (through the C ABI).

With shrinking (Eq. shrink, Algorithms 4-5), a launch over a problem that is
not already one on-chip cluster ends once fewer than three quarters of its
rows are active; the active rows are gathered in index order into a smaller problem
that gets its own launch shape, and the state is scattered back when that
launch ends. Rows keep their order, so the lowest-index tie-break of Eq.
(bminmax) and every step's arithmetic are unchanged: a solve with the
re-layout must equal the solve without it (SVM_FLAG_NO_RELAYOUT) bit for bit,
pair trace, alpha and b. The unrelaid solves are checked against the oracle
in test_gpu_smo.py; here the end state is also checked with the oracle's
KKT test.
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

NO_RELAYOUT = pkg.SVM_FLAG_NO_RELAYOUT


def _pair(p, trace_len, **kw):
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    flags = kw.pop("flags", 0)
    a = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, trace_len=trace_len, flags=flags, active_trace_len=4096, **kw)
    b = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, trace_len=trace_len, flags=flags | NO_RELAYOUT,
                      active_trace_len=4096, **kw)
    return a, b


def _same(a, b):
    assert a["status"] == b["status"] == pkg.SVM_OK
    assert a["iters"] == b["iters"]
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["alpha"].cpu().numpy(), b["alpha"].cpu().numpy())
    assert a["b"] == b["b"]
    assert a["stats"]["shrink_events"] == b["stats"]["shrink_events"]
    assert a["stats"]["reconstructions"] == b["stats"]["reconstructions"]
    assert a["stats"]["row_visits"] == b["stats"]["row_visits"]
    assert b["stats"]["relayouts"] == 0
    # the active-set trajectory (|pi| after each shrink event) is the same too
    assert np.array_equal(a["active_trace"], b["active_trace"])
    assert len(a["active_trace"]) == min(4096, a["stats"]["shrink_events"])


def _kkt(p, r):
    kk = oracle.kkt(p.X, p.y, r["alpha"].cpu().numpy(), p.C, p.gamma)
    assert kk["gap"] <= 2 * p.tau + 1e-9


def _problem(name):
    if name == "bits":
        return synth.onehot_sparse(n=6000, n_test=0, seed=12), {}
    if name == "csr-binary":
        return synth.onehot_sparse(n=6000, n_test=0, seed=12), {"flags": pkg.SVM_FLAG_CSR_ROWS}
    if name == "dense-fp64":
        return synth.gaussian_mixture(n=5000, n_test=0, seed=21), {}
    if name == "dense-mixed":
        return synth.gaussian_mixture(n=5000, n_test=0, seed=21), {"precision": pkg.SVM_MIXED_BF16}
    if name == "dense-mixed-tiles":
        return synth.gaussian_mixture(n=5000, n_test=0, d=64, seed=22, gamma=0.01), {
            "precision": pkg.SVM_MIXED_BF16, "flags": pkg.SVM_FLAG_TENSOR_ROWS}
    if name == "ragged":
        return synth.random_sparse(6001, 300, 0.02, seed=5, binary=False, C=10.0, gamma=0.05), {}
    raise KeyError(name)


@pytest.mark.parametrize("policy", ["Multi5pc", "Multi2", "Single5pc"])
@pytest.mark.parametrize("name", ["bits", "csr-binary", "dense-fp64", "dense-mixed", "dense-mixed-tiles", "ragged"])
def test_relayout_is_the_same_solve(name, policy):
    """Clusters of 8 over the GPU (ctas=152), so that the re-layout engages."""
    p, kw = _problem(name)
    a, b = _pair(p, 100000, shrink=pkg.POLICIES[policy], ctas=152, **kw)
    _same(a, b)
    assert a["stats"]["relayouts"] >= 1
    if kw.get("precision", pkg.SVM_FP64) == pkg.SVM_FP64:
        _kkt(p, a)   # (mixed precision is checked against FP64 in test_gpu_mixed.py)


@pytest.mark.parametrize("name", ["bits", "dense-mixed", "ragged"])
def test_relayout_streamed_and_flat(name):
    """Streamed segments at every level, and the exchange without clusters."""
    p, kw = _problem(name)
    flags = kw.pop("flags", 0)
    for extra in (pkg.SVM_FLAG_STREAM_ROWS, pkg.SVM_FLAG_NO_CLUSTERS):
        a, b = _pair(p, 100000, shrink=pkg.POLICIES["Multi5pc"], ctas=152, flags=flags | extra, **kw)
        _same(a, b)
        assert a["stats"]["relayouts"] >= 1


def test_relayout_with_second_order_selection_and_row_cache():
    p, _ = _problem("dense-fp64")
    a, b = _pair(p, 100000, shrink=pkg.POLICIES["Multi5pc"], ctas=152, flags=pkg.SVM_FLAG_WSS2)
    _same(a, b)
    assert a["stats"]["relayouts"] >= 1
    # FP64 rows keep the kernel-row cache (automatic) across levels
    a, b = _pair(p, 100000, shrink=pkg.POLICIES["Multi5pc"], ctas=152, cache_mb=64)
    _same(a, b)
    assert a["stats"]["relayouts"] >= 1 and a["stats"]["cache_slots"] > 0


def test_relayout_automatic_shape():
    """A covtype-shaped problem too large for one on-chip cluster: the
    automatic shape starts on clusters of 8 and moves to a single cluster
    once the active set has shrunk."""
    p = synth.covtype_like(n=60000, n_test=0, seed=9)
    a, b = _pair(p, 3000, shrink=pkg.POLICIES["Multi5pc"], precision=pkg.SVM_MIXED_BF16)
    assert a["stats"]["cluster_size"] == 8
    _same(a, b)
    assert a["stats"]["relayouts"] >= 1


def test_no_relayout_without_shrinking_or_for_one_cluster():
    p, _ = _problem("bits")
    a, b = _pair(p, 10, ctas=152)
    _same(a, b)
    assert a["stats"]["relayouts"] == 0
    a, b = _pair(p, 10, shrink=pkg.POLICIES["Multi5pc"])
    assert a["stats"]["cluster_size"] == 16
    _same(a, b)
    assert a["stats"]["relayouts"] == 0


@pytest.mark.timeout(600)
def test_automatic_shape_with_relayout_against_the_oracle():
    """FP64, 40,000 covtype-shaped rows: the automatic shape starts on
    clusters of 8 with on-chip segments and, as shrinking proceeds, moves
    through re-laid-out levels to one cluster. Against the oracle (plain
    Algorithm 1): the first 200 pairs (the first shrink test comes later),
    and the end state under the oracle's KKT check and objective."""
    from test_gpu_smo import check_end_state, first_mismatch
    p = synth.covtype_like(n=40000, n_test=0, seed=9)
    oracle.set_threads(oracle.max_threads())
    ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, trace_len=300)
    assert ref["status"] == 0
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, shrink=pkg.POLICIES["Multi5pc"], trace_len=300)
    assert r["status"] == pkg.SVM_OK
    assert r["stats"]["cluster_size"] == 8 and r["stats"]["relayouts"] >= 1
    t = first_mismatch(r["trace"], ref["trace"], ref.get("margin"), 300)
    assert t >= 200
    check_end_state(p, r, ref)


@pytest.mark.parametrize("prec,name,flags", [(pkg.SVM_FP64, "Multi500", 0), (pkg.SVM_FP64, "Multi5pc", 0),
                                             (pkg.SVM_MIXED_BF16_SIMT, "Multi500", pkg.SVM_FLAG_STREAM_ROWS)])
def test_incremental_reconstruction_matches_full_sum(prec, name, flags):
    """After a multiple-reconstruction restart the rows shrunk when the active
    rows are gathered are reconstructed as their f at that moment plus the sum
    over the gathered rows whose alpha changed since (Algorithm 6's sum less
    the unchanged terms): the solve matches the one with Algorithm 6's full
    sum (SVM_FLAG_FULL_RECON) up to rounding order, and in FP64 passes the
    oracle's KKT check (a mixed-precision solve is optimal for the
    BF16-rounded kernel, not for the oracle's)."""
    p = synth.covtype_like(n=40000, n_test=0, seed=17)
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    pol = pkg.POLICIES[name]
    a = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=prec, shrink=pol, flags=flags)
    b = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, precision=prec, shrink=pol,
                      flags=flags | pkg.SVM_FLAG_FULL_RECON)
    assert a["status"] == b["status"] == pkg.SVM_OK
    assert a["stats"]["incremental_recons"] >= 1 and b["stats"]["incremental_recons"] == 0
    assert a["stats"]["reconstructions"] == b["stats"]["reconstructions"]
    wa, wb = a["stats"]["objective"], b["stats"]["objective"]
    assert abs(wa - wb) <= 1e-9 * abs(wb)
    assert abs(a["b"] - b["b"]) <= 1e-6
    if prec == pkg.SVM_FP64:
        _kkt(p, a)
