"""Batched training (svm_train_batch): one persistent launch, jobs from a
device work-list, each job solved by one thread-block cluster.

Each job's result must be the result of the same subproblem trained alone
with svm_train at the same precision (the batched form changes where the
work runs, not what it computes), and, in FP64, pass the oracle's checks."""
import numpy as np
import pytest

import oracle
import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


def ovo_jobs(mc, tau=1e-3):
    jobs = []
    for a, b in mc.ovo_pairs():
        rows, y = mc.subproblem(a, b)
        for C in mc.Cs:
            for g in mc.gammas:
                jobs.append({"rows": rows.astype(np.int32), "y": y, "C": C, "gamma": g, "tau": tau})
    return jobs


def dev_jobs(jobs):
    return [dict(j, rows=torch.as_tensor(j["rows"], device="cuda"),
                 y=torch.as_tensor(j["y"], device="cuda")) for j in jobs]


@pytest.fixture(scope="module")
def small_mc():
    mc = synth.multiclass(n=2400, d=16, classes=4, seed=41, mean_sd=0.6, Cs=(0.5, 2.0),
                          gammas=(0.05, 0.2))
    return mc, ovo_jobs(mc)


def alone(mc, job, precision):
    Xs = mc.X.take(job["rows"])
    return pkg.svm_train(Xs, job["y"], job["C"], job["gamma"], job["tau"], precision=precision)


@pytest.mark.parametrize("precision", [pkg.SVM_FP64, pkg.SVM_MIXED_BF16])
def test_batch_equals_jobs_alone(small_mc, precision):
    mc, jobs = small_mc
    out = pkg.svm_train_batch(pkg.to_device(mc.X), dev_jobs(jobs), precision=precision)
    assert out["status"] == pkg.SVM_OK
    assert out["cluster_size"] >= 1 and out["lanes_per_row"] >= 1
    for job, r in zip(jobs, out["results"]):
        ref = alone(mc, job, precision)
        assert r["status"] == pkg.SVM_OK
        w_ref = ref["stats"]["objective"]
        assert abs(r["objective"] - w_ref) <= 1e-7 * abs(w_ref), (r["objective"], w_ref)
        a = r["alpha"].cpu().numpy()
        assert (a >= 0).all() and (a <= job["C"]).all()
        assert abs((a * job["y"]).sum()) <= 1e-10 * len(a) * job["C"]


def test_batch_fp64_passes_oracle_checks(small_mc):
    mc, jobs = small_mc
    out = pkg.svm_train_batch(mc.X, jobs[:6], precision=pkg.SVM_FP64)   # host buffers
    for job, r in zip(jobs[:6], out["results"]):
        Xs = mc.X.take(job["rows"])
        ref = oracle.smo(Xs, job["y"], job["C"], job["gamma"], job["tau"])
        kk = oracle.kkt(Xs, job["y"], r["alpha"], job["C"], job["gamma"])
        assert kk["gap"] <= 2 * job["tau"] + 1e-9
        assert abs(kk["objective"] - ref["objective"]) <= 1e-5 * abs(ref["objective"])
        assert abs(r["b"] - kk["b"]) <= 1e-6


def test_batch_binary_rows_and_uneven_jobs():
    p = synth.onehot_sparse(n=4000, n_test=0, seed=43)
    rng = np.random.default_rng(1)
    jobs = []
    for k, m in enumerate([500, 1200, 3999, 57, 2500]):
        rows = np.sort(rng.choice(p.X.n, m, replace=False)).astype(np.int32)
        y = p.y[rows].copy()
        if (y > 0).all() or (y < 0).all():
            y[0] = -y[0]
        jobs.append({"rows": rows, "y": y, "C": [1.0, 0.3, 2.0, 1.0, 0.7][k], "gamma": 0.05, "tau": 1e-3})
    jobs.append({"rows": None, "y": p.y.copy(), "C": 1.0, "gamma": 0.1, "tau": 1e-3})
    out = pkg.svm_train_batch(pkg.to_device(p.X), dev_jobs([dict(j, rows=(j["rows"] if j["rows"] is not None else np.arange(p.X.n, dtype=np.int32))) for j in jobs]))
    for job, r in zip(jobs, out["results"]):
        rows = job["rows"] if job["rows"] is not None else np.arange(p.X.n)
        Xs = p.X.take(rows)
        ref = pkg.svm_train(Xs, job["y"], job["C"], job["gamma"], job["tau"])
        assert abs(r["objective"] - ref["stats"]["objective"]) <= 1e-7 * abs(ref["stats"]["objective"])


def test_autotune_returns_a_valid_shape(small_mc):
    mc, jobs = small_mc
    t = pkg.svm_batch_autotune(pkg.to_device(mc.X), dev_jobs(jobs), precision=pkg.SVM_MIXED_BF16)
    assert t["cluster_size"] in (1, 2, 4, 8, 16)
    assert t["lanes_per_row"] in (1, 2, 4, 8, 16, 32)
    out = pkg.svm_train_batch(pkg.to_device(mc.X), dev_jobs(jobs), precision=pkg.SVM_MIXED_BF16,
                              cluster_size=t["cluster_size"], lanes_per_row=t["lanes_per_row"])
    assert out["status"] == pkg.SVM_OK


def test_batch_argument_errors(small_mc):
    mc, jobs = small_mc
    bad = [dict(jobs[0], y=np.ones_like(jobs[0]["y"]))]
    r = pkg.svm_train_batch(mc.X, bad, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG and "both classes" in pkg.svm_last_error()
    bad = [dict(jobs[0], rows=jobs[0]["rows"] + 10**6)]
    r = pkg.svm_train_batch(mc.X, bad, check=False)
    assert r["status"] == pkg.SVM_ERR_ARG


@pytest.mark.parametrize("lanes", [1, 2, 8, 32])
@pytest.mark.parametrize("cluster", [1, 4])
def test_batch_launch_shapes_agree(small_mc, lanes, cluster):
    # every launch shape (including the register-blocked dense row pass at
    # 32 lanes) computes the same per-job solves
    mc, jobs = small_mc
    sub = jobs[:8]
    out = pkg.svm_train_batch(pkg.to_device(mc.X), dev_jobs(sub), precision=pkg.SVM_MIXED_BF16,
                              cluster_size=cluster, lanes_per_row=lanes)
    assert out["cluster_size"] == cluster and out["lanes_per_row"] == lanes
    for job, r in zip(sub, out["results"]):
        ref = alone(mc, job, pkg.SVM_MIXED_BF16)
        w = ref["stats"]["objective"]
        assert abs(r["objective"] - w) <= 1e-7 * abs(w)


def test_batch_tensor_core_tiles_match_alone():
    """Dense BF16 rows with d a multiple of 32 at 16 lanes per row run on the
    tensor cores (mma m16n8k16 tiles of 16 rows x the two targets, FP32
    accumulation in another order than the CUDA-core sums of svm_train):
    each job's objective equals the job trained alone within 1e-5 relative,
    the tolerance the batched form is held to, and its box and equality
    constraints hold."""
    mc = synth.multiclass(n=2400, d=64, classes=3, seed=43, mean_sd=0.6, Cs=(0.5, 2.0),
                          gammas=(0.02, 0.1))
    jobs = ovo_jobs(mc)
    out = pkg.svm_train_batch(pkg.to_device(mc.X), dev_jobs(jobs), precision=pkg.SVM_MIXED_BF16,
                              cluster_size=2, lanes_per_row=16)
    assert out["status"] == pkg.SVM_OK and out["lanes_per_row"] == 16
    for job, r in zip(jobs, out["results"]):
        assert r["status"] == pkg.SVM_OK
        w = alone(mc, job, pkg.SVM_MIXED_BF16)["stats"]["objective"]
        assert abs(r["objective"] - w) <= 1e-5 * abs(w), (r["objective"], w)
        a = r["alpha"].cpu().numpy()
        assert (a >= 0).all() and (a <= job["C"]).all()
        assert abs((a * job["y"]).sum()) <= 1e-10 * len(a) * job["C"]
