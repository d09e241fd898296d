"""Serving: jobs of different n and d submitted over time run concurrently on
the device (continuous batching) under a device-memory budget.

The key property: a job's result is the same alone and in the mix (the
engine computes each job independently and deterministically), and equals
svm_train on the same job at the same precision within the tolerance."""
import time

import numpy as np
import pytest

import oracle
import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)


def mixed_jobs(k, seed=7, nmax=3000):
    specs = synth.serving_stream(n_jobs=k, seed=seed, n_range=(400, nmax), d_range=(16, 300))
    return [synth.serving_job(s) for s in specs]


@pytest.fixture(scope="module")
def jobs():
    return mixed_jobs(10)


def test_same_alone_and_in_mix(jobs):
    with pkg.Server(budget_bytes=2 << 30, max_slots=16) as srv:
        alone = []
        for p in jobs:
            t = srv.submit(p.X, p.y, p.C, p.gamma, p.tau)
            alone.append(srv.wait(t))
        t0, tickets, sub = time.perf_counter(), [], []
        for p in jobs:
            sub.append(1e3 * (time.perf_counter() - t0))
            tickets.append(srv.submit(p.X, p.y, p.C, p.gamma, p.tau))
        mix = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["bytes_in_use"] == 0 and st["running"] == 0
    # the jobs of the mix really ran at the same time: admission-to-done
    # intervals (host clock) of at least two jobs overlap
    spans = [(s + m["queue_ms"], s + m["time_to_model_ms"]) for s, m in zip(sub, mix)]
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1])
    assert overlaps >= 1, spans
    for p, a, m in zip(jobs, alone, mix):
        assert a["status"] == pkg.SVM_OK and m["status"] == pkg.SVM_OK
        # identical computation alone and in the mix
        assert a["iters"] == m["iters"]
        assert np.array_equal(a["alpha"], m["alpha"]) and a["b"] == m["b"]
        # and the job's solve: svm_train alone at the same precision
        ref = pkg.svm_train(p.X, p.y, p.C, p.gamma, p.tau, precision=pkg.SVM_MIXED_BF16)
        w = ref["stats"]["objective"]
        assert abs(m["objective"] - w) <= 1e-5 * abs(w)


def test_fp64_server_matches_oracle():
    ps = mixed_jobs(4, seed=8, nmax=1200)
    with pkg.Server(budget_bytes=1 << 30, precision=pkg.SVM_FP64) as srv:
        tickets = [srv.submit(p.X, p.y, p.C, p.gamma, p.tau) for p in ps]
        outs = [srv.wait(t) for t in tickets]
    for p, o in zip(ps, outs):
        assert o["status"] == pkg.SVM_OK
        kk = oracle.kkt(p.X, p.y, o["alpha"], p.C, p.gamma)
        ref = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau)
        assert kk["gap"] <= 2 * p.tau + 1e-9
        assert abs(kk["objective"] - ref["objective"]) <= 1e-5 * abs(ref["objective"])


def test_budget_admission_and_rejection(jobs):
    sizes = [p.X.n * p.X.d for p in jobs]
    big = jobs[int(np.argmax(sizes))]
    # a budget that holds the largest job but not all jobs at once
    with pkg.Server(budget_bytes=1 << 30, max_slots=2) as srv:
        tickets = [srv.submit(p.X, p.y, p.C, p.gamma, p.tau) for p in jobs]
        seen_queue = False
        for _ in range(200):
            s = srv.stats()
            assert s["running"] <= 2 and s["bytes_in_use"] <= s["budget_bytes"]
            seen_queue |= s["queued"] > 0
            time.sleep(0.002)
        outs = [srv.wait(t) for t in tickets]
    assert seen_queue
    assert all(o["status"] == pkg.SVM_OK for o in outs)
    with pkg.Server(budget_bytes=4096) as srv:
        rc = srv.submit(big.X, big.y, big.C, big.gamma, check=False)
        assert rc == pkg.SVM_ERR_BUDGET and "budget" in pkg.svm_last_error()


def test_cancel_and_bad_job(jobs):
    with pkg.Server(budget_bytes=1 << 30, max_slots=1) as srv:
        tickets = [srv.submit(p.X, p.y, p.C, p.gamma, p.tau) for p in jobs[:3]]
        assert srv.cancel(tickets[2]) == pkg.SVM_OK
        outs = [srv.wait(t) for t in tickets]
        assert outs[0]["status"] == pkg.SVM_OK and outs[1]["status"] == pkg.SVM_OK
        assert outs[2]["status"] == pkg.SVM_ERR_CANCELLED
        p = jobs[0]
        y = p.y.copy()
        y[:] = 1
        t = srv.submit(p.X, y, p.C, p.gamma, p.tau)
        o = srv.wait(t)
        assert o["status"] == pkg.SVM_ERR_ARG and "both classes" in o["error"]
