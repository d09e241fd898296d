"""Failure handling on the GPU without a fault (through the C ABI).

Every wait of the fused step on another CTA is bounded: after its limit of
%globaltimer it gives up, the kernel records the error and returns, and the
call reports SVM_ERR_TIMEOUT with the context still usable. Here the same
bounded wait runs on a barrier that nothing completes (svm_diag_wait_timeout):
it must give up after its limit, not before and not much after, and a
training right afterwards must succeed on the same context.
"""
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


@pytest.mark.parametrize("limit_ms", [20, 200])
def test_wait_that_runs_out_returns_timeout_and_context_stays_usable(limit_ms):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = pkg.svm_diag_wait_timeout(limit_ms * 1_000_000)
    dt = time.perf_counter() - t0
    assert rc == pkg.SVM_ERR_TIMEOUT
    assert "limit" in pkg.svm_last_error()
    assert limit_ms / 1e3 <= dt <= limit_ms / 1e3 + 2.0
    # the context still trains, and correctly
    p = synth.gaussian_mixture(n=500, n_test=0, seed=61)
    r = pkg.svm_train(p.X, p.y, p.C, p.gamma, p.tau)
    assert r["status"] == pkg.SVM_OK
    kk = oracle.kkt(p.X, p.y, np.asarray(r["alpha"]), p.C, p.gamma)
    assert kk["gap"] <= 2 * p.tau + 1e-9


def test_wait_limits_are_checked():
    assert pkg.svm_diag_wait_timeout(10) == pkg.SVM_ERR_ARG
    assert pkg.svm_diag_wait_timeout(10**10) == pkg.SVM_ERR_ARG


def test_sfu_rate_microbenchmark_is_plausible():
    """svm_diag_sfu_rate: ex2.approx instructions per second over the device,
    within a factor of the nominal 16 per clock per SM."""
    r = pkg.svm_diag_sfu_rate()
    props = torch.cuda.get_device_properties(0)
    nominal = 16.0 * props.multi_processor_count * 2.1e9
    assert 0.2 * nominal <= r <= 2.0 * nominal, (r, nominal)
