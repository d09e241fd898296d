"""Checks that pin the FP64 oracle to facts outside itself.

Each check takes an oracle build (``lib``; None = the default build) and
raises AssertionError on failure. ``tests/test_oracle_pins.py`` runs them on
the real oracle; ``tests/test_oracle_mutants.py`` runs them on copies of the
oracle with a planted mistake and requires at least one to fail.

What each check compares against:
* closed forms: the two-point problem (alpha = min(C, 2 / (2 - 2k)), k the
  kernel value) and the RBF kernel of known distances;
* a brute-force exact solver of the dual QP (``qp_reference``) for n <= 12;
* invariants that hold for any correct SMO run: sum y alpha = 0, box
  constraints, monotone dual objective, maintained f equal to Eq. (fcache)
  recomputed densely with numpy, KKT gap at exit;
* numpy dense inner products and Gram matrices;
* structural facts: shrinking does not change the optimum; with a correct
  shrink rule the shrunk run selects the same pairs as the plain run until
  late in the run; the first pair at alpha = 0 is (lowest index with y = +1,
  lowest index with y = -1) by Eq. (bminmax).
"""
import numpy as np

import oracle
from paper_1406_5161_gb300 import synth
import os as _os, sys as _sys
_sys.path.insert(0, _os.path.dirname(__file__))
from qp_reference import dual_bruteforce, dual_objective, kernel_matrix, rbf_matrix


# every run is capped: a wrong oracle may never converge
MAXIT = 200000


def _dense(X):
    return X.to_dense().astype(np.float64)


def check_dot_and_norm(lib=None):
    p = synth.random_sparse(40, 30, 0.3, seed=11, min_nnz=1)
    D = _dense(p.X)
    for i in range(0, 40, 3):
        for j in range(0, 40, 7):
            ref = D[i] @ D[j]
            got = oracle.dot(p.X, i, p.X, j, lib=lib)
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (i, j, got, ref)
        assert abs(oracle.sqnorm(p.X, i, lib=lib) - D[i] @ D[i]) <= 1e-12 * max(1, D[i] @ D[i])


def check_kernel_closed_form(lib=None):
    # K(x,z) = exp(-g ||x-z||^2): distance 2 from norms 1, 3 and dot 1
    for g in (0.05, 0.5, 2.0):
        got = oracle.kernel(g, 1.0, 3.0, 1.0, lib=lib)
        assert abs(got - np.exp(-2.0 * g)) <= 1e-15, (g, got)
        assert oracle.kernel(g, 2.0, 2.0, 2.0, lib=lib) == 1.0
        # rounding below zero is clamped
        assert oracle.kernel(g, 1.0, 1.0, 1.0 + 1e-15, lib=lib) == 1.0


def _two_point(dist, C, gamma):
    x = np.array([[0.0], [dist]], dtype=np.float32)
    X = synth.csr_from_dense(x, keep_zeros=True)
    y = np.array([1, -1], dtype=np.int8)
    return X, y


def check_two_point_closed_form(lib=None):
    for dist, C, gamma in [(1.0, 100.0, 0.5), (0.25, 100.0, 1.0), (3.0, 0.4, 0.1),
                           (2.0, 1.0, 0.05), (0.5, 5.0, 0.3)]:
        X, y = _two_point(dist, C, gamma)
        k = np.exp(-gamma * float(np.float32(dist)) ** 2)
        a_star = min(C, 2.0 / (2.0 - 2.0 * k))
        r = oracle.smo(X, y, C, gamma, 1e-6, max_iter=10, lib=lib)
        assert r["iters"] == 1, r["iters"]
        assert np.allclose(r["alpha"], a_star, rtol=1e-14, atol=0), (r["alpha"], a_star)
        if a_star < C:
            assert np.abs(r["f"]).max() <= 1e-13
            assert abs(r["b"]) <= 1e-13
        else:
            # both at C: b is the midpoint of b_up = f_2 and b_low = f_1
            f1 = C * (1 - k) - 1.0
            assert abs(r["f"][0] - f1) <= 1e-13 and abs(r["f"][1] + f1) <= 1e-13
            assert abs(r["b"]) <= 1e-13


def _tiny(n, seed, C, d=3, gamma=0.5):
    p = synth.small_dense(n, d, seed, sep=0.3, C=C, gamma=gamma, tau=1e-10)
    return p


def check_bruteforce(lib=None, cases=((4, 1, 1.0), (6, 2, 0.5), (7, 3, 10.0),
                                      (8, 4, 1.0), (9, 5, 2.0))):
    for n, seed, C in cases:
        p = _tiny(n, seed, C)
        D = _dense(p.X)
        K = rbf_matrix(D, D, p.gamma)
        w_star, a_star = dual_bruteforce(K, p.y.astype(np.float64), C)
        r = oracle.smo(p.X, p.y, C, p.gamma, 1e-10, max_iter=MAXIT, lib=lib)
        w = dual_objective(r["alpha"], p.y.astype(np.float64), K)
        assert abs(w - w_star) <= 1e-9 * max(1.0, abs(w_star)), (n, seed, w, w_star)
        assert np.abs(r["alpha"] - a_star).max() <= 1e-6, (n, seed, r["alpha"], a_star)
        assert abs(r["objective"] - w_star) <= 1e-9 * max(1.0, abs(w_star))


def check_invariants(lib=None):
    for seed, C, gamma in [(21, 1.0, 0.1), (22, 0.3, 0.5), (23, 5.0, 0.05)]:
        p = synth.small_dense(60, 4, seed, sep=0.4, C=C, gamma=gamma, tau=1e-4)
        D = _dense(p.X)
        K = rbf_matrix(D, D, gamma)
        y = p.y.astype(np.float64)
        r = oracle.smo(p.X, p.y, C, gamma, 1e-4, max_iter=MAXIT, trace_len=MAXIT,
                       record_objective=True, lib=lib)
        a = r["alpha"]
        assert r["status"] == 0
        assert abs(y @ a) <= 1e-12 * len(a) * C
        assert (a >= 0).all() and (a <= C).all()
        objs = r["objectives"]
        assert (np.diff(objs) >= -1e-12 * np.abs(objs[1:]).max()).all(), "objective decreased"
        # maintained f equals Eq. (fcache) from scratch (dense numpy)
        f_ref = K @ (a * y) - y
        assert np.abs(r["f"] - f_ref).max() <= 1e-10 * max(1.0, np.abs(f_ref).max())
        # objective equals the dual objective of alpha (numpy)
        assert abs(r["objective"] - dual_objective(a, y, K)) <= 1e-10 * max(1.0, abs(r["objective"]))
        # KKT at exit over all samples, from the recomputed f
        up = ((a > 0) & (a < C)) | ((y > 0) & (a == 0)) | ((y < 0) & (a == C))
        low = ((a > 0) & (a < C)) | ((y > 0) & (a == C)) | ((y < 0) & (a == 0))
        assert f_ref[low].max() - f_ref[up].min() <= 2e-4 + 1e-12
        # the first pair at alpha = 0 follows Eq. (bminmax) with lowest index
        assert r["trace"][0, 0] == int(np.nonzero(p.y > 0)[0][0])
        assert r["trace"][0, 1] == int(np.nonzero(p.y < 0)[0][0])
        # threshold: mean of f over the free set
        free = (a > 0) & (a < C)
        if free.any():
            assert abs(r["b"] - f_ref[free].mean()) <= 1e-10


def check_gradient_and_decision(lib=None):
    p = synth.random_sparse(80, 25, 0.25, seed=31, min_nnz=1, C=2.0, gamma=0.2)
    r = oracle.smo(p.X, p.y, p.C, p.gamma, 1e-3, max_iter=MAXIT, lib=lib)
    assert r["status"] == 0
    D = _dense(p.X)
    K = rbf_matrix(D, D, p.gamma)
    y = p.y.astype(np.float64)
    a = r["alpha"]
    g = oracle.gradient(p.X, p.y, a, p.gamma, lib=lib)
    assert np.abs(g - (K @ (a * y) - y)).max() <= 1e-12 * max(1, np.abs(g).max())
    # Algorithm 6 on a subset equals the definition; other entries kept
    rows = np.arange(0, 80, 5)
    f_in = np.full(80, 7.0)
    fr = oracle.reconstruct(p.X, p.y, a, p.gamma, rows, f_in, lib=lib)
    assert np.abs(fr[rows] - (K @ (a * y) - y)[rows]).max() <= 1e-12
    keep = np.setdiff1d(np.arange(80), rows)
    assert (fr[keep] == 7.0).all()
    # decision at the training points: sum a y K - b = f + y - b
    dv = oracle.decision(p.X, p.y, a, r["b"], p.gamma, p.X, lib=lib)
    assert np.abs(dv - (K @ (a * y) - r["b"])).max() <= 1e-12 * max(1, np.abs(dv).max())
    # held-out points against a dense Gram matrix
    q = synth.random_sparse(30, 25, 0.25, seed=32, min_nnz=1)
    Kz = rbf_matrix(_dense(q.X), D, p.gamma)
    dz = oracle.decision(p.X, p.y, a, r["b"], p.gamma, q.X, lib=lib)
    assert np.abs(dz - (Kz @ (a * y) - r["b"])).max() <= 1e-12 * max(1, np.abs(dz).max())
    # free support vectors lie on the margin up to the stopping tolerance
    free = (a > 0) & (a < p.C)
    if free.any():
        assert np.abs(dv[free] - y[free]).max() <= 2 * p.tau + 1e-9
    # kkt() agrees with the numpy gap
    kk = oracle.kkt(p.X, p.y, a, p.C, p.gamma, lib=lib)
    assert kk["gap"] <= 2 * p.tau + 1e-12


SHRINK_POLICIES = [
    # Table 3 rows 2-13: (kind, value, reconstruction)
    (oracle.SHRINK_FIXED, 2, oracle.RECON_SINGLE),
    (oracle.SHRINK_FIXED, 500, oracle.RECON_SINGLE),
    (oracle.SHRINK_FIXED, 1000, oracle.RECON_SINGLE),
    (oracle.SHRINK_FRACTION, 0.05, oracle.RECON_SINGLE),
    (oracle.SHRINK_FRACTION, 0.10, oracle.RECON_SINGLE),
    (oracle.SHRINK_FRACTION, 0.50, oracle.RECON_SINGLE),
    (oracle.SHRINK_FIXED, 2, oracle.RECON_MULTI),
    (oracle.SHRINK_FIXED, 500, oracle.RECON_MULTI),
    (oracle.SHRINK_FIXED, 1000, oracle.RECON_MULTI),
    (oracle.SHRINK_FRACTION, 0.05, oracle.RECON_MULTI),
    (oracle.SHRINK_FRACTION, 0.10, oracle.RECON_MULTI),
    (oracle.SHRINK_FRACTION, 0.50, oracle.RECON_MULTI),
]


def _shrink_problem():
    return synth.onehot_sparse(n=1500, n_test=0, seed=41)


def check_shrink_same_optimum(lib=None, policies=SHRINK_POLICIES):
    p = _shrink_problem()
    plain = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=MAXIT, lib=lib)
    assert plain["status"] == 0
    for kind, value, rec in policies:
        s = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, p.tau, kind, value, rec,
                              max_iter=MAXIT, lib=lib)
        assert s["status"] == 0
        kk = oracle.kkt(p.X, p.y, s["alpha"], p.C, p.gamma, lib=lib)
        assert kk["gap"] <= 2 * p.tau + 1e-9, (kind, value, rec, kk["gap"])
        assert abs(kk["objective"] - plain["objective"]) <= 1e-5 * abs(plain["objective"]), \
            (kind, value, rec, kk["objective"], plain["objective"])
        # the f the run ends with equals f recomputed from its alpha
        assert np.abs(s["f"] - kk["f"]).max() <= 1e-9


def check_shrink_none_is_plain(lib=None):
    p = synth.small_dense(200, 5, 51, C=1.0, gamma=0.1)
    a = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=MAXIT, lib=lib)
    b = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, p.tau, oracle.SHRINK_NONE, 0, 0,
                          max_iter=MAXIT, lib=lib)
    assert a["status"] == 0
    assert a["iters"] == b["iters"]
    assert np.array_equal(a["alpha"], b["alpha"]) and np.array_equal(a["f"], b["f"])


def check_shrink_keeps_path(lib=None):
    """A sample removed by Eq. (shrink) is at a bound and on the right side of
    both thresholds, so it is not the next maximal violator: the shrunk run
    must select exactly the plain run's pairs until late in the run."""
    p = _shrink_problem()
    n_it = MAXIT
    plain = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=n_it, trace_len=n_it, lib=lib)
    s = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, p.tau, oracle.SHRINK_FRACTION, 0.05,
                          oracle.RECON_MULTI, max_iter=n_it, trace_len=n_it, lib=lib)
    assert plain["status"] == 0 and s["status"] == 0
    m = min(len(plain["trace"]), len(s["trace"]))
    diff = np.nonzero((plain["trace"][:m] != s["trace"][:m]).any(axis=1))[0]
    first = int(diff[0]) if len(diff) else m
    assert s["n_shrink"] >= 1
    assert s["active"].min() < p.X.n // 2, "shrinking removed too little"
    assert first >= 0.5 * plain["iters"], (first, plain["iters"])


# ------------------------------------------------------------ shrink schedule
# Table 3 / Section III-C: the counter h is a fixed k, or ceil(p N) for a
# fraction p of the N samples. Algorithm 4: the shrink test runs when the
# counter, decremented every step, reaches zero, and the counter is then set
# to the smaller of h and the active-set size. Algorithm 5 (and its multiple
# reconstruction variant): the first reconstruction happens at the first
# selection whose active-set gap b_low - b_up is <= 20 tau, later ones at
# <= 2 tau; after each, the gap over all rows decides: stop at <= 2 tau, else
# continue from the full set, with shrinking restarted at counter h (Multi) or
# switched off (Single). The expected schedule below is derived from these
# definitions alone and compared with the events the oracle records.
SCHEDULE_CASES = [
    # (tau, kind, value, recon): each exercises a part of the definition
    (2e-4, oracle.SHRINK_FIXED, 500, oracle.RECON_MULTI),      # reset to |pi| < h
    (2e-4, oracle.SHRINK_FIXED, 300, oracle.RECON_SINGLE),     # reset; Single stop
    (1e-3, oracle.SHRINK_FRACTION, 0.05, oracle.RECON_MULTI),  # ceil(0.05 * 1501) = 76; Multi restart
    (1e-3, oracle.SHRINK_FRACTION, 0.10, oracle.RECON_SINGLE), # ceil(0.10 * 1501) = 151
    (1e-3, oracle.SHRINK_FIXED, 2, oracle.RECON_MULTI),        # shrink test every other step
]


def _schedule_problem():
    # N = 1501 makes p N non-integer for the fractions above
    return synth.onehot_sparse(n=1501, n_test=0, seed=41)


def _expected_h(kind, value, n):
    # the cases keep p N away from an integer, so ceil is unambiguous
    import math
    if kind == oracle.SHRINK_FIXED:
        return int(value)
    assert abs(value * n - round(value * n)) > 1e-6
    return math.ceil(value * n)


def check_shrink_schedule(lib=None, cases=SCHEDULE_CASES):
    p = _schedule_problem()
    n = p.X.n
    for tau, kind, value, recon in cases:
        run = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, tau, kind, value, recon, max_iter=MAXIT,
                                trace_len=MAXIT, events=100000, lib=lib)
        tag = (tau, kind, value, recon)
        assert run["status"] == 0, tag
        ev, gap, act = run["events"], run["gap"], run["active"]
        assert run["n_events"] == len(ev), tag
        assert len(gap) == run["iters"], tag
        h = _expected_h(kind, value, n)
        assert h >= 1
        next_shrink, thr, phase, shrinking, m = h, 20.0 * tau, 0, True, n
        n_shrink = n_recon = 0
        for j, e in enumerate(ev):
            t = e["step"]
            if e["kind"] == 1:
                # Algorithm 4: a shrink test exactly when the counter expires
                assert shrinking, (tag, "shrink event after shrinking was switched off", e)
                assert t == next_shrink, (tag, "shrink at", t, "expected", next_shrink)
                assert e["active"] <= m, (tag, "Eq. (shrink) only removes rows", e)
                assert e["gap"] == gap[t - 1], tag
                m = e["active"]
                next_shrink = t + max(1, min(h, m))
                n_shrink += 1
            else:
                assert e["kind"] == 2, e
                # Algorithm 5: the phase ends at its first selection with gap <= thr
                assert np.all(gap[phase:t] > thr), (tag, "a selection at or below the threshold "
                                                    "before the reconstruction", phase, t, thr)
                assert e["gap"] <= thr, (tag, e, thr)
                assert not shrinking or next_shrink > t, (tag, "a shrink test was due", next_shrink, t)
                assert e["active"] == n, tag
                n_recon += 1
                phase, m = t, n
                if e["gap_all"] <= 2.0 * tau:
                    assert j == len(ev) - 1 and run["iters"] == t, (tag, "must stop here")
                else:
                    thr = 2.0 * tau
                    if recon == oracle.RECON_MULTI:
                        next_shrink = t + h
                    else:
                        shrinking = False
        # the last phase: no selection reached its threshold before the end,
        # and no shrink test was due
        if not ev or ev[-1]["kind"] != 2:
            assert np.all(gap[phase:] > thr), (tag, "the final phase ran past its threshold")
            assert not shrinking or next_shrink > run["iters"], tag
        assert n_recon >= 1, (tag, "shrinking runs end with a reconstruction")
        assert n_shrink == run["n_shrink"] and n_recon == run["n_recon"], tag
        # the per-step active-set size follows the events
        cur, k = n, 0
        for t in range(run["iters"]):
            while k < len(ev) and ev[k]["step"] <= t:
                cur = ev[k]["active"]
                k += 1
            assert act[t] == cur, (tag, t, act[t], cur)
        # the recorded gaps are those of the state: at exit the gap over all
        # rows recomputed from alpha (Eq. fcache) equals the last one recorded
        kk = oracle.kkt(p.X, p.y, run["alpha"], p.C, p.gamma, lib=lib)
        assert abs(kk["gap"] - (run["b_low"] - run["b_up"])) <= 1e-9, tag
        assert kk["gap"] <= 2.0 * tau + 1e-9, tag
        if ev[-1]["kind"] == 2 and ev[-1]["gap_all"] <= 2.0 * tau:
            assert abs(ev[-1]["gap_all"] - kk["gap"]) <= 1e-9, tag
    return True


# ---------------------------------------------------------------- other kernels
# Section V: other kernels are straightforward to use. Linear <x,z>,
# polynomial (gamma <x,z> + coef0)^degree, sigmoid tanh(gamma <x,z> + coef0).
KERNEL_CASES = [(oracle.KERNEL_LINEAR, 0.0, 1), (oracle.KERNEL_POLY, 1.0, 2),
                (oracle.KERNEL_POLY, 0.5, 3)]


def check_linear_two_point_closed_form(lib=None):
    # two points of opposite labels, linear kernel: the hard-margin optimum is
    # alpha = 2 / ||x1 - x2||^2 (both on the margin), clipped at C
    with oracle.kernel_spec(oracle.KERNEL_LINEAR, lib=lib):
        for x1, x2, C in [((0.0, 0.0), (1.0, 0.0), 100.0), ((0.5, -1.0), (2.0, 1.0), 100.0),
                          ((0.0, 0.0), (0.25, 0.0), 10.0), ((1.0, 2.0), (-1.0, 0.5), 0.3)]:
            x = np.array([x1, x2], dtype=np.float32)
            X = synth.csr_from_dense(x, keep_zeros=True)
            y = np.array([1, -1], dtype=np.int8)
            d2 = float(((x[0].astype(np.float64) - x[1]) ** 2).sum())
            a_star = min(C, 2.0 / d2)
            r = oracle.smo(X, y, C, 1.0, 1e-9, max_iter=10, lib=lib)
            assert r["iters"] == 1, r["iters"]
            assert np.allclose(r["alpha"], a_star, rtol=1e-13, atol=0), (r["alpha"], a_star)
            if a_star < C:   # both points on the margin: f_1 = f_2 = b
                assert abs(r["f"][0] - r["f"][1]) <= 1e-12 * max(1.0, abs(r["f"][0]))
                assert abs(r["b"] - r["f"][0]) <= 1e-12 * max(1.0, abs(r["b"]))


def check_kernels_bruteforce(lib=None):
    for kind, c0, deg in KERNEL_CASES:
        with oracle.kernel_spec(kind, c0, deg, lib=lib):
            for n, seed, C in ((5, 41, 1.0), (7, 42, 3.0), (8, 43, 0.5)):
                p = synth.small_dense(n, 3, seed, sep=0.3, C=C, gamma=0.4, tau=1e-10)
                D = _dense(p.X)
                K = kernel_matrix(D, D, kind, p.gamma, c0, deg)
                w_star, a_star = dual_bruteforce(K, p.y.astype(np.float64), C)
                r = oracle.smo(p.X, p.y, C, p.gamma, 1e-10, max_iter=MAXIT, lib=lib)
                w = dual_objective(r["alpha"], p.y.astype(np.float64), K)
                assert abs(w - w_star) <= 1e-9 * max(1.0, abs(w_star)), (kind, n, w, w_star)
                assert np.abs(r["alpha"] - a_star).max() <= 1e-6, (kind, n, r["alpha"], a_star)


def check_linear_decision_is_primal(lib=None):
    # linear kernel: sum_j a_j y_j <x_j, z> - b = <w, z> - b, w = sum_j a_j y_j x_j
    p = synth.random_sparse(90, 12, 0.4, seed=44, min_nnz=1, C=1.0, gamma=1.0)
    q = synth.random_sparse(40, 12, 0.4, seed=45, min_nnz=1)
    with oracle.kernel_spec(oracle.KERNEL_LINEAR, lib=lib):
        r = oracle.smo(p.X, p.y, p.C, 1.0, 1e-3, max_iter=MAXIT, lib=lib)
        assert r["status"] == 0
        w = (r["alpha"] * p.y) @ _dense(p.X)
        dv = oracle.decision(p.X, p.y, r["alpha"], r["b"], 1.0, q.X, lib=lib)
    ref = _dense(q.X) @ w - r["b"]
    assert np.abs(dv - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def check_kernels_invariants(lib=None):
    # every kernel, sigmoid included (not positive definite): box, equality
    # constraint, maintained f equal to the numpy Gram matrix's, KKT at exit
    for kind, c0, deg in KERNEL_CASES + [(oracle.KERNEL_SIGMOID, -0.5, 0)]:
        with oracle.kernel_spec(kind, c0, deg, lib=lib):
            p = synth.small_dense(70, 4, 46 + kind, sep=0.4, C=1.0, gamma=0.1, tau=1e-4)
            D = _dense(p.X)
            K = kernel_matrix(D, D, kind, p.gamma, c0, deg)
            y = p.y.astype(np.float64)
            r = oracle.smo(p.X, p.y, p.C, p.gamma, 1e-4, max_iter=MAXIT, lib=lib)
            a = r["alpha"]
            assert r["status"] == 0, kind
            assert abs(y @ a) <= 1e-12 * len(a) and (a >= 0).all() and (a <= p.C).all()
            f_ref = K @ (a * y) - y
            assert np.abs(r["f"] - f_ref).max() <= 1e-10 * max(1.0, np.abs(f_ref).max()), kind
            up = ((a > 0) & (a < p.C)) | ((y > 0) & (a == 0)) | ((y < 0) & (a == p.C))
            low = ((a > 0) & (a < p.C)) | ((y > 0) & (a == p.C)) | ((y < 0) & (a == 0))
            assert f_ref[low].max() - f_ref[up].min() <= 2e-4 + 1e-12, kind


def check_wss2(lib=None):
    # second-order choice of i_low: the same optimum as the first-order rule
    # (brute force for tiny n, KKT and objective for larger), and its first
    # choice is the argmax of the gain computed here from the Gram matrix
    for n, seed, C in ((6, 51, 1.0), (8, 52, 3.0)):
        p = synth.small_dense(n, 3, seed, sep=0.3, C=C, gamma=0.5, tau=1e-10)
        K = rbf_matrix(_dense(p.X), _dense(p.X), p.gamma)
        w_star, _ = dual_bruteforce(K, p.y.astype(np.float64), C)
        r = oracle.smo_wss2(p.X, p.y, C, p.gamma, 1e-10, max_iter=MAXIT, lib=lib)
        assert abs(r["objective"] - w_star) <= 1e-9 * max(1.0, abs(w_star))
    p = synth.small_dense(120, 5, 53, sep=0.4, C=1.0, gamma=0.2, tau=1e-4)
    K = rbf_matrix(_dense(p.X), _dense(p.X), p.gamma)
    y = p.y.astype(np.float64)
    r1 = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=MAXIT, lib=lib)
    r2 = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, max_iter=MAXIT, trace_len=5, lib=lib)
    assert r2["status"] == 0
    assert abs(r2["objective"] - r1["objective"]) <= 1e-4 * abs(r1["objective"])
    a = r2["alpha"]
    f = K @ (a * y) - y
    up = ((a > 0) & (a < p.C)) | ((y > 0) & (a == 0)) | ((y < 0) & (a == p.C))
    low = ((a > 0) & (a < p.C)) | ((y > 0) & (a == p.C)) | ((y < 0) & (a == 0))
    assert f[low].max() - f[up].min() <= 2 * p.tau + 1e-12
    # each of the first steps: replay the state after k steps, recompute f,
    # i_up and the gains (f_t - f_i)^2 / (2 - 2 K(i, t)) here, and compare
    # with the pair the oracle chose at step k
    tr = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, max_iter=MAXIT, trace_len=12, lib=lib)["trace"]
    for k in range(12):
        a = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, max_iter=k, lib=lib)["alpha"]
        f = K @ (a * y) - y
        up = ((a > 0) & (a < p.C)) | ((y > 0) & (a == 0)) | ((y < 0) & (a == p.C))
        low = ((a > 0) & (a < p.C)) | ((y > 0) & (a == p.C)) | ((y < 0) & (a == 0))
        i = int(np.nonzero(up)[0][np.argmin(f[up])])
        cand = np.nonzero(low & (f > f[i]))[0]
        gain = (f[cand] - f[i]) ** 2 / np.maximum(2.0 - 2.0 * K[i, cand], 1e-12)
        j = int(cand[np.argmax(gain)])
        assert tuple(tr[k]) == (i, j), (k, tr[k], i, j)


def check_wss2_shrink(lib=None):
    """Second-order i_low with adaptive shrinking. A shrunk row is never a
    candidate of the gain rule (I1/I2 rows are not in I_low; I3/I4 rows lie
    below b_up <= f_up), so the shrunk run follows the unshrunk second-order
    run's pairs until late, and reaches its optimum."""
    p = synth.small_dense(200, 5, 51, C=1.0, gamma=0.1)
    a = oracle.smo_wss2(p.X, p.y, p.C, p.gamma, p.tau, max_iter=MAXIT, lib=lib)
    b = oracle.smo_shrink(p.X, p.y, p.C, p.gamma, p.tau, oracle.SHRINK_NONE, 0, 0,
                          max_iter=MAXIT, wss=2, lib=lib)
    assert a["status"] == 0 and a["iters"] == b["iters"]
    assert np.array_equal(a["alpha"], b["alpha"]) and np.array_equal(a["f"], b["f"])
    q = _shrink_problem()
    plain = oracle.smo_wss2(q.X, q.y, q.C, q.gamma, q.tau, max_iter=MAXIT, trace_len=MAXIT, lib=lib)
    first_order = oracle.smo(q.X, q.y, q.C, q.gamma, q.tau, max_iter=MAXIT, lib=lib)
    assert plain["status"] == 0 and plain["iters"] < first_order["iters"]
    for kind, value, rec in SHRINK_POLICIES:
        s = oracle.smo_shrink(q.X, q.y, q.C, q.gamma, q.tau, kind, value, rec, max_iter=MAXIT,
                              trace_len=MAXIT, wss=2, lib=lib)
        assert s["status"] == 0
        kk = oracle.kkt(q.X, q.y, s["alpha"], q.C, q.gamma, lib=lib)
        assert kk["gap"] <= 2 * q.tau + 1e-9, (kind, value, rec, kk["gap"])
        assert abs(kk["objective"] - first_order["objective"]) <= 1e-5 * abs(first_order["objective"])
        assert np.abs(s["f"] - kk["f"]).max() <= 1e-9
        m = min(len(plain["trace"]), len(s["trace"]))
        diff = np.nonzero((plain["trace"][:m] != s["trace"][:m]).any(axis=1))[0]
        first = int(diff[0]) if len(diff) else m
        assert first >= 0.5 * plain["iters"], (kind, value, rec, first, plain["iters"])
        if (kind, value, rec) == (oracle.SHRINK_FRACTION, 0.05, oracle.RECON_MULTI):
            assert s["n_shrink"] >= 1 and s["active"].min() < q.X.n // 2


ALL_CHECKS = [
    check_dot_and_norm,
    check_kernel_closed_form,
    check_two_point_closed_form,
    check_bruteforce,
    check_invariants,
    check_gradient_and_decision,
    check_shrink_same_optimum,
    check_shrink_none_is_plain,
    check_shrink_keeps_path,
    check_shrink_schedule,
    check_linear_two_point_closed_form,
    check_kernels_bruteforce,
    check_linear_decision_is_primal,
    check_kernels_invariants,
    check_wss2,
    check_wss2_shrink,
]
