"""The seeded synthetic workloads match the recipes they stand for.

The paper's datasets are not available; each benchmark configuration is a
seeded generator (paper_1406_5161_gb300.synth). These checks pin the shape,
structure and value distribution of each one to its stated recipe, so that a
change in a generator cannot silently change the workload every measurement
and parity test runs on.
"""
import math

import numpy as np

from paper_1406_5161_gb300 import synth


def _rows_nnz(X):
    return np.diff(X.indptr)


def test_gaussian_mixture_recipe():
    """2,000 training + 10,000 held-out rows, d = 20 dense, unit variance,
    class means +-0.5 on the first 5 dims, balanced labels; C 1, gamma 0.05,
    tau 1e-3."""
    p = synth.gaussian_mixture()
    assert (p.X.n, p.X.d, p.Z.n) == (2000, 20, 10000)
    assert (_rows_nnz(p.X) == 20).all()
    assert (p.C, p.gamma, p.tau) == (1.0, 0.05, 1e-3)
    assert (p.y == 1).sum() == (p.y == -1).sum() == 1000
    x = np.vstack([p.X.to_dense(), p.Z.to_dense()]).astype(np.float64)
    y = np.concatenate([p.y, p.yz]).astype(np.float64)
    centred = x - y[:, None] * np.r_[np.full(5, 0.5), np.zeros(15)][None, :]
    assert np.abs(centred.mean(0)).max() < 0.04
    assert np.abs(centred.std(0) - 1.0).max() < 0.04
    assert np.abs((x * y[:, None]).mean(0)[:5] - 0.5).max() < 0.04


def test_onehot_sparse_recipe():
    """a9a shape: 32,561 rows, d = 123 binary columns in 14 one-hot groups
    (sizes summing to 123, at least 2 each), exactly one 1 per group per row;
    24% positive before 5% flips; C 1, gamma 0.05."""
    p = synth.onehot_sparse()
    assert (p.X.n, p.X.d, p.Z.n) == (32561, 123, 10000)
    assert (_rows_nnz(p.X) == 14).all()
    assert p.X.values is None or (p.X.values == 1.0).all()
    sizes = np.asarray(p.meta["group_sizes"])
    cols = p.X.indices.reshape(-1, 14)
    assert (np.diff(cols, axis=1) > 0).all()           # sorted, distinct
    assert sizes.sum() == 123 and len(sizes) == 14 and (sizes >= 2).all()
    edges = np.r_[0, np.cumsum(sizes)]
    for g in range(14):
        assert ((cols[:, g] >= edges[g]) & (cols[:, g] < edges[g + 1])).all()
    pos = (np.concatenate([p.y, p.yz]) > 0).mean()
    # 24% positive, then 5% of all labels flipped: 0.24 (0.95) + 0.76 (0.05)
    assert abs(pos - (0.24 * 0.95 + 0.76 * 0.05)) < 0.01
    assert (p.C, p.gamma, p.tau) == (1.0, 0.05, 1e-3)


def test_covtype_like_recipe():
    """covtype shape (per row, checked on a prefix of the generator): d = 54;
    columns 0-9 dense N(0, 1), one of columns 10-13 and one of 14-53 set to
    1 (12 stored entries); 49% positive; C 4, gamma 0.1."""
    p = synth.covtype_like(n=20000, n_test=0, seed=3)
    assert p.X.d == 54 and (_rows_nnz(p.X) == 12).all()
    cols = p.X.indices.reshape(-1, 12)
    vals = p.X.values.reshape(-1, 12)
    assert (cols[:, :10] == np.arange(10)).all()
    assert ((cols[:, 10] >= 10) & (cols[:, 10] < 14)).all()
    assert ((cols[:, 11] >= 14) & (cols[:, 11] < 54)).all()
    assert (vals[:, 10:] == 1.0).all()
    dense = vals[:, :10].astype(np.float64)
    assert abs(dense.mean()) < 0.02 and abs(dense.std() - 1.0) < 0.02
    assert abs((p.y > 0).mean() - 0.49) < 0.01
    assert (p.C, p.gamma) == (4.0, 0.1)


def test_multiclass_recipe():
    """10 classes, n = 50,000, d = 256; class weights U(0.5, 1.5) normalised
    to n give classes of 2,500-7,500 rows and one-vs-one subproblems of
    5k-15k rows; C x gamma grid 3 x 3, so 405 jobs."""
    mc = synth.multiclass()
    assert (mc.X.n, mc.X.d) == (50000, 256)
    counts = np.bincount(mc.labels, minlength=10)
    assert counts.sum() == 50000 and counts.min() >= 2500 and counts.max() <= 7500
    pairs = mc.ovo_pairs()
    assert len(pairs) == 45
    sizes = [len(mc.subproblem(a, b)[0]) for a, b in pairs]
    assert 5000 <= min(sizes) and max(sizes) <= 15000
    assert len(pairs) * len(mc.Cs) * len(mc.gammas) == 405


def test_serving_stream_recipe():
    """2,000 jobs, Poisson arrivals at 20/s; n log-uniform in [1e3, 2e5], d
    log-uniform in [20, 2000], C log-uniform in [0.1, 10]; half dense, half
    sparse; gamma = 1/d; sparse rows hold max(1, round(0.005 d)) entries and
    every row is L2-normalised."""
    js = synth.serving_stream()
    assert len(js) == 2000
    t = np.array([j.arrival_s for j in js])
    gaps = np.diff(np.r_[0.0, t])
    assert (gaps > 0).all() and abs(gaps.mean() - 0.05) < 0.005
    n = np.array([j.n for j in js], dtype=float)
    d = np.array([j.d for j in js], dtype=float)
    C = np.array([j.C for j in js])
    for v, lo, hi in ((n, 1e3, 2e5), (d, 20, 2000), (C, 0.1, 10.0)):
        assert v.min() >= lo * 0.999 and v.max() <= hi * 1.001
        lv = (np.log(v) - math.log(lo)) / (math.log(hi) - math.log(lo))
        assert abs(lv.mean() - 0.5) < 0.03          # uniform in log space
    assert abs(np.mean([j.sparse for j in js]) - 0.5) < 0.04
    assert all(abs(j.gamma - 1.0 / j.d) < 1e-15 for j in js)
    for spec in js[:40]:
        p = synth.serving_job(spec, n=min(spec.n, 300))
        x = p.X.to_dense().astype(np.float64)
        assert np.allclose(np.linalg.norm(x, axis=1), 1.0, atol=1e-5)
        if spec.sparse:
            assert (_rows_nnz(p.X) == max(1, int(round(0.005 * spec.d)))).all()
        else:
            assert (_rows_nnz(p.X) == spec.d).all()
