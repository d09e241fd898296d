"""Seeded synthetic SVM workloads.

This module only draws inputs: feature matrices in CSR form, labels and the
hyper-parameters of each workload. It holds none of the solver's arithmetic
and imports nothing else from the package, so the CUDA path and the FP64
oracle can both take their inputs from it.

The paper evaluates on public datasets (its Table 2: Adult a7a/a9a, Web w7a,
MNIST, USPS, Mushrooms, IJCNN) that are not available here. The generators
below stand in for them with the shapes, sparsity structure and label balance
of the workloads the benchmark is quoted on:

* ``gaussian_mixture``  -- two-class Gaussian mixture, dense rows (20 dims).
* ``onehot_sparse``     -- Adult/a9a-shaped data: 14 one-hot groups over 123
  binary columns, exactly 14 ones per row, labels from an RBF teacher.
* ``covtype_like``      -- 581,012 x 54: 10 dense N(0,1) columns and two
  one-hot blocks (4 and 40 columns), labels from a random tanh MLP.
* ``multiclass``        -- 10-class mixture for one-vs-one batching.
* ``serving_stream``    -- a Poisson stream of training-job descriptors.

Values are drawn in float64 and stored once as float32; every consumer reads
the same float32 values.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class CSR:
    """Compressed sparse rows: int64 row pointer, int32 sorted column indices,
    float32 values (``values is None`` is never produced here)."""

    n: int
    d: int
    indptr: np.ndarray
    indices: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.d), dtype=np.float32)
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        out[rows, self.indices] = self.values
        return out

    def take(self, rows: np.ndarray) -> "CSR":
        rows = np.asarray(rows, dtype=np.int64)
        lens = (self.indptr[rows + 1] - self.indptr[rows]).astype(np.int64)
        indptr = np.zeros(len(rows) + 1, dtype=np.int64)
        np.cumsum(lens, out=indptr[1:])
        src = np.repeat(self.indptr[rows] - indptr[:-1], lens) + np.arange(indptr[-1])
        return CSR(len(rows), self.d, indptr, self.indices[src].copy(),
                   self.values[src].copy())


def csr_from_dense(a: np.ndarray, keep_zeros: bool = False) -> CSR:
    a = np.ascontiguousarray(a, dtype=np.float32)
    n, d = a.shape
    if keep_zeros:
        indptr = np.arange(0, n * d + 1, d, dtype=np.int64)
        indices = np.tile(np.arange(d, dtype=np.int32), n)
        return CSR(n, d, indptr, indices, a.reshape(-1).copy())
    mask = a != 0
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=indptr[1:])
    rows, cols = np.nonzero(mask)
    return CSR(n, d, indptr, cols.astype(np.int32), a[rows, cols].astype(np.float32))


@dataclass
class Problem:
    """One binary training problem plus held-out points."""

    name: str
    X: CSR
    y: np.ndarray          # int8, +1 / -1
    Z: CSR                 # held-out points
    yz: np.ndarray
    C: float
    gamma: float
    tau: float
    meta: dict = field(default_factory=dict)


def _split(X: CSR, y: np.ndarray, n: int):
    idx_tr = np.arange(n)
    idx_te = np.arange(n, X.n)
    return X.take(idx_tr), y[:n].copy(), X.take(idx_te), y[n:].copy()


# --------------------------------------------------------------------------
# Two-class Gaussian mixture (dense)
# --------------------------------------------------------------------------
def gaussian_mixture(n: int = 2000, n_test: int = 10000, d: int = 20,
                     seed: int = 1, mean_dims: int = 5, mean: float = 0.5,
                     C: float = 1.0, gamma: float = 0.05, tau: float = 1e-3) -> Problem:
    """Balanced two-class mixture, unit variance, class means +-``mean`` on the
    first ``mean_dims`` dimensions and 0 elsewhere. Dense rows stored as CSR."""
    rng = np.random.default_rng(seed)
    total = n + n_test

    def labels(m):
        y = np.where(np.arange(m) < m // 2, 1, -1).astype(np.int8)
        rng.shuffle(y)
        return y

    y = np.concatenate([labels(n), labels(n_test)])
    mu = np.zeros((total, d))
    mu[:, :mean_dims] = mean * y[:, None]
    x = (mu + rng.standard_normal((total, d))).astype(np.float32)
    X = csr_from_dense(x, keep_zeros=True)
    Xtr, ytr, Xte, yte = _split(X, y, n)
    return Problem("gaussian_mixture", Xtr, ytr, Xte, yte, C, gamma, tau,
                   {"seed": seed, "d": d})


# --------------------------------------------------------------------------
# Adult-shaped one-hot binary data
# --------------------------------------------------------------------------
def _group_sizes(rng, d: int, groups: int) -> np.ndarray:
    """Split ``d`` columns into ``groups`` one-hot groups of size >= 2."""
    extra = d - 2 * groups
    cuts = np.sort(rng.integers(0, extra + 1, size=groups - 1))
    parts = np.diff(np.concatenate([[0], cuts, [extra]]))
    return (parts + 2).astype(np.int64)


def onehot_rows(rng, m: int, sizes: np.ndarray, zipf_s: float) -> CSR:
    """One active column per group, category drawn Zipf(s) over a fixed random
    ranking of the group's columns; all values 1.0."""
    groups = len(sizes)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    cols = np.empty((m, groups), dtype=np.int32)
    for g, (size, off) in enumerate(zip(sizes, offs)):
        p = 1.0 / np.arange(1, size + 1) ** zipf_s
        p /= p.sum()
        perm = rng.permutation(size)
        cols[:, g] = off + perm[rng.choice(size, size=m, p=p)]
    indptr = np.arange(0, m * groups + 1, groups, dtype=np.int64)
    return CSR(m, int(sizes.sum()), indptr, cols.reshape(-1),
               np.ones(m * groups, dtype=np.float32))


def onehot_sparse(n: int = 32561, n_test: int = 10000, d: int = 123,
                  groups: int = 14, seed: int = 2, zipf_s: float = 1.1,
                  centres: int = 200, teacher_gamma: float = 0.05,
                  positive: float = 0.24, flip: float = 0.05,
                  C: float = 1.0, gamma: float = 0.05, tau: float = 1e-3) -> Problem:
    """a9a-shaped workload: ``groups`` one-hot groups summing to ``d`` columns,
    labels from an RBF teacher over ``centres`` random generated rows with
    random N(0,1) weights, thresholded to ``positive`` positives, then a
    ``flip`` fraction of labels flipped."""
    rng = np.random.default_rng(seed)
    sizes = _group_sizes(rng, d, groups)
    total = n + n_test
    X = onehot_rows(rng, total, sizes, zipf_s)
    M = onehot_rows(rng, centres, sizes, zipf_s)
    w = rng.standard_normal(centres)
    # teacher: sum_c w_c exp(-g ||x - m_c||^2); for one-hot rows the squared
    # distance is 2 * (groups - shared columns)
    xd = X.to_dense().astype(np.float64)
    md = M.to_dense().astype(np.float64)
    score = np.zeros(total)
    for s in range(0, total, 8192):
        shared = xd[s:s + 8192] @ md.T
        score[s:s + 8192] = np.exp(-teacher_gamma * (2 * groups - 2 * shared)) @ w
    thr = np.quantile(score, 1.0 - positive)
    y = np.where(score > thr, 1, -1).astype(np.int8)
    flips = rng.random(total) < flip
    y[flips] = -y[flips]
    Xtr, ytr, Xte, yte = _split(X, y, n)
    return Problem("onehot_sparse", Xtr, ytr, Xte, yte, C, gamma, tau,
                   {"seed": seed, "group_sizes": sizes.tolist()})


# --------------------------------------------------------------------------
# Covtype-shaped mixed dense + one-hot data
# --------------------------------------------------------------------------
def covtype_like(n: int = 581012, n_test: int = 10000, seed: int = 3,
                 dense: int = 10, blocks=(4, 40), hidden: int = 32,
                 positive: float = 0.49, C: float = 4.0, gamma: float = 0.1,
                 tau: float = 1e-3) -> Problem:
    """``dense`` N(0,1) columns followed by one-hot blocks (uniform category);
    labels from the sign of a fixed random 2-layer tanh MLP, thresholded so
    that ``positive`` of the points are positive."""
    rng = np.random.default_rng(seed)
    total = n + n_test
    nb = len(blocks)
    k = dense + nb
    d = dense + int(sum(blocks))
    vals = np.ones((total, k), dtype=np.float32)
    cols = np.empty((total, k), dtype=np.int32)
    vals[:, :dense] = rng.standard_normal((total, dense)).astype(np.float32)
    cols[:, :dense] = np.arange(dense, dtype=np.int32)
    off = dense
    onehot = []
    for j, b in enumerate(blocks):
        c = rng.integers(0, b, size=total)
        cols[:, dense + j] = off + c
        onehot.append(c)
        off += b
    # teacher MLP on the features (dense part + one-hot embedding)
    W1 = rng.standard_normal((d, hidden)) / math.sqrt(dense + nb)
    b1 = 0.5 * rng.standard_normal(hidden)
    w2 = rng.standard_normal(hidden)
    h = vals[:, :dense].astype(np.float64) @ W1[:dense]
    off = dense
    for j, b in enumerate(blocks):
        h += W1[off + onehot[j]]
        off += b
    score = np.tanh(h + b1) @ w2
    thr = np.quantile(score, 1.0 - positive)
    y = np.where(score > thr, 1, -1).astype(np.int8)
    indptr = np.arange(0, total * k + 1, k, dtype=np.int64)
    X = CSR(total, d, indptr, cols.reshape(-1), vals.reshape(-1))
    Xtr, ytr, Xte, yte = _split(X, y, n)
    return Problem("covtype_like", Xtr, ytr, Xte, yte, C, gamma, tau,
                   {"seed": seed})


# --------------------------------------------------------------------------
# Ten-class mixture for one-vs-one batching
# --------------------------------------------------------------------------
@dataclass
class MultiClass:
    X: CSR
    labels: np.ndarray      # int32 class ids
    Cs: tuple
    gammas: tuple
    tau: float

    def ovo_pairs(self):
        k = int(self.labels.max()) + 1
        return [(a, b) for a in range(k) for b in range(a + 1, k)]

    def subproblem(self, a: int, b: int):
        """Rows of classes a and b (ascending) and labels +1 for a, -1 for b."""
        rows = np.nonzero((self.labels == a) | (self.labels == b))[0]
        y = np.where(self.labels[rows] == a, 1, -1).astype(np.int8)
        return rows.astype(np.int64), y


def multiclass(n: int = 50000, d: int = 256, classes: int = 10, seed: int = 4,
               mean_sd: float = 0.3, Cs=(0.1, 1.0, 10.0),
               gammas=(0.002, 0.01, 0.05), tau: float = 1e-3) -> MultiClass:
    """``classes``-class Gaussian mixture: class means N(0, mean_sd^2) per
    dimension, unit noise, class weights U(0.5, 1.5) normalised to ``n``."""
    rng = np.random.default_rng(seed)
    means = mean_sd * rng.standard_normal((classes, d))
    w = rng.uniform(0.5, 1.5, size=classes)
    counts = np.floor(w / w.sum() * n).astype(np.int64)
    counts[: n - counts.sum()] += 1
    labels = np.repeat(np.arange(classes, dtype=np.int32), counts)
    rng.shuffle(labels)
    x = (means[labels] + rng.standard_normal((n, d))).astype(np.float32)
    return MultiClass(csr_from_dense(x, keep_zeros=True), labels, tuple(Cs),
                      tuple(gammas), tau)


# --------------------------------------------------------------------------
# Serving stream
# --------------------------------------------------------------------------
@dataclass
class JobSpec:
    job_id: int
    arrival_s: float
    n: int
    d: int
    sparse: bool
    C: float
    gamma: float
    seed: int


def serving_stream(n_jobs: int = 2000, rate: float = 20.0, seed: int = 5,
                   n_range=(1000, 200000), d_range=(20, 2000),
                   C_range=(0.1, 10.0)) -> list:
    """Poisson arrivals; n, d, C log-uniform; half dense, half sparse;
    gamma = 1/d. Job data are drawn lazily by ``serving_job``."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))

    def logu(lo, hi, size):
        return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))

    ns = np.round(logu(*n_range, n_jobs)).astype(np.int64)
    ds = np.round(logu(*d_range, n_jobs)).astype(np.int64)
    Cs = logu(*C_range, n_jobs)
    sparse = rng.random(n_jobs) < 0.5
    seeds = rng.integers(0, 2**31 - 1, size=n_jobs)
    return [JobSpec(i, float(t[i]), int(ns[i]), int(ds[i]), bool(sparse[i]),
                    float(Cs[i]), 1.0 / float(ds[i]), int(seeds[i]))
            for i in range(n_jobs)]


def serving_job(spec: JobSpec, n: int | None = None, density: float = 0.005) -> Problem:
    """Training data of one serving job: a dense two-class Gaussian mixture,
    or CSR rows with ``max(1, round(density*d))`` distinct random columns and
    lognormal(0,1) values; rows L2-normalised; labels from the mixture class."""
    rng = np.random.default_rng(spec.seed)
    n = spec.n if n is None else n
    d = spec.d
    y = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    if not spec.sparse:
        mu = np.zeros(d)
        mu[: min(5, d)] = 0.5
        x = y[:, None] * mu[None, :] + rng.standard_normal((n, d))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        X = csr_from_dense(x.astype(np.float32), keep_zeros=True)
    else:
        k = max(1, int(round(density * d)))
        # class-dependent column preference so the labels are learnable
        pref = rng.permutation(d)
        half = max(1, d // 2)
        cols = np.empty((n, k), dtype=np.int64)
        for i in range(n):
            pool = pref[:half] if (y[i] > 0) == (rng.random() < 0.8) else pref[half:]
            if len(pool) < k:
                pool = pref
            cols[i] = np.sort(rng.choice(pool, size=k, replace=False))
        v = rng.lognormal(0.0, 1.0, size=(n, k))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        indptr = np.arange(0, n * k + 1, k, dtype=np.int64)
        X = CSR(n, d, indptr, cols.reshape(-1).astype(np.int32),
                v.reshape(-1).astype(np.float32))
    return Problem(f"serving_job_{spec.job_id}", X, y, X.take(np.arange(0)),
                   np.zeros(0, np.int8), spec.C, spec.gamma, 1e-3,
                   {"sparse": spec.sparse})


# --------------------------------------------------------------------------
# Small cases for tests
# --------------------------------------------------------------------------
def small_dense(n: int, d: int, seed: int, sep: float = 0.5,
                C: float = 1.0, gamma: float = 0.1, tau: float = 1e-3) -> Problem:
    """Tiny two-class Gaussian problem with alternating labels."""
    rng = np.random.default_rng(seed)
    y = np.where(np.arange(n) % 2 == 0, 1, -1).astype(np.int8)
    rng.shuffle(y)
    if (y > 0).all() or (y < 0).all():
        y[0] = -y[0]
    x = (sep * y[:, None] + rng.standard_normal((n, d))).astype(np.float32)
    X = csr_from_dense(x, keep_zeros=True)
    return Problem("small_dense", X, y, X.take(np.arange(0)), np.zeros(0, np.int8),
                   C, gamma, tau, {"seed": seed})


def random_sparse(n: int, d: int, density: float, seed: int,
                  C: float = 1.0, gamma: float = 0.1, tau: float = 1e-3,
                  binary: bool = False, min_nnz: int = 0) -> Problem:
    """Random CSR rows with ragged lengths (Bernoulli(density) per column,
    at least ``min_nnz`` per row), labels from a random linear score."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, d)) < density
    for i in range(n):
        if mask[i].sum() < min_nnz:
            mask[i, rng.choice(d, size=min_nnz, replace=False)] = True
    vals = np.ones((n, d)) if binary else rng.standard_normal((n, d))
    x = np.where(mask, vals, 0.0).astype(np.float32)
    w = rng.standard_normal(d)
    s = x.astype(np.float64) @ w
    y = np.where(s > np.median(s), 1, -1).astype(np.int8)
    if (y > 0).all() or (y < 0).all():
        y[0] = -y[0]
    X = csr_from_dense(x)
    return Problem("random_sparse", X, y, X.take(np.arange(0)), np.zeros(0, np.int8),
                   C, gamma, tau, {"seed": seed})
