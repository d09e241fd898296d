"""The FP64 mode's integer-arithmetic kernel values, checked on the device.

`svm_decision` in FP64 with one support vector (alpha = 1, y = +1, b = 0)
returns K(z, x) itself, computed by the CUDA-core contraction with the same
device functions the fused step uses (csrc/fp64_math.cuh: the exact 128-bit
inner products with their funnel shifts and carry chains, the fixed-point
exponential with its 64 x 64 high products). The host build of those
functions is tested in test_fp64_math_cpu.py; this test pins the device
build:

* linear kernel: K = <z, x> equals the exact rational inner product rounded
  to the nearest double (ties to even), bit for bit; for a matrix whose
  values leave the exact format's window, it equals the FP64 sum of fused
  multiply-adds in row order instead;
* RBF kernel: K = exp(-gamma d^2) with d^2 = (||z||^2 + ||x||^2) - 2 <z, x>
  formed from the correctly rounded norms and inner product exactly as the
  kernel forms it, within 0.51 units in the last place of the correctly
  rounded exp (mpmath), 0 where gamma d^2 > 745.
"""
from fractions import Fraction

import numpy as np
import pytest

import paper_1406_5161_gb300 as pkg
from paper_1406_5161_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)
mp = pytest.importorskip("mpmath")
mp.mp.dps = 60


def _matrix(rng, n, d, density, spread, zeros=False):
    """Random float rows: signs mixed, magnitudes 2^[-spread, spread] times
    [1, 2), about `density` of the columns stored (explicit zeros kept when
    `zeros`)."""
    e = rng.integers(-spread, spread + 1, size=(n, d)).astype(np.float64)
    a = rng.choice([-1.0, 1.0], size=(n, d)) * rng.uniform(1, 2, size=(n, d)) * 2.0 ** e
    a[rng.random((n, d)) > density] = 0.0
    a = a.astype(np.float32)
    if zeros:
        a[:, ::7] = 0.0
    return synth.csr_from_dense(a, keep_zeros=zeros)


def _rows(M):
    return [(M.indices[M.indptr[i]:M.indptr[i + 1]], M.values[M.indptr[i]:M.indptr[i + 1]]) for i in range(M.n)]


def _exact_dot(zr, xr):
    zd = dict(zip(zr[0].tolist(), zr[1].tolist()))
    return sum((Fraction(float(v)) * Fraction(zd[c]) for c, v in zip(xr[0].tolist(), xr[1].tolist()) if c in zd),
               Fraction(0))


def _round(fr):
    return fr.numerator / fr.denominator   # correctly rounded, ties to even


def _fma_chain(zr, xr):
    """The FP64 fallback: acc = fma(x_k, z_k, acc) over x's entries in order."""
    zd = dict(zip(zr[0].tolist(), zr[1].tolist()))
    acc = Fraction(0)
    for c, v in zip(xr[0].tolist(), xr[1].tolist()):
        acc = Fraction(_round(Fraction(float(v)) * Fraction(zd.get(c, 0.0)) + acc))
    return float(acc)


def _kernel_values(X, Z, kernel, gamma=1.0):
    y = np.ones(X.n, dtype=np.int8)
    out = np.zeros((X.n, Z.n))
    for j in range(X.n):
        alpha = np.zeros(X.n)
        alpha[j] = 1.0
        out[j] = pkg.svm_decision(X, y, alpha, 0.0, gamma, Z, precision=pkg.SVM_FP64, kernel=kernel)
    return out


@pytest.mark.parametrize("zeros", [False, True])
def test_exact_inner_products_on_the_device(zeros):
    rng = np.random.default_rng(21 + zeros)
    X = _matrix(rng, 12, 40, 0.5, 14, zeros)
    Z = _matrix(rng, 48, 40, 0.5, 14, zeros)
    got = _kernel_values(X, Z, pkg.SVM_KERNEL_LINEAR)
    xr, zr = _rows(X), _rows(Z)
    bad = [(j, q) for j in range(X.n) for q in range(Z.n) if got[j, q] != _round(_exact_dot(zr[q], xr[j]))]
    assert not bad, bad[:5]


def test_inner_products_outside_the_window_are_fp64_row_sums():
    rng = np.random.default_rng(5)
    X = _matrix(rng, 8, 30, 0.6, 6)
    Z = _matrix(rng, 24, 30, 0.6, 6)
    X.values[0] = np.float32(2.0 ** -60)   # 60 binades below the rest: the format is off
    got = _kernel_values(X, Z, pkg.SVM_KERNEL_LINEAR)
    xr, zr = _rows(X), _rows(Z)
    bad = [(j, q) for j in range(X.n) for q in range(Z.n) if got[j, q] != _fma_chain(zr[q], xr[j])]
    assert not bad, bad[:5]


@pytest.mark.parametrize("gamma", [0.05, 1.0, 2.5])
def test_fixed_point_exp_on_the_device(gamma):
    rng = np.random.default_rng(int(gamma * 100))
    X = _matrix(rng, 10, 24, 0.6, 3)
    # the queries: copies of the support rows (d^2 = 0, K = 1) and random rows
    Zd = np.vstack([X.to_dense(), _matrix(rng, 54, 24, 0.6, 3).to_dense()])
    Z = synth.csr_from_dense(Zd)
    got = _kernel_values(X, Z, pkg.SVM_KERNEL_RBF, gamma)
    xr, zr = _rows(X), _rows(Z)
    nx = [_round(_exact_dot(r, r)) for r in xr]
    nz = [_round(_exact_dot(r, r)) for r in zr]
    worst, n_fixed = 0.0, 0
    for j in range(X.n):
        assert got[j, j] == 1.0
        for q in range(Z.n):
            dot = _round(_exact_dot(zr[q], xr[j]))
            d2 = (nz[q] + nx[j]) - 2.0 * dot
            y = gamma * max(d2, 0.0)
            ref = mp.exp(-mp.mpf(y))
            if y > 700.0:   # the library exp: 0 beyond 745, else within 2 ulp
                assert got[j, q] == 0.0 if y > 745.2 else abs(mp.mpf(got[j, q]) - ref) <= 2 * mp.mpf(5e-324) + ref * 2.0 ** -51
                continue
            rd = float(ref)
            err = float(abs(mp.mpf(got[j, q]) - ref) / np.spacing(rd))
            worst = max(worst, err)
            n_fixed += 1
    print("fixed-point values", n_fixed, "max ulp", worst)
    assert n_fixed >= 20
    assert worst <= 0.51
