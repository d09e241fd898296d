"""Independent references used to pin the oracle (test code only).

* ``rbf_matrix``: the RBF Gram matrix from dense float64 rows by numpy,
  exp(-gamma * ||x_i - x_j||^2) with the distance taken directly, not through
  the norm expansion the oracle uses; ``kernel_matrix`` the other kernels
  (linear, polynomial, sigmoid) from the dense inner products.
* ``dual_bruteforce``: exact maximiser of the SVM dual QP for tiny n by
  enumerating, for every sample, the three faces {alpha = 0, alpha = C,
  free} and solving the equality-constrained stationarity system on the
  free set. The feasible candidate with the largest objective is the optimum
  (the dual is a concave QP, so its maximiser lies on one of these faces and
  satisfies that face's stationarity system).
"""
import itertools

import numpy as np


def rbf_matrix(A: np.ndarray, B: np.ndarray, gamma: float) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    diff = A[:, None, :] - B[None, :, :]
    return np.exp(-gamma * np.einsum("ijk,ijk->ij", diff, diff))


def kernel_matrix(A: np.ndarray, B: np.ndarray, kind: int, gamma: float, coef0: float = 0.0,
                  degree: int = 3) -> np.ndarray:
    """Gram matrix of the kernel kind (0 RBF, 1 linear, 2 polynomial,
    3 sigmoid) from dense float64 rows by numpy."""
    if kind == 0:
        return rbf_matrix(A, B, gamma)
    G = np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64).T
    if kind == 1:
        return G
    if kind == 2:
        return np.power(gamma * G + coef0, degree)
    return np.tanh(gamma * G + coef0)


def dual_objective(alpha, y, K) -> float:
    ay = alpha * y
    return float(alpha.sum() - 0.5 * ay @ K @ ay)


def dual_bruteforce(K: np.ndarray, y: np.ndarray, C: float, tol: float = 1e-12):
    n = len(y)
    y = y.astype(np.float64)
    Q = y[:, None] * y[None, :] * K
    best_w, best_a = -np.inf, None
    for assign in itertools.product((0, 1, 2), repeat=n):
        assign = np.array(assign)
        F = np.nonzero(assign == 2)[0]
        Bi = np.nonzero(assign != 2)[0]
        aB = np.where(assign[Bi] == 1, C, 0.0)
        a = np.zeros(n)
        a[Bi] = aB
        if len(F) == 0:
            if abs(y @ a) > 1e-9 * max(1.0, C):
                continue
        else:
            m = len(F)
            M = np.zeros((m + 1, m + 1))
            M[:m, :m] = Q[np.ix_(F, F)]
            M[:m, m] = -y[F]
            M[m, :m] = y[F]
            rhs = np.empty(m + 1)
            rhs[:m] = 1.0 - Q[np.ix_(F, Bi)] @ aB
            rhs[m] = -(y[Bi] @ aB)
            try:
                sol = np.linalg.solve(M, rhs)
            except np.linalg.LinAlgError:
                continue
            aF = sol[:m]
            if (aF < -tol).any() or (aF > C + tol).any():
                continue
            a[F] = np.clip(aF, 0.0, C)
        w = float(a.sum() - 0.5 * a @ Q @ a)
        if w > best_w:
            best_w, best_a = w, a
    return best_w, best_a
