"""Left eigenvectors and the resolvent, plain FP64 (oracle; test infrastructure only).

  * left eigenvector y of lambda: y^* T(lambda) = 0^* (Sec. 2 Eq. (nep-left)), a right
    eigenvector of T(lambda)^*: here the left singular vector of T(lambda) for its smallest
    singular value (a library SVD of the dense matrix, small n);
  * normalisation y^* T'(lambda) x = 1 of Keldysh's theorem (Sec. 2 Eq. (resolvent));
  * left scaled residual eta_L = ||T(lambda)^* y||_2 / (sum_i |f_i(lambda)| ||A_i||_1 ||y||_2), the
    scaled residual of Sec. 2 Eq. (sressplit) for T^* (||A_i^*||_inf = ||A_i||_1);
  * the resolvent's pole part  sum_i (z - lambda_i)^{-1} x_i (y_i^* v)  (Sec. 2 Eq. (resolvent),
    without the holomorphic remainder R(z));
  * the conjugate-transpose solve T(z)^* w = b (a library dense solve).
"""
from __future__ import annotations

import numpy as np

from . import band, fn


def dense_T(problem, z, derivative: bool = False) -> np.ndarray:
    coeffs = [fn.derivatives(f, z) if derivative else fn.values(f, z) for f in problem.fns]
    return band.assemble_dense(problem.mats, np.array(coeffs).reshape(-1))


def adjoint_solve(problem, z, B) -> np.ndarray:
    """W with T(z)^* W = B."""
    return np.linalg.solve(dense_T(problem, z).conj().T, B)


def left_eigenvector(problem, lam) -> np.ndarray:
    """Unit left singular vector of T(lam) for its smallest singular value."""
    U, s, Vh = np.linalg.svd(dense_T(problem, lam))
    return U[:, -1]


def keldysh_normalise(problem, lam, x, y) -> np.ndarray:
    """y scaled so that y^* T'(lam) x = 1."""
    s = np.vdot(y, dense_T(problem, lam, derivative=True) @ x)
    return y / np.conj(s)


def left_residual(problem, lam, y) -> float:
    fv = np.array([fn.values(f, lam) for f in problem.fns]).reshape(-1)
    norms1 = np.array([abs(A).sum(axis=0).max() for A in problem.mats], dtype=np.float64)
    r = dense_T(problem, lam).conj().T @ y
    return float(np.linalg.norm(r) / (np.sum(np.abs(fv) * norms1) * np.linalg.norm(y)))


def apply_resolvent(lams, X, Y, z, V) -> np.ndarray:
    """sum_i (z - lambda_i)^{-1} X[:, i] (Y[:, i]^* V)."""
    out = np.zeros((X.shape[0],) + np.shape(V)[1:], dtype=np.complex128)
    for i, lam in enumerate(lams):
        out += np.multiply.outer(X[:, i], Y[:, i].conj() @ V) / (z - lam)
    return out
