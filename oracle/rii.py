"""Residual inverse iteration (Neumaier's method), plain FP64 (oracle; test infrastructure only).

Sec. 4.1, Algorithm (rii), used to polish an eigenpair (lambda, x) of the contour method whose
scaled residual eta misses the acceptance level:

  lambda^(0) given;  x^(0) normalised
  for k = 0, 1, ...:
      lambda^(k+1) = lambda^(k);  repeat lambda^(k+1) -= mu,
          mu = x^* T(sigma)^{-1} T(lambda^(k+1)) x / x^* T(sigma)^{-1} T'(lambda^(k+1)) x
      until |mu| < sqrt(eps) |lambda^(k+1)|         (Newton on x^* T(sigma)^{-1} T(z) x = 0)
      r = T(lambda^(k+1)) x;  stop if eta(x, lambda^(k+1)) < tol
      solve T(sigma) v = r;   x = (x - v) / ||x - v||

with T(z) = sum_i f_i(z) A_i (Sec. 2 Eq. (split)) and eta of Sec. 2 Eq. (sressplit). T(sigma) is
factored once with the banded LU of the contour method (band_lu.c). The steps are written out
as the algorithm states them (two solves per inner Newton step, one for the update); nothing
here is shared with the device code.

Readings (where the algorithm leaves a choice to the caller):
  * the starting eigenvalue is the contour method's estimate, not sigma itself;
  * sigma is that starting estimate, fixed for the whole iteration (the algorithm's
    "update sigma" line with the update done once, at the start);
  * at most INNER_MAX inner Newton steps and MAX_IT outer iterations; for lambda = 0 the
    inner stopping test is |mu| = 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import band, fn
from .ciss import term_norms_inf

INNER_MAX = 30
MAX_IT = 10
INNER_TOL = math.sqrt(np.finfo(np.float64).eps)


def _apply(mats, coeffs, x):
    out = np.zeros(x.shape[0], dtype=np.complex128)
    for A, f in zip(mats, coeffs):
        out += f * (A @ x)
    return out


def _factor(problem, sigma, kl, ku):
    F = np.array([fn.values(f, sigma) for f in problem.fns]).reshape(-1)
    ab = band.assemble_band(problem.mats, F, kl, ku)
    lu, ipiv, info = band.gbtrf(ab.copy(order="F"), kl, ku)
    return lu, ipiv, info


def rii(problem, lam0: complex, x0: np.ndarray, *, sigma=None, tol: float = 1e-10, max_it: int = MAX_IT,
        kl=None, ku=None):
    """Algorithm (rii) from (lam0, x0). Returns (lambda, x, eta, iterations, converged)."""
    if kl is None or ku is None:
        kl, ku = band.bandwidths(problem.mats)
    sigma = complex(lam0) if sigma is None else complex(sigma)
    lu, ipiv, info = _factor(problem, sigma, kl, ku)
    if info != 0:
        raise ZeroDivisionError(f"T(sigma) is singular in the band LU (info={info})")
    solve = lambda b: band.gbtrs(lu, kl, ku, ipiv, b)[:, 0]
    norms = term_norms_inf(problem.mats)
    x = np.asarray(x0, dtype=np.complex128)
    x = x / np.linalg.norm(x)
    lam = complex(lam0)
    eta = math.inf
    for k in range(max_it + 1):
        # scalar Newton on x^* T(sigma)^{-1} T(z) x = 0
        for _ in range(INNER_MAX):
            fv = [fn.values(f, lam) for f in problem.fns]
            dv = [fn.derivatives(f, lam) for f in problem.fns]
            num = np.vdot(x, solve(_apply(problem.mats, fv, x)))
            den = np.vdot(x, solve(_apply(problem.mats, dv, x)))
            if den == 0:
                break
            mu = num / den
            lam = lam - mu
            if (lam != 0 and abs(mu) < INNER_TOL * abs(lam)) or (lam == 0 and mu == 0):
                break
        fv = np.array([fn.values(f, lam) for f in problem.fns]).reshape(-1)
        r = _apply(problem.mats, fv, x)
        eta = float(np.linalg.norm(r) / (np.sum(np.abs(fv) * norms) * np.linalg.norm(x)))
        if eta < tol:
            return lam, x, eta, k, True
        if k == max_it:
            break
        v = solve(r)
        x = x - v
        x = x / np.linalg.norm(x)
    return lam, x, eta, max_it, False
