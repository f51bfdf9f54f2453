"""Polynomial interpolation solver ("Interpol", Sec. 4.4) in plain FP64 (oracle; test infrastructure only).

For a real interval I = [a, b] (here the real axis of the region's ellipse: a = c - a_r, b = c + a_r,
with a real centre c), T is interpolated in the variable theta of [-1, 1], lambda = alpha theta + beta,
alpha = (b - a)/2, beta = (b + a)/2:

  * Chebyshev nodes nu_j = cos(omega_j), omega_j = (j + 1/2) pi / (d + 1), j = 0 .. d (Eq. (interpolnu));
  * coefficients C_k = 2/(d+1) sum_j T(lambda(nu_j)) cos(k omega_j) (Eq. (polinterpcoef)); in split form
    C_k = sum_i c_ik A_i with c_ik = 2/(d+1) sum_j f_i(lambda(nu_j)) cos(k omega_j);
  * P_d(theta) = C_0/2 tau_0 + sum_{k>=1} C_k tau_k (Eq. (polinterp)), tau_k the Chebyshev polynomials of
    the first kind;
  * the polynomial eigenproblem P_d(theta) x = 0 through a linearisation in the Chebyshev basis: with
    u_k = tau_k(theta) x (k < d), the rows -theta u_0 + u_1 = 0, u_{k-1} - 2 theta u_k + u_{k+1} = 0
    (1 <= k <= d-2, from theta tau_k = (tau_{k+1} + tau_{k-1})/2 and theta tau_0 = tau_1), and the last
    row sum_{k<d} C'_k u_k + C_d (2 theta u_{d-1} - u_{d-2}) = 0 (tau_d = 2 theta tau_{d-1} - tau_{d-2},
    C'_0 = C_0/2, C'_k = C_k otherwise): a pencil (A, B) of d blocks of n, built densely, its eigenvalues
    from a library generalized eigensolver; x is the first block u_0 of the eigenvector;
  * the region filter of Sec. 4.4: eigenvalues lambda = alpha theta + beta strictly inside the
    region's ellipse (the interval and its vicinity, set by the imaginary semi-axis).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import contour


def interval_map(region: dict):
    """alpha, beta of lambda = alpha theta + beta for the real axis of the ellipse."""
    c = complex(region["center"])
    if c.imag != 0.0:
        raise ValueError("the interval is the real axis of a region with a real centre")
    return float(region["a"]), c.real


def chebyshev_nodes(d: int):
    """omega_j and nu_j = cos(omega_j), j = 0 .. d (Eq. (interpolnu))."""
    om = (np.arange(d + 1) + 0.5) * np.pi / (d + 1)
    return om, np.cos(om)


def coefficients(fns, region: dict, d: int) -> np.ndarray:
    """c[i, k], k = 0 .. d: the scalar Chebyshev coefficients of each f_i (Eq. (polinterpcoef)),
    written as the plain double sum."""
    alpha, beta = interval_map(region)
    om, nu = chebyshev_nodes(d)
    lam = alpha * nu + beta
    F = contour.coefficient_table(fns, lam.astype(np.complex128))  # f_i(lambda(nu_j))
    c = np.zeros((len(fns), d + 1), dtype=np.complex128)
    for i in range(len(fns)):
        for k in range(d + 1):
            s = 0.0 + 0.0j
            for j in range(d + 1):
                s += F[i, j] * np.cos(k * om[j])
            c[i, k] = 2.0 / (d + 1) * s
    return c


def chebyshev_values(theta, d: int) -> np.ndarray:
    """tau_0 .. tau_d at theta (three-term recurrence)."""
    theta = np.asarray(theta, dtype=np.complex128)
    t = np.zeros((d + 1,) + theta.shape, dtype=np.complex128)
    t[0] = 1.0
    if d >= 1:
        t[1] = theta
    for k in range(1, d):
        t[k + 1] = 2.0 * theta * t[k] - t[k - 1]
    return t


def interpolant_values(c: np.ndarray, theta) -> np.ndarray:
    """p_i(theta) = c_i0/2 + sum_{k>=1} c_ik tau_k(theta), the interpolant of each f_i."""
    d = c.shape[1] - 1
    t = chebyshev_values(theta, d)
    w = c.copy()
    w[:, 0] *= 0.5
    return np.tensordot(w, t, axes=(1, 0))


def pencil(mats, c: np.ndarray):
    """Dense (A, B) of the Chebyshev-basis linearisation of P_d (d >= 2), order d n."""
    d = c.shape[1] - 1
    if d < 2:
        raise ValueError("the linearisation needs d >= 2")
    n = mats[0].shape[0]
    Cp = []
    for k in range(d + 1):
        w = c[:, k] * (0.5 if k == 0 else 1.0)
        Cp.append(sum(w[i] * mats[i].toarray() for i in range(len(mats))))
    I = np.eye(n)
    A = np.zeros((d * n, d * n), dtype=np.complex128)
    B = np.zeros_like(A)
    blk = lambda r, q: (slice(r * n, (r + 1) * n), slice(q * n, (q + 1) * n))
    # row 0: -theta u_0 + u_1 = 0
    A[blk(0, 1)] = I
    B[blk(0, 0)] = I
    # rows k = 1 .. d-2: u_{k-1} - 2 theta u_k + u_{k+1} = 0
    for k in range(1, d - 1):
        A[blk(k, k - 1)] = I
        A[blk(k, k + 1)] = I
        B[blk(k, k)] = 2.0 * I
    # last row: sum_{k<d} C'_k u_k - C_d u_{d-2} + 2 theta C_d u_{d-1} = 0
    r = d - 1
    for k in range(d):
        A[blk(r, k)] += Cp[k]
    A[blk(r, d - 2)] -= Cp[d]
    B[blk(r, d - 1)] = -2.0 * Cp[d]
    return A, B


def solve(problem, region: dict, d: int):
    """Eigenpairs of P_d(theta) x = 0 mapped to lambda, filtered to the region (Sec. 4.4).
    Returns lambda (sorted by (Re, Im)), the first blocks x (unit 2-norm) and the coefficients."""
    c = coefficients(problem.fns, region, d)
    A, B = pencil(problem.mats, c)
    th, Vv = scipy.linalg.eig(A, B)
    alpha, beta = interval_map(region)
    n = problem.n
    lam, X = [], []
    for e in range(len(th)):
        if not np.isfinite(th[e]):
            continue
        l = alpha * th[e] + beta
        if not contour.inside(region, np.array([l]))[0]:
            continue
        x = Vv[:n, e]
        nx = np.linalg.norm(x)
        if nx == 0:
            continue
        lam.append(l)
        X.append(x / nx)
    order = sorted(range(len(lam)), key=lambda q: (lam[q].real, lam[q].imag))
    lam = np.array([lam[q] for q in order], dtype=np.complex128)
    X = np.stack([X[q] for q in order], axis=1) if order else np.zeros((n, 0), np.complex128)
    return {"lam": lam, "X": X, "coef": c}
