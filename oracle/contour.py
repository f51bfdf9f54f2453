"""Quadrature nodes and weights on an ellipse (oracle; test infrastructure only).

The contour-integral moments approximate (1/(2 pi i)) oint_Gamma ((z-c)/a)^k T(z)^{-1} V dz;
by Keldysh's expansion of the resolvent (Sec. 2 Eq. (resolvent)) these isolate the
eigenvectors of the eigenvalues enclosed by Gamma.

Gamma: z(theta) = c + a cos(theta) + i b sin(theta), trapezoid rule at
theta_j = 2 pi (j + 1/2) / N (no node on the real axis), so that
  (1/(2 pi i)) oint g(z) dz  ~=  sum_j w_j g(z_j),   w_j = (b cos theta_j + i a sin theta_j) / N,
and the scaled variable zeta_j = (z_j - c) / a.

Pinned by the closed form of the discrete moments of z I - diag(d) on a circle
(tests/test_oracle_moments.py).
"""
from __future__ import annotations

import numpy as np

from . import fn


def nodes(region: dict, N: int):
    c = complex(region["center"])
    a = float(region["a"])
    b = float(region["b"])
    theta = 2.0 * np.pi * (np.arange(N) + 0.5) / N
    z = c + a * np.cos(theta) + 1j * b * np.sin(theta)
    w = (b * np.cos(theta) + 1j * a * np.sin(theta)) / N
    zeta = (z - c) / a
    return z, w, zeta


def coefficient_table(fns, z):
    """F[i, j] = f_i(z_j) (split form, Sec. 2 Eq. (split))."""
    return np.array([fn.values(f, z) for f in fns], dtype=np.complex128)


def inside(region: dict, lam):
    """Strictly inside the ellipse: ((Re(l-c))/a)^2 + ((Im(l-c))/b)^2 < 1."""
    d = np.asarray(lam, dtype=np.complex128) - complex(region["center"])
    return (d.real / region["a"]) ** 2 + (d.imag / region["b"]) ** 2 < 1.0
