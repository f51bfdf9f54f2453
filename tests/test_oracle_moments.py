"""Pins of the oracle's quadrature and moments against closed forms (CPU only).

For T(z) = z I - diag(d) on a circle with nodes theta_j = 2 pi (j + 1/2)/N
(zeta_j^N = -1), the discrete moments are exactly
    sum_j w_j zeta_j^k (z_j - d)^{-1} = alpha^k / (1 + alpha^N),  alpha = (d - c)/r,
for 0 <= k < N and |alpha| != 1 (geometric series of 1/(zeta - alpha)); as N grows this
tends to the residue sum of Keldysh's expansion (Sec. 2 Eq. (resolvent)).
"""
import math

import numpy as np
import scipy.sparse as sp

import synth
from oracle import ciss, contour


def _shifted_identity_problem(d, center, radius):
    n = len(d)
    mats = [sp.identity(n, format="csr"), sp.diags(np.asarray(d, float), 0, format="csr")]
    fns = [{"kind": "rational", "num": [1.0, 0.0], "den": None, "alpha": 1.0, "beta": 1.0},
           {"kind": "rational", "num": [-1.0], "den": None, "alpha": 1.0, "beta": 1.0}]
    region = {"center": complex(center), "a": float(radius), "b": float(radius)}
    return synth.Problem("zI-diag", n, mats, fns, region)


def moment_closed_form_error(N=32, M=8):
    c, r = -1.0, 2.0
    alpha = np.array([0.36, 0.95, 1.025, 1.27, -0.6, -1.4])
    d = c + r * alpha
    p = _shifted_identity_problem(d, c, r)
    V = synth.random_probe_block(p.n, 3, seed=7)
    mom = ciss.moments(p, p.region, N, M, V)
    err = 0.0
    for k in range(M):
        ref = (alpha ** k / (1 + alpha ** N))[:, None] * V
        err = max(err, float(np.abs(mom["S"][k] - ref).max()))
    return err


def test_moments_closed_form_circle():
    assert moment_closed_form_error() < 1e-13


def test_raw_moments_binomial_identity():
    """S^raw_k = sum_j w_j z_j^k Y_j equals sum_m C(k, m) c^(k-m) a^m S_m (z = c + a zeta)."""
    p = synth.delay_2d(s=6, seed=1, center=-1.5, radius=2.5)
    V = synth.random_probe_block(p.n, 2, seed=1)
    N, M = 16, 4
    mom = ciss.moments(p, p.region, N, M, V, keep_Y=True)
    z, w = mom["z"], mom["w"]
    c, a = complex(p.region["center"]), p.region["a"]
    for k in range(M):
        raw = sum(w[j] * z[j] ** k * mom["Y"][j] for j in range(N))
        mix = sum(math.comb(k, m) * c ** (k - m) * a ** m * mom["S"][m] for m in range(k + 1))
        assert np.allclose(raw, mix, rtol=1e-12, atol=1e-13 * np.abs(raw).max())


def test_ellipse_weights_integrate_cauchy_kernel():
    """sum_j w_j g(z_j) -> (1/(2 pi i)) oint g dz: 1/(z-p) gives 1 inside, 0 outside; z^k gives 0."""
    region = {"center": 2.0 + 0j, "a": 1.0, "b": 0.2}
    z, w, zeta = contour.nodes(region, 1024)
    for p, ref in [(2.3 + 0.05j, 1.0), (1.5 - 0.1j, 1.0), (3.5 + 0j, 0.0), (2.0 + 0.5j, 0.0)]:
        assert abs(np.sum(w / (z - p)) - ref) < 1e-10
    for k in range(6):
        assert abs(np.sum(w * z ** k)) < 1e-12 * max(1.0, np.abs(z).max() ** k)
    # the scaled variable: zeta = (z - c)/a lies on the ellipse of semi-axes 1 and b/a
    assert np.allclose((zeta.real) ** 2 + (zeta.imag / 0.2) ** 2, 1.0)


def test_hankel_matrix_layout():
    rng = np.random.default_rng(0)
    L, M = 2, 3
    mu = rng.standard_normal((2 * M, L, L)) + 1j * rng.standard_normal((2 * M, L, L))
    H, Hs = ciss.hankel_matrices(mu)
    for i in range(M):
        for j in range(M):
            assert np.array_equal(H[i * L:(i + 1) * L, j * L:(j + 1) * L], mu[i + j])
            assert np.array_equal(Hs[i * L:(i + 1) * L, j * L:(j + 1) * L], mu[i + j + 1])
