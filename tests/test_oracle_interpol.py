"""Pins of the Interpol oracle (Sec. 4.4) against closed forms and independent library routines (CPU).

  * Chebyshev orthogonality: the coefficients of f = tau_3(theta(lambda)) are exactly e_3;
  * interpolation conditions: the interpolant equals f_i at every Chebyshev node, and e^{-lambda}
    to rounding in between at degree 40;
  * an exactly interpolated problem: a quadratic T(lambda) = A0 + lambda A1 + lambda^2 A2 has P_d = T for
    d >= 2, so the linearisation's eigenvalues in the region are the quadratic's (from its own companion
    pencil, a different linearisation);
  * decoupled delay problems with real eigenvalues lambda = a + W_0(b e^{-a}) (Lambert W) on an interval.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
from scipy.special import lambertw

import synth
from oracle import interpol
from synth.problems import Problem, _exp, _rational, _sorted_csr


def test_chebyshev_orthogonality():
    region = {"center": 0.7 + 0j, "a": 1.3, "b": 0.1}
    alpha, beta = 1.3, 0.7
    # tau_3(theta) = 4 theta^3 - 3 theta with theta = (lambda - beta) / alpha, as a polynomial in lambda
    th = np.poly1d([1.0 / alpha, -beta / alpha])
    p = 4 * th ** 3 - 3 * th
    f = _rational(list(p.coeffs))
    for d in (3, 7, 12):
        c = interpol.coefficients([f], region, d)[0]
        e = np.zeros(d + 1)
        e[3] = 1.0
        assert np.abs(c - e).max() <= 1e-13, (d, c)


def test_interpolation_conditions():
    region = {"center": -0.25 + 0j, "a": 2.25, "b": 0.1}
    fns = [_exp(alpha=-1.0), _rational([-1.0, 0.0]), _rational([1.0, 0.5], [1.0, 5.0])]
    for d in (5, 40):
        c = interpol.coefficients(fns, region, d)
        _, nu = interpol.chebyshev_nodes(d)
        lam = 2.25 * nu - 0.25
        P = interpol.interpolant_values(c, nu)
        F = np.array([np.exp(-lam), -lam, (lam + 0.5) / (lam + 5.0)])
        assert np.abs(P - F).max() <= 1e-13 * max(1.0, np.abs(F).max())
    th = np.linspace(-1, 1, 101)
    P = interpol.interpolant_values(c, th)
    assert np.abs(P[0] - np.exp(-(2.25 * th - 0.25))).max() <= 1e-13 * np.exp(2.5)


def quadratic_problem(n=5, seed=0):
    rng = np.random.default_rng(seed)
    A = [(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n) for _ in range(3)]
    A[2] = np.eye(n) + 0.2 * A[2]
    mats = [_sorted_csr(sp.csr_matrix(M)) for M in A]
    fns = [_rational([1.0]), _rational([1.0, 0.0]), _rational([1.0, 0.0, 0.0])]
    return Problem("quadratic", n, mats, fns, {"center": 0.0 + 0j, "a": 1.5, "b": 1.5}), A


def test_exact_interpolation_of_a_quadratic():
    p, A = quadratic_problem()
    n = p.n
    # companion pencil of the quadratic (monomial basis): [[0, I], [-A0, -A1]] - lambda [[I, 0], [0, A2]]
    Z, I = np.zeros((n, n)), np.eye(n)
    ref = scipy.linalg.eigvals(np.block([[Z, I], [-A[0], -A[1]]]), np.block([[I, Z], [Z, A[2]]]))
    ref = ref[(np.abs(ref.real / 1.5) ** 2 + np.abs(ref.imag / 1.5) ** 2) < 1]
    assert len(ref) >= 2
    for d in (2, 3, 6):
        r = interpol.solve(p, p.region, d)
        assert len(r["lam"]) == len(ref), (d, r["lam"], ref)
        for l in ref:
            assert np.min(np.abs(r["lam"] - l)) <= 1e-10 * max(1.0, abs(l))


def real_delay_problem(n=6, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-2.0, 0.0, n)
    b = rng.uniform(0.1, 0.8, n)
    mats = [_sorted_csr(sp.diags(a, 0, format="csr")), _sorted_csr(sp.identity(n, format="csr")),
            _sorted_csr(sp.diags(b, 0, format="csr"))]
    fns = [_rational([1.0]), _rational([-1.0, 0.0]), _exp(alpha=-1.0)]
    region = {"center": -0.25 + 0j, "a": 2.25, "b": 0.1}
    return Problem("real_delay", n, mats, fns, region, meta={"a": a, "b": b})


def lambert_real(p):
    a, b = p.meta["a"], p.meta["b"]
    return np.sort(np.real(a + lambertw(b * np.exp(-a), 0)))


@pytest.mark.parametrize("seed", [0, 1])
def test_real_delay_eigenvalues_on_an_interval(seed):
    p = real_delay_problem(seed=seed)
    ref = lambert_real(p)
    r = interpol.solve(p, p.region, 40)
    assert len(r["lam"]) == len(ref)
    assert np.abs(np.sort(r["lam"].real) - ref).max() <= 1e-10
    assert np.abs(r["lam"].imag).max() <= 1e-10
    # the first block of the eigenvector is the NEP's eigenvector (a unit vector here)
    for k in range(len(r["lam"])):
        assert np.abs(r["X"][:, k]).max() >= 1 - 1e-8
