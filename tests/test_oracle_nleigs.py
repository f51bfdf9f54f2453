"""Pins of the NLEIGS oracle (Sec. 4.5, static variant) (CPU only).

  * the rational interpolant sum_j b_j(z) d_i^j reproduces f_i at its nodes and, within the
    degree test's tolerance, on the boundary and inside Sigma (direct evaluation of f_i);
  * a rational problem is interpolated exactly everywhere once the degree passes its type;
  * the nodes and poles satisfy the Leja-Bagby conditions and the scalings max |b_j| = 1,
    recomputed from scratch by products;
  * the matrix-function divided differences equal those of the interpolation recurrence
    D_j = (T(sigma_j) - R_{j-1}(sigma_j)) / b_j(sigma_j) (a different algorithm);
  * the linearisation's eigenvalues inside Sigma are the closed-form eigenvalues: Lambert W
    (decoupled delay), the companion roots (decoupled Drude), the quadratic roots (decoupled
    square root) and the generalized eigenvalues of a linear pencil.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import contour, fn, nleigs
from tests.test_oracle_pins import _match, drude_reference, lambert_reference, sqrt_reference

PROBLEMS = {
    "delay": lambda: synth.diagonal_delay(n=8, seed=0),
    "drude": lambda: synth.diagonal_drude(n=6, seed=0),
    "sqrt": lambda: synth.diagonal_sqrt(n=6, seed=0),
}


def _fvals(fns, z):
    return np.array([fn.values(f, z) for f in fns])


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_interpolant_reproduces_the_functions(name):
    p = PROBLEMS[name]()
    it = nleigs.interpolation(p.fns, p.region)
    # at the nodes: interpolation conditions
    r = nleigs.interpolant_coeffs(it, it["sigma"])
    f = _fvals(p.fns, it["sigma"])
    assert np.abs(r - f).max() <= 1e-13 * np.abs(f).max()
    # on the boundary and inside (maximum modulus): within the degree test's tolerance
    rng = np.random.default_rng(0)
    rad = np.sqrt(rng.uniform(0, 1, 200))
    th = rng.uniform(0, 2 * np.pi, 200)
    z_in = complex(p.region["center"]) + rad * (p.region["a"] * np.cos(th) + 1j * p.region["b"] * np.sin(th))
    for z in (it["bnd"], z_in):
        r = nleigs.interpolant_coeffs(it, z)
        f = _fvals(p.fns, z)
        assert np.abs(r - f).max() <= 1e-11 * np.abs(f).max(), name


def test_rational_problem_is_interpolated_exactly():
    p = synth.diagonal_drude(n=6, seed=0)
    it = nleigs.interpolation(p.fns, p.region)
    g = p.meta["gamma"]
    assert np.isclose(it["xi"][1], -1j * g)  # the pole of the Drude term, found from its denominator
    assert it["d"] == 4                        # type (3, 1): the degree-3 interpolant is exact
    rng = np.random.default_rng(1)
    z = 4.0 * (rng.standard_normal(100) + 1j * rng.standard_normal(100))
    z = z[np.abs(z + 1j * g) > 0.5]
    r = nleigs.interpolant_coeffs(it, z)
    f = _fvals(p.fns, z)
    assert np.abs(r - f).max() <= 1e-11 * np.abs(f).max()


def test_leja_bagby_conditions_and_scalings():
    p = synth.diagonal_sqrt(n=6, seed=0)
    it = nleigs.interpolation(p.fns, p.region)
    bnd, Xi, sigma, xi, d = it["bnd"], it["Xi"], it["sigma"], it["xi_seq"], it["d"]
    assert len(Xi) == len(nleigs.CUT_T)
    assert np.all(Xi.imag == 0) and Xi.real.max() <= p.meta["sigma"] ** 2  # the cut (-inf, sigma^2]
    used = []
    for j in range(d):
        def s(z):
            num = np.prod([z - sigma[k] for k in range(j + 1)], axis=0)
            den = np.prod([1 - z / xi[k] for k in range(1, j + 1) if np.isfinite(xi[k])], axis=0) \
                if any(np.isfinite(xi[1:j + 1])) else 1.0
            return num / den
        sb = np.abs(s(bnd))
        assert abs(s(np.array([sigma[j + 1]]))[0]) >= sb.max() * (1 - 1e-12)
        if np.isfinite(xi[j + 1]):
            used.append(xi[j + 1])
            cand = np.array([x for x in Xi if not np.any(np.isclose(x, used[:-1], rtol=0, atol=0))])
            assert abs(s(np.array([xi[j + 1]]))[0]) <= np.abs(s(cand)).min() * (1 + 1e-12)
    b = nleigs.basis(bnd, it["sigma"], it["xi"], it["beta"], d)
    assert np.allclose(np.abs(b).max(axis=1), 1.0, rtol=1e-14)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_divided_differences_match_the_interpolation_recurrence(name):
    p = PROBLEMS[name]()
    it = nleigs.interpolation(p.fns, p.region)
    sig, xi, beta, d = it["sigma"], it["xi"], it["beta"], it["d"]
    B = nleigs.basis(sig, sig, xi, beta, d)  # B[k, j] = b_k(sigma_j)
    F = _fvals(p.fns, sig)
    rec = np.zeros_like(it["dd"])
    for j in range(d + 1):
        rec[:, j] = (F[:, j] - rec[:, :j] @ B[:j, j]) / B[j, j]
    scale = np.abs(it["dd"][:, 0]).max()
    assert np.abs(rec - it["dd"]).max() <= 1e-12 * scale


def test_linear_pencil_eigenvalues():
    p = synth.dense_linear_small(n=8, seed=3)
    r = nleigs.solve(p)
    A, B = p.mats[0].toarray(), p.mats[1].toarray()
    ref = [complex(e) for e in scipy.linalg.eig(A, B, right=False) if contour.inside(p.region, e)]
    assert len(ref) > 0
    _match(list(r["lam"]), ref, 1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_delay_eigenvalues_are_lambert_w(seed):
    p = synth.diagonal_delay(n=8, seed=seed)
    r = nleigs.solve(p)
    _match(list(r["lam"]), lambert_reference(p), 1e-12)
    assert r["eta"].max() < 1e-13
    # eigenvectors of a decoupled problem are unit vectors
    assert np.all(np.sort(np.abs(r["X"]), axis=0)[-2] <= 1e-10)


def test_drude_and_sqrt_closed_forms():
    p = synth.diagonal_drude(n=6, seed=0)
    ref = drude_reference(p)
    assert len(ref) > 0
    _match(list(nleigs.solve(p)["lam"]), ref, 1e-11)
    p = synth.diagonal_sqrt(n=6, seed=0)
    ref = sqrt_reference(p)
    assert len(ref) > 0
    _match(list(nleigs.solve(p)["lam"]), ref, 1e-11)
