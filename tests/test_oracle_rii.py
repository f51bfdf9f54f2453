"""Pins of the residual inverse iteration oracle (Sec. 4.1, Algorithm (rii)) against closed forms (CPU only).

  * decoupled delay problems: the iteration converges to lambda = a + W_k(b e^{-a}) (Lambert W)
    from a perturbed start, and the eigenvector to the unit vector of that row;
  * an exact eigenpair is a fixed point (no update, eta at rounding level);
  * a linear problem T(z) = diag(d) - z I: the scalar equation x^* T(sigma)^{-1} T(z) x = 0 is linear
    in z, so the inner Newton loop lands on its root, written out elementwise without a solve;
  * perturbed contour-method eigenpairs of a coupled problem polish back to the unperturbed
    eigenvalues and eigenvectors (those are pinned by the contour method's own tests).
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.special import lambertw

import synth
from oracle import ciss, contour, rii


def _lambert_pairs(p):
    """(lambda, row) of the eigenvalues inside the region of a decoupled delay problem."""
    a, b = p.meta["a"], p.meta["b"]
    out = []
    for i in range(p.n):
        for k in range(-6, 7):
            lam = complex(a[i] + lambertw(b[i] * np.exp(-a[i]), k))
            if contour.inside(p.region, lam):
                out.append((lam, i))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_rii_converges_to_lambert_w(seed):
    p = synth.diagonal_delay(n=8, seed=seed)
    pairs = _lambert_pairs(p)
    assert pairs
    rng = np.random.default_rng(100 + seed)
    for lam_ref, i in pairs:
        x0 = 1e-3 * (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n))
        x0[i] = 1.0
        lam0 = lam_ref + 1e-3 * (1 + 1j) * max(1.0, abs(lam_ref))
        lam, x, eta, its, ok = rii.rii(p, lam0, x0, tol=1e-12)
        assert ok and eta < 1e-12, (lam_ref, eta, its)
        assert abs(lam - lam_ref) <= 1e-12 * max(1.0, abs(lam_ref)), (lam, lam_ref)
        others = np.abs(np.delete(x, i))
        assert others.max() <= 1e-10 and abs(abs(x[i]) - 1.0) <= 1e-12


def test_rii_exact_pair_is_a_fixed_point():
    p = synth.diagonal_delay(n=8, seed=0)
    lam_ref, i = _lambert_pairs(p)[0]
    x0 = np.zeros(p.n, np.complex128)
    x0[i] = 1.0
    lam, x, eta, its, ok = rii.rii(p, lam_ref, x0, sigma=lam_ref + 0.05, tol=1e-10)
    assert ok and its == 0 and eta < 1e-14
    assert abs(lam - lam_ref) <= 1e-14 * max(1.0, abs(lam_ref))
    assert np.array_equal(x, x0)


def test_rii_inner_step_on_a_linear_problem_is_the_root_of_the_scalar_equation():
    n = 6
    rng = np.random.default_rng(7)
    d = rng.uniform(-2.0, 2.0, n) + 1j * rng.uniform(-1.0, 1.0, n)
    mats = [sp.diags(d, 0, format="csr"), sp.identity(n, format="csr", dtype=np.complex128)]
    fns = [{"kind": "rational", "num": [1.0], "den": [1.0], "alpha": 1.0, "beta": 1.0},
           {"kind": "rational", "num": [-1.0, 0.0], "den": [1.0], "alpha": 1.0, "beta": 1.0}]
    p = synth.Problem("diag_linear", n, mats, fns, {"center": 0j, "a": 3.0, "b": 3.0}, N=16, L=2, M=2)
    x0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x0 = x0 / np.linalg.norm(x0)
    sigma = 0.3 - 0.2j
    # x^* T(sigma)^{-1} (D - z I) x = 0 with T(sigma)^{-1} = diag(1 / (d - sigma)):
    # z = sum |x_k|^2 d_k / (d_k - sigma) / sum |x_k|^2 / (d_k - sigma)
    w = np.abs(x0) ** 2 / (d - sigma)
    z_root = np.sum(w * d) / np.sum(w)
    lam, x, eta, its, ok = rii.rii(p, 1.0 + 0.5j, x0, sigma=sigma, tol=1e-30, max_it=0)
    assert abs(lam - z_root) <= 1e-13 * max(1.0, abs(z_root)), (lam, z_root)
    assert np.allclose(x, x0)


def test_rii_recovers_perturbed_contour_pairs_of_a_coupled_problem():
    # the contour method's pairs of a coupled delay problem (eta ~ 1e-16), perturbed to ~1e-5
    p = synth.delay_2d(s=8, seed=1)
    V = synth.random_probe_block(p.n, 16, 0)
    r = ciss.solve(p, N=16, L=16, M=4, V=V)
    assert len(r["lam"]) >= 10 and r["eta"].max() < 1e-14
    rng = np.random.default_rng(11)
    for k in range(len(r["lam"])):
        x0 = r["X"][:, k] + 1e-5 * (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n))
        lam0 = r["lam"][k] * (1 + 1e-5)
        assert ciss.scaled_residual(p.mats, p.fns, ciss.term_norms_inf(p.mats), lam0, x0) > 1e-8
        lam, x, eta, its, ok = rii.rii(p, lam0, x0, tol=1e-12)
        assert ok and eta < 1e-12, (k, eta, its)
        assert abs(lam - r["lam"][k]) <= 1e-11 * max(1.0, abs(r["lam"][k])), (lam, r["lam"][k])
        assert abs(abs(np.vdot(x, r["X"][:, k])) - 1.0) <= 1e-10
