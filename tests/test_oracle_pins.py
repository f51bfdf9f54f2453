"""Whole-pipeline pins of the oracle against closed forms, library routines and counts (CPU only).

  * decoupled delay problems: lambda = a + W_k(b e^{-a}) (Lambert W branches);
  * decoupled Drude problems: roots of the cubic (lambda + i g) t(lambda) (companion matrix);
  * decoupled square-root problems: roots of a quadratic in s = sqrt(lambda - sigma^2);
  * tiny dense problems: linear pencil / cubic companion pencil via scipy.linalg.eig;
  * eigenvalue counts by the argument principle (det T(z) winding, Sec. 2);
  * the scaled residual of Sec. 2 Eq. (sressplit) on a hand-computed example.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
from scipy.special import lambertw

import synth
from oracle import ciss, contour, count

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _match(found, expected, tol):
    found = sorted(found, key=lambda x: (round(x.real, 6), x.imag))
    expected = sorted(expected, key=lambda x: (round(x.real, 6), x.imag))
    assert len(found) == len(expected), (found, expected)
    used = set()
    for e in expected:
        j = min((j for j in range(len(found)) if j not in used), key=lambda j: abs(found[j] - e))
        used.add(j)
        assert abs(found[j] - e) <= tol * max(1.0, abs(e)), (found[j], e)


def lambert_reference(p):
    a, b = p.meta["a"], p.meta["b"]
    out = []
    for i in range(p.n):
        for k in range(-8, 9):
            lam = a[i] + lambertw(b[i] * np.exp(-a[i]), k)
            if contour.inside(p.region, lam):
                out.append(complex(lam))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_diagonal_delay_lambert_w(seed):
    p = synth.diagonal_delay(n=8, seed=seed)
    V = synth.random_probe_block(p.n, p.L, seed)
    r = ciss.solve(p, V=V)
    _match(list(r["lam"]), lambert_reference(p), 1e-12)
    assert r["eta"].max() < 1e-13


def drude_reference(p):
    wp, g = p.meta["omega_p"], p.meta["gamma"]
    out = []
    for k, m, d in zip(p.meta["k"], p.meta["m"], p.meta["d"]):
        coeffs = [-(m + d), -1j * g * (m + d), k + wp ** 2 * d, 1j * g * k]
        for lam in np.roots(coeffs):
            if abs(lam + 1j * g) > 1e-9 and contour.inside(p.region, lam):
                out.append(complex(lam))
    return out


@pytest.mark.parametrize("seed", [0, 4])
def test_diagonal_drude_companion_roots(seed):
    p = synth.diagonal_drude(n=6, seed=seed)
    V = synth.random_probe_block(p.n, p.L, seed)
    r = ciss.solve(p, V=V)
    ref = drude_reference(p)
    assert len(ref) > 0
    _match(list(r["lam"]), ref, 1e-11)


def sqrt_reference(p):
    out = []
    s2 = p.meta["sigma"] ** 2
    for k, m, w in zip(p.meta["k"], p.meta["m"], p.meta["w"]):
        # -m s^2 + i w s + (k - m sigma^2) = 0, s on the principal branch
        for s in np.roots([-m, 1j * w, k - m * s2]):
            if s.real > 0 or (s.real == 0 and s.imag >= 0):
                lam = s * s + s2
                if contour.inside(p.region, lam):
                    out.append(complex(lam))
    return out


def test_diagonal_sqrt_quadratic_roots():
    p = synth.diagonal_sqrt(n=6, seed=0)
    V = synth.random_probe_block(p.n, p.L, 0)
    r = ciss.solve(p, V=V)
    ref = sqrt_reference(p)
    assert len(ref) > 0
    _match(list(r["lam"]), ref, 1e-11)


def test_dense_linear_pencil():
    p = synth.dense_linear_small(n=10, seed=0)
    V = synth.random_probe_block(p.n, p.L, 0)
    r = ciss.solve(p, V=V)
    A, B = p.mats[0].toarray(), p.mats[1].toarray()
    ev = scipy.linalg.eig(A, B, right=False)
    ref = [complex(e) for e in ev if contour.inside(p.region, e)]
    assert len(ref) > 0
    _match(list(r["lam"]), ref, 1e-10)


def test_dense_drude_cubic_linearisation():
    """(lambda + i g) T(lambda) is the cubic matrix polynomial -(M+D) l^3 - i g (M+D) l^2 + (K + wp^2 D) l + i g K."""
    p = synth.dense_drude_small(n=6, seed=0)
    V = synth.random_probe_block(p.n, p.L, 0)
    r = ciss.solve(p, V=V)
    K, Mm, D = (m.toarray().astype(complex) for m in p.mats)
    wp, g = 3.0, 0.1
    A3, A2, A1, A0 = -(Mm + D), -1j * g * (Mm + D), K + wp ** 2 * D, 1j * g * K
    n = p.n
    Z, I = np.zeros((n, n)), np.eye(n)
    Ac = np.block([[Z, I, Z], [Z, Z, I], [-A0, -A1, -A2]])
    Bc = np.block([[I, Z, Z], [Z, I, Z], [Z, Z, A3]])
    ev = scipy.linalg.eig(Ac, Bc, right=False)
    ref = [complex(e) for e in ev if np.isfinite(e) and abs(e + 1j * g) > 1e-8 and contour.inside(p.region, e)]
    assert len(ref) > 0
    _match(list(r["lam"]), ref, 1e-10)


def test_count_matches_returned_delay1d_wide():
    with open(os.path.join(GOLDEN, "counts.json")) as f:
        golden = json.load(f)
    p = synth.config_problem("delay1d_n64_wide")
    V = synth.random_probe_block(p.n, p.L, 0)
    r = ciss.solve(p, V=V)
    assert len(r["lam"]) == golden["delay1d_n64"]["count"]
    assert count.count_inside(p) == golden["delay1d_n64"]["count"]
    assert r["eta"].max() < 1e-12


def test_count_matches_returned_small_grid():
    p = synth.delay_2d(s=12, seed=2, center=-1.5, radius=1.5)
    V = synth.random_probe_block(p.n, 8, 2)
    r = ciss.solve(p, N=64, L=8, M=4, V=V)
    assert not r["saturated"]
    assert len(r["lam"]) == count.count_inside(p)
    assert r["eta"].max() < 1e-10


def test_saturated_flag_when_subspace_too_small():
    p = synth.config_problem("delay1d_n64")  # L*M = 16 < 32 eigenvalues inside
    V = synth.random_probe_block(p.n, p.L, 0)
    r = ciss.solve(p, V=V)
    assert r["saturated"] and r["m"] == p.L * p.M


def test_scaled_residual_hand_example():
    """T(l) = diag(1,2) + l [[0,1],[1,0]] at l = 2, x = e1: ||Tx|| = sqrt(5); sum |f_i| ||A_i||_inf = 1*2 + 2*1."""
    mats = [sp.csr_matrix(np.diag([1.0, 2.0])), sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]]))]
    fns = [{"kind": "rational", "num": [1.0], "den": None},
           {"kind": "rational", "num": [1.0, 0.0], "den": None}]
    norms = ciss.term_norms_inf(mats)
    eta = ciss.scaled_residual(mats, fns, norms, 2.0 + 0j, np.array([1.0 + 0j, 0.0]))
    assert math.isclose(eta, math.sqrt(5.0) / 4.0, rel_tol=1e-15)


def test_invariant_pair_of_returned_eigenpairs():
    """(X, diag(lambda)) is an invariant pair: sum_i A_i X f_i(Lambda) = 0 (Sec. 2 Eq. (invpair) split form)."""
    p = synth.config_problem("delay1d_n64_wide")
    V = synth.random_probe_block(p.n, p.L, 0)
    r = ciss.solve(p, V=V)
    X, lam = r["X"], r["lam"]
    from oracle import fn
    Tsum = np.zeros_like(X)
    scale = 0.0
    for A, f in zip(p.mats, p.fns):
        fv = fn.values(f, lam)
        Tsum += (A @ X) * fv[None, :]
        scale += np.abs(fv).max() * np.abs(A).sum(axis=1).max()
    assert np.linalg.norm(Tsum) / (scale * np.linalg.norm(X)) < 1e-13


def diagonal_linear_on_node(z_node, n=6, seed=0, N=16):
    """T(z) = diag(d) - z I on the unit circle around 0 with d_0 placed exactly on a quadrature node
    (T(z_node) exactly singular) and the other d_i drawn strictly inside or outside the circle."""
    from synth.problems import Problem, _rational, _sorted_csr
    rng = np.random.default_rng(seed)
    rad = np.concatenate([[0.0], rng.uniform(0.1, 0.7, n - 3), rng.uniform(1.3, 1.6, 2)])
    d = rad * np.exp(2j * np.pi * rng.uniform(size=n))
    d[0] = z_node
    mats = [_sorted_csr(sp.diags(d, 0, format="csr")), _sorted_csr(sp.identity(n, format="csr"))]
    fns = [_rational([1.0]), _rational([-1.0, 0.0])]
    region = {"center": 0j, "a": 1.0, "b": 1.0}
    return Problem("diagonal_linear_on_node", n, mats, fns, region, N=N, L=n, M=2, meta={"d": d})


def test_singular_node_drops_out():
    """An eigenvalue exactly on a quadrature node makes T(z_0) singular: that node contributes
    nothing, the result stays finite and the eigenvalues strictly inside are the d_i exactly."""
    z, _, _ = contour.nodes({"center": 0j, "a": 1.0, "b": 1.0}, 16)
    p = diagonal_linear_on_node(z[0])
    V = synth.random_probe_block(p.n, p.L, 0)
    r = ciss.solve(p, V=V)
    assert r["info"][0] != 0 and not np.any(r["info"][1:])
    assert np.all(np.isfinite(r["S"]))
    inside = [complex(x) for x in p.meta["d"][1:] if abs(x) < 1]
    found = [l for l in r["lam"] if abs(l - p.meta["d"][0]) > 1e-8]
    _match(found, inside, 1e-12)
