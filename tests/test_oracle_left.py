"""Pins of the left-eigenvector and resolvent oracle (Sec. 2 Eqs. (nep-left), (resolvent)) (CPU only).

  * a linear pencil T(z) = A - z B with every eigenvalue taken: the resolvent is exactly its pole
    part with Keldysh-normalised left eigenvectors, checked against a dense solve with T(z);
  * decoupled delay problems: the left eigenvector of row i is the unit vector e_i, scaled by the
    normalisation to 1 / conj(T'(lambda)_ii);
  * a coupled delay problem: (z - lambda) T(z)^{-1} -> x y^* as z -> lambda (the residue), an
    independent check of the left vector and of its normalisation;
  * the conjugate-transpose solve satisfies w^* (T v) = b^* v.
"""
import numpy as np
import scipy.linalg
from scipy.special import lambertw

import synth
from oracle import ciss, contour, left


def test_resolvent_of_a_linear_pencil_is_its_pole_part():
    p = synth.dense_linear_small(n=8, seed=3)
    A, B = (m.toarray() for m in p.mats)
    lams, Xr = scipy.linalg.eig(A, B)
    X = Xr / np.linalg.norm(Xr, axis=0)
    Y = np.stack([left.keldysh_normalise(p, lam, X[:, i], left.left_eigenvector(p, lam))
                  for i, lam in enumerate(lams)], axis=1)
    rng = np.random.default_rng(1)
    V = rng.standard_normal((p.n, 3)) + 1j * rng.standard_normal((p.n, 3))
    for z in (0.3 + 0.2j, -1.1 + 0.5j, 2.0 - 0.7j):
        ref = np.linalg.solve(A - z * B, V)
        got = left.apply_resolvent(lams, X, Y, z, V)
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_left_eigenvectors_of_decoupled_delay_problems():
    p = synth.diagonal_delay(n=8, seed=1)
    a, b = p.meta["a"], p.meta["b"]
    for i in range(p.n):
        lam = complex(a[i] + lambertw(b[i] * np.exp(-a[i]), 0))
        y = left.left_eigenvector(p, lam)
        assert abs(abs(y[i]) - 1.0) <= 1e-12 and np.abs(np.delete(y, i)).max() <= 1e-12
        x = np.zeros(p.n, np.complex128)
        x[i] = 1.0
        yn = left.keldysh_normalise(p, lam, x, y)
        dT = -1.0 - b[i] * np.exp(-lam)  # T'(lambda)_ii for T = diag(a) - z I + e^{-z} diag(b)
        assert abs(yn[i] - 1.0 / np.conj(dT)) <= 1e-12 * abs(1.0 / dT)
        assert left.left_residual(p, lam, y) <= 1e-15


def test_residue_of_the_resolvent_of_a_coupled_problem():
    p = synth.delay_2d(s=8, seed=1)
    V = synth.random_probe_block(p.n, 16, 0)
    r = ciss.solve(p, N=16, L=16, M=4, V=V)
    assert len(r["lam"]) >= 3
    for k in range(3):
        lam, x = r["lam"][k], r["X"][:, k]
        y = left.keldysh_normalise(p, lam, x, left.left_eigenvector(p, lam))
        assert left.left_residual(p, lam, y) <= 1e-13
        xy = np.outer(x, y.conj())
        err = []
        for e in (1e-7, 1e-8):
            eps = e * max(1.0, abs(lam))
            Rz = eps * np.linalg.inv(left.dense_T(p, lam + eps))
            err.append(np.abs(Rz - xy).max() / np.abs(xy).max())
        # the remainder is O(eps): one decade of eps, one decade of error (a misscaled y would
        # leave an error that does not shrink)
        assert err[1] <= 1e-5 and 8.0 <= err[0] / err[1] <= 12.0, err


def test_adjoint_solve_identity():
    p = synth.delay_2d(s=5, seed=0)
    rng = np.random.default_rng(4)
    z = -1.5 + 0.4j
    b = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    v = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    w = left.adjoint_solve(p, z, b)
    assert abs(np.vdot(w, left.dense_T(p, z) @ v) - np.vdot(b, v)) <= 1e-12 * np.linalg.norm(b) * np.linalg.norm(v) * 10
