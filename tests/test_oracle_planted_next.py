"""Planted mistakes in the NLEIGS, left-eigenvector and residual-inverse-iteration oracles must be
caught by their pins (CPU only).

Each test monkeypatches one plausible error into the oracle and checks that an independent pin
(closed-form eigenvalues, the linear-pencil resolvent, the exact left vectors of decoupled
problems, the Lambert W fixed point of the iteration) then fails.
"""
import numpy as np
import scipy.linalg
from scipy.special import lambertw

import synth
from oracle import left, nleigs, rii
from tests.test_oracle_pins import _match, lambert_reference


def _nleigs_lambert_error():
    p = synth.diagonal_delay(n=8, seed=0)
    try:
        r = nleigs.solve(p)
    except Exception:
        return np.inf
    ref = lambert_reference(p)
    if len(r["lam"]) != len(ref):
        return np.inf
    return max(min(abs(l - e) for l in r["lam"]) for e in ref)


def _resolvent_error():
    p = synth.dense_linear_small(n=8, seed=3)
    A, B = (m.toarray() for m in p.mats)
    lams, Xr = scipy.linalg.eig(A, B)
    X = Xr / np.linalg.norm(Xr, axis=0)
    Y = np.stack([left.keldysh_normalise(p, lam, X[:, i], left.left_eigenvector(p, lam))
                  for i, lam in enumerate(lams)], axis=1)
    V = np.random.default_rng(1).standard_normal((p.n, 2)) + 0j
    z = 0.3 + 0.2j
    ref = np.linalg.solve(A - z * B, V)
    return np.abs(left.apply_resolvent(lams, X, Y, z, V) - ref).max() / np.abs(ref).max()


def _rii_error():
    p = synth.diagonal_delay(n=8, seed=0)
    a, b = p.meta["a"], p.meta["b"]
    lam_ref = complex(a[0] + lambertw(b[0] * np.exp(-a[0]), 0))
    x0 = np.zeros(p.n, np.complex128)
    x0[0] = 1.0
    x0[1] = 1e-3
    lam, x, eta, its, ok = rii.rii(p, lam_ref + 1e-3, x0, tol=1e-12)
    return abs(lam - lam_ref) if ok else np.inf


def test_unplanted_baselines():
    assert _nleigs_lambert_error() < 1e-12
    assert _resolvent_error() < 1e-11
    assert _rii_error() < 1e-12


def test_nleigs_linearisation_node_index_caught(monkeypatch):
    orig = nleigs.linearization

    def bad(mats, interp):
        A, B = orig(mats, interp)
        n, d, sig = mats[0].shape[0], interp["d"], interp["sigma"]
        for j in range(1, d):  # sigma_j where the recurrence of b_j needs sigma_{j-1}
            A[j * n:(j + 1) * n, (j - 1) * n:j * n] = sig[j] * np.eye(n)
        return A, B
    monkeypatch.setattr(nleigs, "linearization", bad)
    assert _nleigs_lambert_error() > 1e-6


def test_nleigs_linearisation_without_scalings_caught(monkeypatch):
    orig = nleigs.linearization

    def bad(mats, interp):
        it = dict(interp)
        it["beta"] = np.ones_like(interp["beta"])  # the pencil built without the beta_j
        return orig(mats, it)
    monkeypatch.setattr(nleigs, "linearization", bad)
    assert _nleigs_lambert_error() > 1e-6


def test_keldysh_without_conjugate_caught(monkeypatch):
    def bad(problem, lam, x, y):
        s = np.vdot(y, left.dense_T(problem, lam, derivative=True) @ x)
        return y / s  # conj missing
    monkeypatch.setattr(left, "keldysh_normalise", bad)
    assert _resolvent_error() > 1e-6


def test_left_vector_as_right_vector_caught(monkeypatch):
    def bad(problem, lam):
        U, s, Vh = np.linalg.svd(left.dense_T(problem, lam))
        return Vh[-1].conj()  # the right null vector instead of the left one
    monkeypatch.setattr(left, "left_eigenvector", bad)
    assert _resolvent_error() > 1e-6


def test_rii_without_residual_update_caught(monkeypatch):
    orig = rii.rii

    def bad(problem, lam0, x0, **kw):
        kw["max_it"] = 0  # no iteration at all: the start comes back unchanged
        return orig(problem, lam0, x0, **kw)
    monkeypatch.setattr(rii, "rii", bad)
    assert _rii_error() > 1e-6


def _interpol_errors():
    """(delay error vs Lambert W, quadratic error vs its companion eigenvalues), inf on failure."""
    from oracle import interpol
    from tests.test_oracle_interpol import lambert_real, quadratic_problem, real_delay_problem
    out = []
    p = real_delay_problem(seed=0)
    try:
        r = interpol.solve(p, p.region, 40)
        ref = lambert_real(p)
        out.append(np.abs(np.sort(r["lam"].real) - ref).max() if len(r["lam"]) == len(ref) else np.inf)
    except Exception:
        out.append(np.inf)
    p, A = quadratic_problem()
    n = p.n
    Z, I = np.zeros((n, n)), np.eye(n)
    ref = scipy.linalg.eigvals(np.block([[Z, I], [-A[0], -A[1]]]), np.block([[I, Z], [Z, A[2]]]))
    ref = ref[np.abs(ref / 1.5) < 1]
    try:
        r = interpol.solve(p, p.region, 4)
        out.append(max(np.min(np.abs(r["lam"] - l)) for l in ref) if len(r["lam"]) == len(ref) else np.inf)
    except Exception:
        out.append(np.inf)
    return out


def test_interpol_unplanted():
    assert max(_interpol_errors()) < 1e-10


def test_interpol_node_off_by_half_caught(monkeypatch):
    """Chebyshev points of the second kind's spacing (omega_j = j pi / (d+1)) instead of Eq. (interpolnu)."""
    from oracle import interpol

    def bad(d):
        om = np.arange(d + 1) * np.pi / (d + 1)
        return om, np.cos(om)
    monkeypatch.setattr(interpol, "chebyshev_nodes", bad)
    assert max(_interpol_errors()) > 1e-6


def test_interpol_unhalved_c0_caught(monkeypatch):
    """P_d with C_0 instead of C_0 / 2 (Eq. (polinterp))."""
    from oracle import interpol
    orig = interpol.coefficients

    def bad(fns, region, d):
        c = orig(fns, region, d)
        c[:, 0] *= 2.0
        return c
    monkeypatch.setattr(interpol, "coefficients", bad)
    assert max(_interpol_errors()) > 1e-6


def test_interpol_wrong_recurrence_row_caught(monkeypatch):
    """theta tau_k = tau_{k+1} + tau_{k-1} (the factor 1/2 of the Chebyshev recurrence dropped) in the
    linearisation's middle rows."""
    from oracle import interpol
    orig = interpol.pencil

    def bad(mats, c):
        A, B = orig(mats, c)
        n = mats[0].shape[0]
        d = c.shape[1] - 1
        for k in range(1, d - 1):
            B[k * n:(k + 1) * n, k * n:(k + 1) * n] *= 0.5
        return A, B
    monkeypatch.setattr(interpol, "pencil", bad)
    assert max(_interpol_errors()) > 1e-6
