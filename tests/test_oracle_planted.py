"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each test monkeypatches one plausible error into the oracle (a conjugated weight,
a shifted Hankel block, a dropped split-form term, a sign flip in the refinement
residual) and checks that a closed-form pin then fails.
"""
import numpy as np
import pytest

import synth
from oracle import band, ciss, contour
from tests.test_oracle_moments import moment_closed_form_error
from tests.test_oracle_pins import lambert_reference


def _lambert_error():
    p = synth.diagonal_delay(n=8, seed=0)
    V = synth.random_probe_block(p.n, p.L, 0)
    try:
        r = ciss.solve(p, V=V)
    except Exception:
        return np.inf
    ref = lambert_reference(p)
    if len(r["lam"]) != len(ref):
        return np.inf
    return max(min(abs(l - e) for l in r["lam"]) for e in ref)


def test_unplanted_baseline():
    assert moment_closed_form_error() < 1e-13
    assert _lambert_error() < 1e-12


def test_conjugated_weights_caught(monkeypatch):
    orig = contour.nodes

    def bad(region, N):
        z, w, zeta = orig(region, N)
        return z, np.conj(w), zeta
    monkeypatch.setattr(contour, "nodes", bad)
    assert moment_closed_form_error() > 1e-3


def test_hankel_shift_caught(monkeypatch):
    orig = ciss.hankel_matrices

    def bad(mu):
        H, Hs = orig(mu)
        return H, H.copy()
    monkeypatch.setattr(ciss, "hankel_matrices", bad)
    assert _lambert_error() > 1e-6


def test_dropped_term_caught(monkeypatch):
    orig = band.assemble_sparse

    def bad(mats, coeffs):
        return orig(mats[:-1], coeffs[:-1])
    monkeypatch.setattr(band, "assemble_sparse", bad)
    monkeypatch.setattr(band, "assemble_band", lambda mats, coeffs, kl, ku: _band_without_last(mats, coeffs, kl, ku))
    assert _lambert_error() > 1e-6


def _band_without_last(mats, coeffs, kl, ku):
    n = mats[0].shape[0]
    ab = np.zeros((2 * kl + ku + 1, n), dtype=np.complex128, order="F")
    import scipy.sparse as sp
    T = sp.coo_matrix(sum(c * A for A, c in zip(mats[:-1], coeffs[:-1])))
    ab[kl + ku + T.row - T.col, T.col] = T.data
    return ab


def test_wrong_refinement_sign_caught(monkeypatch):
    """A refinement step that adds T Y instead of subtracting must break the moment pin."""
    orig = ciss.solve_point

    def bad(problem, kl, ku, coeffs, V, **kw):
        r = orig(problem, kl, ku, coeffs, V, refine_max=0)
        T = band.assemble_sparse(problem.mats, coeffs)
        ab = band.assemble_band(problem.mats, coeffs, kl, ku)
        ab, ipiv, _ = band.gbtrf(ab, kl, ku)
        Y = r["Y"]
        R = V + T @ Y
        r["Y"] = Y + band.gbtrs(ab, kl, ku, ipiv, R)
        return r
    monkeypatch.setattr(ciss, "solve_point", bad)
    assert moment_closed_form_error() > 1e-3


def _lambert_matched(p, L):
    V = synth.random_probe_block(p.n, L, 0)
    r = ciss.solve(p, V=V, L=L)
    ref = lambert_reference(p)
    return sum(1 for e in ref if len(r["lam"]) and np.min(np.abs(r["lam"] - e)) <= 1e-12 * max(1.0, abs(e)))


def test_eager_newton_abandonment_caught(monkeypatch):
    """Giving up on a Newton iterate that is unconverged and outside Gamma by 10% after 3 steps
    loses a Lambert W eigenvalue: on this decoupled delay problem (probe block of 2 columns) the
    only Newton path that reaches lambda = -0.3211 lies outside Gamma at step 3 and converges
    inside at step 9."""
    p = synth.diagonal_delay(n=8, seed=8)
    plain = _lambert_matched(p, 2)
    assert plain >= 1
    orig = ciss.newton_projected
    c = complex(p.region["center"])
    a, b = p.region["a"], p.region["b"]

    def eager(Bs, fns, lam0, y0, region):
        monkeypatch.setattr(ciss, "NEWTON_MAX", 3)
        lam, y, ok, it = orig(Bs, fns, lam0, y0, region)
        monkeypatch.setattr(ciss, "NEWTON_MAX", 30)
        if ok and it == 3 and ((lam - c).real / a) ** 2 + ((lam - c).imag / b) ** 2 > 1.21:
            return lam, y, False, it
        return orig(Bs, fns, lam0, y0, region)
    monkeypatch.setattr(ciss, "newton_projected", eager)
    assert _lambert_matched(p, 2) < plain
