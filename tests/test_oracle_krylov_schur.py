"""Pins of the oracle's Krylov-Schur restart with locking (the restart on top of Algorithm (nleigs),
Sec. 4.5.3) on the explicit shift-and-invert operator of NLEIGS's linearisation (CPU only):

  * after restarts the Krylov decomposition S V_k = V_{k+1} Hf holds to rounding (up to the locked
    residuals, below the convergence tolerance) and V stays orthonormal;
  * the converged wanted Ritz values give exactly the eigenvalues inside the region: the Lambert W
    values of a decoupled delay problem, all of them;
  * a short cycle with restarts finds the same eigenvalues as one long cycle without.
"""
import numpy as np

import synth
from oracle import contour, nleigs
from tests.test_oracle_pins import lambert_reference


def _setup(seed=0):
    p = synth.diagonal_delay(n=8, seed=seed)
    it = nleigs.interpolation(p.fns, p.region)
    sigma = complex(p.region["center"]) + 0.05j
    S = nleigs.shift_invert_dense(p, it, sigma)
    rng = np.random.default_rng(3)
    v0 = rng.standard_normal(S.shape[0]) + 1j * rng.standard_normal(S.shape[0])
    wanted = lambda th: contour.inside(p.region, np.array([sigma + 1.0 / th]))[0]
    return p, S, v0, sigma, wanted


def _eigs(r, sigma):
    return np.array([sigma + 1.0 / r["theta"][q] for q in r["converged"]])


def test_restarted_decomposition_and_eigenvalues():
    p, S, v0, sigma, wanted = _setup()
    ref = lambert_reference(p)
    r = nleigs.krylov_schur(S, v0, ncv=24, nkeep=14, wanted=wanted, tol=1e-12, max_restarts=40)
    assert r["restarts"] >= 1
    V, Hf = r["V"], r["Hf"]
    k = Hf.shape[1]
    assert np.abs(V.conj().T @ V - np.eye(k + 1)).max() <= 1e-12
    assert np.abs(S @ V[:, :k] - V @ Hf).max() <= 1e-10 * np.abs(S).max()
    lam = _eigs(r, sigma)
    assert len(lam) == len(ref) == len(r["wanted"])
    for e in ref:
        assert np.min(np.abs(lam - e)) <= 1e-10 * max(1.0, abs(e))


def test_restarts_find_what_one_long_cycle_finds():
    p, S, v0, sigma, wanted = _setup(seed=1)
    long = nleigs.krylov_schur(S, v0, ncv=150, nkeep=75, wanted=wanted, tol=1e-12, max_restarts=0)
    short = nleigs.krylov_schur(S, v0, ncv=24, nkeep=14, wanted=wanted, tol=1e-12, max_restarts=40)
    assert short["restarts"] >= 1
    a, b = _eigs(long, sigma), _eigs(short, sigma)
    assert len(a) == len(b) >= 3
    assert max(np.min(np.abs(b - x)) for x in a) <= 1e-10
    assert max(np.min(np.abs(a - x)) for x in b) <= 1e-10


def test_planted_unorthonormalised_restart_caught(monkeypatch):
    """A restart that keeps the selected Ritz vectors as they are (unit length, not orthonormalised)
    breaks the orthonormal basis and the decomposition."""
    p, S, v0, sigma, wanted = _setup()
    real_qr = np.linalg.qr
    monkeypatch.setattr(np.linalg, "qr", lambda A, *a, **k: (A / np.linalg.norm(A, axis=0), None))
    r = nleigs.krylov_schur(S, v0, ncv=24, nkeep=14, wanted=wanted, tol=1e-12, max_restarts=3)
    monkeypatch.setattr(np.linalg, "qr", real_qr)
    V, Hf = r["V"], r["Hf"]
    k = Hf.shape[1]
    bad_orth = np.abs(V.conj().T @ V - np.eye(k + 1)).max()
    bad_rel = np.abs(S @ V[:, :k] - V @ Hf).max() / np.abs(S).max()
    assert bad_orth > 1e-6 or bad_rel > 1e-6


def test_nev_stops_once_that_many_wanted_pairs_converged():
    """With nev set, the run ends once nev wanted pairs have converged: nev = 3 stops earlier than
    the default (all wanted pairs), and its converged pairs are Lambert W eigenvalues."""
    p, S, v0, sigma, wanted = _setup()
    ref = lambert_reference(p)
    few = nleigs.krylov_schur(S, v0, ncv=24, nkeep=14, wanted=wanted, tol=1e-12, max_restarts=40, nev=3)
    full = nleigs.krylov_schur(S, v0, ncv=24, nkeep=14, wanted=wanted, tol=1e-12, max_restarts=40)
    assert len(few["converged"]) >= 3 and few["restarts"] <= full["restarts"]
    for e in _eigs(few, sigma):
        assert np.min(np.abs(np.array(ref) - e)) <= 1e-10 * max(1.0, abs(e))
