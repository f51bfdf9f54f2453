"""Pins of the oracle's compact (TOAR) Arnoldi for NLEIGS (Sec. 4.5.3) (CPU only): its Krylov
vectors, rebuilt as (I_d (x) U) g, and its Hessenberg matrix equal those of a plain full-basis
Arnoldi with the explicit S = (A - sigma B)^{-1} B from the same start; its Ritz values near the
shift are eigenvalues of the linearisation; U keeps orthonormal columns and grows by one per step."""
import numpy as np
import pytest

import synth
from oracle import nleigs


@pytest.mark.parametrize("name", ["delay1d", "delay2d"])
def test_toar_equals_the_full_basis_arnoldi(name):
    # n >= d + k, so that U can grow by one column every step
    p = synth.delay_1d(n=64, seed=0) if name == "delay1d" else synth.delay_2d(s=8, seed=2)
    it = nleigs.interpolation(p.fns, p.region)
    d, n, k = it["d"], p.n, 30
    sigma = complex(p.region["center"]) + 0.1j
    w0 = np.random.default_rng(5).standard_normal((n, d)) + 1j * np.random.default_rng(6).standard_normal((n, d))
    U, G, H = nleigs.arnoldi_toar(p, it, sigma, w0, k)
    assert U.shape == (n, d + k)
    assert np.abs(U.conj().T @ U - np.eye(d + k)).max() <= 1e-12
    S = nleigs.shift_invert_dense(p, it, sigma)
    V, Hf = nleigs.arnoldi_full(S, w0.T.reshape(-1), k)
    Vt = nleigs.toar_vectors(U, G, d)
    assert np.abs(Vt - V).max() <= 1e-10
    assert np.abs(H - Hf).max() <= 1e-10 * np.abs(Hf).max()
    # converged Ritz pairs are eigenpairs of T: the first block of the Ritz vector, rebuilt from
    # the compact representation, has a small scaled residual of the full T
    from oracle import ciss
    theta, s = np.linalg.eig(H[:k, :k])
    res = np.abs(H[k, k - 1] * s[k - 1, :])
    norms = ciss.term_norms_inf(p.mats)
    conv = [q for q in range(k) if res[q] <= 1e-12 * abs(theta[q])]
    assert len(conv) >= 3
    for q in conv:
        lam = sigma + 1.0 / theta[q]
        x = Vt[:n, :k] @ s[:, q]
        assert ciss.scaled_residual(p.mats, p.fns, norms, lam, x) <= 1e-9


def test_toar_with_fewer_rows_than_basis_vectors():
    """n < d + k: y^0 falls into span(U) once U has n columns; U then stops growing (no column of
    NaNs), and the Krylov vectors and Hessenberg matrix still equal the full-basis Arnoldi's."""
    p = synth.diagonal_delay(n=6, seed=1)
    it = nleigs.interpolation(p.fns, p.region)
    d, n, k = it["d"], p.n, 12
    assert n < d + k
    sigma = complex(p.region["center"]) + 0.1j
    rng = np.random.default_rng(7)
    w0 = rng.standard_normal((n, d)) + 1j * rng.standard_normal((n, d))
    U, G, H = nleigs.arnoldi_toar(p, it, sigma, w0, k)
    assert U.shape == (n, n) and np.all(np.isfinite(U))
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= 1e-12
    S = nleigs.shift_invert_dense(p, it, sigma)
    V, Hf = nleigs.arnoldi_full(S, w0.T.reshape(-1), k)
    assert np.abs(nleigs.toar_vectors(U, G, d) - V).max() <= 1e-10
    assert np.abs(H - Hf).max() <= 1e-10 * np.abs(Hf).max()
