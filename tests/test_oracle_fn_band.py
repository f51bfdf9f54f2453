"""Pins of the oracle's scalar functions, band assembly, banded LU and banded solve (CPU only)."""
import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack as lapack
import scipy.sparse as sp

import synth
from oracle import band, contour, fn


def _fd(spec, z, h=1e-6):
    return (fn.values(spec, z + h) - fn.values(spec, z - h)) / (2 * h)


SPECS = [
    {"kind": "rational", "num": [-1.0, 0.0], "den": None, "alpha": 1.0, "beta": 1.0},
    {"kind": "rational", "num": [-1.0, -0.1j, 9.0, 0.0], "den": [1.0, 0.1j], "alpha": 1.0, "beta": 1.0},
    {"kind": "exp", "alpha": -1.0, "beta": 2.0},
    {"kind": "sqrt", "alpha": 1.0, "beta": 1j, "shift": 1.0},
    {"kind": "combine", "op": "mul", "alpha": 1.0, "beta": 1.0,
     "a": {"kind": "exp", "alpha": -1.0, "beta": 1.0},
     "b": {"kind": "rational", "num": [1.0, 2.0], "den": None, "alpha": 1.0, "beta": 1.0}},
    {"kind": "combine", "op": "compose", "alpha": 0.5, "beta": 3.0,
     "a": {"kind": "sqrt", "alpha": 1.0, "beta": 1.0, "shift": 0.0},
     "b": {"kind": "exp", "alpha": 1.0, "beta": 1.0}},
    {"kind": "combine", "op": "div", "alpha": 1.0, "beta": 1.0,
     "a": {"kind": "exp", "alpha": 1.0, "beta": 1.0},
     "b": {"kind": "rational", "num": [1.0, 3.0], "den": None, "alpha": 1.0, "beta": 1.0}},
]


@pytest.mark.parametrize("spec", SPECS)
def test_fn_derivative_matches_finite_difference(spec):
    z = np.array([2.5 + 0.3j, 4.0 - 1.0j, 1.7 + 0.01j])
    d = fn.derivatives(spec, z)
    assert np.allclose(d, _fd(spec, z), rtol=1e-7, atol=1e-8)


def test_fn_values_closed_forms():
    z = np.array([0.5 + 0.5j, -1.0 + 2.0j])
    assert np.allclose(fn.values({"kind": "exp", "alpha": -1.0, "beta": 2.0}, z), 2 * np.exp(-z))
    # principal square root: sqrt(-4 + 0i) = 2i, cut on the negative axis
    assert np.isclose(fn.values({"kind": "sqrt", "alpha": 1.0, "beta": 1.0, "shift": 0.0}, -4.0 + 0j), 2j)
    # Drude: -z^2 eps(z) with eps = 1 - wp^2/(z(z + i g))
    wp, g = 3.0, 0.1
    spec = synth.problems._drude_fns(wp, g)[2]
    eps = 1 - wp ** 2 / (z * (z + 1j * g))
    assert np.allclose(fn.values(spec, z), -z ** 2 * eps, rtol=1e-14)


def test_band_assembly_matches_dense():
    p = synth.delay_2d(s=7, seed=3)
    kl, ku = band.bandwidths(p.mats)
    assert (kl, ku) == (7, 7)
    z = np.array([-1.3 + 0.7j])
    F = contour.coefficient_table(p.fns, z)[:, 0]
    ab = band.assemble_band(p.mats, F, kl, ku)
    T = band.assemble_dense(p.mats, F)
    n = p.n
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            assert ab[kl + ku + i - j, j] == T[i, j]
    # dense reference built entry by entry from the split form
    Tref = sum(F[i] * p.mats[i].toarray() for i in range(len(F)))
    assert np.array_equal(T, Tref)


def _rand_band(n, kl, ku, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            A[i, j] = rng.standard_normal() + 1j * rng.standard_normal()
    return A


@pytest.mark.parametrize("n,kl,ku", [(30, 3, 2), (41, 5, 5), (17, 1, 4), (12, 11, 11)])
def test_band_lu_matches_lapack_zgbtrf(n, kl, ku):
    A = _rand_band(n, kl, ku, seed=n + kl)
    ldab = 2 * kl + ku + 1
    ab = np.zeros((ldab, n), dtype=np.complex128, order="F")
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[kl + ku + i - j, j] = A[i, j]
    lu_ref, piv_ref, info_ref = lapack.zgbtrf(ab.copy(order="F"), kl, ku)
    lu, piv, info = band.gbtrf(ab.copy(order="F"), kl, ku)
    assert info == info_ref == 0
    assert np.array_equal(piv, piv_ref)
    assert np.allclose(lu, lu_ref, rtol=1e-12, atol=1e-12)
    B = np.asfortranarray(np.random.default_rng(1).standard_normal((n, 3)) + 0j)
    X = band.gbtrs(lu, kl, ku, piv, B)
    assert np.allclose(X, np.linalg.solve(A, B), rtol=1e-11, atol=1e-11)


def test_band_lu_zero_pivot_reports_column():
    n, kl, ku = 8, 2, 2
    A = _rand_band(n, kl, ku, seed=5)
    A[:, 4] = 0.0
    ldab = 2 * kl + ku + 1
    ab = np.zeros((ldab, n), dtype=np.complex128, order="F")
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[kl + ku + i - j, j] = A[i, j]
    _, _, info = band.gbtrf(ab, kl, ku)
    _, _, info_ref = lapack.zgbtrf(ab.copy(order="F"), kl, ku)
    assert info == 5 == info_ref


def test_dense_case_is_band_with_full_width():
    n = 9
    rng = np.random.default_rng(2)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    kl = ku = n - 1
    ldab = 2 * kl + ku + 1
    ab = np.zeros((ldab, n), dtype=np.complex128, order="F")
    for j in range(n):
        for i in range(n):
            ab[kl + ku + i - j, j] = A[i, j]
    lu, piv, info = band.gbtrf(ab, kl, ku)
    b = np.asfortranarray(rng.standard_normal((n, 1)) + 0j)
    assert np.allclose(band.gbtrs(lu, kl, ku, piv, b), scipy.linalg.solve(A, b))
