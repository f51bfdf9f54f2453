"""Interpol (Sec. 4.4) on the device, through the C ABI: Chebyshev interpolation on the region's real
axis and shift-and-invert Arnoldi on the Chebyshev-basis linearisation of P_d, against

  * the Lambert W real roots of decoupled delay problems on an interval (closed form);
  * an exactly interpolated quadratic problem against its own companion pencil;
  * the oracle's dense linearisation of a coupled delay problem (same d, same interval);
  * the fast mode (complex64 solves, residual inverse iteration on T) against the same closed form.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import interpol
from tests.gpu_util import match_eigenvalues, torch_cuda
from tests.test_oracle_interpol import lambert_real, quadratic_problem, real_delay_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("fast", [0, 1])
def test_real_delay_lambert(bnd, seed, fast):
    torch_cuda()
    p = real_delay_problem(seed=seed)
    split = bnd.Split.from_problem(p)
    res = bnd.interpol_solve(split, p.region, degree=40, krylov=60, fast_solves=fast)
    ref = lambert_real(p)
    assert len(res["lam"]) == len(ref), (res["lam"], ref)
    assert np.abs(np.sort(res["lam"].real) - ref).max() <= 1e-10
    assert res["eta"].max() <= 1e-10
    ora = interpol.solve(p, p.region, 40)
    err, _ = match_eigenvalues(res["lam"], ora["lam"])
    assert err <= 1e-10


def test_quadratic_exact(bnd):
    torch_cuda()
    p, A = quadratic_problem()
    n = p.n
    Z, I = np.zeros((n, n)), np.eye(n)
    ref = scipy.linalg.eigvals(np.block([[Z, I], [-A[0], -A[1]]]), np.block([[I, Z], [Z, A[2]]]))
    ref = ref[np.abs(ref / 1.5) < 1]
    split = bnd.Split.from_problem(p)
    res = bnd.interpol_solve(split, p.region, degree=4, krylov=16)
    err, _ = match_eigenvalues(res["lam"], ref)
    assert err <= 1e-9


def test_coupled_delay_against_the_oracle_pencil(bnd):
    torch_cuda()
    p = synth.delay_2d(s=5, seed=3, center=-1.5, radius=1.5)
    region = {"center": -1.5 + 0j, "a": 1.5, "b": 0.3}
    d = 30
    ora = interpol.solve(p, region, d)
    assert len(ora["lam"]) >= 1
    split = bnd.Split.from_problem(p)
    res = bnd.interpol_solve(split, region, degree=d, krylov=120)
    err, pairs = match_eigenvalues(res["lam"], ora["lam"])
    assert err <= 1e-9
    for i, j in pairs:
        assert 1.0 - abs(np.vdot(res["X"][:, i], ora["X"][:, j])) <= 1e-8


def test_refusals(bnd):
    torch_cuda()
    p = real_delay_problem(seed=0)
    split = bnd.Split.from_problem(p)
    with pytest.raises(bnd.NepError) as e:
        bnd.interpol_solve(split, {"center": -0.25 + 0.1j, "a": 2.25, "b": 0.1})
    assert e.value.code == bnd.NEP_ERR_ARG
    with pytest.raises(bnd.NepError) as e:
        bnd.interpol_solve(split, p.region, degree=64)
    assert e.value.code == bnd.NEP_ERR_ARG


def test_coupled_delay_with_restarts(bnd):
    """Krylov-Schur restarts (cycles of 40 restarted to 24 vectors, until as many pairs as the oracle
    pencil has inside the region have converged) reach the oracle pencil's eigenvalues that one
    120-step cycle reaches."""
    torch_cuda()
    p = synth.delay_2d(s=5, seed=3, center=-1.5, radius=1.5)
    region = {"center": -1.5 + 0j, "a": 1.5, "b": 0.3}
    d = 30
    ora = interpol.solve(p, region, d)
    split = bnd.Split.from_problem(p)
    res = bnd.interpol_solve(split, region, degree=d, krylov=40, keep=24, max_restarts=30, nev=len(ora["lam"]))
    assert res["info"]["restarts"] >= 1
    assert len(res["lam"]) == len(ora["lam"])
    err, _ = match_eigenvalues(res["lam"], ora["lam"])
    assert err <= 1e-9
