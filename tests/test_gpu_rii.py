"""Residual inverse iteration on the device (nep_rii, nep_plan_polish; Sec. 4.1, Algorithm (rii))
against the oracle's iteration and the closed forms that pin it.

The starting pairs are seeded perturbations of known eigenpairs (Lambert W values of decoupled
delay problems, the oracle's contour pairs of a coupled problem); both sides receive the same
starts. The results are compared after convergence: eigenvalues to 1e-11..1e-12 relative,
eigenvectors up to a phase, and eta below the requested tolerance."""
import numpy as np
import pytest
from scipy.special import lambertw

import synth
from oracle import ciss, contour, rii
from tests.gpu_util import from_dev_c128, match_eigenvalues, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _lambert_pairs(p):
    a, b = p.meta["a"], p.meta["b"]
    out = []
    for i in range(p.n):
        for k in range(-6, 7):
            lam = complex(a[i] + lambertw(b[i] * np.exp(-a[i]), k))
            if contour.inside(p.region, lam):
                out.append((lam, i))
    return out


def _device_rii(bnd, torch, p, precision, lam0, X0, tol, max_it=10):
    P = len(lam0)
    split = bnd.Split.from_problem(p)
    lam_d = to_dev(np.asarray(lam0, np.complex128), torch)
    X_d = to_dev(np.asfortranarray(X0), torch)
    eta_d = torch.zeros(P, dtype=torch.float64, device="cuda")
    its_d = torch.zeros(P, dtype=torch.int32, device="cuda")
    k = bnd.rii(split, precision, P, lam_d, X_d, eta_d, its_d, tol=tol, max_it=max_it)
    torch.cuda.synchronize()
    X = from_dev_c128(X_d).reshape(P, p.n).T
    return from_dev_c128(lam_d), X, eta_d.cpu().numpy(), its_d.cpu().numpy(), k


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_rii_reaches_the_lambert_w_eigenpairs(bnd, precision, seed):
    torch = torch_cuda()
    p = synth.diagonal_delay(n=8, seed=seed)
    pairs = _lambert_pairs(p)
    rng = np.random.default_rng(100 + seed)
    lam0, X0 = [], np.zeros((p.n, len(pairs)), np.complex128)
    for q, (lam_ref, i) in enumerate(pairs):
        X0[:, q] = 1e-3 * (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n))
        X0[i, q] = 1.0
        lam0.append(lam_ref + 1e-3 * (1 + 1j) * max(1.0, abs(lam_ref)))
    lam, X, eta, its, k = _device_rii(bnd, torch, p, precision, lam0, X0, tol=1e-12)
    assert eta.max() < 1e-12, eta
    for q, (lam_ref, i) in enumerate(pairs):
        assert abs(lam[q] - lam_ref) <= 1e-12 * max(1.0, abs(lam_ref)), (q, lam[q], lam_ref)
        assert np.abs(np.delete(X[:, q], i)).max() <= 1e-10
        # the oracle's iteration from the same start lands on the same pair
        lo, xo, eo, _, ok = rii.rii(p, lam0[q], X0[:, q], tol=1e-12)
        assert ok and abs(lam[q] - lo) <= 1e-12 * max(1.0, abs(lo))
        assert abs(abs(np.vdot(X[:, q], xo)) - 1.0) <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_rii_recovers_perturbed_contour_pairs(bnd, precision):
    torch = torch_cuda()
    p = synth.delay_2d(s=8, seed=1)
    V = synth.random_probe_block(p.n, 16, 0)
    r = ciss.solve(p, N=16, L=16, M=4, V=V)
    P = len(r["lam"])
    assert P >= 10
    rng = np.random.default_rng(11)
    X0 = r["X"] + 1e-5 * (rng.standard_normal((p.n, P)) + 1j * rng.standard_normal((p.n, P)))
    lam0 = r["lam"] * (1 + 1e-5)
    lam, X, eta, its, k = _device_rii(bnd, torch, p, precision, lam0, X0, tol=1e-12)
    assert eta.max() < 1e-12, eta
    assert np.all(np.abs(lam - r["lam"]) <= 1e-11 * np.maximum(1.0, np.abs(r["lam"])))
    for q in range(P):
        assert abs(abs(np.vdot(X[:, q], r["X"][:, q])) - 1.0) <= 1e-10
        assert np.linalg.norm(X[:, q]) == pytest.approx(1.0, abs=1e-13)


def test_plan_polish_tightens_the_returned_pairs(bnd):
    torch = torch_cuda()
    p = synth.delay_2d(s=16, seed=3)
    V = synth.random_probe_block(p.n, p.L, 5)
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=1)
    plan.execute(to_dev(np.asfortranarray(V), torch))
    torch.cuda.synchronize()
    before = plan.result()
    tol = 1e-13
    assert before["eta"].max() >= tol  # mixed precision leaves eta at 1e-12 .. 1e-10
    polished, its = plan.polish(tol=tol, max_it=10)
    after = plan.result()
    assert polished == int((before["eta"] >= tol).sum()) and its >= 1
    assert len(after["lam"]) == len(before["lam"])
    assert after["eta"].max() < tol
    # the same pairs, closer to the FP64 oracle's eigenvalues
    ora = ciss.solve(p, V=V)
    err_b, _ = match_eigenvalues(before["lam"], ora["lam"])
    err_a, _ = match_eigenvalues(after["lam"], ora["lam"])
    assert err_a <= 1e-12, (err_a, err_b)
    assert np.all(np.abs(after["lam"] - before["lam"]) <= 1e-8 * np.maximum(1.0, np.abs(before["lam"])))
    # a second polish finds nothing left to do
    assert plan.polish(tol=tol)[0] == 0


def test_rii_refuses_bad_arguments(bnd):
    torch = torch_cuda()
    p = synth.diagonal_delay(n=8, seed=0)
    split = bnd.Split.from_problem(p)
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    for args in [(split, 1, -1, z, z, z), (split, 7, 1, z, z, z), (split, 1, 1, None, z, z)]:
        with pytest.raises(bnd.NepError) as e:
            bnd.rii(*args)
        assert e.value.code == bnd.NEP_ERR_ARG
    with pytest.raises(bnd.NepError) as e:
        bnd.rii(split, 1, 1, z, z, z, max_it=-1)
    assert e.value.code == bnd.NEP_ERR_ARG
