"""NLEIGS, static variant, through the C ABI (nep_nleigs_interpolation, nep_nleigs_solve;
Sec. 4.5) against the oracle and closed forms.

  * the interpolation: the library's divided differences (its own matrix functions) equal the
    oracle's (scipy's) matrix-function divided differences for the library's own nodes, poles and
    scalings; those satisfy the Leja-Bagby conditions and max |b_j| = 1 on the boundary; the
    degree is the oracle's;
  * the eigenvalues: Lambert W (decoupled delay), companion roots (decoupled Drude), quadratic
    roots (decoupled square root), a linear pencil's generalized eigenvalues, and the oracle's
    linearisation eigenvalues of a coupled delay problem;
  * refusals: too many terms, a branch cut inside the region, bad options.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import ciss, contour, fn, nleigs
from tests.gpu_util import match_eigenvalues, torch_cuda
from tests.test_oracle_pins import drude_reference, lambert_reference, sqrt_reference

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


PROBLEMS = {
    "delay": lambda: synth.diagonal_delay(n=8, seed=0),
    "drude": lambda: synth.diagonal_drude(n=6, seed=0),
    "sqrt": lambda: synth.diagonal_sqrt(n=6, seed=0),
    "linear": lambda: synth.dense_linear_small(n=8, seed=3),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_interpolation_matches_the_oracle(bnd, name):
    torch_cuda()
    p = PROBLEMS[name]()
    split = bnd.Split.from_problem(p)
    it = bnd.nleigs_interpolation(split, p.region)
    ora = nleigs.interpolation(p.fns, p.region)
    assert it["converged"]
    assert it["d"] == ora["d"], (it["d"], ora["d"])
    assert it["nsing"] == len(ora["Xi"])
    d = it["d"]
    sig, xi, beta = it["sigma"], it["xi"].copy(), it["beta"]
    xi[~np.isfinite(xi)] = np.inf
    # nodes on the boundary, scalings max |b_j| = 1 there
    bndry = nleigs.boundary(p.region)
    assert all(np.abs(bndry - s).min() <= 1e-12 for s in sig)
    b = nleigs.basis(bndry, sig, xi, beta, d)
    assert np.allclose(np.abs(b).max(axis=1), 1.0, rtol=1e-13)
    # divided differences: the library's matrix functions vs scipy's (oracle) for the same nodes
    ref = nleigs.divided_differences(p.fns, sig, xi, beta, d)
    assert np.abs(it["dd"] - ref).max() <= 1e-11 * np.abs(ref[:, 0]).max()
    # the interpolant reproduces the f_i on the boundary
    r = it["dd"] @ b
    f = np.array([fn.values(g, bndry) for g in p.fns])
    assert np.abs(r - f).max() <= 1e-11 * np.abs(f).max()


def _solve(bnd, p, **kw):
    split = bnd.Split.from_problem(p)
    it = bnd.nleigs_interpolation(split, p.region)
    kw.setdefault("krylov", min(120, it["d"] * p.n))
    return bnd.nleigs_solve(split, p.region, **kw)


@pytest.mark.parametrize("seed", [0, 1])
def test_delay_eigenvalues_are_lambert_w(bnd, seed):
    torch_cuda()
    p = synth.diagonal_delay(n=8, seed=seed)
    r = _solve(bnd, p)
    ref = lambert_reference(p)
    err, _ = match_eigenvalues(r["lam"], ref)
    assert err <= 1e-11, err
    assert r["eta"].max() <= 1e-12


def test_drude_sqrt_and_linear_closed_forms(bnd):
    torch_cuda()
    p = synth.diagonal_drude(n=6, seed=0)
    err, _ = match_eigenvalues(_solve(bnd, p)["lam"], drude_reference(p))
    assert err <= 1e-10, err
    p = synth.diagonal_sqrt(n=6, seed=0)
    err, _ = match_eigenvalues(_solve(bnd, p)["lam"], sqrt_reference(p))
    assert err <= 1e-10, err
    p = synth.dense_linear_small(n=8, seed=3)
    A, B = p.mats[0].toarray(), p.mats[1].toarray()
    ref = [e for e in scipy.linalg.eig(A, B, right=False) if contour.inside(p.region, e)]
    err, _ = match_eigenvalues(_solve(bnd, p)["lam"], ref)
    assert err <= 1e-10, err


def test_coupled_delay_problem_matches_the_oracle_linearisation(bnd):
    torch_cuda()
    p = synth.delay_2d(s=5, seed=1)
    ora = nleigs.solve(p)
    assert len(ora["lam"]) >= 3
    r = _solve(bnd, p, krylov=150)
    err, pairs = match_eigenvalues(r["lam"], ora["lam"])
    assert err <= 1e-10, err
    for i, j in pairs:
        assert abs(abs(np.vdot(r["X"][:, i], ora["X"][:, j])) - 1.0) <= 1e-9
    # the returned pairs are eigenpairs of T itself (oracle residual)
    norms = ciss.term_norms_inf(p.mats)
    for q in range(len(r["lam"])):
        assert ciss.scaled_residual(p.mats, p.fns, norms, r["lam"][q], r["X"][:, q]) <= 1e-11


def test_refusals(bnd):
    torch_cuda()
    p = synth.diagonal_sqrt(n=6, seed=0)
    split = bnd.Split.from_problem(p)
    with pytest.raises(bnd.NepError) as e:  # the cut (-inf, 1] crosses this region
        bnd.nleigs_solve(split, {"center": 1.0, "a": 1.0, "b": 1.0})
    assert e.value.code == bnd.NEP_ERR_REGION
    with pytest.raises(bnd.NepError) as e:
        bnd.nleigs_solve(split, p.region, max_degree=64)
    assert e.value.code == bnd.NEP_ERR_ARG
    with pytest.raises(bnd.NepError) as e:
        bnd.nleigs_solve(split, {"center": 4.0, "a": 0.0, "b": 1.0})
    assert e.value.code == bnd.NEP_ERR_ARG


def test_full_size_delay_problem_agrees_with_the_contour_solver(bnd):
    """n = 4096, bandwidth 64: no dense oracle at this size; every returned pair is checked by the
    oracle's scaled residual on the host, and the eigenvalues against the contour solver's."""
    torch = torch_cuda()
    from tests.gpu_util import to_dev
    p = synth.config_problem("delay2d_s64")
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=0)
    plan.execute(to_dev(np.asfortranarray(synth.random_probe_block(p.n, p.L, 0)), torch))
    torch.cuda.synchronize()
    rc = plan.result()
    r = bnd.nleigs_solve(split, p.region, krylov=150)
    assert len(rc["lam"]) >= 5 and len(r["lam"]) == len(rc["lam"]), (len(r["lam"]), len(rc["lam"]))
    err, _ = match_eigenvalues(r["lam"], rc["lam"])
    assert err <= 1e-9, err
    norms = ciss.term_norms_inf(p.mats)
    for q in range(len(r["lam"])):
        assert ciss.scaled_residual(p.mats, p.fns, norms, r["lam"][q], r["X"][:, q]) <= 1e-11


def test_exact_solve_mode_matches_the_oracle_linearisation(bnd):
    """exact_solves = 1: each Arnoldi solve corrected against the FP64 residual, no polish."""
    torch_cuda()
    p = synth.delay_2d(s=5, seed=1)
    ora = nleigs.solve(p)
    r = _solve(bnd, p, krylov=150, exact_solves=1)
    err, _ = match_eigenvalues(r["lam"], ora["lam"])
    assert err <= 1e-10, err
    assert r["eta"].max() <= 1e-11


@pytest.mark.parametrize("full_basis", [0, 1])
def test_compact_and_full_basis_match_the_oracle_linearisation(bnd, full_basis):
    """n = 36 >= d: the compact (TOAR) basis of Sec. 4.5.3 (default) and the full basis give the
    oracle's linearisation eigenvalues and vectors."""
    torch_cuda()
    p = synth.delay_2d(s=6, seed=1)
    split = bnd.Split.from_problem(p)
    assert p.n >= bnd.nleigs_interpolation(split, p.region)["d"]
    ora = nleigs.solve(p)
    assert len(ora["lam"]) >= 3
    r = _solve(bnd, p, krylov=150, full_basis=full_basis)
    err, pairs = match_eigenvalues(r["lam"], ora["lam"])
    assert err <= 1e-10, err
    for i, j in pairs:
        assert abs(abs(np.vdot(r["X"][:, i], ora["X"][:, j])) - 1.0) <= 1e-9


def test_compact_basis_equals_full_basis_at_full_size(bnd):
    """n = 4096: the same start vector and steps give the same eigenpairs with either basis."""
    torch_cuda()
    p = synth.config_problem("delay2d_s64")
    split = bnd.Split.from_problem(p)
    a = bnd.nleigs_solve(split, p.region, krylov=100)
    b = bnd.nleigs_solve(split, p.region, krylov=100, full_basis=1)
    assert len(a["lam"]) == len(b["lam"]) >= 5
    err, _ = match_eigenvalues(a["lam"], b["lam"])
    assert err <= 1e-10, err


def _oracle_restarted(p, ncv, nkeep):
    """The oracle's Krylov-Schur restart on the explicit S of the linearisation (shift: the centre)."""
    it = nleigs.interpolation(p.fns, p.region)
    sigma = complex(p.region["center"])
    S = nleigs.shift_invert_dense(p, it, sigma)
    rng = np.random.default_rng(3)
    v0 = rng.standard_normal(S.shape[0]) + 1j * rng.standard_normal(S.shape[0])
    wanted = lambda th: contour.inside(p.region, np.array([sigma + 1.0 / th]))[0]
    r = nleigs.krylov_schur(S, v0, ncv=ncv, nkeep=nkeep, wanted=wanted, tol=1e-10, max_restarts=40)
    assert r["restarts"] >= 1 and len(r["converged"]) == len(r["wanted"])
    return np.array([sigma + 1.0 / r["theta"][q] for q in r["converged"]])


@pytest.mark.parametrize("full_basis", [0, 1])
def test_restarted_arnoldi_finds_what_the_oracle_restart_finds(bnd, full_basis):
    """Krylov-Schur restarts with locking (Sec. 4.5.3): cycles of 40 steps restarted to 30 vectors
    find every eigenvalue of the linearisation inside the region (23 of them), the set the oracle's
    restarted Arnoldi on the explicit operator converges to; one cycle of 40 steps alone does not.
    Both bases (n = 36 >= d: the compact basis is compressed at each restart)."""
    torch_cuda()
    p = synth.delay_2d(s=6, seed=1)
    split = bnd.Split.from_problem(p)
    lam_o = _oracle_restarted(p, 40, 30)
    ref = nleigs.solve(p)["lam"]
    assert len(lam_o) == len(ref) == 23
    kw = dict(krylov=40, keep=30, max_restarts=40, restart_tol=1e-10, full_basis=full_basis)
    r = bnd.nleigs_solve(split, p.region, exact_solves=1, **kw)
    assert 1 <= r["info"]["restarts"] <= 40
    assert r["info"]["krylov_steps"] > 40
    assert len(r["lam"]) == len(lam_o), (len(r["lam"]), len(lam_o))
    err, pairs = match_eigenvalues(r["lam"], lam_o)
    assert err <= 1e-10, err
    assert r["eta"].max() <= 1e-10  # the pairs converged to |b^T s| <= 1e-10 |theta|
    # complex64 solves (convergence at 1e-6, then the polish) give the same eigenvalues
    kw["restart_tol"] = 0.0
    f = bnd.nleigs_solve(split, p.region, **kw)
    assert len(f["lam"]) == len(lam_o)
    err, _ = match_eigenvalues(f["lam"], lam_o)
    assert err <= 1e-10, err
    one = bnd.nleigs_solve(split, p.region, krylov=40, exact_solves=1, full_basis=full_basis)
    assert one["info"]["restarts"] == 0 and one["info"]["krylov_steps"] == 40
    assert len(one["lam"]) < len(lam_o)


def test_restarted_compact_basis_at_full_size(bnd):
    """n = 4096: cycles of 40 steps restarted to 20 vectors give the contour solver's eigenvalues
    (FP64 plan) and the same set as one 100-step cycle."""
    torch = torch_cuda()
    from tests.gpu_util import to_dev
    p = synth.config_problem("delay2d_s64")
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=0)
    plan.execute(to_dev(np.asfortranarray(synth.random_probe_block(p.n, p.L, 0)), torch))
    torch.cuda.synchronize()
    rc = plan.result()
    r = bnd.nleigs_solve(split, p.region, krylov=40, keep=20, max_restarts=30)
    assert r["info"]["restarts"] >= 1
    assert len(r["lam"]) == len(rc["lam"]) >= 5, (len(r["lam"]), len(rc["lam"]))
    err, _ = match_eigenvalues(r["lam"], rc["lam"])
    assert err <= 1e-9, err
    norms = ciss.term_norms_inf(p.mats)
    for q in range(len(r["lam"])):
        assert ciss.scaled_residual(p.mats, p.fns, norms, r["lam"][q], r["X"][:, q]) <= 1e-11


def test_restart_option_refusals(bnd):
    torch_cuda()
    p = synth.diagonal_delay(n=8, seed=0)
    split = bnd.Split.from_problem(p)
    for kw in (dict(krylov=20, keep=20, max_restarts=3), dict(krylov=20, max_restarts=-1),
               dict(krylov=1, max_restarts=2)):
        with pytest.raises(bnd.NepError) as e:
            bnd.nleigs_solve(split, p.region, **kw)
        assert e.value.code == bnd.NEP_ERR_ARG
