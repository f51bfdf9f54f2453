"""Failure paths of the device pass, made safely: no fault, trap or endless wait.

  * an eigenvalue exactly on a quadrature node: T(z_0) is singular, the LU meets an exactly zero
    pivot; the call flags NEP_WARN_SINGULAR_NODE, that node contributes nothing and the result is
    finite, with the eigenvalues strictly inside equal to the closed form and to the oracle's;
  * a refinement budget of one sweep on complex64 factors: the backward-error target is missed
    and NEP_WARN_REFINE is raised;
  * a device-side wait bound of zero polls: the grid barriers of the Jacobi SVD give up, the call
    returns NEP_ERR_INTERNAL, and the same call succeeds once the bound is restored.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import ciss
from tests.gpu_util import from_dev_c128, match_eigenvalues, to_dev, torch_cuda
from tests.test_oracle_pins import diagonal_linear_on_node

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _solve(bnd, p, V, precision, **opts):
    torch = torch_cuda()
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=precision, **opts)
    plan.execute(to_dev(np.asfortranarray(V), torch))
    torch.cuda.synchronize()
    return plan.result()


@pytest.mark.parametrize("precision", [0, 1])
def test_eigenvalue_on_a_node(bnd, precision):
    z, _, _ = bnd.nodes({"center": 0.0, "a": 1.0, "b": 1.0}, 16)
    p = diagonal_linear_on_node(z[0])
    V = synth.random_probe_block(p.n, p.L, 0)
    res = _solve(bnd, p, V, precision)
    assert res["flags"] & bnd.NEP_WARN_SINGULAR_NODE
    assert np.all(np.isfinite(res["lam"])) and np.all(np.isfinite(res["X"]))
    assert np.all(np.isfinite(res["sigma"]))
    inside = [complex(x) for x in p.meta["d"][1:] if abs(x) < 1]
    found = [l for l in res["lam"] if abs(l - p.meta["d"][0]) > 1e-8]
    err, _ = match_eigenvalues(found, inside)
    assert err <= 1e-12
    ora = ciss.solve(p, V=V)
    ora_found = [l for l in ora["lam"] if abs(l - p.meta["d"][0]) > 1e-8]
    err, _ = match_eigenvalues(found, ora_found)
    assert err <= 1e-12


def test_one_refinement_sweep_misses_the_target(bnd):
    p = synth.delay_2d(s=12, seed=2, center=-1.5, radius=1.5)
    V = synth.random_probe_block(p.n, 8, 5)
    p.N, p.L, p.M = 32, 8, 4
    res = _solve(bnd, p, V, 1, refine_max=1)
    assert res["flags"] & bnd.NEP_WARN_REFINE
    assert res["info"]["max_backward"] > 1e-10
    ok = _solve(bnd, p, V, 1)
    assert not (ok["flags"] & bnd.NEP_WARN_REFINE)


def test_wait_bound_gives_up_and_context_survives(bnd, monkeypatch):
    # the cooperative grid kernel of the Jacobi SVD, whose grid barriers are the bounded waits
    monkeypatch.setenv("NEP_JACOBI_CLUSTER", "0")
    torch = torch_cuda()
    lib = bnd.load()
    rows = cols = 128
    rng = np.random.default_rng(3)
    A = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))

    def run():
        Ad = to_dev(np.asfortranarray(A), torch)
        Wd = torch.zeros(cols * cols * 2, dtype=torch.float64, device="cuda")
        sd = torch.zeros(cols, dtype=torch.float64, device="cuda")
        rc = lib.nep_jacobi_svd(rows, cols, Ad.data_ptr(), Wd.data_ptr(), sd.data_ptr(), None)
        torch.cuda.synchronize()
        return rc, sd.cpu().numpy()

    prev = ctypes.c_int64()
    assert lib.nep_set_wait_limit(-1, None) == bnd.NEP_ERR_ARG
    assert lib.nep_set_wait_limit(0, ctypes.byref(prev)) == bnd.NEP_OK
    try:
        rc, _ = run()
        assert rc == bnd.NEP_ERR_INTERNAL, rc
        assert b"timed out" in lib.nep_last_error()
    finally:
        assert lib.nep_set_wait_limit(prev.value, None) == bnd.NEP_OK
    rc, sig = run()
    assert rc == bnd.NEP_OK
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.abs(sig - ref).max() <= 1e-13 * ref[0] * rows
