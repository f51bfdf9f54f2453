"""Conjugate-symmetric quadrature (real operator, region symmetric about the real axis, real V):
only the N/2 nodes with Im z > 0 are solved; S_k = 2 Re of their sum. The result must equal the
full quadrature (GPU and oracle) on the same real probe block, and the option must be refused
where the symmetry does not hold."""
import numpy as np
import pytest

import synth
from oracle import ciss
from tests.gpu_util import match_eigenvalues, to_dev, torch_cuda
from tests.test_gpu_pipeline import gpu_buffer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _real_probe(n, L, seed):
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, L)).astype(np.complex128))


def _run(bnd, p, V, precision, symmetric):
    torch = torch_cuda()
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=precision, symmetric=symmetric)
    plan.execute(to_dev(V, torch))
    torch.cuda.synchronize()
    res = plan.result()
    res["plan"], res["split"] = plan, split
    return res


@pytest.mark.parametrize("precision", [0, 1])
def test_symmetric_matches_full_quadrature(bnd, precision):
    p = synth.delay_2d(s=20, seed=7)
    V = _real_probe(p.n, p.L, 3)
    full = _run(bnd, p, V, precision, 0)
    half = _run(bnd, p, V, precision, 1)
    ora = ciss.solve(p, V=V)
    assert half["m"] == full["m"] == ora["m"]
    # moments: the half sum doubled equals the full sum (real for a real problem and a real V)
    S_full = gpu_buffer(full["plan"], "S").reshape(-1, p.L, p.n)[:p.M]
    S_half = gpu_buffer(half["plan"], "S").reshape(-1, p.L, p.n)[:p.M]
    So = ora["S"].transpose(0, 2, 1)
    assert np.abs(S_half.imag).max() == 0.0
    assert np.abs(So.imag).max() <= 1e-12 * np.abs(So).max()
    tol = 1e-10 if precision else 1e-12
    assert np.linalg.norm(S_half - S_full) <= tol * np.linalg.norm(S_full)
    assert np.linalg.norm(S_half - So) <= tol * np.linalg.norm(So)
    err, _ = match_eigenvalues(half["lam"], ora["lam"])
    assert err <= 1e-9, err
    err, _ = match_eigenvalues(half["lam"], full["lam"])
    assert err <= 1e-9, err
    # the same eigenpairs, accepted by the same scaled-residual test (eta <= 1e-8)
    assert len(half["lam"]) == len(full["lam"]) >= 1 and half["eta"].max() <= 1e-8
    assert np.allclose(np.sort(half["eta"]), np.sort(full["eta"]), rtol=1e-3, atol=1e-14)
    # only half the points were factored: the per-point buffers have N/2 entries
    assert gpu_buffer(half["plan"], "sweeps", "i32").size == p.N // 2


def test_symmetric_refused_where_it_does_not_hold(bnd):
    torch = torch_cuda()
    # complex functions (the Drude term carries i*gamma)
    p = synth.drude_2d(s=10, seed=2, block=4)
    split = bnd.Split.from_problem(p)
    with pytest.raises(bnd.NepError) as e:
        bnd.Plan(split, p.region, p.N, p.L, p.M, symmetric=1)
    assert e.value.code == bnd.NEP_ERR_ARG
    # odd N and a centre off the real axis
    q = synth.delay_2d(s=8, seed=1)
    sq = bnd.Split.from_problem(q)
    with pytest.raises(bnd.NepError):
        bnd.Plan(sq, q.region, 31, q.L, q.M, symmetric=1)
    reg = dict(q.region, center=q.region["center"] + 0.1j)
    with pytest.raises(bnd.NepError):
        bnd.Plan(sq, reg, q.N, q.L, q.M, symmetric=1)
    # complex probe block at execute
    plan = bnd.Plan(sq, q.region, q.N, q.L, q.M, symmetric=1)
    Vc = synth.random_probe_block(q.n, q.L, 0)
    with pytest.raises(bnd.NepError) as e:
        plan.execute(to_dev(np.asfortranarray(Vc), torch))
    assert e.value.code == bnd.NEP_ERR_ARG


def test_symmetric_one_shot_draws_real_probe(bnd):
    torch_cuda()
    p = synth.delay_2d(s=12, seed=4)
    split = bnd.Split.from_problem(p)
    res = bnd.ciss_solve(split, p.region, p.N, p.L, p.M, symmetric=1, seed=5)
    assert res["m"] >= 1 and len(res["lam"]) >= 1
    assert res["eta"].max() <= 1e-8
