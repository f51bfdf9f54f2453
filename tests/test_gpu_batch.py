"""Several plans in shared launches (nep_plan_execute_batch): the LU and the sweeps of the points of
problems of uneven n, bandwidth, N and L run together, and every plan's results are bitwise those of
its own nep_plan_execute (same kernel instance and arguments per point)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from tests.gpu_util import to_dev, torch_cuda
from tests.test_gpu_pipeline import gpu_buffer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _band(n, kl, ku, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            rows.append(i)
            cols.append(j)
    A = sp.csr_matrix((rng.standard_normal(len(rows)), (rows, cols)), shape=(n, n))
    B = sp.diags(rng.uniform(0.5, 1.5, n), 0, format="csr")
    fns = [{"kind": "rational", "num": [1.0], "den": None}, {"kind": "rational", "num": [-1.0, 0.0], "den": None}]
    return synth.Problem(f"band{n}", n, [A, B], fns, {"center": 0.3 + 0.2j, "a": 1.0, "b": 0.7}, N=8, L=4, M=2)


def _narrow():
    ps = []
    p = synth.delay_2d(s=12, seed=2, center=-1.5, radius=1.5)
    p.N, p.L, p.M = 32, 8, 4
    ps.append(p)
    p = synth.drude_2d(s=10, seed=2, block=4)
    p.N, p.L, p.M = 16, 6, 3
    ps.append(p)
    p = synth.sqrt_3d(s=5, seed=3)
    p.N, p.L, p.M = 24, 5, 4
    ps.append(p)
    ps.append(_band(150, 40, 23, 5))
    p = synth.delay_1d(n=64, seed=0)
    p.N, p.L, p.M = 32, 16, 4
    ps.append(p)
    return ps


def _wide():
    a = _band(600, 128, 128, 9)
    b = _band(400, 150, 150, 10)
    b.L = 3
    return [a, b]


def _snapshot(plan, p):
    r = plan.result()
    return r, gpu_buffer(plan, "S"), gpu_buffer(plan, "Y")


@pytest.mark.parametrize("kind,precision", [("narrow", 1), ("narrow", 0), ("wide", 1)])
def test_batch_is_bitwise_alone(bnd, kind, precision):
    torch = torch_cuda()
    probs = _narrow() if kind == "narrow" else _wide()
    splits = [bnd.Split.from_problem(p) for p in probs]
    plans = [bnd.Plan(sp_, p.region, p.N, p.L, p.M, precision=precision) for sp_, p in zip(splits, probs)]
    Vs = [to_dev(np.asfortranarray(synth.random_probe_block(p.n, p.L, 7 + i)), torch) for i, p in enumerate(probs)]
    alone = []
    for pl, p, V in zip(plans, probs, Vs):
        pl.execute(V)
        torch.cuda.synchronize()
        alone.append(_snapshot(pl, p))
    bnd.execute_batch(plans, Vs)
    torch.cuda.synchronize()
    for pl, p, (r0, S0, Y0) in zip(plans, probs, alone):
        r1, S1, Y1 = _snapshot(pl, p)
        assert np.array_equal(Y0, Y1) and np.array_equal(S0, S1), p.name
        assert np.array_equal(r0["lam"], r1["lam"]) and np.array_equal(r0["X"], r1["X"])
        assert np.array_equal(r0["eta"], r1["eta"]) and r0["m"] == r1["m"]
        assert np.array_equal(r0["points"]["sweeps"], r1["points"]["sweeps"])
        assert r1["info"]["max_backward"] <= 1e-10


def test_batch_refusals(bnd):
    torch = torch_cuda()
    p = _narrow()[0]
    sp_ = bnd.Split.from_problem(p)
    a = bnd.Plan(sp_, p.region, p.N, p.L, p.M, precision=1)
    b = bnd.Plan(sp_, p.region, p.N, p.L, p.M, precision=0)
    V = to_dev(np.asfortranarray(synth.random_probe_block(p.n, p.L, 1)), torch)
    with pytest.raises(bnd.NepError):
        bnd.execute_batch([a, a], [V, V])
    with pytest.raises(bnd.NepError):
        bnd.execute_batch([a, b], [V, V])
