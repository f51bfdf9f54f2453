"""Host-supplied functions in the split form (the callback interface of Sec. 3.2.1, and functions
tabulated at the quadrature nodes), and the per-point status of a result, through the C ABI.

The delay problem's e^{-z} term is given (a) as the built-in NEP_FN_EXP, (b) as a host callback
returning e^{-z} and -e^{-z}, (c) as a table of its values at the quadrature nodes with the callback
for the Newton iterates; all three return the same eigenpairs, which also match the oracle's.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import ciss
from tests.gpu_util import match_eigenvalues, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CALLS = {"count": 0, "points": 0}


def exp_minus(z):
    CALLS["count"] += 1
    CALLS["points"] += len(z)
    e = np.exp(-z)
    return e, -e


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _problem():
    p = synth.delay_2d(s=12, seed=2, center=-1.5, radius=1.5)
    p.N, p.L, p.M = 32, 8, 4
    return p


def _with_fn(p, spec):
    fns = list(p.fns)
    assert fns[2]["kind"] == "exp" and complex(fns[2]["alpha"]) == -1
    fns[2] = spec
    return fns


def _solve(bnd, mats, fns, p, V, precision, **opts):
    torch = torch_cuda()
    split = bnd.Split(mats, fns)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=precision, **opts)
    plan.execute(to_dev(np.asfortranarray(V), torch))
    torch.cuda.synchronize()
    res = plan.result()
    return res, split


@pytest.mark.parametrize("precision", [0, 1])
def test_callback_term_gives_the_builtin_pairs(bnd, precision):
    p = _problem()
    V = synth.random_probe_block(p.n, p.L, 5)
    ref, _ = _solve(bnd, p.mats, p.fns, p, V, precision)
    CALLS["count"] = 0
    res, split = _solve(bnd, p.mats, _with_fn(p, {"kind": "callback", "fn": exp_minus}), p, V, precision)
    assert CALLS["count"] >= 3  # the nodes, Newton steps, the residuals
    assert len(res["lam"]) == len(ref["lam"]) > 0
    err, pairs = match_eigenvalues(res["lam"], ref["lam"])
    assert err <= 1e-12
    for i, j in pairs:
        assert 1.0 - abs(np.vdot(res["X"][:, i], ref["X"][:, j])) <= 1e-10
    assert res["eta"].max() <= 1e-10
    assert not (res["flags"] & bnd.NEP_WARN_NEWTON)
    ora = ciss.solve(p, V=V)
    err, _ = match_eigenvalues(res["lam"], ora["lam"])
    assert err <= 1e-9
    # the coefficient entry point goes through the callback too
    z = np.array([0.3 + 0.1j, -1.0 - 0.5j])
    F, dF = bnd.coefficients(split, z)
    assert np.allclose(F[2], np.exp(-z), rtol=1e-15) and np.allclose(dF[2], -np.exp(-z), rtol=1e-15)


def test_table_term_with_callback_off_the_nodes(bnd):
    p = _problem()
    V = synth.random_probe_block(p.n, p.L, 5)
    z, _, _ = bnd.nodes(p.region, p.N)
    ref, _ = _solve(bnd, p.mats, p.fns, p, V, 1)
    res, _ = _solve(bnd, p.mats, _with_fn(p, {"kind": "table", "values": np.exp(-z), "fn": exp_minus}), p, V, 1)
    err, _ = match_eigenvalues(res["lam"], ref["lam"])
    assert err <= 1e-12
    # the moment block is built from the table: identical to the built-in exp at the nodes
    assert res["m"] == ref["m"]


def test_table_term_refusals(bnd):
    p = _problem()
    z, _, _ = bnd.nodes(p.region, p.N)
    torch_cuda()
    split = bnd.Split(p.mats, _with_fn(p, {"kind": "table", "values": np.exp(-z)}))
    with pytest.raises(bnd.NepError) as e:
        bnd.Plan(split, p.region, p.N, p.L, p.M)
    assert e.value.code == bnd.NEP_ERR_UNSUPPORTED
    split2 = bnd.Split(p.mats, _with_fn(p, {"kind": "table", "values": np.exp(-z[:-2]), "fn": exp_minus}))
    with pytest.raises(bnd.NepError) as e:
        bnd.Plan(split2, p.region, p.N, p.L, p.M)
    assert e.value.code == bnd.NEP_ERR_ARG


def test_device_only_entry_points_refuse_host_functions(bnd):
    torch = torch_cuda()
    p = _problem()
    split = bnd.Split(p.mats, _with_fn(p, {"kind": "callback", "fn": exp_minus}))
    lam = torch.zeros(2, dtype=torch.float64, device="cuda")
    X = torch.zeros(2 * p.n, dtype=torch.float64, device="cuda")
    eta = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = bnd.load()
    assert lib.nep_rii(split.handle, 1, 1, lam.data_ptr(), X.data_ptr(), eta.data_ptr(), None, 1e-10, 3, None,
                       None) == bnd.NEP_ERR_UNSUPPORTED
    region = bnd.region_struct(p.region)
    out = ctypes.c_void_p()
    assert lib.nep_nleigs_solve(split.handle, ctypes.byref(region), None, ctypes.byref(out), None,
                                None) == bnd.NEP_ERR_UNSUPPORTED


def test_callback_request_through_the_server(bnd):
    p = _problem()
    V = synth.random_probe_block(p.n, p.L, 5)
    torch_cuda()
    split = bnd.Split(p.mats, _with_fn(p, {"kind": "callback", "fn": exp_minus}))
    ref, _ = _solve(bnd, p.mats, p.fns, p, V, 1)
    srv = bnd.Server(workers=2)
    tk = [srv.submit(split, p.region, p.N, p.L, p.M, V=V, precision=1) for _ in range(3)]
    outs = [srv.wait(t) for t in tk]
    srv.close()
    for res in outs:
        err, _ = match_eigenvalues(res["lam"], ref["lam"])
        assert err <= 1e-12


@pytest.mark.parametrize("symmetric", [0, 1])
def test_per_point_status(bnd, symmetric):
    p = _problem()
    V = np.asfortranarray(synth.random_probe_block(p.n, p.L, 5).real.astype(np.complex128)) if symmetric else \
        synth.random_probe_block(p.n, p.L, 5)
    res, _ = _solve(bnd, p.mats, p.fns, p, V, 1, symmetric=symmetric)
    pts = res["points"]
    npts = p.N // 2 if symmetric else p.N
    assert len(pts["sweeps"]) == len(pts["lu_info"]) == len(pts["backward"]) == npts
    assert np.all(pts["sweeps"] >= 1) and np.all(pts["sweeps"] <= 10)
    assert np.all(pts["lu_info"] == 0)
    assert pts["backward"].max() <= 1e-10 and pts["backward"].max() == res["info"]["max_backward"]
    assert pts["sweeps"].max() == res["info"]["max_sweeps"]
