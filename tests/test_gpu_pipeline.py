"""Whole contour-integral pass on the GPU (C ABI) against the oracle and the closed-form pins.

Tolerances (eigenvalues <= 1e-9 relative, scaled residual <= 1e-10, moment Frobenius
error <= 1e-12 for the FP64 path and <= 1e-10 for the refined mixed path) are the acceptance
gates of the method; both sides take the same probe block V.
"""
import numpy as np
import pytest

import synth
from oracle import ciss, contour, count
from tests.gpu_util import from_dev_c128, match_eigenvalues, to_dev, torch_cuda
from tests.test_oracle_pins import drude_reference, lambert_reference, sqrt_reference

pytestmark = pytest.mark.gpu

EIG_TOL = 1e-9
ETA_TOL = 1e-10
MOM_TOL = {0: 1e-12, 1: 1e-10}


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def gpu_buffer(plan, name, dtype="c128"):
    """Host copy of a plan's device buffer (wrapped for torch through __cuda_array_interface__)."""
    torch = torch_cuda()
    ptr, nbytes = plan.buffer(name)

    class _View:
        pass
    v = _View()
    v.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}
    torch.cuda.synchronize()
    host = torch.as_tensor(v, device="cuda").cpu().numpy().copy()
    if dtype == "c128":
        return host.view(np.complex128)
    if dtype == "f64":
        return host.view(np.float64)
    return host.view(np.int32)


def check_against_oracle(res, ora, precision, plan=None, p=None, eig_tol=EIG_TOL):
    assert res["m"] == ora["m"], (res["m"], ora["m"])
    sig_g, sig_o = res["sigma"], ora["sigma"]
    assert np.abs(sig_g - sig_o).max() <= (1e-10 if precision else 1e-12) * sig_o[0]
    err, pairs = match_eigenvalues(res["lam"], ora["lam"])
    assert err <= eig_tol, err
    if len(res["eta"]):
        assert res["eta"].max() <= ETA_TOL
    for i, j in pairs:
        x, y = res["X"][:, i], ora["X"][:, j]
        assert 1.0 - abs(np.vdot(x, y)) <= 1e-8
    if plan is not None:
        S = gpu_buffer(plan, "S").reshape(-1, p.L, p.n)[:p.M]
        So = ora["S"].transpose(0, 2, 1)
        rel = np.linalg.norm(S - So) / np.linalg.norm(So)
        assert rel <= MOM_TOL[precision], rel


@pytest.mark.parametrize("precision", [0, 1])
def test_delay1d_wide_matches_oracle(bnd, precision):
    p = synth.config_problem("delay1d_n64_wide")
    V = synth.random_probe_block(p.n, p.L, 0)
    ora = ciss.solve(p, V=V)
    res = run_gpu_plain(bnd, p, V, precision)
    check_against_oracle(res, ora, precision, res["plan"], p)
    assert len(res["lam"]) == 32
    assert not (res["flags"] & bnd.NEP_WARN_REFINE)


def run_gpu_plain(bnd, p, V, precision, N=None, L=None, M=None):
    torch = torch_cuda()
    N, L, M = N or p.N, L or p.L, M or p.M
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, N, L, M, precision=precision)
    Vd = to_dev(np.asfortranarray(V), torch)
    plan.execute(Vd)
    torch.cuda.synchronize()
    res = plan.result()
    res["plan"], res["split"] = plan, split
    return res


@pytest.mark.parametrize("precision", [0, 1])
def test_delay1d_saturated_flag(bnd, precision):
    p = synth.config_problem("delay1d_n64")
    V = synth.random_probe_block(p.n, p.L, 0)
    ora = ciss.solve(p, V=V)
    res = run_gpu_plain(bnd, p, V, precision)
    assert res["flags"] & bnd.NEP_WARN_SATURATED
    assert res["m"] == ora["m"] == 16
    S = gpu_buffer(res["plan"], "S").reshape(-1, p.L, p.n)[:p.M]
    So = ora["S"].transpose(0, 2, 1)
    assert np.linalg.norm(S - So) / np.linalg.norm(So) <= MOM_TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_diagonal_delay_lambert_w_on_gpu(bnd, precision):
    for seed in (0, 1, 2):
        p = synth.diagonal_delay(n=8, seed=seed)
        V = synth.random_probe_block(p.n, p.L, seed)
        res = run_gpu_plain(bnd, p, V, precision)
        err, _ = match_eigenvalues(res["lam"], lambert_reference(p))
        assert err <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_diagonal_drude_and_sqrt_on_gpu(bnd, precision):
    p = synth.diagonal_drude(n=6, seed=0)
    res = run_gpu_plain(bnd, p, synth.random_probe_block(p.n, p.L, 0), precision)
    err, _ = match_eigenvalues(res["lam"], drude_reference(p))
    assert err <= 1e-11
    p = synth.diagonal_sqrt(n=6, seed=0)
    res = run_gpu_plain(bnd, p, synth.random_probe_block(p.n, p.L, 0), precision)
    err, _ = match_eigenvalues(res["lam"], sqrt_reference(p))
    assert err <= 1e-11


SMALL = {
    "delay2d_s12": (lambda: synth.delay_2d(s=12, seed=2, center=-1.5, radius=1.5), 64, 8, 4),
    "delay2d_s20": (lambda: synth.delay_2d(s=20, seed=3), 48, 12, 6),
    "drude2d_s16": (lambda: synth.drude_2d(s=16, seed=1, block=5), 96, 8, 4),
    "sqrt3d_s6": (lambda: synth.sqrt_3d(s=6, seed=1, center=4.0, radius=1.5), 48, 8, 4),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(SMALL))
def test_small_problems_match_oracle(bnd, name, precision):
    make, N, L, M = SMALL[name]
    p = make()
    p.N, p.L, p.M = N, L, M
    V = synth.random_probe_block(p.n, L, 5)
    ora = ciss.solve(p, V=V)
    res = run_gpu_plain(bnd, p, V, precision)
    check_against_oracle(res, ora, precision, res["plan"], p)


@pytest.mark.parametrize("precision", [0, 1])
def test_delay2d_s64_full_size(bnd, precision):
    """The n = 4096, bandwidth 64 delay workload (N=64, L=16, M=8) at full size, both precisions."""
    p = synth.config_problem("delay2d_s64")
    V = synth.random_probe_block(p.n, p.L, 0)
    ora = ciss.solve(p, V=V)
    res = run_gpu_plain(bnd, p, V, precision)
    check_against_oracle(res, ora, precision, res["plan"], p)
    assert len(res["lam"]) == 9
    # sampled quadrature solves against the oracle's solves at the same nodes
    Y = gpu_buffer(res["plan"], "Y").reshape(p.N, p.L, p.n)
    for j, r in zip([0, 17, 63], ciss.solve_points(p, p.region, p.N, V, [0, 17, 63])):
        err = np.abs(Y[j].T - r["Y"]).max() / np.abs(r["Y"]).max()
        assert err <= (1e-12 if precision == 0 else 1e-10), err


def test_host_buffer_solve_matches_plan(bnd):
    """nep_ciss_solve (host buffers) returns the same eigenpairs as the device-resident plan."""
    p = synth.delay_2d(s=12, seed=2, center=-1.5, radius=1.5)
    V = synth.random_probe_block(p.n, 8, 5)
    split = bnd.Split.from_problem(p)
    a = bnd.ciss_solve(split, p.region, 64, 8, 4, V=V, precision=1)
    b = run_gpu_plain(bnd, p, V, 1, N=64, L=8, M=4)
    err, _ = match_eigenvalues(a["lam"], b["lam"])
    assert err == 0.0
    assert np.array_equal(a["eta"], b["eta"])


def test_region_crossing_branch_cut_rejected(bnd):
    p = synth.sqrt_3d(s=4, seed=0)
    split = bnd.Split.from_problem(p)
    with pytest.raises(bnd.NepError) as e:
        bnd.Plan(split, {"center": 0.5, "a": 1.0, "b": 1.0}, 16, 2, 2)
    assert e.value.code == bnd.NEP_ERR_REGION


def test_invalid_arguments_rejected(bnd):
    p = synth.delay_2d(s=4, seed=0)
    split = bnd.Split.from_problem(p)
    for N, L, M in [(1, 2, 2), (16, 0, 2), (16, 2, 0), (16, p.n + 1, 1)]:
        with pytest.raises(bnd.NepError) as e:
            bnd.Plan(split, p.region, N, L, M)
        assert e.value.code == bnd.NEP_ERR_ARG


def _run_opts(bnd, p, V, precision, L=None, **opts):
    torch = torch_cuda()
    L = L or p.L
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, L, p.M, precision=precision, **opts)
    plan.execute(to_dev(np.asfortranarray(V), torch))
    torch.cuda.synchronize()
    res = plan.result()
    res["plan"] = plan
    return res


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["diag_delay_s8_L2", "delay1d_n64_wide", "drude_small"])
def test_device_shortcuts_do_not_change_results(bnd, precision, case):
    """The device's two shortcuts (Newton iterates given up outside Gamma after 8 steps; a refinement
    sweep saved when the observed contraction puts the next correction below the step tolerance)
    return the same eigenvalues as the device without them and as the plain oracle, which has
    neither. The first case is the one whose only Newton path to lambda = -0.3211 lies outside
    Gamma at step 3; a shortcut taken too early would lose it."""
    if case == "diag_delay_s8_L2":
        p, L = synth.diagonal_delay(n=8, seed=8), 2
    elif case == "delay1d_n64_wide":
        p, L = synth.config_problem("delay1d_n64_wide"), None
    else:
        p, L = synth.dense_drude_small(n=6, seed=0), None
    L = L or p.L
    V = synth.random_probe_block(p.n, L, 0)
    ora = ciss.solve(p, V=V, L=L)
    fast = _run_opts(bnd, p, V, precision, L=L)
    plain = _run_opts(bnd, p, V, precision, L=L, newton_abandon=0, refine_extrapolate=0)
    for res in (fast, plain):
        err, _ = match_eigenvalues(res["lam"], ora["lam"])
        assert err <= EIG_TOL, err
        assert not (res["flags"] & bnd.NEP_WARN_NEWTON), res["info"]
    err, _ = match_eigenvalues(fast["lam"], plain["lam"])
    assert err <= EIG_TOL
    assert fast["info"]["max_sweeps"] <= plain["info"]["max_sweeps"]


def test_double_float_refinement_reaches_fp64_level(bnd):
    """With complex64 factors the refinement residual and the accumulated solution are double-float
    (about 48 bits). Asked for a backward error of 5e-14, every quadrature solve gets there, far below
    what an FP32 residual can resolve (about 1e-7), and the solves agree with the oracle's FP64
    solves to 1e-12."""
    torch = torch_cuda()
    p = synth.delay_2d(s=20, seed=1)
    N, L, M = 32, 8, 4
    V = synth.random_probe_block(p.n, L, 3)
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, N, L, M, precision=1, refine_tol=5e-14, step_tol=1e-18, refine_max=15)
    plan.execute(to_dev(np.asfortranarray(V), torch))
    torch.cuda.synchronize()
    res = plan.result()
    assert not res["flags"] & bnd.NEP_WARN_REFINE
    bw = res["points"]["backward"]
    assert len(bw) == N and bw.max() <= 5e-14, bw.max()
    Y = gpu_buffer(plan, "Y").reshape(N, L, p.n)
    for j, r in zip([0, 11, 31], ciss.solve_points(p, p.region, N, V, [0, 11, 31])):
        err = np.abs(Y[j].T - r["Y"]).max() / np.abs(r["Y"]).max()
        assert err <= 1e-12, err
