"""Full-size wide-band workloads on the GPU, checked on outputs the oracle computes one by one.

* Drude, 128 x 128 grid (n = 16384, bandwidth 128), ellipse c=2, a=1, b=0.2, N=128, L=32, M=8;
* square root, 24^3 grid (n = 13824, bandwidth 576), circle c=4, r=1.5, N=64, L=24, M=8.

The oracle's whole pass on both workloads (minutes on the host) is stored in tests/golden/ by
tests/golden/make_golden_fullsize.py, which calls only the oracle: the eigenvalues, the Hankel
rank and singular values, and the moment block on a fixed set of rows. The tests gate on the
method's acceptance tolerances against it: eigenvalues <= 1e-9 relative, the same Hankel rank,
and the moment Frobenius error <= 1e-10 (mixed path), estimated from the stored rows as
sqrt(n / rows) ||(S - S_oracle)[rows]||_F / ||S_oracle||_F. They also compare sampled quadrature
solves Y_j node by node with the oracle's, recompute the scaled residual of every returned
eigenpair with the oracle (Sec. 2 Eq. (sressplit)), and check properties that hold at any size
(eigenvalues strictly inside the contour, every solve refined to backward error <= 1e-10).
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import ciss, contour
from tests.gpu_util import match_eigenvalues, to_dev, torch_cuda
from tests.test_gpu_pipeline import gpu_buffer

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _run(bnd, p, precision=1):
    torch = torch_cuda()
    V = synth.random_probe_block(p.n, p.L, 0)
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=precision)
    plan.execute(to_dev(np.asfortranarray(V), torch))
    torch.cuda.synchronize()
    res = plan.result()
    return res, plan, V


def _check(bnd, p, res, plan, V, sample_nodes):
    info = res["info"]
    assert not (res["flags"] & bnd.NEP_WARN_REFINE), info
    assert info["max_backward"] <= 1e-10
    # sampled quadrature solves against the oracle's solves at the same nodes
    Y = gpu_buffer(plan, "Y").reshape(p.N, p.L, p.n)
    for j, r in zip(sample_nodes, ciss.solve_points(p, p.region, p.N, V, sample_nodes)):
        err = np.abs(Y[j].T - r["Y"]).max() / np.abs(r["Y"]).max()
        assert err <= 1e-10, (j, err)
    # every returned eigenpair: inside the contour and scaled residual <= 1e-10 (oracle's eta)
    norms = ciss.term_norms_inf(p.mats)
    assert np.all(contour.inside(p.region, res["lam"]))
    for k in range(len(res["lam"])):
        eta = ciss.scaled_residual(p.mats, p.fns, norms, res["lam"][k], res["X"][:, k])
        assert eta <= 1e-10, (res["lam"][k], eta)
        assert abs(eta - res["eta"][k]) <= 1e-12 + 1e-6 * eta


def _check_golden(p, res, plan, name, mom_tol=1e-10):
    g = json.load(open(os.path.join(GOLDEN, f"fullsize_{name}.json")))
    assert (g["n"], g["N"], g["L"], g["M"]) == (p.n, p.N, p.L, p.M)
    lam_o = np.array(g["lam_re"]) + 1j * np.array(g["lam_im"])
    assert len(lam_o) >= 1
    err, _ = match_eigenvalues(res["lam"], lam_o)
    assert err <= 1e-9, (err, res["lam"], lam_o)
    assert res["m"] == g["hankel_rank"], (res["m"], g["hankel_rank"])
    sig_o = np.array(g["sigma"])
    assert np.abs(res["sigma"][:len(sig_o)] - sig_o).max() <= 1e-10 * sig_o[0]
    rows = np.array(g["rows"])
    S_o = np.load(os.path.join(GOLDEN, f"fullsize_{name}.npz"))["S_rows"]  # M x rows x L
    S = gpu_buffer(plan, "S").reshape(-1, p.L, p.n)[:p.M][:, :, rows].transpose(0, 2, 1)
    est = np.sqrt(p.n / len(rows)) * np.linalg.norm(S - S_o) / g["S_fro"]
    assert est <= mom_tol, est


def test_drude_128x128_full_size(bnd):
    p = synth.config_problem("drude2d_s128")
    res, plan, V = _run(bnd, p)
    _check(bnd, p, res, plan, V, [0, 77])
    _check_golden(p, res, plan, "drude2d_s128")


def test_sqrt_24cubed_full_size(bnd):
    p = synth.config_problem("sqrt3d_s24")
    res, plan, V = _run(bnd, p)
    _check(bnd, p, res, plan, V, [5])
    _check_golden(p, res, plan, "sqrt3d_s24")
