"""The autotuner (nep_autotune, nep_tune_load): candidates timed on the problem itself, accuracy as a gate
(every quadrature solve at the backward-error target), the choice kept per shape and in a cache file."""
import numpy as np
import pytest

import synth
from tests.gpu_util import match_eigenvalues, to_dev, torch_cuda
from tests.test_gpu_batch import _band
from tests.test_gpu_pipeline import gpu_buffer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _run(bnd, split, p, V, **opts):
    torch = torch_cuda()
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=1, **opts)
    plan.execute(V)
    torch.cuda.synchronize()
    return plan.result(), gpu_buffer(plan, "Y")


def test_narrow_band_sweep_width(bnd, tmp_path):
    torch = torch_cuda()
    p = synth.delay_2d(s=12, seed=2, center=-1.5, radius=1.5)
    p.N, p.L, p.M = 32, 8, 4
    split = bnd.Split.from_problem(p)
    V = to_dev(np.asfortranarray(synth.random_probe_block(p.n, p.L, 5)), torch)
    cache = tmp_path / "tune.txt"
    t = bnd.autotune(split, p.region, p.N, p.L, p.M, V, cache_path=str(cache), precision=1)
    assert t["candidates"] == 3 and t["accurate"] == 3 and t["solve_rh"] in (1, 2, 4) and t["ms"] > 0
    line = cache.read_text().strip().splitlines()[-1]
    assert line.startswith("nep-tune ") and f"n={p.n} kl={split.kl}" in line and f"solve_rh={t['solve_rh']}" in line
    assert bnd.tune_load(str(cache)) == 1
    # the sweep width is a launch shape only: every choice gives the same solves, and a plan of this shape
    # created with default options now runs the tuned one
    ref, Yref = _run(bnd, split, p, V, solve_rh=1)
    for rh in (2, 4, 0):
        r, Y = _run(bnd, split, p, V, solve_rh=rh)
        assert np.array_equal(Y, Yref) and np.array_equal(r["lam"], ref["lam"])


def test_wide_band_lu_kernel_with_accuracy_gate(bnd):
    torch = torch_cuda()
    p = _band(600, 128, 128, 9)
    p.N, p.L, p.M = 16, 4, 2
    split = bnd.Split.from_problem(p)
    V = to_dev(np.asfortranarray(synth.random_probe_block(p.n, p.L, 3)), torch)
    t = bnd.autotune(split, p.region, p.N, p.L, p.M, V, precision=1)
    assert t["candidates"] == 9  # three LU kernels x three sweep widths
    assert t["accurate"] >= 6    # the tensor core with the hi/lo split and the SIMT kernel always qualify
    assert t["lu_kernel"] in (1, 2, 3)
    ref, _ = _run(bnd, split, p, V, lu_kernel=3)  # FP32 SIMT factors
    for lu in (1, 2, 0):
        r, _ = _run(bnd, split, p, V, lu_kernel=lu)
        if lu == 2 and (r["flags"] & bnd.NEP_WARN_REFINE):
            continue  # TF32 operands that refinement cannot repair: the tuner's gate excludes this
        assert r["info"]["max_backward"] <= 1e-10
        err, _ = match_eigenvalues(r["lam"], ref["lam"])
        assert err <= 1e-9


def test_narrow_band_tensor_core_lu_by_name(bnd):
    """lu_kernel 1 or 2 on a band the register-window LU takes (32 <= kl <= 64) runs the tensor-core LU:
    the same eigenpairs to rounding, every solve at the target, and the shared-launch path equal to the
    plan's own pass."""
    torch = torch_cuda()
    p = synth.delay_2d(s=40, seed=4, center=-1.5, radius=1.5)
    p.N, p.L, p.M = 16, 4, 4
    split = bnd.Split.from_problem(p)
    assert 32 <= split.kl <= 64
    V = to_dev(np.asfortranarray(synth.random_probe_block(p.n, p.L, 6)), torch)
    ref, _ = _run(bnd, split, p, V)  # register-window LU
    for lu in (1, 2):
        r, Y = _run(bnd, split, p, V, lu_kernel=lu)
        if lu == 2 and (r["flags"] & bnd.NEP_WARN_REFINE):
            continue  # TF32 operands that refinement cannot repair
        assert r["info"]["max_backward"] <= 1e-10
        err, _ = match_eigenvalues(r["lam"], ref["lam"])
        assert err <= 1e-9
        if lu == 1:
            a = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=1, lu_kernel=1)
            b = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=1)
            bnd.execute_batch([a, b], [V, V])
            torch.cuda.synchronize()
            assert np.array_equal(gpu_buffer(a, "Y"), Y)
            assert np.array_equal(a.result()["lam"], r["lam"])
