"""The library's NLEIGS interpolation setup, a host computation, against the oracle without a GPU
(nep_nleigs_interpolation_fns; Sec. 4.5.1): same degree and count of singular points, nodes on
the boundary, scalings max |b_j| = 1 there, and divided differences (the library's own matrix functions)
equal to the oracle's (scipy's) matrix-function divided differences on the library's own nodes and poles."""
import numpy as np
import pytest

import synth
from oracle import fn, nleigs

PROBLEMS = {
    "delay": lambda: synth.diagonal_delay(n=8, seed=0),
    "drude": lambda: synth.diagonal_drude(n=6, seed=0),
    "sqrt": lambda: synth.diagonal_sqrt(n=6, seed=0),
    "linear": lambda: synth.dense_linear_small(n=8, seed=3),
    "delay2d": lambda: synth.delay_2d(s=6, seed=0),
}


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_host_interpolation_matches_the_oracle(bnd, name):
    p = PROBLEMS[name]()
    it = bnd.nleigs_interpolation_fns(p.fns, p.region)
    ora = nleigs.interpolation(p.fns, p.region)
    assert it["converged"]
    assert it["d"] == ora["d"] and it["nsing"] == len(ora["Xi"])
    d = it["d"]
    sig, xi, beta = it["sigma"], it["xi"].copy(), it["beta"]
    xi[~np.isfinite(xi)] = np.inf
    assert np.isinf(xi[d]) and np.isinf(xi[0])
    bndry = nleigs.boundary(p.region)
    assert all(np.abs(bndry - s).min() <= 1e-12 for s in sig)
    b = nleigs.basis(bndry, sig, xi, beta, d)
    assert np.allclose(np.abs(b).max(axis=1), 1.0, rtol=1e-13)
    ref = nleigs.divided_differences(p.fns, sig, xi, beta, d)
    assert np.abs(it["dd"] - ref).max() <= 1e-11 * np.abs(ref[:, 0]).max()
    r = it["dd"] @ b
    f = np.array([fn.values(g, bndry) for g in p.fns])
    assert np.abs(r - f).max() <= 1e-11 * np.abs(f).max()


def test_host_interpolation_refusals(bnd):
    p = synth.diagonal_sqrt(n=6, seed=0)
    with pytest.raises(bnd.NepError) as e:  # the branch cut (-inf, 1] crosses this region
        bnd.nleigs_interpolation_fns(p.fns, {"center": 1.0, "a": 1.0, "b": 1.0})
    assert e.value.code == bnd.NEP_ERR_REGION
    with pytest.raises(bnd.NepError) as e:
        bnd.nleigs_interpolation_fns(p.fns, p.region, max_degree=70)
    assert e.value.code == bnd.NEP_ERR_ARG
