"""Left eigenvectors and the resolvent on the device (nep_band_solve_adjoint, nep_left_eigvecs,
nep_plan_left, nep_apply_resolvent; Sec. 2 Eqs. (nep-left), (resolvent)) against the oracle.

  * the conjugate-transpose band solve against a dense solve with T^* on every band shape of the
    kernel tests (register-window bands, the staged kernel, the global-memory kernel for wide
    FP64 bands) plus an upper-triangular band (no L, no interchanges);
  * left eigenvectors against closed forms (decoupled delay problems: e_i / conj T'(lambda)_ii; an
    upper-bidiagonal pencil whose factor has an exactly zero pivot) and against the oracle's SVD
    left vectors of a coupled problem, element by element after the Keldysh normalisation;
  * the resolvent's pole part: equal to T(z)^{-1} for a linear pencil with all its eigenvalues,
    and to the oracle's sum for given pairs.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
from scipy.special import lambertw

import synth
from oracle import band, ciss, contour, left, rii
from tests.gpu_util import from_dev_c64, from_dev_c128, to_dev, torch_cuda
from tests.test_gpu_kernels import PROBLEMS, _random_band_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


ADJ_PROBLEMS = dict(PROBLEMS)
ADJ_PROBLEMS["band_90_0_7"] = lambda: _random_band_problem(90, 0, 7, 12)  # upper triangular band


def _factor(bnd, torch, p, split, z, precision):
    npts = len(z)
    F, _ = bnd.coefficients(split, z)
    fdt = torch.float64 if precision == 0 else torch.float32
    ab = torch.zeros(npts * p.n * split.ldab * 2, dtype=fdt, device="cuda")
    bnd.assemble_band(split, npts, to_dev(np.asfortranarray(F), torch), precision, ab)
    ipiv = torch.zeros(npts * p.n, dtype=torch.int32, device="cuda")
    info = torch.zeros(npts, dtype=torch.int32, device="cuda")
    bnd.band_factor(split, npts, precision, ab, ipiv, info)
    return ab, ipiv, info


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(ADJ_PROBLEMS))
def test_adjoint_solve_matches_dense(bnd, name, precision):
    torch = torch_cuda()
    p = ADJ_PROBLEMS[name]()
    split = bnd.Split.from_problem(p)
    npts, L, n = 3, 4, p.n
    z, _, _ = contour.nodes(p.region, npts)
    ab, ipiv, info = _factor(bnd, torch, p, split, z, precision)
    V = synth.random_probe_block(n, L, seed=21)
    Vrep = np.concatenate([np.asfortranarray(V).ravel(order="F")] * npts)
    B = to_dev(Vrep, torch) if precision == 0 else \
        torch.from_numpy(Vrep.astype(np.complex64).view(np.float32).copy()).cuda()
    bnd.band_solve_adjoint(split, npts, precision, ab, ipiv, L, B)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    W = (from_dev_c128(B) if precision == 0 else from_dev_c64(B).astype(np.complex128)).reshape(npts, L, n)
    Fo = contour.coefficient_table(p.fns, z)
    for j in range(npts):
        T = band.assemble_dense(p.mats, Fo[:, j])
        Wo = np.linalg.solve(T.conj().T, V)
        err = np.abs(W[j].T - Wo).max() / np.abs(Wo).max()
        cond = np.linalg.cond(T)
        tol = 1e-13 * cond if precision == 0 else 5e-6 * cond
        assert err <= max(tol, 1e-12), (err, cond)


def _device_left(bnd, torch, p, precision, lam, X, tol=1e-13, max_it=6):
    P = len(lam)
    split = bnd.Split.from_problem(p)
    lam_d = to_dev(np.asarray(lam, np.complex128), torch)
    X_d = to_dev(np.asfortranarray(X), torch)
    Y_d = torch.zeros(2 * p.n * P, dtype=torch.float64, device="cuda")
    eta_d = torch.zeros(P, dtype=torch.float64, device="cuda")
    its_d = torch.zeros(P, dtype=torch.int32, device="cuda")
    k = bnd.left_eigvecs(split, precision, P, lam_d, X_d, Y_d, eta_d, its_d, tol=tol, max_it=max_it)
    torch.cuda.synchronize()
    return from_dev_c128(Y_d).reshape(P, p.n).T, eta_d.cpu().numpy(), its_d.cpu().numpy(), k


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_left_eigenvectors_of_decoupled_delay_problems(bnd, precision, seed):
    torch = torch_cuda()
    p = synth.diagonal_delay(n=8, seed=seed)
    a, b = p.meta["a"], p.meta["b"]
    lam, X, rows = [], [], []
    for i in range(p.n):
        for k in (-1, 0, 1):
            lam.append(complex(a[i] + lambertw(b[i] * np.exp(-a[i]), k)))
            x = np.zeros(p.n, np.complex128)
            x[i] = 1.0
            X.append(x)
            rows.append(i)
    Y, eta, its, _ = _device_left(bnd, torch, p, precision, lam, np.array(X).T, tol=1e-16)
    for q, (l, i) in enumerate(zip(lam, rows)):
        dT = -1.0 - b[i] * np.exp(-l)  # T'(lambda)_ii for T(z) = diag(a) - z I + e^{-z} diag(b)
        ref = np.zeros(p.n, np.complex128)
        ref[i] = 1.0 / np.conj(dT)
        assert np.abs(Y[:, q] - ref).max() <= 1e-12 * abs(ref[i]), (q, Y[:, q], ref)
    assert eta.max() <= 1e-14


def test_left_eigenvector_through_an_exactly_zero_pivot(bnd):
    """T(z) = A - z I, A upper bidiagonal with integer diagonal: at lambda = a_ii the factor has an
    exactly zero pivot (info != 0), which the solve replaces by a tiny one."""
    torch = torch_cuda()
    n = 40
    rng = np.random.default_rng(3)
    d = np.arange(1, n + 1, dtype=np.float64)
    A = sp.diags([d, 0.3 * rng.standard_normal(n - 1)], [0, 1], format="csr")
    I = sp.identity(n, format="csr")
    fns = [{"kind": "rational", "num": [1.0], "den": None}, {"kind": "rational", "num": [-1.0, 0.0], "den": None}]
    p = synth.Problem("bidiag40", n, [A, I], fns, {"center": 10.0 + 0j, "a": 1.0, "b": 1.0})
    for precision in (0, 1):
        lam = [7.0 + 0j, 23.0 + 0j]
        X = []
        for l in lam:
            T = left.dense_T(p, l)
            x = np.linalg.svd(T)[2][-1].conj()
            X.append(x / np.linalg.norm(x))
        X = np.array(X).T
        Y, eta, its, _ = _device_left(bnd, torch, p, precision, lam, X, tol=1e-16)
        for q, l in enumerate(lam):
            ref = left.keldysh_normalise(p, l, X[:, q], left.left_eigenvector(p, l))
            assert np.abs(Y[:, q] - ref).max() <= 1e-12 * np.abs(ref).max(), precision
        assert eta.max() <= 1e-14


@pytest.mark.parametrize("precision", [0, 1])
def test_left_eigenvectors_of_a_coupled_problem_match_the_oracle(bnd, precision):
    torch = torch_cuda()
    p = synth.delay_2d(s=8, seed=1)
    V = synth.random_probe_block(p.n, 16, 0)
    r = ciss.solve(p, N=16, L=16, M=4, V=V)
    assert len(r["lam"]) >= 10
    # pairs polished by the oracle's residual inverse iteration: lambda to ~1e-15, so that the
    # left residual has no floor from the eigenvalue's error
    lam, X = [], []
    for q in range(len(r["lam"])):
        lo, xo, eo, _, ok = rii.rii(p, r["lam"][q], r["X"][:, q], tol=1e-14)
        assert ok
        lam.append(lo)
        X.append(xo / np.linalg.norm(xo))
    lam, X = np.array(lam), np.array(X).T
    Y, eta, its, k = _device_left(bnd, torch, p, precision, lam, X)
    assert k <= 6
    for q in range(len(lam)):
        ref = left.keldysh_normalise(p, lam[q], X[:, q], left.left_eigenvector(p, lam[q]))
        assert np.abs(Y[:, q] - ref).max() <= 1e-9 * np.abs(ref).max(), q
        # the normalisation and the left residual, recomputed on the host
        dT = left.dense_T(p, lam[q], derivative=True)
        assert abs(np.vdot(Y[:, q], dT @ X[:, q]) - 1.0) <= 1e-12
        assert left.left_residual(p, lam[q], Y[:, q]) <= 1e-13
        assert eta[q] <= 1e-13


def test_plan_left_returns_the_left_vectors_of_the_returned_pairs(bnd):
    torch = torch_cuda()
    p = synth.delay_2d(s=16, seed=3)
    V = synth.random_probe_block(p.n, p.L, 5)
    split = bnd.Split.from_problem(p)
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=1)
    plan.execute(to_dev(np.asfortranarray(V), torch))
    plan.polish(tol=1e-13)
    res = plan.result()
    m = len(res["lam"])
    assert m >= 5
    cap = m + 3
    Y_d = torch.zeros(2 * p.n * cap, dtype=torch.float64, device="cuda")
    eta_d = torch.full((cap,), -1.0, dtype=torch.float64, device="cuda")
    nc, k = plan.left(Y_d, eta_d, cap, tol=1e-13)
    torch.cuda.synchronize()
    assert nc == m and 1 <= k <= 6
    Y = from_dev_c128(Y_d).reshape(cap, p.n).T
    eta = eta_d.cpu().numpy()
    assert np.all(eta[m:] == -1.0)  # columns beyond the returned pairs are untouched
    for q in range(m):
        lam, x = res["lam"][q], res["X"][:, q]
        ref = left.keldysh_normalise(p, lam, x, left.left_eigenvector(p, lam))
        assert np.abs(Y[:, q] - ref).max() <= 1e-8 * np.abs(ref).max(), q
    # too little room is refused
    with pytest.raises(bnd.NepError) as e:
        plan.left(Y_d, eta_d, m - 1)
    assert e.value.code == bnd.NEP_ERR_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_resolvent_of_a_linear_pencil(bnd, precision):
    """With every eigenvalue of A - z B, T(z)^{-1} is exactly its pole part."""
    torch = torch_cuda()
    p = synth.dense_linear_small(n=8, seed=3)
    A, B = (m.toarray() for m in p.mats)
    lams, Xr = scipy.linalg.eig(A, B)
    X = Xr / np.linalg.norm(Xr, axis=0)
    Y, eta, _, _ = _device_left(bnd, torch, p, precision, lams, X)
    zs = np.array([0.3 + 0.2j, -1.1 + 0.5j, 2.0 - 0.7j])
    rng = np.random.default_rng(1)
    V = rng.standard_normal((p.n, 3)) + 1j * rng.standard_normal((p.n, 3))
    out = torch.zeros(2 * p.n * len(zs) * 3, dtype=torch.float64, device="cuda")
    bnd.apply_resolvent(p.n, len(lams), to_dev(lams, torch), to_dev(np.asfortranarray(X), torch),
                        to_dev(np.asfortranarray(Y), torch), len(zs), to_dev(zs, torch), 3,
                        to_dev(np.asfortranarray(V), torch), out)
    torch.cuda.synchronize()
    got = from_dev_c128(out).reshape(len(zs) * 3, p.n).T
    for j, z in enumerate(zs):
        ref = np.linalg.solve(A - z * B, V)
        assert np.abs(got[:, 3 * j:3 * j + 3] - ref).max() <= 1e-10 * np.abs(ref).max(), j


def test_resolvent_matches_the_oracle_sum(bnd):
    """Kernel parity on given pairs: random (lambda, x, y), ragged sizes."""
    torch = torch_cuda()
    rng = np.random.default_rng(7)
    n, P, nz, nv = 301, 13, 5, 7
    lam = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    X = rng.standard_normal((n, P)) + 1j * rng.standard_normal((n, P))
    Y = rng.standard_normal((n, P)) + 1j * rng.standard_normal((n, P))
    zs = 3.0 * (rng.standard_normal(nz) + 1j * rng.standard_normal(nz))
    V = rng.standard_normal((n, nv)) + 1j * rng.standard_normal((n, nv))
    out = torch.zeros(2 * n * nz * nv, dtype=torch.float64, device="cuda")
    bnd.apply_resolvent(n, P, to_dev(lam, torch), to_dev(np.asfortranarray(X), torch),
                        to_dev(np.asfortranarray(Y), torch), nz, to_dev(zs, torch), nv,
                        to_dev(np.asfortranarray(V), torch), out)
    torch.cuda.synchronize()
    got = from_dev_c128(out).reshape(nz * nv, n).T
    for j, z in enumerate(zs):
        ref = left.apply_resolvent(lam, X, Y, z, V)
        assert np.abs(got[:, nv * j:nv * (j + 1)] - ref).max() <= 1e-13 * np.abs(ref).max(), j
    # no pairs: zero; no points: nothing written
    bnd.apply_resolvent(n, 0, None, None, None, nz, to_dev(zs, torch), nv, to_dev(np.asfortranarray(V), torch), out)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0


def test_left_refuses_bad_arguments(bnd):
    torch = torch_cuda()
    p = synth.diagonal_delay(n=8, seed=0)
    split = bnd.Split.from_problem(p)
    z = torch.zeros(32, dtype=torch.float64, device="cuda")
    for kw in [dict(P=-1), dict(precision=7), dict(max_it=0)]:
        args = dict(precision=1, P=1, max_it=4)
        args.update(kw)
        with pytest.raises(bnd.NepError) as e:
            bnd.left_eigvecs(split, args["precision"], args["P"], z, z, z, z, max_it=args["max_it"])
        assert e.value.code == bnd.NEP_ERR_ARG
    with pytest.raises(bnd.NepError) as e:
        bnd.left_eigvecs(split, 1, 1, z, None, z, z)
    assert e.value.code == bnd.NEP_ERR_ARG
    with pytest.raises(bnd.NepError) as e:
        bnd.apply_resolvent(0, 1, z, z, z, 1, z, 1, z, z)
    assert e.value.code == bnd.NEP_ERR_ARG
    # nothing to do is not an error
    assert bnd.left_eigvecs(split, 1, 0, None, None, None, None) == 0
