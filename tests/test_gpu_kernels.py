"""Kernel-level parity of the CUDA path (through the C ABI) against the oracle.

Assembly, banded LU (pivots bit-exact in FP64 where no near-tie decides them), banded
solves, the FP64 split residual, the moment sums, the Jacobi SVD and the small eigensolver.
Sizes span several register/warp tiles and ragged tails.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import band, ciss, contour
from tests.gpu_util import (dense_from_rowband, factors_from_gbtrf, factors_from_rowband, from_dev_c64,
                            from_dev_c128, match_eigenvalues, to_dev, torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _random_band_problem(n, kl, ku, seed):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            rows.append(i)
            cols.append(j)
            vals.append(rng.standard_normal())
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    B = sp.diags(rng.uniform(0.5, 1.5, n), 0, format="csr")
    fns = [{"kind": "rational", "num": [1.0], "den": None}, {"kind": "rational", "num": [-1.0, 0.0], "den": None}]
    return synth.Problem(f"band{n}_{kl}_{ku}", n, [A, B], fns, {"center": 0.3 + 0.2j, "a": 1.0, "b": 0.7})


PROBLEMS = {
    "delay2d_s9": lambda: synth.delay_2d(s=9, seed=1),
    "drude2d_s10": lambda: synth.drude_2d(s=10, seed=2, block=4),
    "sqrt3d_s5": lambda: synth.sqrt_3d(s=5, seed=3),
    "band_97_5_12": lambda: _random_band_problem(97, 5, 12, 4),
    "band_150_40_23": lambda: _random_band_problem(150, 40, 23, 5),
    "band_70_64_64": lambda: _random_band_problem(70, 64, 64, 6),
    "band_300_70_9": lambda: _random_band_problem(300, 70, 9, 7),
    "band_33_1_1": lambda: _random_band_problem(33, 1, 1, 8),
    "band_600_128_128": lambda: _random_band_problem(600, 128, 128, 9),   # widest register-window sweeps
    "band_400_150_150": lambda: _random_band_problem(400, 150, 150, 10),  # beyond them: shared-memory solve
}


def _points(p, npts):
    z, _, _ = contour.nodes(p.region, npts)
    return z


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_coefficients_match_oracle(bnd, name):
    p = PROBLEMS[name]()
    split = bnd.Split.from_problem(p)
    z = _points(p, 7)
    F, dF = bnd.coefficients(split, z)
    Fo = contour.coefficient_table(p.fns, z)
    from oracle import fn
    dFo = np.array([fn.derivatives(f, z) for f in p.fns])
    assert np.allclose(F, Fo, rtol=1e-14, atol=1e-14)
    assert np.allclose(dF, dFo, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_assemble_band(bnd, name, precision):
    torch = torch_cuda()
    p = PROBLEMS[name]()
    split = bnd.Split.from_problem(p)
    npts = 5
    z = _points(p, npts)
    F, _ = bnd.coefficients(split, z)
    Fd = to_dev(np.asfortranarray(F), torch)  # F[i + l*j]
    n, ldab = p.n, split.ldab
    ab = torch.zeros(npts * n * ldab * 2, dtype=torch.float64 if precision == 0 else torch.float32, device="cuda")
    tn = torch.zeros(npts, dtype=torch.float64, device="cuda")
    bnd.assemble_band(split, npts, Fd, precision, ab, tn)
    torch.cuda.synchronize()
    abh = from_dev_c128(ab) if precision == 0 else from_dev_c64(ab).astype(np.complex128)
    Fo = contour.coefficient_table(p.fns, z)
    kl, ku = band.bandwidths(p.mats)
    assert (kl, ku) == (split.kl, split.ku)
    for j in range(npts):
        T = band.assemble_dense(p.mats, Fo[:, j])
        G = dense_from_rowband(abh[j * n * ldab:(j + 1) * n * ldab], n, kl, ku, ldab)
        tol = 1e-14 if precision == 0 else 2e-7
        assert np.abs(G - T).max() <= tol * np.abs(T).max()
        tref = float(np.abs(T).sum(axis=1).max())
        assert abs(tn.cpu().numpy()[j] - tref) <= 1e-13 * tref


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_band_factor_fp64_matches_oracle(bnd, name):
    torch = torch_cuda()
    p = PROBLEMS[name]()
    split = bnd.Split.from_problem(p)
    npts = 3
    z = _points(p, npts)
    F, _ = bnd.coefficients(split, z)
    n, ldab, kl, ku = p.n, split.ldab, split.kl, split.ku
    ab = torch.zeros(npts * n * ldab * 2, dtype=torch.float64, device="cuda")
    bnd.assemble_band(split, npts, to_dev(np.asfortranarray(F), torch), 0, ab)
    ipiv = torch.zeros(npts * n, dtype=torch.int32, device="cuda")
    info = torch.zeros(npts, dtype=torch.int32, device="cuda")
    bnd.band_factor(split, npts, 0, ab, ipiv, info)
    torch.cuda.synchronize()
    abh = from_dev_c128(ab)
    piv = ipiv.cpu().numpy().reshape(npts, n)
    assert np.all(info.cpu().numpy() == 0)
    Fo = contour.coefficient_table(p.fns, z)
    for j in range(npts):
        ab_o = band.assemble_band(p.mats, Fo[:, j], kl, ku)
        lu_o, piv_o, info_o = band.gbtrf(ab_o.copy(order="F"), kl, ku)
        assert info_o == 0
        if not np.array_equal(piv[j], piv_o):
            first = int(np.argmax(piv[j] != piv_o))
            pytest.fail(f"pivot sequence differs from column {first}")
        Ug, Lg = factors_from_rowband(abh[j * n * ldab:(j + 1) * n * ldab], n, kl, ku, ldab)
        Uo, Lo = factors_from_gbtrf(lu_o, n, kl, ku)
        # entries beyond column n-1 are not part of the factors
        for c in range(n):
            Ug[c, max(0, n - c):] = 0
        scale = max(np.abs(Uo).max(), 1.0)
        assert np.abs(Ug - Uo).max() <= 1e-12 * scale
        # a multiplier is (rounded entry)/(pivot): its rounding differences scale with 1/|pivot|
        piv_mag = np.maximum(np.abs(Uo[:, 0]), 1e-300)
        lerr = np.abs(Lg - Lo).max(axis=1)
        assert np.all(lerr <= 1e-12 * scale / piv_mag), float((lerr * piv_mag / scale).max())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_band_solve_matches_oracle(bnd, name, precision):
    torch = torch_cuda()
    p = PROBLEMS[name]()
    split = bnd.Split.from_problem(p)
    npts, L = 3, 5
    z = _points(p, npts)
    F, _ = bnd.coefficients(split, z)
    n, ldab, kl, ku = p.n, split.ldab, split.kl, split.ku
    fdt = torch.float64 if precision == 0 else torch.float32
    ab = torch.zeros(npts * n * ldab * 2, dtype=fdt, device="cuda")
    bnd.assemble_band(split, npts, to_dev(np.asfortranarray(F), torch), precision, ab)
    ipiv = torch.zeros(npts * n, dtype=torch.int32, device="cuda")
    info = torch.zeros(npts, dtype=torch.int32, device="cuda")
    bnd.band_factor(split, npts, precision, ab, ipiv, info)
    V = synth.random_probe_block(n, L, seed=11)
    Vrep = np.concatenate([np.asfortranarray(V).ravel(order="F")] * npts)
    if precision == 0:
        B = to_dev(Vrep, torch)
    else:
        B = torch.from_numpy(Vrep.astype(np.complex64).view(np.float32).copy()).cuda()
    bnd.band_solve(split, npts, precision, ab, ipiv, L, B)
    torch.cuda.synchronize()
    Xg = (from_dev_c128(B) if precision == 0 else from_dev_c64(B).astype(np.complex128)).reshape(npts, L, n)
    Fo = contour.coefficient_table(p.fns, z)
    for j in range(npts):
        T = band.assemble_dense(p.mats, Fo[:, j])
        Xo = np.linalg.solve(T, V)
        err = np.abs(Xg[j].T - Xo).max() / np.abs(Xo).max()
        cond = np.linalg.cond(T)
        tol = 1e-13 * cond if precision == 0 else 5e-6 * cond
        assert err <= max(tol, 1e-12), (err, cond)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["band_150_40_23", "band_600_128_128", "delay2d_s9", "band_400_150_150"])
def test_transpose_u_and_solve_cols(bnd, name, precision):
    """U by columns is a pure copy of the factored band; solving with it is bitwise the plain solve."""
    torch = torch_cuda()
    p = PROBLEMS[name]()
    split = bnd.Split.from_problem(p)
    npts, L = 2, 3
    z = _points(p, npts)
    F, _ = bnd.coefficients(split, z)
    n, ldab, kl, ku = p.n, split.ldab, split.kl, split.ku
    kv = kl + ku
    fdt = torch.float64 if precision == 0 else torch.float32
    ab = torch.zeros(npts * n * ldab * 2, dtype=fdt, device="cuda")
    bnd.assemble_band(split, npts, to_dev(np.asfortranarray(F), torch), precision, ab)
    ipiv = torch.zeros(npts * n, dtype=torch.int32, device="cuda")
    info = torch.zeros(npts, dtype=torch.int32, device="cuda")
    bnd.band_factor(split, npts, precision, ab, ipiv, info)
    ut = torch.full((npts * n * (kv + 1) * 2,), float("nan"), dtype=fdt, device="cuda")
    bnd.band_transpose_u(split, npts, precision, ab, ut)
    rb = ab.cpu().numpy().view(np.complex128 if precision == 0 else np.complex64).reshape(npts, n, ldab)
    uc = ut.cpu().numpy().view(np.complex128 if precision == 0 else np.complex64).reshape(npts, n, kv + 1)
    for c in range(n):
        d = np.arange(kv + 1)
        ok = c - d >= 0
        assert np.array_equal(uc[:, c, d[ok]], rb[:, c - d[ok], d[ok]])
        assert np.all(uc[:, c, d[~ok]] == 0)
    V = synth.random_probe_block(n, L, seed=12)
    Vrep = np.concatenate([np.asfortranarray(V).ravel(order="F")] * npts)
    B1 = to_dev(Vrep, torch) if precision == 0 else \
        torch.from_numpy(Vrep.astype(np.complex64).view(np.float32).copy()).cuda()
    B2 = B1.clone()
    bnd.band_solve(split, npts, precision, ab, ipiv, L, B1)
    wide = kl + 1 > 288 or kv + 1 > 288
    bnd.band_solve_cols(split, npts, precision, ab, None if wide else ut, ipiv, L, B2)
    torch.cuda.synchronize()
    assert torch.equal(B1, B2)
    assert torch.isfinite(B1).all()


def test_split_residual_matches_oracle(bnd):
    torch = torch_cuda()
    p = synth.drude_2d(s=12, seed=3, block=4)
    split = bnd.Split.from_problem(p)
    npts, L = 4, 3
    z = _points(p, npts)
    F, _ = bnd.coefficients(split, z)
    rng = np.random.default_rng(0)
    V = synth.random_probe_block(p.n, L, 3)
    Y = rng.standard_normal((npts, L, p.n)) + 1j * rng.standard_normal((npts, L, p.n))
    R = torch.zeros(npts * L * p.n * 2, dtype=torch.float64, device="cuda")
    bnd.split_residual(split, npts, to_dev(np.asfortranarray(F), torch), L, to_dev(np.asfortranarray(V), torch),
                       to_dev(Y, torch), R)
    torch.cuda.synchronize()
    Rg = from_dev_c128(R).reshape(npts, L, p.n)
    Fo = contour.coefficient_table(p.fns, z)
    for j in range(npts):
        T = band.assemble_sparse(p.mats, Fo[:, j])
        Ro = V - T @ Y[j].T
        assert np.abs(Rg[j].T - Ro).max() <= 1e-13 * (np.abs(T).sum(axis=1).max() * np.abs(Y).max() + 1)


@pytest.mark.parametrize("K", [8, 16, 5])
def test_moments_kernel(bnd, K):
    torch = torch_cuda()
    rng = np.random.default_rng(K)
    n, L, N = 301, 7, 24
    Y = rng.standard_normal((N, L, n)) + 1j * rng.standard_normal((N, L, n))
    region = {"center": -1.0, "a": 2.0, "b": 1.0}
    z, w, zeta = contour.nodes(region, N)
    coef = np.array([[w[j] * zeta[j] ** k for k in range(K)] for j in range(N)])  # N x K
    S = torch.zeros(K * L * n * 2, dtype=torch.float64, device="cuda")
    bnd.moments(n, L, N, K, to_dev(np.asfortranarray(coef), torch), to_dev(Y, torch), S)
    torch.cuda.synchronize()
    Sg = from_dev_c128(S).reshape(K, L, n)
    for k in range(K):
        ref = sum(coef[j, k] * Y[j] for j in range(N))
        assert np.abs(Sg[k] - ref).max() <= 1e-14 * np.abs(Y).max() * np.abs(coef).sum(axis=0).max()


# shapes span both work splits (one pair per CTA of four warps up to 256 rows and columns, one
# pair per warp beyond), two elements per thread (rows > 128), odd column counts (a padding
# column in the round-robin) and a single column
@pytest.mark.parametrize("shape,rank", [((40, 40), None), ((128, 128), None), ((96, 96), 30), ((200, 64), None),
                                        ((17, 17), None), ((129, 65), None), ((300, 120), None), ((257, 33), 20),
                                        ((5, 1), None)])
@pytest.mark.parametrize("kernel", ["cluster", "grid"])
def test_jacobi_svd_matches_lapack(bnd, shape, rank, kernel, monkeypatch):
    # "grid": the cooperative grid kernel with bounded grid barriers (the default); "cluster": one
    # thread-block cluster with the columns in distributed shared memory (NEP_JACOBI_CLUSTER=1)
    monkeypatch.setenv("NEP_JACOBI_CLUSTER", "1" if kernel == "cluster" else "0")
    torch = torch_cuda()
    rows, cols = shape
    rng = np.random.default_rng(rows + cols)
    A = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if rank:
        A = A[:, :rank] @ (rng.standard_normal((rank, cols)) + 1j * rng.standard_normal((rank, cols)))
        A *= np.logspace(0, -8, cols)[None, :]
    Ad = to_dev(np.asfortranarray(A), torch)
    Wd = torch.zeros(cols * cols * 2, dtype=torch.float64, device="cuda")
    sd = torch.zeros(cols, dtype=torch.float64, device="cuda")
    bnd.jacobi_svd(rows, cols, Ad, Wd, sd)
    torch.cuda.synchronize()
    sig = sd.cpu().numpy()
    U = from_dev_c128(Ad).reshape(cols, rows).T
    W = from_dev_c128(Wd).reshape(cols, cols).T
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.diff(sig) <= 0)
    assert np.abs(sig - ref).max() <= 1e-13 * ref[0] * max(rows, cols)
    # A W = U Sigma and W unitary
    assert np.abs(A @ W - U * sig[None, :]).max() <= 1e-12 * ref[0]
    assert np.abs(W.conj().T @ W - np.eye(cols)).max() <= 1e-12


@pytest.mark.parametrize("m", [1, 2, 9, 33, 64])
def test_small_eig_matches_lapack(bnd, m):
    torch = torch_cuda()
    rng = np.random.default_rng(m)
    A = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    Ad = to_dev(np.asfortranarray(A), torch)
    ev = torch.zeros(2 * m, dtype=torch.float64, device="cuda")
    evec = torch.zeros(2 * m * m, dtype=torch.float64, device="cuda")
    bnd.small_eig(m, Ad, ev, evec)
    torch.cuda.synchronize()
    lam = from_dev_c128(ev)
    Vv = from_dev_c128(evec).reshape(m, m).T
    err, _ = match_eigenvalues(lam, np.linalg.eigvals(A))
    assert err <= 1e-11
    for i in range(m):
        v = Vv[:, i]
        assert np.linalg.norm(A @ v - lam[i] * v) <= 1e-10 * np.linalg.norm(v) * max(1.0, np.linalg.norm(A, 2))


@pytest.mark.parametrize("n,kl,ku,L", [(403, 150, 150, 5), (320, 300, 10, 3), (517, 300, 40, 20), (400, 20, 300, 17),
                                       (1000, 576, 576, 24), (45, 0, 0, 4), (50, 0, 6, 3)])
def test_blocked_band_solve_matches_oracle(bnd, n, kl, ku, L):
    """The blocked complex64 substitution for bands beyond the register-window sweeps (16-step blocks):
    n not a multiple of the block, n below the backward window, several CTAs per point (L > 16), kl much
    larger or smaller than ku, the bandwidth-576 shape, and bands narrower than a block (kl = 0); the
    oracle's dense FP64 solve."""
    torch = torch_cuda()
    p = _random_band_problem(n, kl, ku, n + kl)
    split = bnd.Split.from_problem(p)
    assert (split.kl, split.ku) == (kl, ku)
    assert kl == 0 or not (kl + 1 <= 288 and kl + ku + 1 <= 288)  # kl = 0: never the register sweeps
    npts = 2
    z = _points(p, npts)
    F, _ = bnd.coefficients(split, z)
    ab = torch.zeros(npts * n * split.ldab * 2, dtype=torch.float32, device="cuda")
    bnd.assemble_band(split, npts, to_dev(np.asfortranarray(F), torch), 1, ab)
    ipiv = torch.zeros(npts * n, dtype=torch.int32, device="cuda")
    info = torch.zeros(npts, dtype=torch.int32, device="cuda")
    bnd.band_factor(split, npts, 1, ab, ipiv, info)
    assert not info.cpu().numpy().any()
    piv = ipiv.cpu().numpy().reshape(npts, n)
    if kl > 0:
        assert (piv != np.arange(n)).sum() > n // 4  # row interchanges are exercised
    V = synth.random_probe_block(n, L, seed=12)
    Vrep = np.concatenate([np.asfortranarray(V).ravel(order="F")] * npts)
    B = torch.from_numpy(Vrep.astype(np.complex64).view(np.float32).copy()).cuda()
    bnd.band_solve(split, npts, 1, ab, ipiv, L, B)
    torch.cuda.synchronize()
    Xg = from_dev_c64(B).astype(np.complex128).reshape(npts, L, n)
    Fo = contour.coefficient_table(p.fns, z)
    for j in range(npts):
        T = band.assemble_dense(p.mats, Fo[:, j])
        Xo = np.linalg.solve(T, V)
        err = np.abs(Xg[j].T - Xo).max() / np.abs(Xo).max()
        cond = np.linalg.cond(T)
        assert err <= max(5e-6 * cond, 1e-12), (err, cond)
