"""Contour-integral (block Sakurai-Sugiura / Beyn-type) solver, plain FP64 (oracle; test infrastructure only).

The steps, in the order the method takes them:
  O1  nodes z_j, weights w_j, scaled zeta_j and F[i,j] = f_i(z_j)        (contour.py)
  O2  band storage of T(z_j) = sum_i F[i,j] A_i                            (Sec. 2 Eq. (split); band.py)
  O3  banded LU with partial pivoting                                      (band_lu.c)
  O4  Y_j = T(z_j)^{-1} V, refined with FP64 residuals V - T(z_j) Y_j      (solve_point)
  O5  S_k = sum_j w_j zeta_j^k Y_j (k < M);  mu_k = sum_j w_j zeta_j^k V^H Y_j (k < 2M)
      -- quadrature of the resolvent, whose poles are the eigenvalues inside
         Gamma by Keldysh's theorem (Sec. 2 Eq. (resolvent))                (moments)
  O6  block Hankel H = [mu_{i+j}], H< = [mu_{i+j+1}]; SVD, numerical rank m;
      eigenvalues theta of U_m^H H< W_m Sigma_m^{-1}; lambda = c + a theta;
      Hankel eigenvector estimates X_H = [S_0 .. S_{M-1}] W_m Sigma_m^{-1} T   (hankel_extract)
  O7  Q = orthonormal basis of the normalised X_H (truncated SVD)           (rayleigh_ritz)
  O8  projected split form B_i = Q^H A_i Q (Sec. 4.2 Eq. (narnoldi-split)), Newton's
      method on sum_i f_i(lambda) B_i y = 0 (Sec. 4.1 Eq. (newton), normalised by u^H y = 1)
      from every Hankel candidate; x = Q y                                   (newton_projected)
  O9  keep lambda strictly inside Gamma with eta <= eig_tol, drop duplicates
  O10 eta = ||T(lambda) x||_2 / (sum_i |f_i(lambda)| ||A_i||_inf ||x||_2)  (Sec. 2 Eq. (sressplit),
      infinity norms of the A_i as in Sec. 6)                               (scaled_residual)

Readings where the paper is silent are stated in the repository's design notes;
the constants below carry them.
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os

import numpy as np
import scipy.sparse as sp

from . import band, contour, fn

DELTA_HANKEL = 1e-12      # numerical rank of H: sigma_i > DELTA_HANKEL * sigma_1
DELTA_BASIS = 1e-6        # rank of the normalised Hankel eigenvector block: sigma_i > DELTA_BASIS * sigma_1
REFINE_TOL = 1e-10        # per-solve backward error target
REFINE_STEP_TOL = 1e-14   # relative correction at which the solve is converged in the forward sense
REFINE_MAX = 10
NEWTON_MAX = 30
NEWTON_TOL = 1e-15        # |dlambda| <= NEWTON_TOL * max(1, |lambda|)
EIG_TOL = 1e-8            # eta acceptance of a returned eigenpair
DEDUP_LAMBDA = 1e-10
DEDUP_VECTOR = 1e-8


def _threads():
    return max(1, min(32, os.cpu_count() or 1))


def term_norms_inf(mats):
    """||A_i||_inf (max absolute row sum), the matrix norms of Eq. (sressplit) as used in Sec. 6."""
    return np.array([float(abs(A).sum(axis=1).max()) if A.nnz else 0.0 for A in mats])


def backward_error(T: sp.csr_matrix, Tnorm: float, V: np.ndarray, Y: np.ndarray, R: np.ndarray) -> float:
    """max over columns of ||v - T y||_inf / (||T||_inf ||y||_inf + ||v||_inf) (normwise backward error)."""
    num = np.abs(R).max(axis=0)
    den = Tnorm * np.abs(Y).max(axis=0) + np.abs(V).max(axis=0)
    return float((num / den).max())


def solve_point(problem, kl: int, ku: int, coeffs, V: np.ndarray, *, refine_max: int = REFINE_MAX,
                return_factors: bool = False):
    """O2-O4 at one quadrature point: Y = T^{-1} V by banded LU, then FP64 iterative refinement.

    Refinement sweep: R = V - T Y (FP64 split-form product), D = T^{-1} R, Y += D;
    stop once the backward error of the iterate is <= REFINE_TOL and the relative
    correction is <= REFINE_STEP_TOL or stopped halving, at most refine_max sweeps.
    A node at which the LU meets an exactly zero pivot (T(z_j) singular: an eigenvalue on the
    contour at the node) has no resolvent to sample; it contributes Y = 0 to the moments and
    takes no refinement (the paper is silent; the repository's design notes list this reading).
    Returns a dict.
    """
    T = band.assemble_sparse(problem.mats, coeffs)
    Tnorm = float(abs(T).sum(axis=1).max())
    ab0 = band.assemble_band(problem.mats, coeffs, kl, ku)
    ab, ipiv, info = band.gbtrf(ab0.copy(order="F"), kl, ku)
    if info:
        out = {"Y": np.zeros_like(V, order="F"), "info": info, "beta": 0.0, "sweeps": 0, "Tnorm": Tnorm}
        if return_factors:
            out.update(ab_in=ab0, ab=ab, ipiv=ipiv)
        return out
    Y = band.gbtrs(ab, kl, ku, ipiv, V)
    prev = math.inf
    beta = math.inf
    sweeps = 0
    for _ in range(refine_max):
        R = V - T @ Y
        beta = backward_error(T, Tnorm, V, Y, R)
        D = band.gbtrs(ab, kl, ku, ipiv, R)
        Y = Y + D
        sweeps += 1
        d = float(np.abs(D).max() / max(np.abs(Y).max(), 1e-300))
        if beta <= REFINE_TOL and (d <= REFINE_STEP_TOL or d > 0.5 * prev):
            break
        prev = d
    out = {"Y": np.asfortranarray(Y), "info": info, "beta": beta, "sweeps": sweeps, "Tnorm": Tnorm}
    if return_factors:
        out.update(ab_in=ab0, ab=ab, ipiv=ipiv)
    return out


def solve_points(problem, region, N: int, V: np.ndarray, js, *, kl=None, ku=None, **kw):
    """O1-O4 at selected quadrature points (threads over points; the C core releases the GIL)."""
    z, w, zeta = contour.nodes(region, N)
    F = contour.coefficient_table(problem.fns, z)
    if kl is None:
        kl, ku = band.bandwidths(problem.mats)
    with cf.ThreadPoolExecutor(_threads()) as ex:
        res = list(ex.map(lambda j: solve_point(problem, kl, ku, F[:, j], V, **kw), js))
    return res


def moments(problem, region, N: int, M: int, V: np.ndarray, *, kl=None, ku=None, keep_Y: bool = False):
    """O1-O5: S_k (k < M), mu_k (k < 2M), summed over j in ascending order."""
    n, L = V.shape
    z, w, zeta = contour.nodes(region, N)
    F = contour.coefficient_table(problem.fns, z)
    if kl is None:
        kl, ku = band.bandwidths(problem.mats)
    S = np.zeros((M, n, L), dtype=np.complex128)
    mu = np.zeros((2 * M, L, L), dtype=np.complex128)
    info = np.zeros(N, dtype=np.int64)
    beta = np.zeros(N)
    sweeps = np.zeros(N, dtype=np.int64)
    Ys = [] if keep_Y else None
    VH = V.conj().T
    chunk = max(1, _threads())
    with cf.ThreadPoolExecutor(_threads()) as ex:
        for j0 in range(0, N, chunk):
            js = list(range(j0, min(N, j0 + chunk)))
            res = list(ex.map(lambda j: solve_point(problem, kl, ku, F[:, j], V), js))
            for j, r in zip(js, res):
                Y = r["Y"]
                info[j], beta[j], sweeps[j] = r["info"], r["beta"], r["sweeps"]
                P = VH @ Y
                for k in range(2 * M):
                    c = w[j] * zeta[j] ** k
                    if k < M:
                        S[k] += c * Y
                    mu[k] += c * P
                if keep_Y:
                    Ys.append(Y)
    return {"z": z, "w": w, "zeta": zeta, "F": F, "S": S, "mu": mu, "info": info, "beta": beta,
            "sweeps": sweeps, "Y": Ys, "kl": kl, "ku": ku}


def hankel_matrices(mu: np.ndarray):
    """H = [mu_{i+j}], H< = [mu_{i+j+1}] (block i, j < M), each LM x LM."""
    M2, L, _ = mu.shape
    M = M2 // 2
    H = np.zeros((L * M, L * M), dtype=np.complex128)
    Hs = np.zeros_like(H)
    for i in range(M):
        for j in range(M):
            H[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j]
            Hs[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j + 1]
    return H, Hs


def hankel_extract(S: np.ndarray, mu: np.ndarray, region: dict, delta: float = DELTA_HANKEL):
    """O6: rank-revealing SVD of the block Hankel matrix and the reduced eigenproblem."""
    H, Hs = hankel_matrices(mu)
    U, sig, Wh = np.linalg.svd(H)
    m = int(np.count_nonzero(sig > delta * sig[0])) if sig[0] > 0 else 0
    Wm = Wh[:m].conj().T
    Bred = U[:, :m].conj().T @ Hs @ Wm @ np.diag(1.0 / sig[:m])
    theta, Tv = np.linalg.eig(Bred)
    lam = complex(region["center"]) + float(region["a"]) * theta
    M, n, L = S.shape
    Scat = np.concatenate([S[k] for k in range(M)], axis=1)  # n x LM, block k = S_k
    XH = Scat @ (Wm @ np.diag(1.0 / sig[:m]) @ Tv)
    return {"H": H, "Hs": Hs, "sigma": sig, "m": m, "Bred": Bred, "theta": theta, "cand": lam, "XH": XH}


def orth_basis(XH: np.ndarray, delta: float = DELTA_BASIS):
    """O7: orthonormal basis of the column-normalised Hankel eigenvector block (truncated SVD)."""
    if XH.shape[1] == 0:
        return XH.copy()
    Xn = XH / np.linalg.norm(XH, axis=0, keepdims=True)
    U, sig, _ = np.linalg.svd(Xn, full_matrices=False)
    k = int(np.count_nonzero(sig > delta * sig[0]))
    return U[:, :k]


def project(mats, Q):
    """B_i = Q^H A_i Q (Sec. 4.2 Eq. (narnoldi-split))."""
    return [Q.conj().T @ (A @ Q) for A in mats]


def newton_projected(Bs, fns, lam0: complex, y0: np.ndarray, region: dict):
    """Newton's method (Sec. 4.1 Eq. (newton)) on the projected NEP sum_i f_i(lam) B_i y = 0.

    Bordered system with normalisation u^H y = 1, u the current unit iterate:
        [ B(lam)  B'(lam) y ] [dy  ]     [ B(lam) y ]
        [ u^H     0         ] [dlam] = - [    0     ]
    Stops when |dlam| <= NEWTON_TOL * max(1, |lam|) or after NEWTON_MAX steps; a
    step leaving the disc |lam - c| <= 4 max(a, b) marks the candidate invalid (its
    iterate has left every neighbourhood of the region, where the acceptance test of O9
    would drop it anyway).
    """
    k = Bs[0].shape[0]
    y = y0 / np.linalg.norm(y0)
    lam = complex(lam0)
    c = complex(region["center"])
    rad = 4.0 * max(region["a"], region["b"])
    ok = True
    it = 0
    for it in range(1, NEWTON_MAX + 1):
        fv = np.array([fn.evaluate(f, lam) for f in fns])
        Bl = sum(fv[i, 0] * Bs[i] for i in range(len(Bs)))
        dB = sum(fv[i, 1] * Bs[i] for i in range(len(Bs)))
        J = np.zeros((k + 1, k + 1), dtype=np.complex128)
        J[:k, :k] = Bl
        J[:k, k] = dB @ y
        J[k, :k] = y.conj()
        rhs = np.concatenate([-(Bl @ y), [0.0]])
        try:
            d = np.linalg.solve(J, rhs)
        except np.linalg.LinAlgError:
            ok = False
            break
        y = y + d[:k]
        lam = lam + d[k]
        y = y / np.linalg.norm(y)
        if not np.isfinite(lam) or abs(lam - c) > rad:
            ok = False
            break
        if abs(d[k]) <= NEWTON_TOL * max(1.0, abs(lam)):
            break
    return lam, y, ok, it


def normalise_vector(x: np.ndarray) -> np.ndarray:
    """Unit 2-norm, phase fixed so that the first entry of largest modulus is real positive."""
    x = x / np.linalg.norm(x)
    i = int(np.argmax(np.abs(x)))
    return x * (abs(x[i]) / x[i])


def scaled_residual(mats, fns, norms, lam: complex, x: np.ndarray) -> float:
    """eta = ||T(lam) x||_2 / (sum_i |f_i(lam)| ||A_i||_inf ||x||_2), Sec. 2 Eq. (sressplit)."""
    fv = np.array([fn.values(f, lam) for f in fns]).reshape(-1)
    r = np.zeros(x.shape[0], dtype=np.complex128)
    for A, f in zip(mats, fv):
        r += f * (A @ x)
    return float(np.linalg.norm(r) / (np.sum(np.abs(fv) * norms) * np.linalg.norm(x)))


def solve(problem, region=None, N=None, L=None, M=None, V=None, *, eig_tol: float = EIG_TOL,
          delta: float = DELTA_HANKEL, keep: bool = False):
    """Full CISS pass O1-O10. Returns eigenvalues, eigenvectors, residuals and diagnostics."""
    region = region or problem.region
    N = N or problem.N
    L = L or problem.L
    M = M or problem.M
    if V is None:
        raise ValueError("the oracle takes the probe block V as an input")
    mom = moments(problem, region, N, M, V, keep_Y=keep)
    hk = hankel_extract(mom["S"], mom["mu"], region, delta)
    Q = orth_basis(hk["XH"])
    Bs = project(problem.mats, Q)
    norms = term_norms_inf(problem.mats)
    lam_list, x_list, eta_list = [], [], []
    newton_info = []
    for k in range(hk["m"]):
        y0 = Q.conj().T @ hk["XH"][:, k]
        if np.linalg.norm(y0) == 0:
            newton_info.append((False, 0))
            continue
        lam, y, ok, it = newton_projected(Bs, problem.fns, hk["cand"][k], y0, region)
        newton_info.append((ok, it))
        if not ok:
            continue
        x = normalise_vector(Q @ y)
        eta = scaled_residual(problem.mats, problem.fns, norms, lam, x)
        lam_list.append(lam)
        x_list.append(x)
        eta_list.append(eta)
    lam_a = np.array(lam_list, dtype=np.complex128)
    eta_a = np.array(eta_list)
    keep_mask = contour.inside(region, lam_a) & (eta_a <= eig_tol) if len(lam_a) else np.zeros(0, bool)
    order = np.argsort(eta_a, kind="stable") if len(lam_a) else np.zeros(0, int)
    acc = []
    for i in order:
        if not keep_mask[i]:
            continue
        dup = False
        for j in acc:
            if abs(lam_a[i] - lam_a[j]) <= DEDUP_LAMBDA * max(1.0, abs(lam_a[i])) and \
                    abs(np.vdot(x_list[i], x_list[j])) >= 1.0 - DEDUP_VECTOR:
                dup = True
                break
        if not dup:
            acc.append(i)
    acc.sort(key=lambda i: (lam_a[i].real, lam_a[i].imag))
    lam_out = lam_a[acc] if acc else np.zeros(0, np.complex128)
    X_out = np.stack([x_list[i] for i in acc], axis=1) if acc else np.zeros((problem.n, 0), np.complex128)
    eta_out = eta_a[acc] if acc else np.zeros(0)
    out = {"lam": lam_out, "X": X_out, "eta": eta_out, "m": hk["m"], "sigma": hk["sigma"],
           "cand": hk["cand"], "rank_basis": Q.shape[1], "saturated": hk["m"] == L * M,
           "S": mom["S"], "mu": mom["mu"], "beta": mom["beta"], "sweeps": mom["sweeps"], "info": mom["info"],
           "z": mom["z"], "w": mom["w"], "F": mom["F"], "kl": mom["kl"], "ku": mom["ku"], "newton": newton_info}
    if keep:
        out.update(Y=mom["Y"], H=hk["H"], Hs=hk["Hs"], XH=hk["XH"], Q=Q)
    return out
