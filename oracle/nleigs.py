"""NLEIGS, static variant (Sec. 4.5), in plain FP64 (oracle; test infrastructure only).

  * target set Sigma: the region's ellipse, its boundary discretised at NB points
    z_k = c + a cos(2 pi k/NB) + i b sin(2 pi k/NB);
  * singularity set Xi (Sec. 4.5.1): poles of the rational parts of the f_i (denominator roots
    from the companion matrix, zeros of a quotient's rational denominator), the branch cut of a
    square root discretised at CUT_T; exp has none; the outer function of a composition is
    not searched;
  * Leja-Bagby nodes sigma_j on the boundary and poles xi_j in Xi (Sec. 4.5.1 Eq.
    (nleigsleja)): sigma_0 = z_0; sigma_{j+1} maximises |s_j| on the boundary, xi_{j+1}
    minimises it over the points of Xi not taken yet (infinity once none is left);
  * basis b_0 = 1, b_j = b_{j-1} (z - sigma_{j-1}) / (beta_j (1 - z/xi_j)) with beta_j making
    max |b_j| = 1 on the boundary (Sec. 4.5.1 Eq. (nleigsbj));
  * rational divided differences d_i^j = e_j^T f_i(H K^{-1}) e_1 (Sec. 4.5.1 Eq. (nleigsfdd)),
    f_i of the matrix formed from its function tree (scipy expm / sqrtm, matrix polynomials);
  * degree d: the first d >= 1 whose last pole, taken as infinity, gives
    max_i |d_i^d| < tol max_i |d_i^0| (Sec. 4.5.1; the last pole is infinity, Sec. 4.5.1
    Eq. (nleigsmatlin));
  * the linearisation pencil (A, B) of Eq. (nleigsmatlin) built densely, its eigenvalues by a
    library generalized eigensolver: the eigenvalues of R_d(lambda) x = 0, with x the first
    block of the eigenvector.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import contour, fn

NB = 1024                      # boundary points of Sigma
CUT_T = np.concatenate([[0.0], 10.0 ** np.linspace(-4.0, 4.0, 48)])  # square-root cut samples
DMAX = 60
TOL = 1e-13


def boundary(region: dict, nb: int = NB) -> np.ndarray:
    th = 2.0 * np.pi * np.arange(nb) / nb
    return complex(region["center"]) + region["a"] * np.cos(th) + 1j * region["b"] * np.sin(th)


def _sing(spec: dict, scale: complex) -> list:
    """Singular points in z of a node whose input is scale * z."""
    alpha = complex(spec.get("alpha", 1.0))
    s = alpha * scale  # the node's inner argument is u = s z
    kind = spec["kind"]
    out = []
    if kind == "rational":
        den = spec.get("den")
        if den is not None and len(den) > 1:
            out += [r / s for r in np.roots(np.asarray(den, dtype=np.complex128))]
    elif kind == "sqrt":
        out += [(complex(spec.get("shift", 0.0)) - t) / s for t in CUT_T]
    elif kind == "combine":
        op = spec["op"]
        if op == "compose":
            out += _sing(spec["b"], s)
        else:
            out += _sing(spec["a"], s) + _sing(spec["b"], s)
            b = spec["b"]
            if op == "div" and b["kind"] == "rational" and len(b["num"]) > 1:
                sb = complex(b.get("alpha", 1.0)) * s
                out += [r / sb for r in np.roots(np.asarray(b["num"], dtype=np.complex128))]
    return out


def singularities(fns) -> np.ndarray:
    pts = []
    for f in fns:
        pts += _sing(f, 1.0)
    return np.array(pts, dtype=np.complex128)


def leja_bagby(bnd: np.ndarray, Xi: np.ndarray, dmax: int):
    """Nodes sigma[0..dmax], poles xi[0..dmax] (xi[0] unused, inf = none)."""
    sigma = np.zeros(dmax + 1, np.complex128)
    xi = np.full(dmax + 1, np.inf + 0j)
    sigma[0] = bnd[0]
    used = np.zeros(len(Xi), bool)
    sb = bnd - sigma[0]           # s_0 on the boundary
    sx = Xi - sigma[0]            # s_0 on Xi
    for j in range(dmax):
        sigma[j + 1] = bnd[int(np.argmax(np.abs(sb)))]
        ax = np.abs(sx)
        ok = np.isfinite(ax) & ~used
        if ok.any():
            k = int(np.flatnonzero(ok)[np.argmin(ax[ok])])
            xi[j + 1] = Xi[k]
            used[k] = True
        # s_{j+1} = s_j (z - sigma_{j+1}) / (1 - z/xi_{j+1}), rescaled to max 1 on the boundary
        den_b = 1.0 - bnd / xi[j + 1] if np.isfinite(xi[j + 1]) else 1.0
        den_x = 1.0 - Xi / xi[j + 1] if np.isfinite(xi[j + 1]) else 1.0
        with np.errstate(divide="ignore", invalid="ignore"):
            sb = sb * (bnd - sigma[j + 1]) / den_b
            sx = sx * (Xi - sigma[j + 1]) / den_x
        if len(Xi) and np.isfinite(xi[j + 1]):
            sx[Xi == xi[j + 1]] = np.inf
        m = np.abs(sb).max()
        with np.errstate(invalid="ignore"):
            sb, sx = sb / m, sx / m
    return sigma, xi


def basis_scalings(bnd, sigma, xi, d):
    """beta[0..d] with max |b_j| = 1 on the boundary (beta_0 = 1)."""
    beta = np.ones(d + 1)
    b = np.ones(len(bnd), np.complex128)
    for j in range(1, d + 1):
        g = b * (bnd - sigma[j - 1])
        if np.isfinite(xi[j]):
            g = g / (1.0 - bnd / xi[j])
        beta[j] = np.abs(g).max()
        b = g / beta[j]
    return beta


def basis(z, sigma, xi, beta, d) -> np.ndarray:
    """b_0(z) .. b_d(z) (rows) for points z."""
    z = np.atleast_1d(np.asarray(z, np.complex128))
    out = np.zeros((d + 1, len(z)), np.complex128)
    out[0] = 1.0 / beta[0]
    for j in range(1, d + 1):
        g = out[j - 1] * (z - sigma[j - 1]) / beta[j]
        if np.isfinite(xi[j]):
            g = g / (1.0 - z / xi[j])
        out[j] = g
    return out


def matrix_function(spec: dict, M: np.ndarray) -> np.ndarray:
    """f(M) for a function tree: beta h(alpha M), h from the node kind."""
    n = M.shape[0]
    I = np.eye(n, dtype=np.complex128)
    X = complex(spec.get("alpha", 1.0)) * M
    kind = spec["kind"]
    if kind == "rational":
        def poly(c):
            R = np.zeros_like(X)
            for a in c:
                R = R @ X + complex(a) * I
            return R
        H = poly(spec["num"])
        if spec.get("den") is not None:
            H = np.linalg.solve(poly(spec["den"]), H)
    elif kind == "exp":
        H = scipy.linalg.expm(X)
    elif kind == "sqrt":
        H = scipy.linalg.sqrtm(X - complex(spec.get("shift", 0.0)) * I)
    elif kind == "combine":
        op = spec["op"]
        if op == "compose":
            H = matrix_function(spec["a"], matrix_function(spec["b"], X))
        else:
            A, B = matrix_function(spec["a"], X), matrix_function(spec["b"], X)
            H = {"add": lambda: A + B, "mul": lambda: A @ B, "div": lambda: np.linalg.solve(B, A)}[op]()
    else:
        raise ValueError(kind)
    return complex(spec.get("beta", 1.0)) * H


def divided_differences(fns, sigma, xi, beta, d) -> np.ndarray:
    """dd[i, j] = d_i^j = beta_0 e_j^T f_i(H K^{-1}) e_1 (Eq. (nleigsfdd))."""
    H = np.diag(sigma[:d + 1].astype(np.complex128))
    K = np.eye(d + 1, dtype=np.complex128)
    for j in range(1, d + 1):
        H[j, j - 1] = beta[j]
        K[j, j - 1] = beta[j] / xi[j] if np.isfinite(xi[j]) else 0.0
    M = H @ np.linalg.inv(K)
    return np.array([beta[0] * matrix_function(f, M)[:, 0] for f in fns])


def interpolation(fns, region: dict, tol: float = TOL, dmax: int = DMAX, nb: int = NB) -> dict:
    bnd = boundary(region, nb)
    Xi = singularities(fns)
    sigma, xi_nat = leja_bagby(bnd, Xi, dmax)
    for d in range(1, dmax + 1):
        xi = xi_nat[:d + 1].copy()
        xi[d] = np.inf  # the last pole of the interpolant is infinity
        beta = basis_scalings(bnd, sigma, xi, d)
        dd = divided_differences(fns, sigma, xi, beta, d)
        delta = np.abs(dd).max(axis=0)
        if delta[d] < tol * delta[0]:
            break
    return {"d": d, "sigma": sigma[:d + 1], "xi": xi, "beta": beta, "dd": dd, "Xi": Xi, "bnd": bnd,
            "xi_seq": xi_nat}


def interpolant_coeffs(interp: dict, z) -> np.ndarray:
    """r_i(z) = sum_j b_j(z) d_i^j: R_d(z) = sum_i r_i(z) A_i."""
    return interp["dd"] @ basis(z, interp["sigma"], interp["xi"], interp["beta"], interp["d"])


def linearization(mats, interp: dict):
    """Dense (A, B) of Eq. (nleigsmatlin), d blocks of n."""
    d, sigma, xi, beta, dd = interp["d"], interp["sigma"], interp["xi"], interp["beta"], interp["dd"]
    dense = [m.toarray() if hasattr(m, "toarray") else np.asarray(m) for m in mats]
    n = dense[0].shape[0]
    D = [sum(dd[i, j] * dense[i] for i in range(len(dense))) for j in range(d + 1)]
    A = np.zeros((d * n, d * n), np.complex128)
    B = np.zeros_like(A)
    I = np.eye(n)
    blk = lambda r, c: (slice(r * n, (r + 1) * n), slice(c * n, (c + 1) * n))
    for j in range(d - 1):
        A[blk(0, j)] = D[j]
    A[blk(0, d - 1)] = D[d - 1] - sigma[d - 1] / beta[d] * D[d]
    B[blk(0, d - 1)] = -D[d] / beta[d]
    for j in range(1, d):
        A[blk(j, j - 1)] = sigma[j - 1] * I
        A[blk(j, j)] = beta[j] * I
        B[blk(j, j - 1)] = I
        B[blk(j, j)] = (beta[j] / xi[j] if np.isfinite(xi[j]) else 0.0) * I
    return A, B


def solve(problem, region=None, *, tol: float = TOL, dmax: int = DMAX, eig_tol: float = 1e-8):
    """Eigenvalues of the linearisation inside Sigma with their first blocks, eta <= eig_tol."""
    from .ciss import normalise_vector, scaled_residual, term_norms_inf
    region = region or problem.region
    interp = interpolation(problem.fns, region, tol, dmax)
    A, B = linearization(problem.mats, interp)
    lam, Y = scipy.linalg.eig(A, B)
    n = problem.n
    norms = term_norms_inf(problem.mats)
    keep = np.isfinite(lam) & contour.inside(region, np.where(np.isfinite(lam), lam, 0.0))
    out_l, out_x, out_e = [], [], []
    for k in np.flatnonzero(keep):
        x = normalise_vector(Y[:n, k])
        eta = scaled_residual(problem.mats, problem.fns, norms, lam[k], x)
        if eta <= eig_tol:
            out_l.append(lam[k])
            out_x.append(x)
            out_e.append(eta)
    order = sorted(range(len(out_l)), key=lambda i: (out_l[i].real, out_l[i].imag))
    return {"lam": np.array([out_l[i] for i in order], np.complex128),
            "X": np.stack([out_x[i] for i in order], axis=1) if order else np.zeros((n, 0), np.complex128),
            "eta": np.array([out_e[i] for i in order]), "interp": interp}
