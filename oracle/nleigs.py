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
    block of the eigenvector;
  * Arnoldi on S = (A - sigma B)^{-1} B in the compact (TOAR) representation of Sec. 4.5.3
    (Eqs. (nleigs-toar1)-(nleigs-toar4)), next to a plain full-basis Arnoldi on the explicit S.
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


def shift_invert_dense(problem, interp: dict, sigma: complex):
    """The explicit S = (A - sigma B)^{-1} B of the dense pencil (small problems only)."""
    A, B = linearization(problem.mats, interp)
    return np.linalg.solve(A - sigma * B, B)


def arnoldi_full(S: np.ndarray, v0: np.ndarray, k: int):
    """Plain Arnoldi (classical Gram-Schmidt twice) on an explicit matrix: V (N x k+1), H (k+1 x k)."""
    N = S.shape[0]
    V = np.zeros((N, k + 1), np.complex128)
    H = np.zeros((k + 1, k), np.complex128)
    V[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(k):
        w = S @ V[:, j]
        for _ in range(2):
            h = V[:, :j + 1].conj().T @ w
            w = w - V[:, :j + 1] @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


def arnoldi_toar(problem, interp: dict, sigma: complex, w0: np.ndarray, k: int):
    """Arnoldi on S in the compact (TOAR) representation of Sec. 4.5.3: every Krylov vector's d
    blocks are U g^i for one orthonormal U (n x (k+d)) and coefficient vectors g^i. The expansion
    follows Eqs. (nleigs-toar1)-(nleigs-toar4): the coefficient recurrence for y^1 .. y^{d-1}, the
    solve with R_d(sigma) for y^0 in split form, its orthogonalisation against U (which extends U
    by one vector), then the coefficients of S v. The Arnoldi orthogonalisation runs on the
    stacked coefficients (U has orthonormal columns). w0: n x d start blocks.
    Returns U, G (list of k+1 stacked coefficient vectors), H (k+1 x k)."""
    from . import band
    d, sig, xi, beta, dd = interp["d"], interp["sigma"], interp["xi"], interp["beta"], interp["dd"]
    mats = problem.mats
    inv_xi = np.array([1.0 / x if np.isfinite(x) else 0.0 for x in xi], np.complex128)
    bs = basis(sigma, sig, xi, beta, d)[:, 0]                     # b_j(sigma)
    Rd = sum(complex(dd[t] @ bs) * mats[t] for t in range(len(mats)))  # R_d(sigma), split form
    Rd = Rd.toarray() if hasattr(Rd, "toarray") else np.asarray(Rd)
    Q, R = np.linalg.qr(w0)                                       # U_d and g_1 (Algorithm, first lines)
    U = Q
    g = R.T.reshape(-1)                                           # blocks g^i = R[:, i], stacked
    g = g / np.linalg.norm(g)
    G = [g]
    H = np.zeros((k + 1, k), np.complex128)
    for j in range(k):
        m = U.shape[1]
        gb = G[-1].reshape(d, m)                                  # g^0 .. g^{d-1}
        # Eq. (nleigs-toar1): gt^{d-1} .. gt^1 (gt^i stands for y^i in the coefficients)
        gt = np.zeros((d, m), np.complex128)
        for i in range(d - 1, 0, -1):
            z = gb[i - 1] + beta[i] * inv_xi[i] * gb[i]
            nxt = gt[i + 1] if i + 1 < d else 0.0
            gt[i] = (z - beta[i] * (1.0 - sigma * inv_xi[i]) * nxt) / (sig[i - 1] - sigma)
        # Eq. (nleigs-toar2) in split form: y^0 = R_d(sigma)^{-1} (-sum_t A_t U c_t)
        rhs = np.zeros(problem.n, np.complex128)
        for t, A in enumerate(mats):
            c = sum(dd[t, i] * gt[i + 1] for i in range(d - 1)) + dd[t, d] / beta[d] * gb[d - 1]
            rhs -= A @ (U @ c)
        y0 = np.linalg.solve(Rd, rhs)
        # Eq. (nleigs-toar3): orthogonalise y^0 against U, extend U
        h = U.conj().T @ y0
        r = y0 - U @ h
        h2 = U.conj().T @ r
        r = r - U @ h2
        h = h + h2
        rho = np.linalg.norm(r)
        if rho <= 64 * np.finfo(float).eps * max(np.linalg.norm(y0), np.finfo(float).tiny):
            # y^0 already lies in span(U) (at the latest once U has n columns): U is not extended
            mp, gt0 = m, h
        else:
            mp = m + 1
            U = np.column_stack([U, r / rho])
            gt0 = np.concatenate([h, [rho]])
        # Eq. (nleigs-toar4): coefficients of S v in the (possibly extended) basis
        gn = np.zeros((d, mp), np.complex128)
        for i in range(d - 1):
            gn[i, :m] = gt[i + 1]
            gn[i] += bs[i] * gt0
        gn[d - 1] = bs[d - 1] * gt0
        gvec = gn.reshape(-1)
        # Arnoldi on the stacked coefficients (old vectors padded with zeros for a new column of U)
        Gm = np.column_stack([np.pad(x.reshape(d, -1), ((0, 0), (0, mp - x.size // d))).reshape(-1)
                              for x in G])
        for _ in range(2):
            hh = Gm.conj().T @ gvec
            gvec = gvec - Gm @ hh
            H[:j + 1, j] += hh
        H[j + 1, j] = np.linalg.norm(gvec)
        G.append(gvec / H[j + 1, j])
    return U, G, H


def toar_vectors(U: np.ndarray, G: list, d: int) -> np.ndarray:
    """The full Krylov vectors (I_d (x) U) g of the compact representation, as columns."""
    m = U.shape[1]
    cols = []
    for g in G:
        gb = g.reshape(d, -1)
        gb = np.pad(gb, ((0, 0), (0, m - gb.shape[1])))
        cols.append(np.concatenate([U @ gb[i] for i in range(d)]))
    return np.column_stack(cols)



def krylov_schur(S: np.ndarray, v0: np.ndarray, ncv: int, nkeep: int, wanted, tol: float = 1e-12,
                 max_restarts: int = 20, nev: int = 0):
    """Shift-and-invert Arnoldi on an explicit S with thick restarts in Krylov-Schur form and locking
    (the restart the paper runs on top of Algorithm (nleigs), Sec. 4.5.3), plain FP64.

    The decomposition S V[:, :k] = V[:, :k+1] Hf[:k+1, :k] is extended to k = ncv by Arnoldi steps
    (classical Gram-Schmidt twice). With H = Hf[:ncv, :ncv] and b = Hf[ncv, :], a Ritz pair (theta, y)
    of H (unit y) has the residual estimate |b^T y|; `wanted(theta)` marks the pairs sought, converged
    when |b^T y| <= tol |theta|. The run stops once nev wanted pairs have converged (the number of
    eigenvalues sought, which also sets the basis size in the experiments of Sec. 6; nev = 0: every
    wanted pair of the cycle, at least one) or after max_restarts restarts. A restart keeps an orthonormal basis Q of the selected Ritz
    vectors (converged wanted ones first, then the other wanted ones, then the rest, each by decreasing
    |theta|, i.e. nearest the shift first; nkeep of them, at least one more than the converged ones):
    V[:, :p] <- V[:, :ncv] Q, V[:, p] <- V[:, ncv], Hf[:p, :p] <- Q^H H Q and Hf[p, :p] <- b^T Q with the
    entries of the converged (locked) vectors set to zero, so they stay an invariant subspace.
    Returns V, Hf, the restarts run, the Ritz values and vectors of the last cycle, the residual
    estimates, and the wanted and converged indices."""
    N = S.shape[0]
    V = np.zeros((N, ncv + 1), np.complex128)
    Hf = np.zeros((ncv + 1, ncv), np.complex128)
    V[:, 0] = v0 / np.linalg.norm(v0)
    k0, restarts = 0, 0
    while True:
        for j in range(k0, ncv):
            w = S @ V[:, j]
            for _ in range(2):
                hh = V[:, :j + 1].conj().T @ w
                w = w - V[:, :j + 1] @ hh
                Hf[:j + 1, j] += hh
            Hf[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / Hf[j + 1, j]
        H, b = Hf[:ncv, :ncv], Hf[ncv, :]
        theta, Y = np.linalg.eig(H)
        Y = Y / np.linalg.norm(Y, axis=0, keepdims=True)
        res = np.abs(b @ Y)
        want = [q for q in range(ncv) if wanted(theta[q])]
        conv = [q for q in want if res[q] <= tol * abs(theta[q])]
        done = len(conv) >= nev if nev > 0 else (want and len(conv) == len(want))
        if done or restarts >= max_restarts:
            return {"V": V, "Hf": Hf, "restarts": restarts, "theta": theta, "Y": Y, "res": res,
                    "wanted": want, "converged": conv}
        by_size = lambda qs: sorted(qs, key=lambda q: -abs(theta[q]))
        conv_s = by_size(conv)
        rest = by_size([q for q in want if q not in conv])
        others = by_size([q for q in range(ncv) if q not in want])
        p = min(ncv - 1, max(nkeep, len(conv) + 1))
        sel = (conv_s + rest + others)[:p]
        Q, _ = np.linalg.qr(Y[:, sel])
        Hn = Q.conj().T @ H @ Q
        bn = b @ Q
        bn[:len(conv_s)] = 0.0
        Vn = V[:, :ncv] @ Q
        vlast = V[:, ncv].copy()
        V[:] = 0.0
        V[:, :p] = Vn
        V[:, p] = vlast
        Hf[:] = 0.0
        Hf[:p, :p] = Hn
        Hf[p, :p] = bn
        k0 = p
        restarts += 1
