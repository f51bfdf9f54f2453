"""Seeded generators for split-form nonlinear eigenproblems and probe blocks.

Every problem is T(z) = sum_i A_i f_i(z) (Sec. 2, Eq. (split)) with:
  * ``mats``: list of scipy.sparse CSR matrices (float64 or complex128), one per term;
  * ``fns``: list of function descriptions (plain dicts) understood by both the
    C-ABI binding and the oracle. Kinds (the FN classes of Sec. 3.2.2):
      {"kind": "rational", "num": [...], "den": [...] or None, "alpha": a, "beta": b}
            g(z) = b * p(a z) / q(a z), coefficients highest degree first;
      {"kind": "exp", "alpha": a, "beta": b}            g(z) = b * exp(a z);
      {"kind": "sqrt", "alpha": a, "beta": b, "shift": s}
            g(z) = b * sqrt(a z - s), principal branch;
      {"kind": "combine", "op": "add"|"mul"|"div"|"compose", "a": fa, "b": fb,
       "alpha": a, "beta": b}
            g(z) = b * h(a z), h = fa + fb, fa * fb, fa / fb or fa(fb(.)).
  * ``region``: ellipse {"center": c, "a": real semi-axis, "b": imaginary semi-axis}.

The problem families follow the experiments of Sec. 6 (delay, Drude-type rational
and square-root problems), on synthetic finite-difference grids with x fastest.
No quadrature, factorisation or moment arithmetic lives here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

# Seed streams: problem randomness uses default_rng(seed); the probe block V uses
# default_rng(seed + V_STREAM_OFFSET), so eigenvalue-determining data and V are
# independent streams.
V_STREAM_OFFSET = 1_000_003


@dataclasses.dataclass
class Problem:
    name: str
    n: int
    mats: list
    fns: list
    region: dict
    N: int = 32
    L: int = 4
    M: int = 4
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nterms(self) -> int:
        return len(self.mats)


def _rational(num, den=None, alpha=1.0, beta=1.0):
    return {"kind": "rational", "num": [complex(c) for c in num],
            "den": None if den is None else [complex(c) for c in den],
            "alpha": complex(alpha), "beta": complex(beta)}


def _exp(alpha=1.0, beta=1.0):
    return {"kind": "exp", "alpha": complex(alpha), "beta": complex(beta)}


def _sqrt(shift=0.0, alpha=1.0, beta=1.0):
    return {"kind": "sqrt", "alpha": complex(alpha), "beta": complex(beta), "shift": complex(shift)}


def _lap1d(s: int) -> sp.csr_matrix:
    e = np.ones(s)
    return sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], format="csr")


def _lap2d(s: int) -> sp.csr_matrix:
    """5-point stencil (+1 neighbours, -4 centre), Dirichlet, x fastest (index ix + s*iy)."""
    I = sp.identity(s, format="csr")
    T = _lap1d(s)
    return (sp.kron(I, T) + sp.kron(T, I)).tocsr()


def _lap3d(s: int) -> sp.csr_matrix:
    """7-point stencil (+1 neighbours, -6 centre), x fastest (index ix + s*iy + s^2*iz)."""
    I = sp.identity(s, format="csr")
    T = _lap1d(s)
    return (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).tocsr()


def _sorted_csr(A) -> sp.csr_matrix:
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    A.sort_indices()
    return A


def delay_1d(n: int = 64, seed: int = 0, tau: float = 1.0) -> Problem:
    """Delay problem T = -z I + A + e^{-tau z} B with A = 5 tridiag(1,-2,1), B = diag(U[-1,1]).

    Term order follows the split-form example of Sec. 3.2.2: (A, 1), (I, -z), (B, e^{-tau z}).
    Circle centre -1, radius 2; N=32, L=4, M=4.
    """
    rng = np.random.default_rng(seed)
    A = 5.0 * _lap1d(n)
    B = sp.diags(rng.uniform(-1.0, 1.0, n), 0, format="csr")
    I = sp.identity(n, format="csr")
    fns = [_rational([1.0]), _rational([-1.0, 0.0]), _exp(alpha=-tau)]
    return Problem("delay_1d", n, [_sorted_csr(A), _sorted_csr(I), _sorted_csr(B)], fns,
                   {"center": -1.0 + 0j, "a": 2.0, "b": 2.0}, N=32, L=4, M=4,
                   meta={"seed": seed, "tau": tau, "bandwidth": 1})


def delay_2d(s: int = 64, seed: int = 0, tau: float = 1.0, center=-2.0, radius=3.0) -> Problem:
    """Delay problem on an s x s grid: A = Lap_h / pi^2 (h = 1/(s+1)), B = diag(U[-1,1]).

    n = s^2, bandwidth s. Circle centre -2, radius 3; N=64, L=16, M=8 at s = 64.
    """
    n = s * s
    h = 1.0 / (s + 1)
    rng = np.random.default_rng(seed)
    A = _lap2d(s) * (1.0 / (math.pi ** 2 * h * h))
    B = sp.diags(rng.uniform(-1.0, 1.0, n), 0, format="csr")
    I = sp.identity(n, format="csr")
    fns = [_rational([1.0]), _rational([-1.0, 0.0]), _exp(alpha=-tau)]
    return Problem("delay_2d", n, [_sorted_csr(A), _sorted_csr(I), _sorted_csr(B)], fns,
                   {"center": complex(center), "a": float(radius), "b": float(radius)}, N=64, L=16, M=8,
                   meta={"seed": seed, "tau": tau, "grid": s, "bandwidth": s})


def _drude_fns(omega_p: float, gamma: float):
    # -z^2 eps(z) with eps(z) = 1 - wp^2/(z (z + i g)):  -z^2 + wp^2 z/(z + i g)
    #   = (-z^3 - i g z^2 + wp^2 z) / (z + i g)   (the pole at 0 cancels).
    num = [-1.0, -1j * gamma, omega_p ** 2, 0.0]
    den = [1.0, 1j * gamma]
    return [_rational([1.0]), _rational([-1.0, 0.0, 0.0]), _rational(num, den)]


def drude_2d(s: int = 128, seed: int = 0, omega_p: float = 3.0, gamma: float = 0.1,
             block: int | None = None, center=2.0, a=1.0, b=0.2) -> Problem:
    """Drude-type rational problem T = K - z^2 M - z^2 eps(z) D on an s x s grid.

    K = -Lap_h / pi^2 (positive stiffness), M = diag(U[1,2]), D = indicator of the
    central block (40 x 40 at s = 128: grid indices 44..83), eps(z) = 1 - wp^2/(z(z+i g)).
    Ellipse centre 2, semi-axes 1 (real) and 0.2 (imaginary); N=128, L=32, M=8 at s = 128.
    """
    n = s * s
    h = 1.0 / (s + 1)
    rng = np.random.default_rng(seed)
    K = _lap2d(s) * (-1.0 / (math.pi ** 2 * h * h))
    Mm = sp.diags(rng.uniform(1.0, 2.0, n), 0, format="csr")
    if block is None:
        block = int(round(40 * s / 128))
    lo = (s - block) // 2
    mask = np.zeros((s, s))
    mask[lo:lo + block, lo:lo + block] = 1.0
    D = sp.diags(mask.reshape(-1), 0, format="csr")
    return Problem("drude_2d", n, [_sorted_csr(K), _sorted_csr(Mm), _sorted_csr(D)], _drude_fns(omega_p, gamma),
                   {"center": complex(center), "a": float(a), "b": float(b)}, N=128, L=32, M=8,
                   meta={"seed": seed, "grid": s, "bandwidth": s, "omega_p": omega_p, "gamma": gamma,
                         "block": (lo, lo + block - 1)})


def sqrt_3d(s: int = 24, seed: int = 0, sigma1: float = 0.0, sigma2: float = 1.0,
            center=4.0, radius=1.5) -> Problem:
    """Square-root problem T = K - z M + i sqrt(z - s1^2) W1 + i sqrt(z - s2^2) W2 on an s^3 grid.

    K = -Lap3D_h / pi^2, M = diag(U[0.5,1.5]), W1/W2 = indicators of the x = 0 and x = s-1
    faces. n = s^3, bandwidth s^2. Circle centre 4, radius 1.5; N=64, L=24, M=8 at s = 24.
    """
    n = s ** 3
    h = 1.0 / (s + 1)
    rng = np.random.default_rng(seed)
    K = _lap3d(s) * (-1.0 / (math.pi ** 2 * h * h))
    Mm = sp.diags(rng.uniform(0.5, 1.5, n), 0, format="csr")
    ix = np.arange(n) % s
    W1 = sp.diags((ix == 0).astype(float), 0, format="csr")
    W2 = sp.diags((ix == s - 1).astype(float), 0, format="csr")
    fns = [_rational([1.0]), _rational([-1.0, 0.0]), _sqrt(shift=sigma1 ** 2, beta=1j), _sqrt(shift=sigma2 ** 2, beta=1j)]
    return Problem("sqrt_3d", n, [_sorted_csr(K), _sorted_csr(Mm), _sorted_csr(W1), _sorted_csr(W2)], fns,
                   {"center": complex(center), "a": float(radius), "b": float(radius)}, N=64, L=24, M=8,
                   meta={"seed": seed, "grid": s, "bandwidth": s * s, "sigma1": sigma1, "sigma2": sigma2})


# ---------------------------------------------------------------- diagonal (decoupled) problems
def diagonal_delay(n: int = 8, seed: int = 0, center=-1.0, radius=2.0, tau: float = 1.0) -> Problem:
    """T = -z I + diag(a) + e^{-tau z} diag(b): n decoupled scalar delay equations."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-2.5, 0.5, n)
    b = rng.uniform(-1.0, 1.0, n)
    fns = [_rational([1.0]), _rational([-1.0, 0.0]), _exp(alpha=-tau)]
    mats = [sp.diags(a, 0, format="csr"), sp.identity(n, format="csr"), sp.diags(b, 0, format="csr")]
    return Problem("diagonal_delay", n, [_sorted_csr(m) for m in mats], fns,
                   {"center": complex(center), "a": float(radius), "b": float(radius)}, N=64, L=4, M=4,
                   meta={"seed": seed, "tau": tau, "a": a, "b": b})


def diagonal_drude(n: int = 6, seed: int = 0, omega_p: float = 3.0, gamma: float = 0.1,
                   center=2.0, a=1.0, b=0.5) -> Problem:
    """T = diag(k) - z^2 diag(m) - z^2 eps(z) diag(d): decoupled scalar rational equations."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(2.0, 12.0, n)
    m = rng.uniform(1.0, 2.0, n)
    d = (rng.uniform(0, 1, n) < 0.5).astype(float)
    mats = [sp.diags(k, 0, format="csr"), sp.diags(m, 0, format="csr"), sp.diags(d, 0, format="csr")]
    return Problem("diagonal_drude", n, [_sorted_csr(x) for x in mats], _drude_fns(omega_p, gamma),
                   {"center": complex(center), "a": float(a), "b": float(b)}, N=128, L=4, M=4,
                   meta={"seed": seed, "k": k, "m": m, "d": d, "omega_p": omega_p, "gamma": gamma})


def diagonal_sqrt(n: int = 6, seed: int = 0, sigma: float = 1.0, center=4.0, radius=1.5) -> Problem:
    """T = diag(k) - z diag(m) + i sqrt(z - sigma^2) diag(w): decoupled square-root equations."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(3.0, 6.0, n)
    m = rng.uniform(0.8, 1.2, n)
    w = rng.uniform(0.0, 0.5, n)
    mats = [sp.diags(k, 0, format="csr"), sp.diags(m, 0, format="csr"), sp.diags(w, 0, format="csr")]
    fns = [_rational([1.0]), _rational([-1.0, 0.0]), _sqrt(shift=sigma ** 2, beta=1j)]
    return Problem("diagonal_sqrt", n, [_sorted_csr(x) for x in mats], fns,
                   {"center": complex(center), "a": float(radius), "b": float(radius)}, N=64, L=4, M=4,
                   meta={"seed": seed, "k": k, "m": m, "w": w, "sigma": sigma})


def dense_drude_small(n: int = 6, seed: int = 0, omega_p: float = 3.0, gamma: float = 0.1,
                      center=2.0, a=1.5, b=0.6) -> Problem:
    """Tiny coupled Drude problem with dense symmetric K, diagonal M, D (for linearisation checks)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    K = G @ G.T / n + np.diag(rng.uniform(2.0, 8.0, n))
    m = rng.uniform(1.0, 2.0, n)
    d = (rng.uniform(0, 1, n) < 0.5).astype(float)
    mats = [sp.csr_matrix(K), sp.diags(m, 0, format="csr"), sp.diags(d, 0, format="csr")]
    return Problem("dense_drude_small", n, [_sorted_csr(x) for x in mats], _drude_fns(omega_p, gamma),
                   {"center": complex(center), "a": float(a), "b": float(b)}, N=128, L=6, M=4,
                   meta={"seed": seed})


def dense_linear_small(n: int = 10, seed: int = 0, center=0.0 + 0j, radius=1.2) -> Problem:
    """Tiny linear problem T(z) = A - z B with dense random A and diagonally dominant B."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A /= math.sqrt(n)
    B = np.eye(n) + 0.1 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(n)
    mats = [sp.csr_matrix(A), sp.csr_matrix(B)]
    fns = [_rational([1.0]), _rational([-1.0, 0.0])]
    return Problem("dense_linear_small", n, [_sorted_csr(x) for x in mats], fns,
                   {"center": complex(center), "a": float(radius), "b": float(radius)}, N=64, L=6, M=4,
                   meta={"seed": seed})


# ---------------------------------------------------------------- named workloads
CONFIGS = {
    # delay, n=64, dense/tridiagonal, circle c=-1 r=2, N=32, L=4, M=4, plain FP64
    "delay1d_n64": dict(builder="delay_1d", kwargs=dict(n=64), N=32, L=4, M=4),
    # same problem with a wider probe block (L*M = 64 exceeds the eigenvalue count)
    "delay1d_n64_wide": dict(builder="delay_1d", kwargs=dict(n=64), N=32, L=16, M=4),
    # delay, 64x64 grid, n=4096, band 64, circle c=-2 r=3, N=64, L=16, M=8
    "delay2d_s64": dict(builder="delay_2d", kwargs=dict(s=64), N=64, L=16, M=8),
    # Drude, 128x128 grid, n=16384, band 128, ellipse c=2 a=1 b=0.2, N=128, L=32, M=8
    "drude2d_s128": dict(builder="drude_2d", kwargs=dict(s=128), N=128, L=32, M=8),
    # square-root, 24^3 grid, n=13824, band 576, circle c=4 r=1.5, N=64, L=24, M=8
    "sqrt3d_s24": dict(builder="sqrt_3d", kwargs=dict(s=24), N=64, L=24, M=8),
}

_BUILDERS = {"delay_1d": delay_1d, "delay_2d": delay_2d, "drude_2d": drude_2d, "sqrt_3d": sqrt_3d}


def config_problem(name: str, seed: int = 0) -> Problem:
    cfg = CONFIGS[name]
    p = _BUILDERS[cfg["builder"]](seed=seed, **cfg["kwargs"])
    p.N, p.L, p.M = cfg["N"], cfg["L"], cfg["M"]
    p.name = name
    return p


def random_probe_block(n: int, L: int, seed: int = 0) -> np.ndarray:
    """V (n x L, column-major) with Re and Im iid N(0,1) from numpy's PCG64 stream seed + offset."""
    rng = np.random.default_rng(seed + V_STREAM_OFFSET)
    re = rng.standard_normal((L, n))
    im = rng.standard_normal((L, n))
    return np.asfortranarray((re + 1j * im).T)


def serving_requests(count: int = 2000, seed: int = 0, rate_hz: float = 100.0,
                     s_min: int = 16, s_max: int = 128):
    """Request stream for continuous-batching serving: Poisson arrivals, delay or Drude on s x s grids.

    n log-uniform in [s_min^2, s_max^2] (s = round(sqrt(n))), N in {32,64,128}, L in {8,16,32},
    M = 8, contour centre shifted by U[-0.5, 0.5] from the family's centre.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, count))
    out = []
    for r in range(count):
        n = math.exp(rng.uniform(math.log(s_min ** 2), math.log(s_max ** 2)))
        s = int(round(math.sqrt(n)))
        fam = "delay" if rng.uniform() < 0.5 else "drude"
        N = int(rng.choice([32, 64, 128]))
        L = int(rng.choice([8, 16, 32]))
        shift = float(rng.uniform(-0.5, 0.5))
        pseed = int(rng.integers(0, 2 ** 31))
        out.append(dict(arrival=float(t[r]), family=fam, s=s, N=N, L=L, M=8, shift=shift, seed=pseed))
    return out


def serving_problem(req: dict) -> Problem:
    if req["family"] == "delay":
        p = delay_2d(s=req["s"], seed=req["seed"], center=-2.0 + req["shift"])
    else:
        p = drude_2d(s=req["s"], seed=req["seed"], center=2.0 + req["shift"])
    p.N, p.L, p.M = req["N"], min(req["L"], p.n), req["M"]
    return p
