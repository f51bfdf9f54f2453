"""Eigenvalue count inside the contour by the argument principle (oracle; test infrastructure only).

The eigenvalues are the roots of det T(z) (Sec. 2, after Eq. (nep)), counted with
algebraic multiplicity (Sec. 2). For T holomorphic inside Gamma the count is the
winding number of det T(z) along Gamma. arg det T(z) is read off the banded LU
with partial pivoting: sum of arg u_jj plus pi per row interchange. Nodes are
doubled until every phase step along the contour is below pi/4.
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os

import numpy as np

from . import band, contour


def _phase(problem, kl, ku, z):
    coeffs = contour.coefficient_table(problem.fns, np.array([z]))[:, 0]
    ab = band.assemble_band(problem.mats, coeffs, kl, ku)
    ab, ipiv, info = band.gbtrf(ab, kl, ku)
    if info:
        raise ZeroDivisionError("det T(z) = 0 on the contour")
    kv = kl + ku
    diag = ab[kv, :]
    swaps = int(np.count_nonzero(ipiv != np.arange(len(ipiv))))
    return (float(np.sum(np.angle(diag))) + math.pi * swaps) % (2.0 * math.pi)


def count_inside(problem, region=None, K0: int = 256, Kmax: int = 1 << 16, threads=None) -> int:
    region = region or problem.region
    kl, ku = band.bandwidths(problem.mats)
    c = complex(region["center"])
    a, b = float(region["a"]), float(region["b"])
    threads = threads or max(1, min(32, os.cpu_count() or 1))
    cache = {}

    def phases(K):
        th = 2.0 * math.pi * (np.arange(K) + 0.25) / K
        zs = c + a * np.cos(th) + 1j * b * np.sin(th)
        todo = [zz for zz in zs if zz not in cache]
        with cf.ThreadPoolExecutor(threads) as ex:
            for zz, ph in zip(todo, ex.map(lambda q: _phase(problem, kl, ku, q), todo)):
                cache[zz] = ph
        return np.array([cache[zz] for zz in zs])

    K = K0
    while True:
        ph = phases(K)
        d = np.diff(np.concatenate([ph, ph[:1]]))
        d = (d + math.pi) % (2.0 * math.pi) - math.pi
        if np.all(np.abs(d) < math.pi / 4) or K >= Kmax:
            return int(round(float(np.sum(d)) / (2.0 * math.pi)))
        K *= 2
