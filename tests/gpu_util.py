"""Helpers shared by the GPU tests: device buffers via torch, layout conversions, matching."""
import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("needs a CUDA GPU")
    return torch


def to_dev(a, torch):
    """complex128 numpy -> float64 torch view on cuda (interleaved re, im), keeping memory order."""
    a = np.asarray(a)
    if np.iscomplexobj(a):
        flat = np.ascontiguousarray(a.ravel(order="K")).astype(np.complex128).view(np.float64)
    else:
        flat = np.ascontiguousarray(a.ravel(order="K"))
    return torch.from_numpy(flat.copy()).cuda()


def from_dev_c128(t):
    return t.cpu().numpy().view(np.complex128)


def from_dev_c64(t):
    return t.cpu().numpy().view(np.complex64)


def dense_from_rowband(ab_row, n, kl, ku, ldab):
    """Dense matrix from the library's row-oriented band input layout."""
    T = np.zeros((n, n), dtype=np.complex128)
    for r in range(n):
        for t in range(kl + ku + 1):
            k = r - kl + t
            if 0 <= k < n:
                T[r, k] = ab_row[r * ldab + t]
    return T


def factors_from_rowband(ab_row, n, kl, ku, ldab):
    """(U, L multipliers) from the library's factored layout: U[c, t] = U(c, c+t), L[c, i] = L(c+1+i, c)."""
    kv = kl + ku
    A = ab_row.reshape(n, ldab)
    return A[:, :kv + 1].copy(), A[:, kv + 1:kv + 1 + kl].copy()


def factors_from_gbtrf(ab, n, kl, ku):
    """Same (U, L) arrays from the oracle's LAPACK-layout factors."""
    kv = kl + ku
    U = np.zeros((n, kv + 1), dtype=np.complex128)
    L = np.zeros((n, kl), dtype=np.complex128)
    for c in range(n):
        for t in range(kv + 1):
            k = c + t
            if k < n:
                U[c, t] = ab[kv + c - k, k]
        for i in range(kl):
            r = c + 1 + i
            if r < n:
                L[c, i] = ab[kv + r - c, c]
    return U, L


def match_eigenvalues(a, b):
    """Pairs a[i] with b[j] by a greedy nearest assignment (sets of equal size); returns max rel error."""
    a, b = list(a), list(b)
    assert len(a) == len(b), (a, b)
    used = set()
    err = 0.0
    pairs = []
    for i, x in enumerate(a):
        j = min((j for j in range(len(b)) if j not in used), key=lambda j: abs(b[j] - x))
        used.add(j)
        pairs.append((i, j))
        err = max(err, abs(b[j] - x) / max(1.0, abs(x)))
    return err, pairs
