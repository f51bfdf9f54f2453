"""Band storage assembly of T(z) and ctypes glue for band_lu.c (oracle; test infrastructure only).

T(z) = sum_i f_i(z) A_i (Sec. 2 Eq. (split)); Sec. 3.2.2 builds it from the f_i(z)
values with l-1 sparse matrix axpy operations, which is what ``assemble_dense``
and ``assemble_band`` do (scipy sparse sums as the axpy primitive).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "band_lu.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_band.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile band_lu.c with the host C compiler (plain -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            zp = np.ctypeslib.ndpointer(np.complex128, flags="F_CONTIGUOUS")
            ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            lib.oracle_gbtrf.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, zp, ctypes.c_int, ip]
            lib.oracle_gbtrf.restype = ctypes.c_int
            lib.oracle_gbtrs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, zp, ctypes.c_int,
                                         ip, zp, ctypes.c_int]
            lib.oracle_gbtrs.restype = None
            _lib = lib
    return _lib


def bandwidths(mats):
    """(kl, ku) of the union sparsity pattern of all A_i."""
    kl = ku = 0
    for A in mats:
        C = sp.coo_matrix(A)
        if C.nnz:
            d = C.row.astype(np.int64) - C.col.astype(np.int64)
            kl = max(kl, int(d.max()))
            ku = max(ku, int(-d.min()))
    return kl, ku


def assemble_dense(mats, coeffs) -> np.ndarray:
    T = np.zeros(mats[0].shape, dtype=np.complex128)
    for A, f in zip(mats, coeffs):
        T += f * A.toarray()
    return T


def assemble_sparse(mats, coeffs) -> sp.csr_matrix:
    T = coeffs[0] * mats[0].astype(np.complex128)
    for A, f in zip(mats[1:], coeffs[1:]):
        T = T + f * A
    return sp.csr_matrix(T)


def assemble_band(mats, coeffs, kl: int, ku: int) -> np.ndarray:
    """Band array (ldab = 2 kl + ku + 1) x n, column-major, of T = sum_i coeffs[i] A_i."""
    n = mats[0].shape[0]
    ldab = 2 * kl + ku + 1
    ab = np.zeros((ldab, n), dtype=np.complex128, order="F")
    T = sp.coo_matrix(assemble_sparse(mats, coeffs))
    ab[kl + ku + T.row - T.col, T.col] = T.data
    return ab


def gbtrf(ab: np.ndarray, kl: int, ku: int):
    """In-place banded LU with partial pivoting; returns (ipiv, info)."""
    lib = _load()
    ab = np.asfortranarray(ab)
    n = ab.shape[1]
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib.oracle_gbtrf(n, kl, ku, ab, ab.shape[0], ipiv)
    return ab, ipiv, info


def gbtrs(ab: np.ndarray, kl: int, ku: int, ipiv: np.ndarray, B: np.ndarray) -> np.ndarray:
    lib = _load()
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    n, nrhs = X.shape
    lib.oracle_gbtrs(n, kl, ku, nrhs, ab, ab.shape[0], ipiv, X, n)
    return X
