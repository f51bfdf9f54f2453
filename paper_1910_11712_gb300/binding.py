"""ctypes binding of libnepciss.so: the same entry points as include/nep_ciss.h.

Argument marshalling only: every numerical step runs inside the CUDA library. If the
library is missing, ``load()`` raises; there is no CPU fallback. Device buffers are passed
as raw pointers (e.g. ``torch.Tensor.data_ptr()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# Hardware work queues of the CUDA context (read once, when the process creates it; 8 by default).
# Streams beyond that count share queues, so with a server's worker streams busy a short copy on
# one stream can wait behind another stream's whole pass. 32 is the largest value; a process that
# set it, or created its context before this import, keeps what it has.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

c_int32, c_int64, c_double, c_void_p, c_size_t = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
P_double = ctypes.POINTER(c_double)

NEP_OK = 0
NEP_PENDING = 1
NEP_ERR_ARG, NEP_ERR_CUDA, NEP_ERR_REGION, NEP_ERR_NOMEM, NEP_ERR_UNSUPPORTED, NEP_ERR_INTERNAL = -1, -2, -3, -4, -5, -6
NEP_WARN_SATURATED, NEP_WARN_REFINE, NEP_WARN_SINGULAR_NODE, NEP_WARN_NEWTON = 1, 2, 4, 8
NEP_PREC_FP64, NEP_PREC_MIXED = 0, 1
FN_KIND = {"rational": 0, "exp": 1, "sqrt": 2, "combine": 3, "callback": 4, "table": 5}
FN_OP = {"add": 0, "mul": 1, "div": 2, "compose": 3}


class NepCsr(ctypes.Structure):
    _fields_ = [("n_rows", c_int32), ("n_cols", c_int32), ("rowptr", ctypes.POINTER(c_int64)),
                ("col", ctypes.POINTER(c_int32)), ("val_re", P_double), ("val_im", P_double)]


class NepFn(ctypes.Structure):
    pass


# void eval(const double* z, int32_t count, double* f, double* df, void* ctx)
NEP_FN_EVAL = ctypes.CFUNCTYPE(None, P_double, c_int32, P_double, P_double, c_void_p)

NepFn._fields_ = [("kind", c_int32), ("alpha_re", c_double), ("alpha_im", c_double), ("beta_re", c_double),
                  ("beta_im", c_double), ("shift_re", c_double), ("shift_im", c_double), ("nnum", c_int32),
                  ("nden", c_int32), ("num", P_double), ("den", P_double), ("op", c_int32),
                  ("a", ctypes.POINTER(NepFn)), ("b", ctypes.POINTER(NepFn)), ("eval", NEP_FN_EVAL),
                  ("ctx", c_void_p), ("table", P_double), ("table_count", c_int32)]


class NepRegion(ctypes.Structure):
    _fields_ = [("center_re", c_double), ("center_im", c_double), ("a", c_double), ("b", c_double)]


class NepOpts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("rank_tol", c_double), ("basis_tol", c_double), ("refine_tol", c_double),
                ("step_tol", c_double), ("refine_max", c_int32), ("eig_tol", c_double), ("newton_max", c_int32),
                ("newton_tol", c_double), ("seed", ctypes.c_uint64), ("symmetric", c_int32),
                ("newton_abandon", c_int32), ("refine_extrapolate", c_int32), ("lu_kernel", c_int32),
                ("solve_rh", c_int32)]


class NepNleigsOpts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_degree", c_int32), ("nboundary", c_int32), ("krylov", c_int32),
                ("has_shift", c_int32), ("shift_re", c_double), ("shift_im", c_double), ("seed", ctypes.c_uint64),
                ("eig_tol", c_double), ("exact_solves", c_int32), ("full_basis", c_int32),
                ("max_restarts", c_int32), ("keep", c_int32), ("restart_tol", c_double), ("nev", c_int32)]


class NepInterpolOpts(ctypes.Structure):
    _fields_ = [("degree", c_int32), ("krylov", c_int32), ("has_shift", c_int32), ("shift_re", c_double),
                ("shift_im", c_double), ("seed", ctypes.c_uint64), ("eig_tol", c_double), ("fast_solves", c_int32),
                ("max_restarts", c_int32), ("keep", c_int32), ("restart_tol", c_double), ("nev", c_int32)]


class NepTuneResult(ctypes.Structure):
    _fields_ = [("lu_kernel", c_int32), ("solve_rh", c_int32), ("ms", c_double), ("candidates", c_int32),
                ("accurate", c_int32)]


class NepResultInfo(ctypes.Structure):
    _fields_ = [("n", c_int32), ("N", c_int32), ("L", c_int32), ("M", c_int32), ("precision", c_int32),
                ("hankel_rank", c_int32), ("basis_rank", c_int32), ("ncandidates", c_int32),
                ("max_sweeps", c_int32), ("svd_sweeps", c_int32), ("flags", c_int32), ("max_backward", c_double),
                ("ms_assemble", c_double), ("ms_factor", c_double), ("ms_solve", c_double),
                ("ms_moments", c_double), ("ms_extract", c_double), ("ms_total", c_double),
                ("ms_queued", c_double), ("ms_latency", c_double), ("newton_failed", c_int32),
                ("newton_left", c_int32), ("krylov_steps", c_int32), ("restarts", c_int32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "nep_opts_default": (None, [ctypes.POINTER(NepOpts)]),
    "nep_create_split": (c_int32, [c_int32, c_int32, ctypes.POINTER(NepCsr), ctypes.POINTER(NepFn), ctypes.POINTER(c_void_p)]),
    "nep_destroy": (c_int32, [c_void_p]),
    "nep_split_info": (c_int32, [c_void_p] + [ctypes.POINTER(c_int32)] * 5),
    "nep_ciss_solve": (c_int32, [c_void_p, ctypes.POINTER(NepRegion), c_int32, c_int32, c_int32, ctypes.POINTER(NepOpts),
                                 c_void_p, ctypes.POINTER(c_void_p)]),
    "nep_result_get": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(P_double), ctypes.POINTER(P_double),
                                 ctypes.POINTER(P_double), ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "nep_result_info": (c_int32, [c_void_p, ctypes.POINTER(NepResultInfo)]),
    "nep_result_hankel_sigma": (c_int32, [c_void_p, ctypes.POINTER(P_double), ctypes.POINTER(c_int32)]),
    "nep_result_free": (c_int32, [c_void_p]),
    "nep_last_error": (ctypes.c_char_p, []),
    "nep_kernel_launches": (ctypes.c_uint64, []),
    "nep_set_wait_limit": (c_int32, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "nep_server_create": (c_int32, [c_int32, ctypes.c_uint64, ctypes.POINTER(c_void_p)]),
    "nep_server_create_batched": (c_int32, [c_int32, c_int32, ctypes.c_uint64, ctypes.POINTER(c_void_p)]),
    "nep_submit": (c_int32, [c_void_p, c_void_p, ctypes.POINTER(NepRegion), c_int32, c_int32, c_int32,
                             ctypes.POINTER(NepOpts), c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "nep_poll": (c_int32, [c_void_p, ctypes.c_uint64, ctypes.POINTER(c_void_p)]),
    "nep_server_wait": (c_int32, [c_void_p, ctypes.c_uint64, ctypes.POINTER(c_void_p)]),
    "nep_server_destroy": (c_int32, [c_void_p]),
    "nep_plan_bytes": (ctypes.c_uint64, [c_void_p, c_int32, c_int32, c_int32, c_int32]),
    "nep_plan_create": (c_int32, [c_void_p, ctypes.POINTER(NepRegion), c_int32, c_int32, c_int32, ctypes.POINTER(NepOpts),
                                  ctypes.POINTER(c_void_p)]),
    "nep_plan_execute": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "nep_autotune": (c_int32, [c_void_p, ctypes.POINTER(NepRegion), c_int32, c_int32, c_int32, ctypes.POINTER(NepOpts),
                               c_void_p, ctypes.c_char_p, ctypes.POINTER(NepTuneResult), c_void_p]),
    "nep_tune_load": (c_int32, [ctypes.c_char_p, ctypes.POINTER(c_int32)]),
    "nep_plan_execute_batch": (c_int32, [c_int32, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_void_p]),
    "nep_plan_result": (c_int32, [c_void_p, ctypes.POINTER(c_void_p)]),
    "nep_plan_destroy": (c_int32, [c_void_p]),
    "nep_plan_buffer": (c_int32, [c_void_p, ctypes.c_char_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_size_t)]),
    "nep_nodes": (c_int32, [ctypes.POINTER(NepRegion), c_int32, c_void_p, c_void_p, c_void_p]),
    "nep_coefficients": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "nep_result_points": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(ctypes.POINTER(c_int32)),
                                    ctypes.POINTER(ctypes.POINTER(c_int32)), ctypes.POINTER(P_double)]),
    "nep_assemble_band": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "nep_band_factor": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nep_band_solve": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "nep_band_transpose_u": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p]),
    "nep_band_solve_cols": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                      c_void_p]),
    "nep_split_residual": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nep_moments": (c_int32, [c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nep_jacobi_svd": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nep_jacobi_svd_noalloc": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nep_small_eig": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "nep_rii": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_double, c_int32,
                          ctypes.POINTER(c_int32), c_void_p]),
    "nep_plan_polish": (c_int32, [c_void_p, ctypes.c_double, c_int32, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                  c_void_p]),
    "nep_band_solve_adjoint": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_int32, c_void_p,
                                         c_void_p]),
    "nep_left_eigvecs": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   ctypes.c_double, c_int32, ctypes.POINTER(c_int32), c_void_p]),
    "nep_plan_left": (c_int32, [c_void_p, ctypes.c_double, c_int32, c_int32, c_void_p, c_void_p,
                                ctypes.POINTER(c_int32), ctypes.POINTER(c_int32), c_void_p]),
    "nep_nleigs_interpolation": (c_int32, [c_void_p, ctypes.POINTER(NepRegion), ctypes.POINTER(NepNleigsOpts), c_int32,
                                           c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_int32),
                                           ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "nep_nleigs_interpolation_fns": (c_int32, [c_int32, c_void_p, ctypes.POINTER(NepRegion),
                                               ctypes.POINTER(NepNleigsOpts), c_int32, c_void_p, c_void_p, c_void_p,
                                               c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                               ctypes.POINTER(c_int32)]),
    "nep_nleigs_solve": (c_int32, [c_void_p, ctypes.POINTER(NepRegion), ctypes.POINTER(NepNleigsOpts),
                                   ctypes.POINTER(c_void_p), ctypes.POINTER(c_int32), c_void_p]),
    "nep_interpol_coefficients": (c_int32, [c_int32, ctypes.POINTER(NepFn), ctypes.POINTER(NepRegion), c_int32,
                                            c_void_p]),
    "nep_interpol_solve": (c_int32, [c_void_p, ctypes.POINTER(NepRegion), ctypes.POINTER(NepInterpolOpts),
                                     ctypes.POINTER(c_void_p), c_void_p]),
    "nep_apply_resolvent": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_int32,
                                      c_void_p, c_void_p, c_void_p]),
}

_lib = None


class NepError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nep error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libnepciss.so (building it first when asked). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with paper_1910_11712_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fnc = getattr(lib, name)
        fnc.restype = res
        fnc.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != NEP_OK:
        raise NepError(rc, load().nep_last_error().decode())
    return rc


def ptr(x) -> int:
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


# ------------------------------------------------------------------ marshalling helpers
class _Keep:
    """Keeps numpy buffers referenced while a C call reads them."""

    def __init__(self):
        self.refs = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(a)
        return a


def _cplx_array(keep, vals):
    a = keep.arr(np.array([complex(v) for v in vals], dtype=np.complex128).view(np.float64), np.float64)
    return a.ctypes.data_as(P_double)


def _fn_struct(keep, spec) -> NepFn:
    f = NepFn()
    f.kind = FN_KIND[spec["kind"]]
    al, be = complex(spec.get("alpha", 1.0)), complex(spec.get("beta", 1.0))
    sh = complex(spec.get("shift", 0.0))
    f.alpha_re, f.alpha_im, f.beta_re, f.beta_im = al.real, al.imag, be.real, be.imag
    f.shift_re, f.shift_im = sh.real, sh.imag
    if spec["kind"] == "rational":
        f.nnum = len(spec["num"])
        f.num = _cplx_array(keep, spec["num"])
        den = spec.get("den")
        f.nden = 0 if den is None else len(den)
        f.den = _cplx_array(keep, den) if den is not None else P_double()
    if spec.get("fn") is not None:
        # host function: fn(z) -> (f, df) for a complex array z (the library calls it on the host only)
        fn = spec["fn"]

        def trampoline(zp, count, fp, dfp, ctx, fn=fn):
            z = np.ctypeslib.as_array(zp, (2 * count,)).view(np.complex128)
            fv, dfv = fn(z.copy())
            np.ctypeslib.as_array(fp, (2 * count,))[:] = np.asarray(fv, np.complex128).view(np.float64)
            if dfp:
                np.ctypeslib.as_array(dfp, (2 * count,))[:] = np.asarray(dfv, np.complex128).view(np.float64)
        cb = NEP_FN_EVAL(trampoline)
        keep.refs.append(cb)
        f.eval = cb
    if spec["kind"] == "table":
        vals = np.ascontiguousarray(spec["values"], dtype=np.complex128)
        f.table = _cplx_array(keep, list(vals))
        f.table_count = len(vals)
    if spec["kind"] == "combine":
        f.op = FN_OP[spec["op"]]
        fa, fb = _fn_struct(keep, spec["a"]), _fn_struct(keep, spec["b"])
        keep.refs += [fa, fb]
        f.a = ctypes.pointer(fa)
        f.b = ctypes.pointer(fb)
    return f


def region_struct(region) -> NepRegion:
    c = complex(region["center"])
    return NepRegion(c.real, c.imag, float(region["a"]), float(region["b"]))


def opts_struct(**kw) -> NepOpts:
    o = NepOpts()
    load().nep_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


class Split:
    """Split operator T(z) = sum_i A_i f_i(z) on the device (nep_create_split)."""

    def __init__(self, mats, fns):
        import scipy.sparse as sp
        lib = load()
        keep = _Keep()
        n = mats[0].shape[0]
        csrs = (NepCsr * len(mats))()
        for i, A in enumerate(mats):
            A = sp.csr_matrix(A)
            A.sort_indices()
            rp = keep.arr(A.indptr, np.int64)
            ci = keep.arr(A.indices, np.int32)
            re = keep.arr(np.real(A.data), np.float64)
            csrs[i].n_rows, csrs[i].n_cols = A.shape
            csrs[i].rowptr = rp.ctypes.data_as(ctypes.POINTER(c_int64))
            csrs[i].col = ci.ctypes.data_as(ctypes.POINTER(c_int32))
            csrs[i].val_re = re.ctypes.data_as(P_double)
            if np.iscomplexobj(A.data) and np.any(np.imag(A.data) != 0):
                im = keep.arr(np.imag(A.data), np.float64)
                csrs[i].val_im = im.ctypes.data_as(P_double)
        fs = (NepFn * len(fns))()
        for i, spec in enumerate(fns):
            fs[i] = _fn_struct(keep, spec)
        h = c_void_p()
        check(lib.nep_create_split(n, len(mats), csrs, fs, ctypes.byref(h)))
        self.handle = h
        self._keep = keep  # host callbacks must outlive the split
        self.n = n
        self.nterms = len(mats)
        info = [c_int32() for _ in range(5)]
        check(lib.nep_split_info(h, *[ctypes.byref(x) for x in info]))
        _, _, self.kl, self.ku, self.ldab = (x.value for x in info)

    @classmethod
    def from_problem(cls, problem):
        return cls(problem.mats, problem.fns)

    def close(self):
        if self.handle:
            load().nep_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _result_dict(res) -> dict:
    lib = load()
    nconv, m, flags = c_int32(), c_int32(), c_int32()
    lam_p, X_p, eta_p = P_double(), P_double(), P_double()
    check(lib.nep_result_get(res, ctypes.byref(nconv), ctypes.byref(lam_p), ctypes.byref(X_p), ctypes.byref(eta_p),
                             ctypes.byref(m), ctypes.byref(flags)))
    info = NepResultInfo()
    check(lib.nep_result_info(res, ctypes.byref(info)))
    k = nconv.value
    n = info.n
    lam = np.ctypeslib.as_array(lam_p, (2 * k,)).copy().view(np.complex128) if k else np.zeros(0, np.complex128)
    X = (np.ctypeslib.as_array(X_p, (2 * n * k,)).copy().view(np.complex128).reshape(k, n).T
         if k else np.zeros((n, 0), np.complex128))
    eta = np.ctypeslib.as_array(eta_p, (k,)).copy() if k else np.zeros(0)
    sp_, cnt = P_double(), c_int32()
    check(lib.nep_result_hankel_sigma(res, ctypes.byref(sp_), ctypes.byref(cnt)))
    sigma = np.ctypeslib.as_array(sp_, (cnt.value,)).copy() if cnt.value else np.zeros(0)
    npts, sw_p, li_p, be_p = c_int32(), ctypes.POINTER(c_int32)(), ctypes.POINTER(c_int32)(), P_double()
    check(lib.nep_result_points(res, ctypes.byref(npts), ctypes.byref(sw_p), ctypes.byref(li_p), ctypes.byref(be_p)))
    q = npts.value
    points = {"sweeps": np.ctypeslib.as_array(sw_p, (q,)).copy() if q else np.zeros(0, np.int32),
              "lu_info": np.ctypeslib.as_array(li_p, (q,)).copy() if q else np.zeros(0, np.int32),
              "backward": np.ctypeslib.as_array(be_p, (q,)).copy() if q else np.zeros(0)}
    out = {"lam": lam, "X": np.asfortranarray(X), "eta": eta, "m": m.value, "flags": flags.value, "sigma": sigma,
           "info": {f: getattr(info, f) for f, _ in NepResultInfo._fields_}, "points": points}
    lib.nep_result_free(res)
    return out


def ciss_solve(split: Split, region, N, L, M, V=None, **opts) -> dict:
    """nep_ciss_solve with host buffers: V (n x L complex128) or None (seeded draw)."""
    lib = load()
    r = region_struct(region)
    o = opts_struct(**opts)
    vptr = None
    if V is not None:
        Vf = np.asfortranarray(V, dtype=np.complex128)
        vptr = Vf.ctypes.data
    res = c_void_p()
    check(lib.nep_ciss_solve(split.handle, ctypes.byref(r), N, L, M, ctypes.byref(o), vptr, ctypes.byref(res)))
    return _result_dict(res)


class Plan:
    """Device-resident solve (nep_plan_*): allocate once, execute many times."""

    def __init__(self, split: Split, region, N, L, M, **opts):
        lib = load()
        self.split = split
        r = region_struct(region)
        o = opts_struct(**opts)
        h = c_void_p()
        check(lib.nep_plan_create(split.handle, ctypes.byref(r), N, L, M, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    def execute(self, V_dev, stream=0):
        check(load().nep_plan_execute(self.handle, ptr(V_dev), stream))

    def result(self) -> dict:
        res = c_void_p()
        check(load().nep_plan_result(self.handle, ctypes.byref(res)))
        return _result_dict(res)

    def polish(self, tol=1e-10, max_it=10, stream=0):
        """nep_plan_polish: residual inverse iteration on the returned pairs with eta >= tol.
        Returns (pairs polished, iterations run)."""
        done, its = c_int32(), c_int32()
        check(load().nep_plan_polish(self.handle, tol, max_it, ctypes.byref(done), ctypes.byref(its), stream))
        return done.value, its.value

    def left(self, Y_dev, eta_dev, capacity, tol=1e-13, max_it=6, stream=0):
        """nep_plan_left: Keldysh-normalised left eigenvectors of the returned pairs into Y_dev
        (n x capacity complex128). Returns (pairs, steps run)."""
        nc, its = c_int32(), c_int32()
        check(load().nep_plan_left(self.handle, tol, max_it, capacity, ptr(Y_dev), ptr(eta_dev), ctypes.byref(nc),
                                   ctypes.byref(its), stream))
        return nc.value, its.value

    def buffer(self, name: str):
        p, b = c_void_p(), c_size_t()
        check(load().nep_plan_buffer(self.handle, name.encode(), ctypes.byref(p), ctypes.byref(b)))
        return p.value, b.value

    def close(self):
        if self.handle:
            load().nep_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (nep_server_*): submit, poll or wait."""

    def __init__(self, workers: int = 4, hbm_budget_bytes: int = 0, max_batch: int = 1):
        h = c_void_p()
        if max_batch > 1:
            check(load().nep_server_create_batched(workers, max_batch, hbm_budget_bytes, ctypes.byref(h)))
        else:
            check(load().nep_server_create(workers, hbm_budget_bytes, ctypes.byref(h)))
        self.handle = h

    def submit(self, split: Split, region, N, L, M, V=None, **opts) -> int:
        r = region_struct(region)
        o = opts_struct(**opts)
        vptr = None
        if V is not None:
            Vf = np.asfortranarray(V, dtype=np.complex128)
            vptr = Vf.ctypes.data
        t = ctypes.c_uint64()
        check(load().nep_submit(self.handle, split.handle, ctypes.byref(r), N, L, M, ctypes.byref(o), vptr,
                                ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        res = c_void_p()
        rc = load().nep_poll(self.handle, ticket, ctypes.byref(res))
        if rc == NEP_PENDING:
            return None
        check(rc)
        return _result_dict(res)

    def wait(self, ticket: int) -> dict:
        res = c_void_p()
        check(load().nep_server_wait(self.handle, ticket, ctypes.byref(res)))
        return _result_dict(res)

    def close(self):
        if self.handle:
            load().nep_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_bytes(split: Split, N, L, M, precision=NEP_PREC_MIXED) -> int:
    return int(load().nep_plan_bytes(split.handle, N, L, M, precision))


# ------------------------------------------------------------------ step entry points
def nodes(region, N):
    z, w, zeta = (np.zeros(N, np.complex128) for _ in range(3))
    r = region_struct(region)
    check(load().nep_nodes(ctypes.byref(r), N, z.ctypes.data, w.ctypes.data, zeta.ctypes.data))
    return z, w, zeta


def coefficients(split: Split, z):
    z = np.ascontiguousarray(z, dtype=np.complex128)
    F = np.zeros((len(z), split.nterms), np.complex128)
    dF = np.zeros_like(F)
    check(load().nep_coefficients(split.handle, len(z), z.ctypes.data, F.ctypes.data, dF.ctypes.data))
    return F.T.copy(), dF.T.copy()


def assemble_band(split, npts, F_dev, precision, ab_dev, tnorm_dev=None, stream=0):
    check(load().nep_assemble_band(split.handle, npts, ptr(F_dev), precision, ptr(ab_dev), ptr(tnorm_dev), stream))


def band_factor(split, npts, precision, ab_dev, ipiv_dev, info_dev, stream=0):
    check(load().nep_band_factor(split.handle, npts, precision, ptr(ab_dev), ptr(ipiv_dev), ptr(info_dev), stream))


def band_solve(split, npts, precision, ab_dev, ipiv_dev, L, B_dev, stream=0):
    check(load().nep_band_solve(split.handle, npts, precision, ptr(ab_dev), ptr(ipiv_dev), L, ptr(B_dev), stream))


def band_transpose_u(split, npts, precision, ab_dev, ut_dev, stream=0):
    check(load().nep_band_transpose_u(split.handle, npts, precision, ptr(ab_dev), ptr(ut_dev), stream))


def band_solve_cols(split, npts, precision, ab_dev, ut_dev, ipiv_dev, L, B_dev, stream=0):
    check(load().nep_band_solve_cols(split.handle, npts, precision, ptr(ab_dev), ptr(ut_dev), ptr(ipiv_dev), L,
                                     ptr(B_dev), stream))


def split_residual(split, npts, F_dev, L, V_dev, Y_dev, R_dev, stream=0):
    check(load().nep_split_residual(split.handle, npts, ptr(F_dev), L, ptr(V_dev), ptr(Y_dev), ptr(R_dev), stream))


def moments(n, L, N, K, coef_dev, Y_dev, S_dev, stream=0):
    check(load().nep_moments(n, L, N, K, ptr(coef_dev), ptr(Y_dev), ptr(S_dev), stream))


def jacobi_svd(rows, cols, A_dev, W_dev, sigma_dev, stream=0):
    check(load().nep_jacobi_svd(rows, cols, ptr(A_dev), ptr(W_dev), ptr(sigma_dev), stream))


def jacobi_svd_noalloc(rows, cols, A_dev, W_dev, sigma_dev, stream=0):
    """nep_jacobi_svd without device allocations (fixed scratch compiled into the library)."""
    check(load().nep_jacobi_svd_noalloc(rows, cols, ptr(A_dev), ptr(W_dev), ptr(sigma_dev), stream))


def rii(split, precision, P, lam_dev, X_dev, eta_dev, its_dev=None, tol=1e-10, max_it=10, stream=0):
    """nep_rii: residual inverse iteration from P (lambda, x) estimates on the device, in place.
    Returns the number of iterations run."""
    its = c_int32()
    check(load().nep_rii(split.handle, precision, P, ptr(lam_dev), ptr(X_dev), ptr(eta_dev), ptr(its_dev), tol,
                         max_it, ctypes.byref(its), stream))
    return its.value


def band_solve_adjoint(split, npts, precision, ab_dev, ipiv_dev, L, B_dev, stream=0):
    check(load().nep_band_solve_adjoint(split.handle, npts, precision, ptr(ab_dev), ptr(ipiv_dev), L, ptr(B_dev),
                                        stream))


def left_eigvecs(split, precision, P, lam_dev, X_dev, Y_dev, eta_dev, its_dev=None, tol=1e-13, max_it=6, stream=0):
    """nep_left_eigvecs: Keldysh-normalised left eigenvectors of P pairs. Returns the steps run."""
    its = c_int32()
    check(load().nep_left_eigvecs(split.handle, precision, P, ptr(lam_dev), ptr(X_dev), ptr(Y_dev), ptr(eta_dev),
                                  ptr(its_dev), tol, max_it, ctypes.byref(its), stream))
    return its.value


def apply_resolvent(n, P, lam_dev, X_dev, Y_dev, nz, z_dev, nv, V_dev, out_dev, stream=0):
    """nep_apply_resolvent: out[:, j*nv + k] = sum_i x_i (y_i^* v_k) / (z_j - lambda_i)."""
    check(load().nep_apply_resolvent(n, P, ptr(lam_dev), ptr(X_dev), ptr(Y_dev), nz, ptr(z_dev), nv, ptr(V_dev),
                                     ptr(out_dev), stream))


def nleigs_opts(tol=0.0, max_degree=0, nboundary=0, krylov=0, shift=None, seed=0, eig_tol=0.0,
                exact_solves=0, full_basis=0, max_restarts=0, keep=0, restart_tol=0.0, nev=0) -> NepNleigsOpts:
    o = NepNleigsOpts()
    o.tol, o.max_degree, o.nboundary, o.krylov, o.seed, o.eig_tol = tol, max_degree, nboundary, krylov, seed, eig_tol
    o.exact_solves, o.full_basis = exact_solves, full_basis
    o.max_restarts, o.keep, o.restart_tol, o.nev = max_restarts, keep, restart_tol, nev
    if shift is not None:
        o.has_shift, o.shift_re, o.shift_im = 1, complex(shift).real, complex(shift).imag
    return o


def _interp_call(call, nterms, region, opts) -> dict:
    r, o = region_struct(region), nleigs_opts(**opts)
    d, conv, ns = c_int32(), c_int32(), c_int32()
    check(call(ctypes.byref(r), ctypes.byref(o), 0, None, None, None, None, ctypes.byref(d), ctypes.byref(conv),
               ctypes.byref(ns)))
    cap = d.value + 1
    sig = np.zeros(cap, np.complex128)
    xi = np.zeros(cap, np.complex128)
    beta = np.zeros(cap)
    dd = np.zeros(nterms * cap, np.complex128)
    check(call(ctypes.byref(r), ctypes.byref(o), cap, sig.ctypes.data, xi.ctypes.data, beta.ctypes.data,
               dd.ctypes.data, ctypes.byref(d), ctypes.byref(conv), ctypes.byref(ns)))
    return {"d": d.value, "converged": bool(conv.value), "nsing": ns.value, "sigma": sig, "xi": xi, "beta": beta,
            "dd": dd.reshape(cap, nterms).T.copy()}


def nleigs_interpolation(split, region, **opts) -> dict:
    """nep_nleigs_interpolation: nodes, poles (inf for none), scalings, divided differences dd[i, j]."""
    lib = load()
    return _interp_call(lambda *a: lib.nep_nleigs_interpolation(split.handle, *a), split.nterms, region, opts)


def nleigs_interpolation_fns(fns, region, **opts) -> dict:
    """nep_nleigs_interpolation_fns: the same from the function descriptions alone (host only)."""
    lib = load()
    keep = _Keep()
    fs = (NepFn * len(fns))()
    for i, spec in enumerate(fns):
        fs[i] = _fn_struct(keep, spec)
    return _interp_call(lambda *a: lib.nep_nleigs_interpolation_fns(len(fns), fs, *a), len(fns), region, opts)


def nleigs_solve(split, region, stream=0, **opts) -> dict:
    """nep_nleigs_solve: the result dict of ciss_solve plus the interpolation degree."""
    lib = load()
    r, o = region_struct(region), nleigs_opts(**opts)
    res, d = c_void_p(), c_int32()
    check(lib.nep_nleigs_solve(split.handle, ctypes.byref(r), ctypes.byref(o), ctypes.byref(res), ctypes.byref(d),
                               stream))
    out = _result_dict(res)
    out["degree"] = d.value
    return out


def autotune(split, region, N, L, M, V_dev, cache_path=None, stream=0, **opts) -> dict:
    """nep_autotune: the fastest accurate (lu_kernel, solve_rh) for this shape, kept for later plans."""
    r, o, t = region_struct(region), opts_struct(**opts), NepTuneResult()
    cp = cache_path.encode() if cache_path else None
    check(load().nep_autotune(split.handle, ctypes.byref(r), N, L, M, ctypes.byref(o), ptr(V_dev), cp,
                              ctypes.byref(t), stream))
    return {f: getattr(t, f) for f, _ in NepTuneResult._fields_}


def tune_load(path) -> int:
    n = c_int32()
    check(load().nep_tune_load(path.encode(), ctypes.byref(n)))
    return n.value


def execute_batch(plans, V_devs, stream=0):
    """nep_plan_execute_batch: several plans' passes with the LU and the sweeps in shared launches."""
    k = len(plans)
    ph = (c_void_p * k)(*[pl.handle.value if isinstance(pl.handle, c_void_p) else pl.handle for pl in plans])
    vh = (c_void_p * k)(*[ptr(v) for v in V_devs])
    check(load().nep_plan_execute_batch(k, ph, vh, stream))


def interpol_coefficients(fns, region, degree) -> np.ndarray:
    """nep_interpol_coefficients (host only): c[i, k] = c_ik, the Chebyshev coefficients of each f_i."""
    lib = load()
    keep = _Keep()
    fs = (NepFn * len(fns))()
    for i, spec in enumerate(fns):
        fs[i] = _fn_struct(keep, spec)
    r = region_struct(region)
    out = np.zeros(len(fns) * (degree + 1), np.complex128)
    check(lib.nep_interpol_coefficients(len(fns), fs, ctypes.byref(r), degree, out.ctypes.data))
    return out.reshape(degree + 1, len(fns)).T.copy()


def interpol_solve(split, region, stream=0, **opts) -> dict:
    """nep_interpol_solve (Sec. 4.4): the result dict of ciss_solve."""
    lib = load()
    r = region_struct(region)
    o = NepInterpolOpts()
    for k, v in opts.items():
        setattr(o, k, v)
    res = c_void_p()
    check(lib.nep_interpol_solve(split.handle, ctypes.byref(r), ctypes.byref(o), ctypes.byref(res), stream))
    return _result_dict(res)


def kernel_launches() -> int:
    return int(load().nep_kernel_launches())


def small_eig(m, A_dev, eval_dev, evec_dev=None, stream=0):
    check(load().nep_small_eig(m, ptr(A_dev), ptr(eval_dev), ptr(evec_dev), stream))
