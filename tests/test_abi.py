"""C-ABI library: builds, loads without a GPU, and exports every function include/nep_ciss.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nep_ciss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(nep_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_1910_11712_gb300 import build
    return build.build()


def test_library_exports_all_declared_symbols(built):
    lib = ctypes.CDLL(built)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(built):
    from paper_1910_11712_gb300 import binding
    assert set(declared_functions()) == set(binding.SIGNATURES)


def test_struct_layouts_match_c(built, tmp_path):
    """sizeof of the ABI structs as compiled by the C compiler equals the ctypes mirrors."""
    import subprocess
    from paper_1910_11712_gb300 import binding
    c = tmp_path / "sz.c"
    c.write_text('#include <stdio.h>\n#include "nep_ciss.h"\nint main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu",'
                 'sizeof(nep_fn), sizeof(nep_opts), sizeof(nep_result_info_t), sizeof(nep_csr), sizeof(nep_region),'
                 'sizeof(nep_nleigs_opts), sizeof(nep_interpol_opts), sizeof(nep_tune_result));}')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    sizes = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert sizes == [ctypes.sizeof(binding.NepFn), ctypes.sizeof(binding.NepOpts),
                     ctypes.sizeof(binding.NepResultInfo), ctypes.sizeof(binding.NepCsr),
                     ctypes.sizeof(binding.NepRegion), ctypes.sizeof(binding.NepNleigsOpts),
                     ctypes.sizeof(binding.NepInterpolOpts), ctypes.sizeof(binding.NepTuneResult)]


def test_host_entry_points_without_gpu(built):
    """Host-only entry points (defaults, nodes, argument checks) work on a machine without a GPU."""
    import numpy as np
    from paper_1910_11712_gb300 import binding
    o = binding.opts_struct()
    assert o.precision == binding.NEP_PREC_MIXED and o.rank_tol == 1e-12 and o.refine_max == 10
    z, w, zeta = binding.nodes({"center": -1.0, "a": 2.0, "b": 2.0}, 16)
    assert np.allclose(np.abs(zeta), 1.0)
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.nep_create_split(0, 1, None, None, ctypes.byref(h)) == binding.NEP_ERR_ARG
    assert b"nep_create_split" in lib.nep_last_error()


def test_new_entry_points_refuse_bad_arguments_without_gpu(built):
    """Argument checks of the left-vector, resolvent and NLEIGS entry points run on the host."""
    from paper_1910_11712_gb300 import binding
    lib = binding.load()
    E = binding.NEP_ERR_ARG
    assert lib.nep_band_solve_adjoint(None, 1, 1, None, None, 1, None, None) == E
    assert lib.nep_left_eigvecs(None, 1, 1, None, None, None, None, None, 1e-13, 4, None, None) == E
    assert lib.nep_plan_left(None, 1e-13, 4, 0, None, None, None, None, None) == E
    assert lib.nep_apply_resolvent(0, 1, None, None, None, 1, None, 1, None, None, None) == E
    assert lib.nep_apply_resolvent(8, -1, None, None, None, 1, None, 1, None, None, None) == E
    region = binding.region_struct({"center": 0.0, "a": 1.0, "b": 1.0})
    assert lib.nep_nleigs_solve(None, ctypes.byref(region), None, None, None, None) == E
    assert lib.nep_nleigs_interpolation_fns(0, None, ctypes.byref(region), None, 0, None, None, None, None,
                                            None, None, None) == E
    # nothing to do is not an error: no pairs, no points
    assert lib.nep_apply_resolvent(8, 0, None, None, None, 0, None, 0, None, None, None) == binding.NEP_OK
    # pairs without their arrays are refused even with nothing to apply them to
    assert lib.nep_apply_resolvent(8, 3, None, None, None, 0, None, 0, None, None, None) == E


def test_host_function_terms_are_validated_without_gpu(built):
    """A callback term needs eval, a table term needs values, and neither may sit inside a combination:
    nep_create_split refuses these before touching a device."""
    import numpy as np
    from paper_1910_11712_gb300 import binding
    lib = binding.load()
    keep = binding._Keep()
    n = 4
    rp = keep.arr(np.arange(n + 1), np.int64)
    ci = keep.arr(np.arange(n), np.int32)
    va = keep.arr(np.ones(n), np.float64)
    csr = binding.NepCsr(n, n, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), va.ctypes.data_as(binding.P_double), None)
    h = ctypes.c_void_p()
    f = binding._fn_struct(keep, {"kind": "callback"})  # no eval
    assert lib.nep_create_split(n, 1, ctypes.byref(csr), ctypes.byref(f), ctypes.byref(h)) == binding.NEP_ERR_ARG
    f = binding._fn_struct(keep, {"kind": "table", "values": []})
    assert lib.nep_create_split(n, 1, ctypes.byref(csr), ctypes.byref(f), ctypes.byref(h)) == binding.NEP_ERR_ARG
    inner = {"kind": "callback", "fn": lambda z: (np.exp(-z), -np.exp(-z))}
    f = binding._fn_struct(keep, {"kind": "combine", "op": "add", "a": inner, "b": {"kind": "exp"}})
    assert lib.nep_create_split(n, 1, ctypes.byref(csr), ctypes.byref(f), ctypes.byref(h)) == binding.NEP_ERR_ARG
    assert b"top level" in lib.nep_last_error()


def test_tune_cache_loader_without_gpu(built, tmp_path):
    """nep_tune_load reads the autotuner's cache lines (later lines win, others ignored) on the host."""
    from paper_1910_11712_gb300 import binding
    f = tmp_path / "tune.txt"
    f.write_text("nep-tune n=4096 kl=64 ku=64 L=16 precision=1 lu_kernel=0 solve_rh=2 ms=22.5\n"
                 "a comment line\n"
                 "nep-tune n=16384 kl=128 ku=128 L=32 precision=1 lu_kernel=1 solve_rh=4 ms=151.0\n")
    assert binding.tune_load(str(f)) == 2
    with pytest.raises(binding.NepError):
        binding.tune_load(str(tmp_path / "missing.txt"))
