"""The C-ABI library builds, loads without a GPU, exports every entry point
that include/*.h declares, and rejects bad arguments before touching CUDA.
CPU only."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(cheb_\w+)\s*\(", src))
    return names


def _build_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_cheb_build", os.path.join(ROOT, "paper_2606_21410_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_library_builds_and_exports_every_declared_symbol():
    path = _build_module().build()
    lib = C.CDLL(path)
    declared = _declared()
    assert len(declared) >= 10
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_without_gpu():
    import paper_2606_21410_b300 as P
    assert P.lib.cheb_status_str(0) == b"ok"
    assert b"singular" in P.lib.cheb_status_str(-5)


def test_plan_create_rejects_bad_arguments_without_cuda():
    import paper_2606_21410_b300 as P
    lib = P.lib
    h = C.c_void_p()
    n = (C.c_int * 3)(9, 9, 9)
    lo = (C.c_double * 3)(-1, -1, -1)
    hi = (C.c_double * 3)(1, 1, 1)
    bc = (C.c_int * 6)(0, 0, 0, 0, 0, 0)
    assert lib.cheb_plan_create(None, 3, n, lo, hi, bc, None) == -1
    assert lib.cheb_plan_create(C.byref(h), 4, n, lo, hi, bc, None) == -1
    assert lib.cheb_plan_create(C.byref(h), 3, (C.c_int * 3)(9, 2, 9), lo, hi, bc, None) == -1
    assert lib.cheb_plan_create(C.byref(h), 2, (C.c_int * 3)(9, 9, 9), lo, hi, bc, None) == -1
    assert lib.cheb_plan_create(C.byref(h), 3, n, lo, (C.c_double * 3)(1, -1, 1), bc, None) == -1
    assert lib.cheb_plan_create(C.byref(h), 3, n, lo, hi, (C.c_int * 6)(0, 0, 3, 0, 0, 0), None) == -1
    assert b"bc_type" in lib.cheb_last_error()
    assert lib.cheb_apply(None, 0, None, None, None) == -1
    assert lib.cheb_plan_destroy(None) == 0


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    """The binding has no CPU fallback: a missing library is an ImportError."""
    import importlib.util
    src = os.path.join(ROOT, "paper_2606_21410_b300", "_lib.py")
    spec = importlib.util.spec_from_file_location("_lib_probe", str(tmp_path / "_lib.py"))
    (tmp_path / "_lib.py").write_text(open(src).read())
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_solve_opts_mirror_matches_the_c_struct():
    """ctypes' SolveOpts has the size and field defaults of cheb_solve_opts:
    cheb_solve_opts_default clears sizeof(cheb_solve_opts) bytes and fills
    the defaults, so on a buffer larger than the mirror pre-filled with 0xAB
    it must touch exactly the mirror's bytes."""
    import paper_2606_21410_b300 as P
    size = C.sizeof(P.SolveOpts)
    buf = (C.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    P.lib.cheb_solve_opts_default(C.cast(buf, C.POINTER(P.SolveOpts)))
    raw = bytes(buf)
    assert raw[size:] == b"\xab" * 64
    assert raw[size - 8:size] != b"\xab" * 8
    o = P.solve_opts()
    assert (o.mode, o.rtol, o.restart, o.augment, o.inner_rtol) == (P.SOLVE_MIXED, 1e-12, 30, 3, 1e-4)
    assert (o.precond, o.batch_mode, o.precond_matrices) == (P.PRECOND_FDM, P.BATCH_AUTO, P.PMAT_TF32)


def test_precond_apply_m_rejects_bad_arguments_without_cuda():
    import paper_2606_21410_b300 as P
    lib = P.lib
    assert lib.cheb_precond_apply_m(None, 1, P.PMAT_TF32, 1.0, None, None) == -1
    assert lib.cheb_precond_apply(None, 1, 1.0, None, None) == -1
