"""ctypes loader of the in-tree ``libcheb_b300.so`` and its C signatures.

There is no fallback: importing this module fails loudly when the library
is missing (build it with ``python -m paper_2606_21410_b300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcheb_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} not found: the CUDA library is required (no CPU fallback); "
        "build it with `python -m paper_2606_21410_b300.build`")

lib = C.CDLL(LIB_PATH)

vp = C.c_void_p
i32 = C.c_int
f64p = C.POINTER(C.c_double)
i32p = C.POINTER(C.c_int)


class SolveOpts(C.Structure):
    """Mirror of ``cheb_solve_opts`` (include/cheb.h)."""
    _fields_ = [
        ("mode", i32),
        ("rtol", C.c_double),
        ("atol", C.c_double),
        ("restart", i32),
        ("augment", i32),
        ("maxiter", i32),
        ("inner_rtol", C.c_double),
        ("inner_maxiter", i32),
        ("max_refinements", i32),
        ("reorth", i32),
        ("precond", i32),
        ("kref", C.c_double),
        ("verbose", i32),
        ("use_graph", i32),
        ("recycle", i32),
        ("formulation", i32),
        ("coarse_rtol", C.c_double),
        ("batch_mode", C.c_int),
        ("precond_matrices", i32),
    ]


class SolveInfo(C.Structure):
    """Mirror of ``cheb_solve_info``."""
    _fields_ = [
        ("status", i32),
        ("iterations", i32),
        ("cycles", i32),
        ("refinements", i32),
        ("applies_fp64", i32),
        ("applies_fp32", i32),
        ("rel_residual", C.c_double),
        ("rel_residual_inner", C.c_double),
        ("seconds", C.c_double),
        ("kref", C.c_double),
        ("graph_captures", i32),
        ("host_syncs", i32),
        ("discarded_steps", i32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS = {
    "cheb_plan_create": (i32, [C.POINTER(vp), i32, i32p, f64p, f64p, i32p, vp]),
    "cheb_plan_destroy": (i32, [vp]),
    "cheb_plan_set_stream": (i32, [vp, vp]),
    "cheb_plan_set_route": (i32, [vp, i32, i32]),
    "cheb_plan_get_route": (i32, [vp, i32, i32p]),
    "cheb_plan_set_route32": (i32, [vp, i32, i32]),
    "cheb_plan_get_route32": (i32, [vp, i32, i32p]),
    "cheb_plan_set_tile": (i32, [vp, i32, i32, i32]),
    "cheb_plan_get_tile": (i32, [vp, i32, i32, i32p]),
    "cheb_nodes": (i32, [vp, i32, f64p]),
    "cheb_autotune": (i32, [vp, C.c_char_p, i32p]),
    "cheb_plan_size": (C.c_size_t, [vp]),
    "cheb_deriv": (i32, [vp, i32, i32, vp, vp]),
    "cheb_deriv_t": (i32, [vp, i32, i32, vp, vp]),
    "cheb_apply": (i32, [vp, i32, vp, vp, vp]),
    "cheb_adjoint_apply": (i32, [vp, i32, vp, vp, vp]),
    "cheb_rhs": (i32, [vp, vp, C.POINTER(vp), vp]),
    "cheb_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
    "cheb_solve": (i32, [vp, vp, vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "cheb_precond_apply": (i32, [vp, i32, C.c_double, vp, vp]),
    "cheb_precond_apply_m": (i32, [vp, i32, i32, C.c_double, vp, vp]),
    "cheb_picard_solve": (i32, [vp, vp, vp, vp, C.c_double, C.c_double, C.c_double, i32,
                                C.POINTER(SolveOpts), C.POINTER(SolveInfo), i32p, f64p]),
    "cheb_solve_batched": (i32, [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                 C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "cheb_picard_batched": (i32, [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                  C.c_double, C.c_double, C.c_double, i32, C.POINTER(SolveOpts),
                                  C.POINTER(SolveInfo), i32p]),
    "cheb_precond_apply_t": (i32, [vp, i32, C.c_double, vp, vp]),
    "cheb_adjoint_solve": (i32, [vp, vp, vp, vp, C.POINTER(SolveOpts), vp, vp, C.POINTER(SolveInfo)]),
    "cheb_prolong": (i32, [vp, vp, i32, vp, vp]),
    "cheb_prolong_noalloc": (i32, [vp, vp, i32, vp, vp]),
    "cheb_rel_diff": (i32, [vp, vp, vp, f64p]),
    "cheb_solve_hierarchy": (i32, [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                   C.POINTER(SolveOpts), C.POINTER(SolveInfo), f64p]),
    "cheb_flux_average": (i32, [vp, i32, vp, vp, f64p]),
    "cheb_jacobian_apply": (i32, [vp, i32, vp, C.POINTER(vp), vp, vp]),
    "cheb_newton_solve": (i32, [vp, vp, C.c_double, vp, vp, C.c_double, i32, C.POINTER(SolveOpts),
                                C.POINTER(SolveInfo), i32p, f64p]),
    "cheb_solve_hierarchy_fine": (i32, [i32, C.POINTER(vp), vp, vp, vp, C.POINTER(SolveOpts),
                                        C.POINTER(SolveInfo), f64p]),
    "cheb_selftest_bounded_wait": (i32, [C.c_longlong]),
    "cheb_launch_count": (C.c_longlong, []),
    "cheb_fma_peak": (i32, [i32, f64p, f64p]),
    "cheb_profile_enable": (i32, [i32]),
    "cheb_profile_read": (i32, [f64p, C.POINTER(C.c_longlong)]),
    "cheb_status_str": (C.c_char_p, [i32]),
    "cheb_last_error": (C.c_char_p, []),
}

OPTIONAL = {}


def _bind():
    missing = []
    for name, (res, args) in {**_SIGS, **OPTIONAL}.items():
        fn = getattr(lib, name, None)
        if fn is None:
            if name in _SIGS:
                missing.append(name)
            continue
        fn.restype = res
        fn.argtypes = args
    if missing:
        raise ImportError(f"{LIB_PATH} lacks symbols {missing}; rebuild it")


_bind()


class ChebError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.cheb_status_str(status).decode()
        detail = lib.cheb_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


def check(status: int, where: str) -> int:
    if status < 0:
        raise ChebError(status, where)
    return status
