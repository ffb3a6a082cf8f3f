"""B300-native Chebyshev-collocation solver for stationary diffusion.

Python binding of ``libcheb_b300.so`` (the C ABI in ``include/cheb.h``).
PyTorch supplies device memory and streams only; every numerical step runs
in the library's CUDA kernels.  There is no CPU fallback: importing this
package fails when the library is missing.

``Plan`` wraps one grid.  Fields are CUDA tensors shaped ``(nz, ny, nx)``
(x fastest), float64 or float32; the tensor dtype selects the arithmetic.
"""
from __future__ import annotations

import ctypes as C
import ctypes as C_

import numpy as np
import torch

from ._lib import ChebError, SolveInfo, SolveOpts, check, lib  # noqa: F401

DIRICHLET, NEUMANN, FLUX = 0, 1, 2
FP64, FP32 = 0, 1
SOLVE_FP64, SOLVE_MIXED = 0, 1
ROUTE_AUTO, ROUTE_TRANSFORM, ROUTE_DENSE, ROUTE_TENSOR = -1, 0, 1, 2
PRECOND_NONE, PRECOND_FDM = 0, 2
FORM_REPLACE, FORM_ELIMINATE = 0, 1
BATCH_AUTO, BATCH_LOCKSTEP, BATCH_CONCURRENT = 0, 1, 2
PMAT_TF32, PMAT_FP32 = 0, 1


def solve_opts(**kw) -> SolveOpts:
    """``cheb_solve_opts`` with the library defaults, fields overridden by kw."""
    o = SolveOpts()
    lib.cheb_solve_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown solve option {k}")
        setattr(o, k, v)
    return o

_PREC = {torch.float64: FP64, torch.float32: FP32}


def _vp(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _stream_ptr() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Plan:
    """A CGL grid with per-face boundary types (``cheb_plan``)."""

    def __init__(self, n, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), bc=(0, 0, 0, 0, 0, 0)):
        n = [int(v) for v in n] + [1] * (3 - len(n))
        self.n = tuple(n)
        self.dim = sum(1 for v in n if v > 1)
        lo = list(lo) + [-1.0] * (3 - len(lo))
        hi = list(hi) + [1.0] * (3 - len(hi))
        self.lo, self.hi = tuple(float(v) for v in lo), tuple(float(v) for v in hi)
        self.bc = tuple(int(v) for v in bc)
        self.shape = (n[2], n[1], n[0])
        self._h = C.c_void_p()
        check(lib.cheb_plan_create(C.byref(self._h), self.dim, (C.c_int * 3)(*n),
                                   (C.c_double * 3)(*self.lo), (C.c_double * 3)(*self.hi),
                                   (C.c_int * 6)(*self.bc), None), "cheb_plan_create")

    # ---------------------------------------------------------------- basics
    @property
    def handle(self) -> C.c_void_p:
        return self._h

    @property
    def size(self) -> int:
        return int(np.prod(self.shape))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.cheb_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        check(lib.cheb_plan_set_stream(self._h, _stream_ptr()), "cheb_plan_set_stream")

    def nodes(self, axis: int) -> np.ndarray:
        out = np.zeros(self.n[axis], dtype=np.float64)
        check(lib.cheb_nodes(self._h, axis, out.ctypes.data_as(C.POINTER(C.c_double))), "cheb_nodes")
        return out

    def mesh(self):
        """Node coordinates (X, Y, Z), numpy arrays shaped (nz, ny, nx)."""
        Z, Y, X = np.meshgrid(self.nodes(2), self.nodes(1), self.nodes(0), indexing="ij")
        return X, Y, Z

    def set_route(self, axis: int, route: int):
        check(lib.cheb_plan_set_route(self._h, axis, route), "cheb_plan_set_route")

    def set_route32(self, axis: int, route: int):
        """FP32 route of one axis alone (ROUTE_TENSOR: the operator apply on
        the tensor cores)."""
        check(lib.cheb_plan_set_route32(self._h, axis, route), "cheb_plan_set_route32")

    def route32(self, axis: int) -> int:
        r = C.c_int()
        check(lib.cheb_plan_get_route32(self._h, axis, C.byref(r)), "cheb_plan_get_route32")
        return r.value

    def autotune(self, cache: str | None = None) -> dict:
        """Pick the faster line-derivative route per axis and precision
        (``cheb_autotune``); cache: optional decision file."""
        out = (C.c_int * 6)()
        self._sync_stream()
        check(lib.cheb_autotune(self._h, cache.encode() if cache else None, out), "cheb_autotune")
        names = {0: "transform", 1: "dense", 2: "tensor"}
        return {"fp64": [names[out[a]] for a in range(self.dim)],
                "fp32": [names[out[3 + a]] for a in range(self.dim)],
                "tile64": [self.tile(a, FP64) for a in range(self.dim)],
                "tile32": [self.tile(a, FP32) for a in range(self.dim)]}

    def set_tile(self, axis: int, prec: int, lines: int):
        """Lines per CTA (8 or 16) of the line passes of one axis (``cheb_plan_set_tile``)."""
        check(lib.cheb_plan_set_tile(self._h, axis, prec, lines), "cheb_plan_set_tile")

    def tile(self, axis: int, prec: int) -> int:
        r = C.c_int()
        check(lib.cheb_plan_get_tile(self._h, axis, prec, C.byref(r)), "cheb_plan_get_tile")
        return r.value

    def route(self, axis: int) -> int:
        r = C.c_int()
        check(lib.cheb_plan_get_route(self._h, axis, C.byref(r)), "cheb_plan_get_route")
        return r.value

    def _field(self, t: torch.Tensor, name: str, dtype=None) -> torch.Tensor:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if tuple(t.shape) != self.shape and t.numel() != self.size:
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {self.shape}")
        if dtype is not None and t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}")
        if t.dtype not in _PREC:
            raise TypeError(f"{name} must be float64 or float32")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _out(self, out, like: torch.Tensor) -> torch.Tensor:
        if out is None:
            return torch.empty(self.shape, dtype=like.dtype, device=like.device)
        return self._field(out, "out", like.dtype)

    # ---------------------------------------------------------------- ops
    def deriv(self, u: torch.Tensor, axis: int, out=None, transpose: bool = False) -> torch.Tensor:
        """d u / d t_axis (``cheb_deriv``) or D_axis^T u (``cheb_deriv_t``)."""
        u = self._field(u, "u")
        out = self._out(out, u)
        self._sync_stream()
        fn = lib.cheb_deriv_t if transpose else lib.cheb_deriv
        check(fn(self._h, _PREC[u.dtype], axis, _vp(u), _vp(out)), "cheb_deriv")
        return out

    def apply(self, K: torch.Tensor, u: torch.Tensor, out=None) -> torch.Tensor:
        """A u with boundary rows (``cheb_apply``)."""
        u = self._field(u, "u")
        K = self._field(K, "K", u.dtype)
        out = self._out(out, u)
        self._sync_stream()
        check(lib.cheb_apply(self._h, _PREC[u.dtype], _vp(K), _vp(u), _vp(out)), "cheb_apply")
        return out

    def adjoint_apply(self, K: torch.Tensor, lam: torch.Tensor, out=None) -> torch.Tensor:
        """A^T lam (``cheb_adjoint_apply``)."""
        lam = self._field(lam, "lam")
        K = self._field(K, "K", lam.dtype)
        out = self._out(out, lam)
        self._sync_stream()
        check(lib.cheb_adjoint_apply(self._h, _PREC[lam.dtype], _vp(K), _vp(lam), _vp(out)),
              "cheb_adjoint_apply")
        return out

    def rhs(self, f: torch.Tensor, faces, out=None) -> torch.Tensor:
        """b: f inside, owner-face data on boundary nodes (``cheb_rhs``), FP64."""
        f = self._field(f, "f", torch.float64)
        out = self._out(out, f)
        ptrs = (C.c_void_p * 6)()
        keep = []
        for i in range(6):
            if i < 2 * self.dim:
                t = faces[i]
                if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                        and t.is_contiguous()):
                    raise TypeError("face data must be contiguous float64 CUDA tensors")
                keep.append(t)
                ptrs[i] = t.data_ptr()
            else:
                ptrs[i] = None
        self._sync_stream()
        check(lib.cheb_rhs(self._h, _vp(f), ptrs, _vp(out)), "cheb_rhs")
        return out


    def solve(self, K: torch.Tensor, b: torch.Tensor, u: torch.Tensor | None = None,
              check_status: bool = True, **opts):
        """Solve A u = b (``cheb_solve``); u (FP64) holds the initial guess and
        receives the solution.  Returns (u, info dict)."""
        K = self._field(K, "K", torch.float64)
        b = self._field(b, "b", torch.float64)
        if u is None:
            u = torch.zeros(self.shape, dtype=torch.float64, device=b.device)
        u = self._field(u, "u", torch.float64)
        o = solve_opts(**opts)
        info = SolveInfo()
        self._sync_stream()
        st = lib.cheb_solve(self._h, _vp(K), _vp(b), _vp(u), C.byref(o), C.byref(info))
        check(st, "cheb_solve")
        d = info.as_dict()
        if check_status and st != 0:
            raise ChebError(st, "cheb_solve")
        return u, d

    def picard_solve(self, K0: torch.Tensor, b: torch.Tensor, u: torch.Tensor | None = None,
                     beta: float = 0.5, tol: float = 1e-9, maxit: int = 30, omega: float = 1.0,
                     check_status: bool = True, **opts):
        """Picard iteration for K = K0 (1 + beta |grad u|^2), relaxation omega
        (``cheb_picard_solve``).
        Returns (u, info, picard_iters, last relative change)."""
        K0 = self._field(K0, "K0", torch.float64)
        b = self._field(b, "b", torch.float64)
        if u is None:
            u = torch.zeros(self.shape, dtype=torch.float64, device=b.device)
        u = self._field(u, "u", torch.float64)
        o = solve_opts(**opts)
        info = SolveInfo()
        its, dlt = C.c_int(), C.c_double()
        self._sync_stream()
        st = lib.cheb_picard_solve(self._h, _vp(K0), _vp(b), _vp(u), float(beta), float(omega),
                                   float(tol), int(maxit), C.byref(o), C.byref(info), C.byref(its),
                                   C.byref(dlt))
        check(st, "cheb_picard_solve")
        if check_status and st != 0:
            raise ChebError(st, "cheb_picard_solve")
        return u, info.as_dict(), its.value, dlt.value

    def jacobian_apply(self, K: torch.Tensor, C, du: torch.Tensor, out=None) -> torch.Tensor:
        """J du of Newton's linearisation (``cheb_jacobian_apply``): K = k(u),
        C = [k'(u) d_a u for each axis]."""
        du = self._field(du, "du")
        K = self._field(K, "K", du.dtype)
        Cs = [self._field(c, "C", du.dtype) for c in C[: self.dim]]
        out = self._out(out, du)
        ptrs = (C_.c_void_p * 3)(*[c.data_ptr() for c in Cs] + [Cs[0].data_ptr()] * (3 - len(Cs)))
        self._sync_stream()
        check(lib.cheb_jacobian_apply(self._h, _PREC[du.dtype], _vp(K), ptrs, _vp(du), _vp(out)),
              "cheb_jacobian_apply")
        return out

    def newton_solve(self, K0: torch.Tensor, b: torch.Tensor, u: torch.Tensor | None = None,
                     alpha: float = 0.5, tol: float = 1e-12, maxit: int = 30, check_status: bool = True,
                     **opts):
        """Newton's method for k(u) = K0 / (1 + alpha u) (``cheb_newton_solve``).
        Returns (u, info, newton iterations, last relative step)."""
        K0 = self._field(K0, "K0", torch.float64)
        b = self._field(b, "b", torch.float64)
        if u is None:
            u = torch.zeros(self.shape, dtype=torch.float64, device=b.device)
        u = self._field(u, "u", torch.float64)
        o = solve_opts(**opts)
        info = SolveInfo()
        its, dlt = C.c_int(), C.c_double()
        self._sync_stream()
        st = lib.cheb_newton_solve(self._h, _vp(K0), float(alpha), _vp(b), _vp(u), float(tol), int(maxit),
                                   C.byref(o), C.byref(info), C.byref(its), C.byref(dlt))
        check(st, "cheb_newton_solve")
        if check_status and st != 0:
            raise ChebError(st, "cheb_newton_solve")
        return u, info.as_dict(), its.value, dlt.value

    def adjoint_solve(self, K: torch.Tensor, dJdu: torch.Tensor, u: torch.Tensor | None = None,
                      lam: torch.Tensor | None = None, dJdK: torch.Tensor | None = None,
                      check_status: bool = True, **opts):
        """lam = A^{-T} dJdu (``cheb_adjoint_solve``); when dJdK is given it is
        incremented by the K-gradient for the forward solution u.  Returns
        (lam, dJdK, info)."""
        K = self._field(K, "K", torch.float64)
        dJdu = self._field(dJdu, "dJdu", torch.float64)
        if lam is None:
            lam = torch.zeros(self.shape, dtype=torch.float64, device=K.device)
        lam = self._field(lam, "lam", torch.float64)
        up = None
        if dJdK is not None:
            dJdK = self._field(dJdK, "dJdK", torch.float64)
            u = self._field(u, "u", torch.float64)
            up = _vp(u)
        o = solve_opts(**opts)
        info = SolveInfo()
        self._sync_stream()
        st = lib.cheb_adjoint_solve(self._h, _vp(K), up, _vp(dJdu), C.byref(o), _vp(lam),
                                    _vp(dJdK) if dJdK is not None else None, C.byref(info))
        check(st, "cheb_adjoint_solve")
        if check_status and st != 0:
            raise ChebError(st, "cheb_adjoint_solve")
        return lam, dJdK, info.as_dict()

    def flux_average(self, K: torch.Tensor, u: torch.Tensor, axis: int = 0) -> float:
        """(1/|Omega|) int K d_axis u by Clenshaw-Curtis quadrature
        (``cheb_flux_average``); K_num = flux_average / G."""
        K = self._field(K, "K", torch.float64)
        u = self._field(u, "u", torch.float64)
        out = C.c_double()
        self._sync_stream()
        check(lib.cheb_flux_average(self._h, int(axis), _vp(K), _vp(u), C.byref(out)), "cheb_flux_average")
        return out.value

    def precond_apply_t(self, y: torch.Tensor, kref: float, out=None) -> torch.Tensor:
        """z = M^{-T} y (``cheb_precond_apply_t``)."""
        y = self._field(y, "y")
        out = self._out(out, y)
        self._sync_stream()
        check(lib.cheb_precond_apply_t(self._h, _PREC[y.dtype], float(kref), _vp(y), _vp(out)),
              "cheb_precond_apply_t")
        return out

    def precond_apply(self, r: torch.Tensor, kref: float, out=None, matrices: int = PMAT_FP32) -> torch.Tensor:
        """z = M^{-1} r for the fast-diagonalization preconditioner
        (``cheb_precond_apply_m``); matrices = PMAT_FP32 (eigenvector matrices
        to FP32 accuracy) or PMAT_TF32 (rounded to TF32, the FP32 inner
        solves' default) for FP32 fields."""
        r = self._field(r, "r")
        out = self._out(out, r)
        self._sync_stream()
        check(lib.cheb_precond_apply_m(self._h, _PREC[r.dtype], int(matrices), float(kref), _vp(r), _vp(out)),
              "cheb_precond_apply_m")
        return out


def prolong(coarse: Plan, fine: Plan, u_c: torch.Tensor, out=None) -> torch.Tensor:
    """Modal prolongation of u_c onto the fine plan's grid (``cheb_prolong``)."""
    u_c = coarse._field(u_c, "u_c")
    out = fine._out(out, u_c)
    fine._sync_stream()
    check(lib.cheb_prolong(coarse.handle, fine.handle, _PREC[u_c.dtype], _vp(u_c), _vp(out)),
          "cheb_prolong")
    return out


def rel_diff(plan: Plan, a: torch.Tensor, b: torch.Tensor) -> float:
    """||a - b|| / ||a|| (``cheb_rel_diff``), FP64 fields."""
    a = plan._field(a, "a", torch.float64)
    b = plan._field(b, "b", torch.float64)
    out = C.c_double()
    plan._sync_stream()
    check(lib.cheb_rel_diff(plan.handle, _vp(a), _vp(b), C.byref(out)), "cheb_rel_diff")
    return out.value


def solve_hierarchy(plans, K, b, u0=None, check_status: bool = True, **opts):
    """Hierarchical refinement (``cheb_solve_hierarchy``): plans of doubling N,
    per-level FP64 K and b.  Returns (list of per-level solutions, infos, e_ref)."""
    L = len(plans)
    us = [torch.zeros(p.shape, dtype=torch.float64, device="cuda") for p in plans]
    if u0 is not None:
        us[0].copy_(u0)
    for i, p in enumerate(plans):
        p._field(K[i], "K", torch.float64)
        p._field(b[i], "b", torch.float64)
        p._sync_stream()
    hp = (C.c_void_p * L)(*[p.handle.value for p in plans])
    Kp = (C.c_void_p * L)(*[t.data_ptr() for t in K])
    bp = (C.c_void_p * L)(*[t.data_ptr() for t in b])
    up = (C.c_void_p * L)(*[t.data_ptr() for t in us])
    infos = (SolveInfo * L)()
    eref = (C.c_double * L)()
    o = solve_opts(**opts)
    st = lib.cheb_solve_hierarchy(L, hp, Kp, bp, up, C.byref(o), infos, eref)
    check(st, "cheb_solve_hierarchy")
    if check_status and st != 0:
        raise ChebError(st, "cheb_solve_hierarchy")
    return us, [i.as_dict() for i in infos], list(eref)


def solve_hierarchy_fine(plans, K, b, u=None, check_status: bool = True, **opts):
    """Hierarchical refinement from the finest level's K and b alone
    (``cheb_solve_hierarchy_fine``: coarse levels recomputed by injection).
    Returns (fine solution, infos, e_ref)."""
    L = len(plans)
    pf = plans[-1]
    K = pf._field(K, "K", torch.float64)
    b = pf._field(b, "b", torch.float64)
    if u is None:
        u = torch.zeros(pf.shape, dtype=torch.float64, device="cuda")
    u = pf._field(u, "u", torch.float64)
    for p in plans:
        p._sync_stream()
    hp = (C.c_void_p * L)(*[p.handle.value for p in plans])
    infos = (SolveInfo * L)()
    eref = (C.c_double * L)()
    st = lib.cheb_solve_hierarchy_fine(L, hp, _vp(K), _vp(b), _vp(u), C.byref(solve_opts(**opts)), infos, eref)
    check(st, "cheb_solve_hierarchy_fine")
    if check_status and st != 0:
        raise ChebError(st, "cheb_solve_hierarchy_fine")
    return u, [i.as_dict() for i in infos], list(eref)


def _batch_args(plans, A, b, u):
    L = len(plans)
    for i, p in enumerate(plans):
        p._field(A[i], "K", torch.float64)
        p._field(b[i], "b", torch.float64)
    if u is None:
        u = [torch.zeros(p.shape, dtype=torch.float64, device="cuda") for p in plans]
    hp = (C.c_void_p * L)(*[p.handle.value for p in plans])
    Ap = (C.c_void_p * L)(*[t.data_ptr() for t in A])
    bp = (C.c_void_p * L)(*[t.data_ptr() for t in b])
    up = (C.c_void_p * L)(*[t.data_ptr() for t in u])
    return L, hp, Ap, bp, up, u


def solve_batched(plans, K, b, u=None, check_status: bool = True, **opts):
    """Independent solves of a batch (``cheb_solve_batched``; ``batch_mode``
    = BATCH_AUTO / BATCH_LOCKSTEP / BATCH_CONCURRENT).  Returns (solutions, infos)."""
    torch.cuda.synchronize()
    L, hp, Kp, bp, up, u = _batch_args(plans, K, b, u)
    infos = (SolveInfo * L)()
    st = lib.cheb_solve_batched(L, hp, Kp, bp, up, C.byref(solve_opts(**opts)), infos)
    check(st, "cheb_solve_batched")
    if check_status and st != 0:
        raise ChebError(st, "cheb_solve_batched")
    return u, [i.as_dict() for i in infos]


def picard_batched(plans, K0, b, u=None, beta: float = 0.5, tol: float = 1e-9, maxit: int = 30,
                   omega: float = 1.0, check_status: bool = True, **opts):
    """Independent Picard solves of a batch (``cheb_picard_batched``, same
    ``batch_mode`` choice).  Returns (solutions, infos, picard iteration counts)."""
    torch.cuda.synchronize()
    L, hp, Kp, bp, up, u = _batch_args(plans, K0, b, u)
    infos = (SolveInfo * L)()
    its = (C.c_int * L)()
    st = lib.cheb_picard_batched(L, hp, Kp, bp, up, float(beta), float(omega), float(tol), int(maxit),
                                 C.byref(solve_opts(**opts)), infos, its)
    check(st, "cheb_picard_batched")
    if check_status and st != 0:
        raise ChebError(st, "cheb_picard_batched")
    return u, [i.as_dict() for i in infos], list(its)


# thin same-name wrappers of the C entry points -------------------------------

def cheb_apply(plan: Plan, K, u, Au):
    return plan.apply(K, u, Au)


def cheb_adjoint_apply(plan: Plan, K, lam, out):
    return plan.adjoint_apply(K, lam, out)


def cheb_deriv(plan: Plan, axis: int, u, du):
    return plan.deriv(u, axis, du)


def cheb_rhs(plan: Plan, f, faces, b):
    return plan.rhs(f, faces, b)


def cheb_solve(plan: Plan, K, b, u, **opts):
    return plan.solve(K, b, u, **opts)


def cheb_prolong(coarse: Plan, fine: Plan, u_c, u_f):
    return prolong(coarse, fine, u_c, u_f)
