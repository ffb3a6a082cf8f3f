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

import numpy as np
import torch

from ._lib import ChebError, SolveInfo, SolveOpts, check, lib  # noqa: F401

DIRICHLET, NEUMANN = 0, 1
FP64, FP32 = 0, 1
SOLVE_FP64, SOLVE_MIXED = 0, 1
ROUTE_AUTO, ROUTE_TRANSFORM, ROUTE_DENSE = -1, 0, 1

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


# thin same-name wrappers of the C entry points -------------------------------

def cheb_apply(plan: Plan, K, u, Au):
    return plan.apply(K, u, Au)


def cheb_adjoint_apply(plan: Plan, K, lam, out):
    return plan.adjoint_apply(K, lam, out)


def cheb_deriv(plan: Plan, axis: int, u, du):
    return plan.deriv(u, axis, du)


def cheb_rhs(plan: Plan, f, faces, b):
    return plan.rhs(f, faces, b)
