"""Constant-coefficient preconditioner for the oracle's GMRES (test
infrastructure; see the package docstring).

Plain restarted GMRES does not converge on the collocation systems beyond
small grids (the paper reports the same for its unpreconditioned LGMRES
beyond N = 48, Sec. 3.2).  The oracle therefore runs GMRES on M^{-1} A u =
M^{-1} b, with M the collocation operator for a constant conductivity
``kref`` and the same boundary rows.  The oracle's answer is still checked
only through its plain dense ``apply``; M merely accelerates convergence.

M^{-1} r, written with dense numpy operations (a flux row -kref s (d_a u) = r
is the Neumann row with datum -r / kref, so flux rows are rescaled first):
1. per axis, the two end rows of every line (Dirichlet: u = g, Neumann:
   +-(D u) = g) give the end values from the line interior,
   u_b = G u_int + Binv g (the boundary elimination of Sec. 2.3.1 in 1-D);
2. the interior equations then read kref (A_x (+) A_y (+) A_z) u_int = rhs, a
   Kronecker sum of 1-D operators, solved through numpy's eigendecomposition
   A_a = S_a diag(lam_a) S_a^{-1};
3. nodes on two or more faces (edges, corners) satisfy their own boundary
   rows, assembled here as a small dense system and solved directly.
Pinned against dense direct solves in tests/test_oracle_precond.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .core import DIRICHLET, FLUX, Grid, apply, owners


def _axis_tables(grid: Grid, a: int):
    D = grid.D(a)
    N = grid.n[a] - 1
    Bm = np.zeros((2, 2))
    Cm = np.zeros((2, N - 1))
    if grid.bc[2 * a + 1] == DIRICHLET:  # index 0 is the hi face
        Bm[0, 0] = 1.0
    else:
        Bm[0] = [D[0, 0], D[0, N]]
        Cm[0] = D[0, 1:N]
    if grid.bc[2 * a] == DIRICHLET:      # index N is the lo face
        Bm[1, 1] = 1.0
    else:
        Bm[1] = [-D[N, 0], -D[N, N]]
        Cm[1] = -D[N, 1:N]
    Binv = np.linalg.inv(Bm)
    G = -Binv @ Cm
    D2 = D @ D
    A_ib = D2[1:N][:, [0, N]]
    Ared = -(D2[1:N, 1:N] + A_ib @ G)
    lam, S = np.linalg.eig(Ared)
    if np.abs(lam.imag).max() > 1e-9 * np.abs(lam).max():
        raise ValueError("complex eigenvalues in the reduced 1-D operator")
    lam, S = lam.real, S.real
    return dict(N=N, G=G, Binv=Binv, Lh=A_ib @ Binv, lam=lam, S=S, Sinv=np.linalg.inv(S))


class FDMPreconditioner:
    """x = M^{-1} r for conductivity kref (see the module docstring)."""

    def __init__(self, grid: Grid, kref: float):
        self.g = grid
        self.kref = float(kref)
        self.t = {a: _axis_tables(grid, a) for a in grid.axes}
        own = owners(grid)
        nfaces = np.zeros(grid.shape, dtype=int)
        for a in grid.axes:
            for idx in (0, grid.n[a] - 1):
                sl = [slice(None)] * 3
                sl[2 - a] = idx
                nfaces[tuple(sl)] += 1
        self.edge = nfaces >= 2
        self.E = np.argwhere(self.edge)             # (k, j, i) rows
        self.own = own
        # dense system of the edge/corner rows restricted to edge/corner columns
        pos = -np.ones(grid.shape, dtype=int)
        for r, (k, j, i) in enumerate(self.E):
            pos[k, j, i] = r
        nE = len(self.E)
        A22 = np.zeros((nE, nE))
        self.rows = []
        for r, (k, j, i) in enumerate(self.E):
            f = own[k, j, i]
            if grid.bc[f] == DIRICHLET:
                A22[r, r] = 1.0
                self.rows.append(None)
                continue
            a, side = divmod(int(f), 2)
            s = 1.0 if side == 1 else -1.0
            D = grid.D(a)
            idx = [i, j, k][a]
            line = []
            for q in range(grid.n[a]):
                node = [k, j, i]
                node[2 - a] = q
                line.append(tuple(node))
                if pos[tuple(node)] >= 0:
                    A22[r, pos[tuple(node)]] += s * D[idx, q]
            self.rows.append((s, D[idx], line))
        self.lu = sla.lu_factor(A22) if nE else None

    def _interior(self):
        sl = []
        for a in (2, 1, 0):
            sl.append(slice(1, -1) if a < self.g.dim else slice(None))
        return tuple(sl)

    def __call__(self, r: np.ndarray) -> np.ndarray:
        g, kref = self.g, self.kref
        r = np.asarray(r, float)
        # a flux row -kref s (d_a u) = r_p is the Neumann row s (d_a u) = -r_p / kref
        flux = np.isin(self.own, [f for f in range(2 * g.dim) if g.bc[f] == FLUX])
        if flux.any():
            r = np.where(flux, -r / kref, r)
        x = np.zeros(g.shape)
        I = self._interior()
        rhs = r[I].copy()
        for a in g.axes:
            t = self.t[a]
            npax = 2 - a
            e0 = list(I)
            e0[npax] = 0
            eN = list(I)
            eN[npax] = -1
            g0, gN = r[tuple(e0)], r[tuple(eN)]
            lift = np.multiply.outer(t["Lh"][:, 0], g0) + np.multiply.outer(t["Lh"][:, 1], gN)
            rhs += kref * np.moveaxis(lift, 0, npax)
        v = rhs
        for a in g.axes:
            v = np.moveaxis(np.tensordot(self.t[a]["Sinv"], v, axes=([1], [2 - a])), 0, 2 - a)
        lam = np.zeros(v.shape)
        for a in g.axes:
            shp = [1, 1, 1]
            shp[2 - a] = -1
            lam = lam + self.t[a]["lam"].reshape(shp)
        v = v / (kref * lam)
        for a in g.axes:
            v = np.moveaxis(np.tensordot(self.t[a]["S"], v, axes=([1], [2 - a])), 0, 2 - a)
        x[I] = v
        for a in g.axes:
            t = self.t[a]
            npax = 2 - a
            e0 = list(I)
            e0[npax] = 0
            eN = list(I)
            eN[npax] = -1
            g0, gN = r[tuple(e0)], r[tuple(eN)]
            ub = np.tensordot(t["G"], v, axes=([1], [npax]))
            x[tuple(e0)] = ub[0] + t["Binv"][0, 0] * g0 + t["Binv"][0, 1] * gN
            x[tuple(eN)] = ub[1] + t["Binv"][1, 0] * g0 + t["Binv"][1, 1] * gN
        if self.lu is not None:
            rhsE = np.zeros(len(self.E))
            for rr, (k, j, i) in enumerate(self.E):
                rhsE[rr] = r[k, j, i]
                row = self.rows[rr]
                if row is None:
                    continue
                s, Drow, line = row
                acc = 0.0
                for q, node in enumerate(line):
                    if not self.edge[node]:
                        acc += Drow[q] * x[node]
                rhsE[rr] -= s * acc
            xE = sla.lu_solve(self.lu, rhsE)
            for rr, (k, j, i) in enumerate(self.E):
                x[k, j, i] = xE[rr]
        return x


    def transpose(self, y: np.ndarray) -> np.ndarray:
        """z = M^{-T} y: the transposes of the steps of __call__ in reverse
        order (edge and corner rows, face values, interior eigen-solve with
        its lifting, flux-row scaling).  Pinned against the dense transpose of
        M^{-1} in tests/test_oracle_precond.py."""
        g, kref = self.g, self.kref
        y = np.array(y, float, copy=True)
        I = self._interior()
        zr = np.zeros(g.shape)          # adjoint of r' (the flux-scaled input)
        # edge / corner rows: xE = A22^{-1} (r'[E] - sum_q s Drow[q] x[q]) over
        # the non-edge nodes q of each edge row's owner-axis line
        if self.lu is not None:
            yE = np.array([y[k, j, i] for (k, j, i) in self.E])
            wE = sla.lu_solve(self.lu, yE, trans=1)
            for rr, (k, j, i) in enumerate(self.E):
                zr[k, j, i] += wE[rr]
                y[k, j, i] = 0.0
                row = self.rows[rr]
                if row is None:
                    continue
                s, Drow, line = row
                for q, node in enumerate(line):
                    if not self.edge[node]:
                        y[node] -= s * Drow[q] * wE[rr]
        # face values: x[e0] = G[0] v + Binv[0,0] g0 + Binv[0,1] gN, x[eN] likewise,
        # with g0, gN the face values of r'
        vbar = y[I].copy()
        for a in g.axes:
            t = self.t[a]
            npax = 2 - a
            e0 = list(I)
            e0[npax] = 0
            eN = list(I)
            eN[npax] = -1
            y0, yN = y[tuple(e0)], y[tuple(eN)]
            vbar += np.moveaxis(np.multiply.outer(t["G"][0], y0) + np.multiply.outer(t["G"][1], yN), 0, npax)
            zr[tuple(e0)] += t["Binv"][0, 0] * y0 + t["Binv"][1, 0] * yN
            zr[tuple(eN)] += t["Binv"][0, 1] * y0 + t["Binv"][1, 1] * yN
        # v = S_all diag(1 / (kref lam)) S_all^{-1} rhs  ->  rhs_bar = S_all^{-T} diag S_all^T vbar
        v = vbar
        for a in g.axes:
            v = np.moveaxis(np.tensordot(self.t[a]["S"].T, v, axes=([1], [2 - a])), 0, 2 - a)
        lam = np.zeros(v.shape)
        for a in g.axes:
            shp = [1, 1, 1]
            shp[2 - a] = -1
            lam = lam + self.t[a]["lam"].reshape(shp)
        v = v / (kref * lam)
        for a in g.axes:
            v = np.moveaxis(np.tensordot(self.t[a]["Sinv"].T, v, axes=([1], [2 - a])), 0, 2 - a)
        # rhs = r'[I] + sum_a kref (Lh[:, 0] g0 + Lh[:, 1] gN) along a
        zr[I] += v
        for a in g.axes:
            t = self.t[a]
            npax = 2 - a
            e0 = list(I)
            e0[npax] = 0
            eN = list(I)
            eN[npax] = -1
            vm = np.moveaxis(v, npax, 0)
            zr[tuple(e0)] += kref * np.tensordot(t["Lh"][:, 0], vm, axes=([0], [0]))
            zr[tuple(eN)] += kref * np.tensordot(t["Lh"][:, 1], vm, axes=([0], [0]))
        flux = np.isin(self.own, [f for f in range(2 * g.dim) if g.bc[f] == FLUX])
        if flux.any():
            zr = np.where(flux, -zr / kref, zr)
        return zr


def geometric_mean(K: np.ndarray) -> float:
    return float(np.exp(np.log(np.asarray(K, float)).mean()))


def solve_preconditioned(K: np.ndarray, b: np.ndarray, grid: Grid, x0=None, rtol: float = 1e-13,
                         restart: int = 50, maxiter: int = 5000, kref: float | None = None):
    """GMRES on M^{-1} A u = M^{-1} b (FP64).  info reports the preconditioned
    relative residual and the plain relative residual ||b - A u|| / ||b||."""
    from .core import gmres
    M = FDMPreconditioner(grid, geometric_mean(K) if kref is None else kref)
    Mb = M(b)
    u, info = gmres(lambda v: M(apply(v, K, grid)), Mb, x0, rtol=rtol, restart=restart,
                    maxiter=maxiter)
    r = b - apply(u, K, grid)
    info["plain_rel_residual"] = float(np.linalg.norm(r) / np.linalg.norm(b))
    info["kref"] = M.kref
    return u, info


def solve_hierarchy(Ks, bs, grids, rtol: float = 1e-12, restart: int = 50, maxiter: int = 5000,
                    x0=None):
    """Hierarchical refinement (Alg. 4, Sec. 2.3.3) with the oracle's own pieces:
    solve the coarsest level (from ``x0`` or zero), then for every finer level
    prolong the previous solution by barycentric interpolation (the same
    polynomial as the paper's coefficient zero-padding) and use it as the
    initial guess of that level's preconditioned GMRES.

    ``Ks``, ``bs``: per-level conductivity and right-hand side sampled on that
    level's grid; ``grids``: oracle Grids of doubling N.  Returns (solutions,
    infos, e_ref) with e_ref[l] = ||u_l - P u_{l-1}|| / ||u_l|| (e_ref[0] = 0)."""
    from .core import e_ref as _e_ref, prolong
    us, infos, eref = [], [], []
    u0 = x0
    for lvl, (K, b, g) in enumerate(zip(Ks, bs, grids)):
        guess = None
        if lvl > 0:
            guess = prolong(us[-1], grids[lvl - 1], g)
        elif u0 is not None:
            guess = u0
        u, info = solve_preconditioned(K, b, g, x0=guess, rtol=rtol, restart=restart, maxiter=maxiter)
        us.append(u)
        infos.append(info)
        eref.append(0.0 if guess is None or lvl == 0 else _e_ref(u, guess))
    return us, infos, eref


def adjoint_solve_preconditioned(K: np.ndarray, c: np.ndarray, grid: Grid, x0=None, rtol: float = 1e-13,
                                 restart: int = 50, maxiter: int = 5000, kref: float | None = None):
    """A^T lam = c by GMRES on M^{-T} A^T lam = M^{-T} c (FP64; the discrete
    adjoint of the collocation system).  info reports the plain relative
    residual ||c - A^T lam|| / ||c|| beside the preconditioned one."""
    from .core import adjoint_apply, gmres
    M = FDMPreconditioner(grid, geometric_mean(K) if kref is None else kref)
    lam, info = gmres(lambda v: M.transpose(adjoint_apply(v, K, grid)), M.transpose(c), x0, rtol=rtol,
                      restart=restart, maxiter=maxiter)
    r = c - adjoint_apply(lam, K, grid)
    info["plain_rel_residual"] = float(np.linalg.norm(r) / np.linalg.norm(c))
    return lam, info
