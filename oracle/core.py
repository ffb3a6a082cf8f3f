"""Plain FP64 definitions of the collocation operator, its solves, prolongation
and adjoint (test infrastructure; see the package docstring).

Index and face conventions
--------------------------
* Axis a = 0, 1, 2 is x, y, z.  Fields are arrays shaped (nz, ny, nx), so axis
  a is numpy axis ``2 - a``.  Unused axes of 1-D/2-D problems have length 1.
* Node j of an axis with N + 1 points sits at the reference coordinate
  x_j = cos(pi j / N) (Sec. 2.2), mapped affinely to [lo, hi] (Sec. 2.2,
  affine mapping), so node 0 is the ``hi`` end and node N the ``lo`` end.
* Face id f = 2a + side, side 0 = ``lo``, side 1 = ``hi`` (x-, x+, y-, y+, z-, z+).
  Neumann data is the outward normal derivative n . grad u; flux data (the
  heat-flux condition of Sec. 3.4) is -K n . grad u.
* Every boundary node has one owner face: a Dirichlet face beats a Neumann
  or flux face, and among the others the lowest axis wins.  (The paper only
  says the equations at boundary nodes are replaced by the boundary
  conditions, Sec. 2 "Extension to the three-dimensional setting"; it does
  not say which face owns an edge or corner node.)
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "DIRICHLET", "NEUMANN", "FLUX", "Grid", "cgl_nodes", "diff_matrix", "cc_weights",
    "grad", "interior_operator", "owners", "apply", "rhs", "assemble",
    "solve_direct", "gmres", "solve", "barycentric_matrix", "prolong", "e_ref",
    "adjoint_apply", "adjoint_solve_direct", "grad_K", "picard_conductivity",
    "picard_solve", "eliminate_solve", "restrict_inject", "volume_average",
    "effective_conductivity", "maxwell_estimate", "reciprocal_law", "jacobian_apply",
    "newton_residual", "newton_solve", "linearized_apply", "eliminated_system",
]

DIRICHLET = 0
NEUMANN = 1
FLUX = 2   # flux data: -K (n . grad u) = g, the heat-flux condition of Sec. 3.4


# ----------------------------------------------------------------------------
# grid
# ----------------------------------------------------------------------------

def cgl_nodes(N: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Chebyshev-Gauss-Lobatto nodes t_j, j = 0..N (Sec. 2.2 and its affine map).

    x_j = cos(pi j / N) is evaluated as sin(pi (N - 2j) / (2N)), the same
    number by the identity cos(a) = sin(pi/2 - a), which makes the nodes
    exactly antisymmetric and x_{N/2} exactly 0.
    """
    j = np.arange(N + 1)
    x = np.sin(np.pi * (N - 2 * j) / (2 * N))
    return 0.5 * (hi - lo) * x + 0.5 * (hi + lo)


def diff_matrix(N: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Dense CGL first-derivative matrix D_jm = l'_m(x_j) (Sec. 2, 1-D) on [lo, hi].

    Off-diagonal entries take the closed form
    D_ij = (cbar_i / cbar_j) (-1)^(i+j) / (x_i - x_j), cbar_0 = cbar_N = 2, else 1
    (Trefethen, Spectral Methods in MATLAB, ch. 6), with the node difference
    computed as x_i - x_j = 2 sin(pi (i+j)/(2N)) sin(pi (j-i)/(2N)) (exact
    identity, avoids cancellation).  The diagonal is the negative row sum
    (D annihilates constants).  Scaled by 2/(hi - lo) for the physical
    coordinate (Sec. 2.2, chain rule of the affine map).
    """
    if N < 1:
        raise ValueError("N >= 1 required")
    i = np.arange(N + 1)[:, None]
    j = np.arange(N + 1)[None, :]
    cbar = np.ones(N + 1)
    cbar[0] = cbar[N] = 2.0
    diff = 2.0 * np.sin(np.pi * (i + j) / (2 * N)) * np.sin(np.pi * (j - i) / (2 * N))
    sign = np.where((i + j) % 2 == 0, 1.0, -1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        D = (cbar[:, None] / cbar[None, :]) * sign / diff
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, -D.sum(axis=1))
    return D * (2.0 / (hi - lo))


def cc_weights(N: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Clenshaw-Curtis quadrature weights at the CGL nodes (Trefethen's clencurt
    formula): w_j = (c_j/N) [1 - sum_{k=1}^{N/2} b_k cos(2 pi j k / N) / (4k^2 - 1)],
    c_0 = c_N = 1 else 2, b_k = 1 if 2k = N else 2; scaled by (hi - lo)/2."""
    w = np.zeros(N + 1)
    for jj in range(N + 1):
        s = 0.0
        for k in range(1, N // 2 + 1):
            b = 1.0 if 2 * k == N else 2.0
            s += b * math.cos(2.0 * math.pi * jj * k / N) / (4.0 * k * k - 1.0)
        c = 1.0 if jj in (0, N) else 2.0
        w[jj] = c / N * (1.0 - s)
    return w * (0.5 * (hi - lo))


class Grid:
    """Tensor CGL grid with per-axis points n = (nx, ny, nz) (unused axes: 1),
    per-axis intervals [lo, hi] and six per-face BC types."""

    def __init__(self, n, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), bc=(0, 0, 0, 0, 0, 0)):
        n = list(n) + [1] * (3 - len(n))
        self.n = tuple(int(v) for v in n)
        self.dim = sum(1 for v in self.n if v > 1)
        if any(v == 1 for v in self.n[: self.dim]) or any(v != 1 for v in self.n[self.dim:]):
            raise ValueError("active axes must come first and have >= 2 points")
        if any(v < 3 for v in self.n[: self.dim]):
            raise ValueError("each active axis needs N + 1 >= 3 points")
        lo = list(lo) + [-1.0] * (3 - len(lo))
        hi = list(hi) + [1.0] * (3 - len(hi))
        self.lo = tuple(float(v) for v in lo)
        self.hi = tuple(float(v) for v in hi)
        self.bc = tuple(int(v) for v in bc)
        self.shape = (self.n[2], self.n[1], self.n[0])
        self.axes = list(range(self.dim))
        self._D = {}

    @property
    def size(self) -> int:
        return int(np.prod(self.shape))

    def nodes(self, a: int) -> np.ndarray:
        if a >= self.dim:
            return np.array([0.0])
        return cgl_nodes(self.n[a] - 1, self.lo[a], self.hi[a])

    def mesh(self):
        """(X, Y, Z) node coordinates, each shaped (nz, ny, nx)."""
        Z, Y, X = np.meshgrid(self.nodes(2), self.nodes(1), self.nodes(0), indexing="ij")
        return X, Y, Z

    def D(self, a: int) -> np.ndarray:
        if a not in self._D:
            self._D[a] = diff_matrix(self.n[a] - 1, self.lo[a], self.hi[a])
        return self._D[a]


# ----------------------------------------------------------------------------
# operator (Alg. 3, Eq. (eq1)) with boundary rows (Sec. 2, boundary nodes)
# ----------------------------------------------------------------------------

def grad(u: np.ndarray, grid: Grid, a: int) -> np.ndarray:
    """Partial derivative along axis a: [d_a u]_pqr = sum_m D^(a) U (separable
    differentiation, Sec. 2 "Extension to the three-dimensional setting")."""
    npax = 2 - a
    return np.moveaxis(np.tensordot(grid.D(a), u, axes=([1], [npax])), 0, npax)


def interior_operator(u: np.ndarray, K: np.ndarray, grid: Grid) -> np.ndarray:
    """L(u) = -sum_a C_a(K * C_a(u)) at every node (Alg. 3; Eq. (eq1) of Sec. 3.3)."""
    out = np.zeros_like(u, dtype=float)
    for a in grid.axes:
        out -= grad(K * grad(u, grid, a), grid, a)
    return out


def owners(grid: Grid) -> np.ndarray:
    """Owner face id of every node (-1 for interior nodes).

    Dirichlet faces are claimed before Neumann and flux faces; within each
    rank, axes in increasing order.  Node index 0 lies on the ``hi`` face (side 1), index
    n - 1 on the ``lo`` face (side 0).
    """
    own = -np.ones(grid.shape, dtype=np.int64)
    for rank in (0, 1):   # Dirichlet faces first, then Neumann and flux faces
        for a in grid.axes:
            for side in (0, 1):
                f = 2 * a + side
                if (grid.bc[f] == DIRICHLET) != (rank == 0):
                    continue
                sl = [slice(None)] * 3
                sl[2 - a] = grid.n[a] - 1 if side == 0 else 0
                view = own[tuple(sl)]
                view[view < 0] = f
    return own


def apply(u: np.ndarray, K: np.ndarray, grid: Grid) -> np.ndarray:
    """A u: collocation rows L(u) at interior nodes (Eq. (eq:residualN)); at a
    boundary node the row is replaced by its owner face's condition
    (Eq. (eq:boundaryN)): Dirichlet u_p, Neumann s (d_a u)_p with s = +1 on the
    ``hi`` face and -1 on the ``lo`` face (outward normal), flux -K_p s (d_a u)_p
    (Sec. 3.4, q_N = -k grad T . n)."""
    out = interior_operator(u, K, grid)
    own = owners(grid)
    out[own >= 0] = 0.0
    for f in range(2 * grid.dim):
        m = own == f
        if not m.any():
            continue
        if grid.bc[f] == DIRICHLET:
            out[m] = u[m]
        else:
            a, side = divmod(f, 2)
            s = 1.0 if side == 1 else -1.0
            row = s * grad(u, grid, a)[m]
            out[m] = -np.asarray(K, float)[m] * row if grid.bc[f] == FLUX else row
    return out


def _face_slice(grid: Grid, f: int):
    a, side = divmod(f, 2)
    sl = [slice(None)] * 3
    sl[2 - a] = grid.n[a] - 1 if side == 0 else 0
    return tuple(sl)


def rhs(f: np.ndarray, faces, grid: Grid) -> np.ndarray:
    """b: f at interior nodes, the owner face's datum g at boundary nodes
    (Eqs. (eq:residualN), (eq:boundaryN)).  ``faces[F]`` is shaped like a field
    with face F's axis removed."""
    b = np.array(f, dtype=float, copy=True)
    own = owners(grid)
    for F in range(2 * grid.dim):
        sl = _face_slice(grid, F)
        bview = b[sl]
        m = own[sl] == F
        bview[m] = np.asarray(faces[F], float)[m]
    return b


def assemble(K: np.ndarray, grid: Grid) -> np.ndarray:
    """Dense A with Kronecker-product derivatives (Sec. 2, vectorised form
    d u/dx = (D^x (x) I (x) I) u, written for C-order (z, y, x) flattening) and
    replaced boundary rows.  Tiny grids only."""
    nx, ny, nz = grid.n
    I = [np.eye(nx), np.eye(ny), np.eye(nz)]
    Dh = []
    for a in grid.axes:
        mats = [I[2], I[1], I[0]]  # z, y, x factors
        mats[2 - a] = grid.D(a)
        Dh.append(np.kron(mats[0], np.kron(mats[1], mats[2])))
    Kd = np.diag(np.asarray(K, float).ravel())
    A = np.zeros((grid.size, grid.size))
    for M in Dh:
        A -= M @ Kd @ M
    own = owners(grid).ravel()
    for f in range(2 * grid.dim):
        rows = np.nonzero(own == f)[0]
        if grid.bc[f] == DIRICHLET:
            A[rows, :] = 0.0
            A[rows, rows] = 1.0
        else:
            a, side = divmod(f, 2)
            s = 1.0 if side == 1 else -1.0
            A[rows, :] = s * Dh[a][rows, :]
            if grid.bc[f] == FLUX:
                A[rows, :] *= -np.asarray(K, float).ravel()[rows][:, None]
    return A


def solve_direct(K: np.ndarray, b: np.ndarray, grid: Grid) -> np.ndarray:
    """Direct dense solve of A u = b (tiny grids).

    Rows are first scaled to unit max-norm (same solution): interior rows
    grow like N^4 while Dirichlet rows are O(1), and an unscaled LU would
    perturb the small rows by eps * ||A||."""
    A = assemble(K, grid)
    s = 1.0 / np.abs(A).max(axis=1)
    x = np.linalg.solve(A * s[:, None], np.asarray(b, float).ravel() * s)
    return x.reshape(grid.shape)


# ----------------------------------------------------------------------------
# restarted GMRES (the oracle's iterative route; not the paper's LGMRES)
# ----------------------------------------------------------------------------

def gmres(matvec, b: np.ndarray, x0=None, rtol: float = 1e-13, atol: float = 0.0,
          restart: int = 50, maxiter: int = 20000, stagnation: int = 5):
    """Restarted GMRES(restart) with modified Gram-Schmidt and Givens rotations,
    FP64.  Stops when the true residual satisfies ||r|| <= max(rtol ||b||, atol),
    after ``maxiter`` inner iterations, or after ``stagnation`` restarts that
    fail to reduce the true residual.  Returns (x, info)."""
    shape = b.shape
    bv = np.asarray(b, float).ravel()
    x = np.zeros_like(bv) if x0 is None else np.array(x0, float).ravel()
    bnorm = np.linalg.norm(bv)
    target = max(rtol * bnorm, atol)
    its = 0
    best = math.inf
    stall = 0
    history = []
    while True:
        r = bv - matvec(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
        history.append(beta)
        if beta <= target or its >= maxiter:
            break
        if beta < 0.999 * best:
            best = beta
            stall = 0
        else:
            stall += 1
            if stall >= stagnation:
                break
        m = restart
        V = np.zeros((m + 1, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for k in range(m):
            w = matvec(V[k].reshape(shape)).ravel()
            its += 1
            for i in range(k + 1):
                H[i, k] = w @ V[i]
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den if den else 1.0
            sn[k] = H[k + 1, k] / den if den else 0.0
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            if abs(g[k + 1]) <= target or its >= maxiter or H[k, k] == 0:
                break
        kk = k + 1
        y = np.zeros(kk)
        for i in range(kk - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:kk] @ y[i + 1:kk]) / H[i, i]
        x = x + V[:kk].T @ y
    return x.reshape(shape), {"iterations": its, "residual": float(beta),
                              "rel_residual": float(beta / bnorm) if bnorm else float(beta),
                              "history": history}


def solve(K: np.ndarray, b: np.ndarray, grid: Grid, x0=None, rtol: float = 1e-13,
          restart: int = 50, maxiter: int = 20000):
    """A u = b: direct for tiny grids (<= 4096 unknowns), else restarted GMRES."""
    if grid.size <= 4096:
        u = solve_direct(K, b, grid)
        r = np.linalg.norm(b - apply(u, K, grid)) / max(np.linalg.norm(b), 1e-300)
        return u, {"iterations": 0, "rel_residual": float(r), "direct": True}
    return gmres(lambda v: apply(v, K, grid), b, x0, rtol=rtol, restart=restart, maxiter=maxiter)


# ----------------------------------------------------------------------------
# prolongation (Sec. 2.3.3): the same polynomial by barycentric interpolation
# ----------------------------------------------------------------------------

def barycentric_matrix(N_c: int, N_f: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """P (N_f+1 x N_c+1): values at the fine CGL nodes of the degree-N_c
    interpolant through the coarse CGL nodes, by the barycentric formula with
    CGL weights w_j = (-1)^j delta_j, delta_0 = delta_N = 1/2 (Berrut and
    Trefethen 2004).  The paper zero-pads Chebyshev coefficients instead
    (Sec. 2.3.3); both evaluate the same unique interpolating polynomial."""
    s = cgl_nodes(N_c, lo, hi)
    t = cgl_nodes(N_f, lo, hi)
    w = np.where(np.arange(N_c + 1) % 2 == 0, 1.0, -1.0)
    w[0] *= 0.5
    w[-1] *= 0.5
    P = np.zeros((N_f + 1, N_c + 1))
    for i, ti in enumerate(t):
        d = ti - s
        hit = np.nonzero(d == 0.0)[0]
        if hit.size:
            P[i, hit[0]] = 1.0
            continue
        q = w / d
        P[i] = q / q.sum()
    return P


def prolong(u_c: np.ndarray, grid_c: Grid, grid_f: Grid) -> np.ndarray:
    """Prolong a nodal field from grid_c to grid_f (per-axis barycentric)."""
    out = np.asarray(u_c, float)
    for a in grid_c.axes:
        P = barycentric_matrix(grid_c.n[a] - 1, grid_f.n[a] - 1, grid_c.lo[a], grid_c.hi[a])
        npax = 2 - a
        out = np.moveaxis(np.tensordot(P, out, axes=([1], [npax])), 0, npax)
    return out


def restrict_inject(u_f: np.ndarray, grid_c: Grid, grid_f: Grid) -> np.ndarray:
    """Injection to the coarse grid: for N_f = 2 N_c, CGL nodes nest,
    x_j^(N_c) = x_{2j}^(N_f), so coarse node j is fine node 2j."""
    sl = []
    for a in (2, 1, 0):
        if a < grid_c.dim:
            r = (grid_f.n[a] - 1) // (grid_c.n[a] - 1)
            sl.append(slice(None, None, r))
        else:
            sl.append(slice(None))
    return np.asarray(u_f)[tuple(sl)].copy()


def e_ref(u_fine: np.ndarray, u_prolonged: np.ndarray) -> float:
    """Refinement indicator ||U_Nf - U_{N->Nf}||_2 / ||U_Nf||_2 (Sec. 2.3.3)."""
    return float(np.linalg.norm(u_fine - u_prolonged) / np.linalg.norm(u_fine))


# ----------------------------------------------------------------------------
# adjoint (discrete, dense transposes)
# ----------------------------------------------------------------------------

def _grad_T(v: np.ndarray, grid: Grid, a: int) -> np.ndarray:
    npax = 2 - a
    return np.moveaxis(np.tensordot(grid.D(a).T, v, axes=([1], [npax])), 0, npax)


def adjoint_apply(lam: np.ndarray, K: np.ndarray, grid: Grid) -> np.ndarray:
    """A^T lam for A = P_int L + R_bc:
    -sum_a D_a^T (K * D_a^T (P_int lam)) + P_dir lam + sum_a D_a^T (S_a lam),
    with S_a = +-1 on Neumann rows owned by an axis-a face (sign of the
    outward normal; -+K_p on flux rows), P_int / P_dir the interior /
    Dirichlet-row masks."""
    own = owners(grid)
    lam = np.asarray(lam, float)
    lam_int = np.where(own < 0, lam, 0.0)
    out = np.zeros_like(lam)
    for a in grid.axes:
        out -= _grad_T(K * _grad_T(lam_int, grid, a), grid, a)
    for f in range(2 * grid.dim):
        m = own == f
        if not m.any():
            continue
        if grid.bc[f] == DIRICHLET:
            out[m] += lam[m]
        else:
            a, side = divmod(f, 2)
            s = 1.0 if side == 1 else -1.0
            w = -np.asarray(K, float) * lam if grid.bc[f] == FLUX else lam
            out += _grad_T(np.where(m, s * w, 0.0), grid, a)
    return out


def adjoint_solve_direct(K: np.ndarray, dJdu: np.ndarray, grid: Grid) -> np.ndarray:
    """lam = A^{-T} dJ/du by a dense solve (tiny grids)."""
    A = assemble(K, grid)
    s = 1.0 / np.abs(A).max(axis=0)
    # column scaling of A^T (= row scaling of A) for the same reason as solve_direct
    y = np.linalg.solve(A.T * s[None, :], np.asarray(dJdu, float).ravel())
    return (y * s).reshape(grid.shape)


def grad_K(u: np.ndarray, lam: np.ndarray, grid: Grid) -> np.ndarray:
    """dJ/dK for J(u(K)) with A(K) u = b and A^T lam = dJ/du (no explicit K in J):
    dJ/dK_p = -lam^T (dA/dK_p) u = sum_a (D_a^T P_int lam)_p (D_a u)_p, because
    A depends on K through the interior rows -sum_a D_a diag(K) D_a, plus
    s lam_p (D_a u)_p on flux rows (row -K_p s (D_a u)_p)."""
    own = owners(grid)
    lam_int = np.where(own < 0, np.asarray(lam, float), 0.0)
    g = np.zeros(grid.shape)
    for a in grid.axes:
        g += _grad_T(lam_int, grid, a) * grad(u, grid, a)
    # flux rows -K_p s (d_a u)_p depend on K_p too: -lam_p * (-s (d_a u)_p)
    for f in range(2 * grid.dim):
        if grid.bc[f] != FLUX:
            continue
        m = own == f
        a, side = divmod(f, 2)
        s = 1.0 if side == 1 else -1.0
        g[m] += s * np.asarray(lam, float)[m] * grad(u, grid, a)[m]
    return g


# ----------------------------------------------------------------------------
# Picard outer loop (Sec. 2.3, Picard iteration) for K = K0 (1 + 0.5 |grad u|^2)
# ----------------------------------------------------------------------------

def picard_conductivity(K0: np.ndarray, u: np.ndarray, grid: Grid, beta: float = 0.5) -> np.ndarray:
    """K = K0 (1 + beta |grad u|^2), gradient by the dense D."""
    s = np.zeros(grid.shape)
    for a in grid.axes:
        s += grad(u, grid, a) ** 2
    return K0 * (1.0 + beta * s)


def picard_solve(K0: np.ndarray, b: np.ndarray, grid: Grid, tol: float = 1e-11,
                 maxit: int = 50, beta: float = 0.5, u0=None, lin_rtol: float = 1e-13,
                 omega: float = 1.0):
    """Picard iteration with the nonlinearity frozen at the previous iterate
    (Sec. 2.3 Picard iteration): u* solves A(K(u^m)) u* = b and
    u^{m+1} = (1 - omega) u^m + omega u* (omega = 1 is the plain iteration);
    stops when ||u^{m+1} - u^m|| / ||u^{m+1}|| <= tol."""
    u = np.zeros(grid.shape) if u0 is None else np.array(u0, float)
    hist = []
    for it in range(1, maxit + 1):
        K = picard_conductivity(K0, u, grid, beta)
        if grid.size <= 4096:
            un, _ = solve(K, b, grid, x0=u, rtol=lin_rtol)
        else:
            from .precond import solve_preconditioned
            un, _ = solve_preconditioned(K, b, grid, x0=u, rtol=lin_rtol)
        un = (1.0 - omega) * u + omega * un
        d = np.linalg.norm(un - u) / max(np.linalg.norm(un), 1e-300)
        hist.append(d)
        u = un
        if d <= tol:
            break
    return u, {"iterations": it, "history": hist}


# ----------------------------------------------------------------------------
# the paper's own BC formulation (Sec. 2.3.1) on tiny grids
# ----------------------------------------------------------------------------

def _elimination_parts(K: np.ndarray, grid: Grid):
    """Pieces of the paper's boundary elimination (Eqs. (eq:BuildSystemBCs),
    (eq:ReducedSystemBCs), (eq:RestrictBCs)): the collocation operator A
    without row replacement, the boundary rows B (one per boundary node, from
    its owner face), the index sets of boundary (r) and interior (k) nodes,
    and G = -B_r^{-1} B_k, H = B_r^{-1} so that x_r = G x_k + H g."""
    nx, ny, nz = grid.n
    I = [np.eye(nx), np.eye(ny), np.eye(nz)]
    Dh = []
    for a in grid.axes:
        mats = [I[2], I[1], I[0]]
        mats[2 - a] = grid.D(a)
        Dh.append(np.kron(mats[0], np.kron(mats[1], mats[2])))
    Kd = np.diag(np.asarray(K, float).ravel())
    A = np.zeros((grid.size, grid.size))
    for M in Dh:
        A -= M @ Kd @ M
    own = owners(grid).ravel()
    r_idx = np.nonzero(own >= 0)[0]
    k_idx = np.nonzero(own < 0)[0]
    B = np.zeros((r_idx.size, grid.size))
    for row, p in enumerate(r_idx):
        fce = own[p]
        if grid.bc[fce] == DIRICHLET:
            B[row, p] = 1.0
        else:
            a, side = divmod(int(fce), 2)
            B[row] = (1.0 if side == 1 else -1.0) * Dh[a][p]
            if grid.bc[fce] == FLUX:
                B[row] *= -float(np.asarray(K, float).ravel()[p])
    Br_inv = np.linalg.inv(B[:, r_idx])
    G = -Br_inv @ B[:, k_idx]
    return A, B, r_idx, k_idx, G, Br_inv


def eliminated_system(K: np.ndarray, grid: Grid) -> np.ndarray:
    """The reduced interior operator A_kk + A_kr G of the elimination
    formulation (tiny grids), for conditioning comparisons with the
    row-replaced matrix of ``assemble``."""
    A, _, r_idx, k_idx, G, _ = _elimination_parts(K, grid)
    return A[np.ix_(k_idx, k_idx)] + A[np.ix_(k_idx, r_idx)] @ G


def eliminate_solve(K: np.ndarray, f: np.ndarray, faces, grid: Grid) -> np.ndarray:
    """Solve by eliminating the boundary unknowns (Eqs. (eq:BuildSystemBCs),
    (eq:ReducedSystemBCs), (eq:RestrictBCs)): B x = g split as
    x_r = G x_k + H g with G = -B_r^{-1} B_k, H = B_r^{-1}; reduced system
    (A_kk + A_kr G) x_k = f_k - A_kr H g; then x_r recovered.  A is the
    collocation operator without row replacement, B the boundary rows (one
    per boundary node, from its owner face)."""
    A, B, r_idx, k_idx, G, H = _elimination_parts(K, grid)
    own = owners(grid).ravel()
    gfull = rhs(np.zeros(grid.shape), faces, grid).ravel()
    g = gfull[r_idx]
    Akk, Akr = A[np.ix_(k_idx, k_idx)], A[np.ix_(k_idx, r_idx)]
    fk = np.asarray(f, float).ravel()[k_idx]
    xk = np.linalg.solve(Akk + Akr @ G, fk - Akr @ (H @ g))
    x = np.zeros(grid.size)
    x[k_idx] = xk
    x[r_idx] = G @ xk + H @ g
    return x.reshape(grid.shape)


# ----------------------------------------------------------------------------
# homogenised response (Sec. 3.3, effective conductivity and the contrast study)
# ----------------------------------------------------------------------------

def volume_average(v: np.ndarray, grid: Grid) -> float:
    """<v> = (1/|Omega|) integral of v, by the tensor Clenshaw-Curtis rule on
    the CGL nodes (exact for polynomials of per-axis degree <= N)."""
    w = [cc_weights(grid.n[a] - 1, grid.lo[a], grid.hi[a]) if a < grid.dim else np.ones(1)
         for a in range(3)]
    vol = 1.0
    for a in grid.axes:
        vol *= grid.hi[a] - grid.lo[a]
    return float(np.einsum("k,j,i,kji->", w[2], w[1], w[0], np.asarray(v, float)) / vol)


def effective_conductivity(u: np.ndarray, K: np.ndarray, grid: Grid, G: float, axis: int = 0) -> float:
    """K_num = -<q_a> / G with the flux q = -K grad u (Sec. 3.3): the volume
    average of K d_a u over the imposed macroscopic gradient G.  The paper
    writes q_y and L_y while imposing u = -+g on the x faces; the gradient is
    taken along the axis that carries the Dirichlet data (here ``axis``), with
    G = 2 g / L_axis."""
    return volume_average(np.asarray(K, float) * grad(u, grid, axis), grid) / G


def maxwell_estimate(k_m: float, k_i: float, phi: float) -> float:
    """Maxwell's dilute estimate of the effective conductivity of spheres of
    conductivity k_i at volume fraction phi in a matrix k_m (Sec. 3.3)."""
    return k_m * (2 * k_m + k_i + 2 * phi * (k_i - k_m)) / (2 * k_m + k_i - phi * (k_i - k_m))


# ----------------------------------------------------------------------------
# Newton's method for a temperature-dependent conductivity (Sec. 2.3 Newton,
# Sec. 3.4): k(T) = K0 / (1 + alpha T)
# ----------------------------------------------------------------------------

def reciprocal_law(K0, T, alpha: float):
    """k(T) = K0 / (1 + alpha T) and dk/dT = -alpha K0 / (1 + alpha T)^2
    (the normalised reciprocal law of Sec. 3.4, with a nodal prefactor K0)."""
    d = 1.0 + alpha * np.asarray(T, float)
    k = np.asarray(K0, float) / d
    return k, -alpha * k / d


def newton_residual(T, K0, alpha: float, b, grid: Grid) -> np.ndarray:
    """R(T) = A(k(T)) T - b: the collocation rows with the conductivity
    evaluated at T, boundary rows included (flux rows carry k(T_p))."""
    k, _ = reciprocal_law(K0, T, alpha)
    return apply(np.asarray(T, float), k, grid) - np.asarray(b, float)


def jacobian_apply(dT, T, K0, alpha: float, grid: Grid) -> np.ndarray:
    """J(T) dT, the derivative of R at T along dT (Sec. 3.4, Jacobian action
    div(-k grad dT - k' dT grad T)): A(k(T)) dT plus, with h = k'(T) dT,
    -sum_a D_a (h D_a T) on interior rows and -s h_p (D_a T)_p on flux rows."""
    T = np.asarray(T, float)
    dT = np.asarray(dT, float)
    k, dk = reciprocal_law(K0, T, alpha)
    h = dk * dT
    out = apply(dT, k, grid)
    own = owners(grid)
    extra = np.zeros(grid.shape)
    for a in grid.axes:
        extra -= grad(h * grad(T, grid, a), grid, a)
    out[own < 0] += extra[own < 0]
    for f in range(2 * grid.dim):
        if grid.bc[f] != FLUX:
            continue
        m = own == f
        a, side = divmod(f, 2)
        s = 1.0 if side == 1 else -1.0
        out[m] += -s * h[m] * grad(T, grid, a)[m]
    return out


def linearized_apply(du, K, C, grid: Grid) -> np.ndarray:
    """The linearised operator with given coefficient fields: A(K) du, plus
    -sum_a D_a (C_a du) on interior rows and -s C_a,p du_p on flux rows of
    axis a.  jacobian_apply is this operator at K = k(T), C_a = k'(T) d_a T."""
    du = np.asarray(du, float)
    out = apply(du, K, grid)
    own = owners(grid)
    extra = np.zeros(grid.shape)
    for a in grid.axes:
        extra -= grad(np.asarray(C[a], float) * du, grid, a)
    out[own < 0] += extra[own < 0]
    for f in range(2 * grid.dim):
        if grid.bc[f] != FLUX:
            continue
        m = own == f
        a, side = divmod(f, 2)
        s = 1.0 if side == 1 else -1.0
        out[m] += -s * (np.asarray(C[a], float) * du)[m]
    return out


def _jacobian_dense(T, K0, alpha: float, grid: Grid) -> np.ndarray:
    """J(T) assembled column by column from jacobian_apply (tiny grids)."""
    n = grid.size
    J = np.zeros((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[c] = 1.0
        J[:, c] = jacobian_apply(e.reshape(grid.shape), T, K0, alpha, grid).ravel()
        e[c] = 0.0
    return J


def newton_solve(K0, alpha: float, b, grid: Grid, T0=None, tol: float = 1e-13, maxit: int = 30,
                 lin_rtol: float = 1e-13):
    """Newton's method (Sec. 2.3 and Sec. 3.4): J(T^m) dT = -R(T^m),
    T^{m+1} = T^m + dT, until ||dT||_inf <= tol max(||T||_inf, 1).  Each
    linear solve is direct on tiny grids, else GMRES on the Jacobian action
    preconditioned by the constant-coefficient inverse at the geometric mean
    of k(T^m).  Returns (T, info) with the iteration count and the history of
    ||dT||_inf."""
    T = np.zeros(grid.shape) if T0 is None else np.array(T0, float)
    hist = []
    it = 0
    for it in range(1, maxit + 1):
        R = newton_residual(T, K0, alpha, b, grid)
        if grid.size <= 4096:
            J = _jacobian_dense(T, K0, alpha, grid)
            s = 1.0 / np.abs(J).max(axis=1)
            dT = np.linalg.solve(J * s[:, None], -R.ravel() * s).reshape(grid.shape)
        else:
            from .precond import FDMPreconditioner, geometric_mean
            k, _ = reciprocal_law(K0, T, alpha)
            M = FDMPreconditioner(grid, geometric_mean(k))
            dT, _ = gmres(lambda v: M(jacobian_apply(v, T, K0, alpha, grid)), M(-R),
                          rtol=lin_rtol, restart=50)
        T = T + dT
        step = float(np.abs(dT).max())
        hist.append(step)
        if step <= tol * max(float(np.abs(T).max()), 1.0):
            break
    return T, {"iterations": it, "history": hist}
