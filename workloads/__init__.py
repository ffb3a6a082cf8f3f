"""Seeded synthetic inputs for the Chebyshev-collocation diffusion problems.

This module only *generates data*: analytic fields evaluated at points the
caller supplies, random fields, and sphere microstructures.  It holds none of
the collocation method's arithmetic (no nodes, no differentiation, no
transforms, no boundary-row logic): both the FP64 CPU oracle and the CUDA path
take their inputs from here, each evaluating on the node coordinates it
computes itself.

Conventions
-----------
* Fields are numpy arrays shaped ``(nz, ny, nx)`` (x fastest); unused axes of
  1-D/2-D problems have length 1.
* A *face* is named by axis and side: face id ``2*axis + side`` with side 0 the
  low coordinate (``lo``) and side 1 the high coordinate (``hi``): ids 0..5 are
  x-, x+, y-, y+, z-, z+.
* ``face_values`` lays out the data of face ``(axis, side)`` as the field's
  array with that axis removed, in the order of the node arrays given.

Workloads (synthetic stand-ins for the paper's analytic test problems; the
paper uses no dataset):
* 1-D Poisson with ``u = exp(x) sin(3x)``;
* the paper's 1-D problem ``u'' = exp(4x)`` (Sec. 3.1) and 3-D manufactured
  solution ``exp(x+y+z) + x^2 + 2y - z^2`` (Sec. 3.2);
* 3-D ``u = sin(pi x/2) cos(pi y) exp(z)``;
* two-phase sphere microstructures by random sequential addition (Sec. 3.3
  uses one sphere; the dense packing is a synthetic microstructure of the
  same kind);
* a lognormal conductivity from a Gaussian random field (random Fourier
  features).
"""
from __future__ import annotations

import math

import numpy as np

DIRICHLET = 0
NEUMANN = 1
FLUX = 2


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed``."""
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# random fields for parity tests
# ----------------------------------------------------------------------------

def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform i.i.d. values in [lo, hi), float64."""
    return rng(seed).uniform(lo, hi, size=shape)


def random_positive_field(shape, seed: int, kmin: float = 0.5, kmax: float = 2.0) -> np.ndarray:
    """Uniform i.i.d. conductivity values in [kmin, kmax), float64."""
    return rng(seed).uniform(kmin, kmax, size=shape)


def random_bc_types(seed: int, dim: int = 3, require_dirichlet: bool = True) -> list[int]:
    """Six per-face BC types (unused axes get Dirichlet); at least one Dirichlet
    face among the active ones when ``require_dirichlet``."""
    g = rng(seed)
    while True:
        t = [int(v) for v in g.integers(0, 2, size=6)]
        for a in range(dim, 3):
            t[2 * a] = t[2 * a + 1] = DIRICHLET
        if not require_dirichlet or any(t[f] == DIRICHLET for f in range(2 * dim)):
            return t


def mesh(x, y, z):
    """Broadcast 1-D coordinate arrays to (nz, ny, nx) grids (Z, Y, X)."""
    Z, Y, X = np.meshgrid(np.asarray(z, float), np.asarray(y, float), np.asarray(x, float),
                          indexing="ij")
    return X, Y, Z


# ----------------------------------------------------------------------------
# analytic manufactured solutions: each returns (u, (ux, uy, uz), lap)
# ----------------------------------------------------------------------------

def exp_sin3_1d(X, Y, Z):
    """u = exp(x) sin(3x) (1-D; Y, Z ignored)."""
    e = np.exp(X)
    s, c = np.sin(3 * X), np.cos(3 * X)
    u = e * s
    ux = e * (s + 3 * c)
    uxx = e * (s + 3 * c) + e * (3 * c - 9 * s)
    zero = np.zeros_like(X)
    return u, (ux, zero, zero), uxx


def paper_exp4x_1d(X, Y, Z):
    """u = (exp(4x) - sinh(4) x - cosh(4)) / 16, u'' = exp(4x) (paper Sec. 3.1)."""
    u = (np.exp(4 * X) - math.sinh(4.0) * X - math.cosh(4.0)) / 16.0
    ux = (4 * np.exp(4 * X) - math.sinh(4.0)) / 16.0
    uxx = np.exp(4 * X)
    zero = np.zeros_like(X)
    return u, (ux, zero, zero), uxx


def paper_exp_poly_3d(X, Y, Z):
    """u = exp(x+y+z) + x^2 + 2y - z^2, lap u = 3 exp(x+y+z) (paper Sec. 3.2)."""
    e = np.exp(X + Y + Z)
    u = e + X ** 2 + 2 * Y - Z ** 2
    return u, (e + 2 * X, e + 2.0, e - 2 * Z), 3 * e


def sin_cos_exp_3d(X, Y, Z):
    """u = sin(pi x/2) cos(pi y) exp(z); lap u = (1 - 5 pi^2/4) u."""
    a = 0.5 * math.pi
    sx, cx = np.sin(a * X), np.cos(a * X)
    sy, cy = np.sin(math.pi * Y), np.cos(math.pi * Y)
    ez = np.exp(Z)
    u = sx * cy * ez
    grad = (a * cx * cy * ez, -math.pi * sx * sy * ez, u)
    lap = (1.0 - 1.25 * math.pi ** 2) * u
    return u, grad, lap


def paper_nonlinear_3d(X, Y, Z, alpha: float = 0.5):
    """The manufactured nonlinear heat problem of Sec. 3.4 on (0,1)^3:
    Phi = sin(pi x) sin(pi y) sin(pi z), T = (exp(alpha Phi) - 1) / alpha solves
    -div(k(T) grad T) = f with k(T) = 1 / (1 + alpha T) and f = -lap Phi =
    3 pi^2 Phi.  Returns (T, grad T, f) -- the third entry is the source term
    of this nonlinear problem, not a Laplacian."""
    sx, sy, sz = np.sin(np.pi * X), np.sin(np.pi * Y), np.sin(np.pi * Z)
    cx, cy, cz = np.cos(np.pi * X), np.cos(np.pi * Y), np.cos(np.pi * Z)
    phi = sx * sy * sz
    e = np.exp(alpha * phi)
    T = (e - 1.0) / alpha
    grad = (e * np.pi * cx * sy * sz, e * np.pi * sx * cy * sz, e * np.pi * sx * sy * cz)
    return T, grad, 3.0 * np.pi ** 2 * phi


def reciprocal_conductivity(alpha: float = 0.5):
    """k(T) = 1 / (1 + alpha T) as a face-data helper ``k_fn(X, Y, Z, T)``."""
    return lambda X, Y, Z, T: 1.0 / (1.0 + alpha * T)


def polynomial_3d(coeffs: dict, X, Y, Z):
    """u = sum c * x^i y^j z^k for ``coeffs = {(i, j, k): c}``; returns u, grad, lap."""
    u = np.zeros_like(X)
    gx, gy, gz, lap = (np.zeros_like(X) for _ in range(4))
    for (i, j, k), c in coeffs.items():
        px, py, pz = X ** i, Y ** j, Z ** k
        u += c * px * py * pz
        if i:
            gx += c * i * X ** (i - 1) * py * pz
        if j:
            gy += c * j * px * Y ** (j - 1) * pz
        if k:
            gz += c * k * px * py * Z ** (k - 1)
        if i >= 2:
            lap += c * i * (i - 1) * X ** (i - 2) * py * pz
        if j >= 2:
            lap += c * j * (j - 1) * px * Y ** (j - 2) * pz
        if k >= 2:
            lap += c * k * (k - 1) * px * py * Z ** (k - 2)
    return u, (gx, gy, gz), lap


def face_values(bc, x, y, z, u_fn, dim: int = 3, k_fn=None):
    """Boundary data of the analytic field ``u_fn`` on the six faces.

    Dirichlet faces carry ``u``; Neumann faces carry the outward normal
    derivative ``n . grad u`` (``-d_a u`` on the low face of axis a, ``+d_a u`` on
    the high face); flux faces (type 2) carry ``-k n . grad u`` with
    ``k = k_fn(X, Y, Z, u)``.  The face of axis a lies at ``min`` (side 0) or ``max``
    (side 1) of that axis' node array.  Returns a list of six arrays shaped
    like a (nz, ny, nx) field with axis a removed; faces of unused axes are
    returned as zero arrays of that shape.
    """
    axes = [np.asarray(x, float), np.asarray(y, float), np.asarray(z, float)]
    out = []
    for f in range(6):
        a, side = divmod(f, 2)
        coords = list(axes)
        npax = 2 - a
        if a >= dim:
            shp = [len(axes[2]), len(axes[1]), len(axes[0])]
            del shp[npax]
            out.append(np.zeros(shp))
            continue
        coords[a] = np.array([axes[a].max() if side else axes[a].min()])
        X, Y, Z = mesh(*coords)
        u, grad, _ = u_fn(X, Y, Z)
        if bc[f] == DIRICHLET:
            v = u
        else:
            v = grad[a] if side else -grad[a]
            if bc[f] == FLUX:
                v = -k_fn(X, Y, Z, u) * v
        out.append(np.take(v, 0, axis=npax).copy())
    return out


# ----------------------------------------------------------------------------
# two-phase sphere microstructures
# ----------------------------------------------------------------------------

def sphere_packing(seed: int = 0, rmin: float = 0.08, rmax: float = 0.15,
                   volume_fraction: float = 0.2, lo: float = -1.0, hi: float = 1.0,
                   max_tries: int = 2_000_000) -> np.ndarray:
    """Non-overlapping spheres by random sequential addition.

    Radii uniform in [rmin, rmax), centres uniform in [lo + r, hi - r]^3 (the
    sphere lies fully inside the box), a candidate is rejected when it
    overlaps an accepted sphere (centre distance < r_i + r_j); stops once the
    summed sphere volume reaches ``volume_fraction`` of the box.  Returns an
    (m, 4) array of (cx, cy, cz, r).
    """
    g = rng(seed)
    target = volume_fraction * (hi - lo) ** 3
    spheres = np.zeros((0, 4))
    vol = 0.0
    tries = 0
    while vol < target:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("sphere packing did not reach the volume fraction")
        r = g.uniform(rmin, rmax)
        c = g.uniform(lo + r, hi - r, size=3)
        if len(spheres):
            d = np.sqrt(((spheres[:, :3] - c) ** 2).sum(axis=1))
            if np.any(d < spheres[:, 3] + r):
                continue
        spheres = np.vstack([spheres, np.r_[c, r]])
        vol += 4.0 / 3.0 * math.pi * r ** 3
    return spheres


def single_sphere(center=(0.5, 0.5, 0.5), radius: float = 0.2) -> np.ndarray:
    """One sphere (the centred inclusion of the unit-cell study, Sec. 3.3)."""
    return np.array([[center[0], center[1], center[2], radius]], dtype=float)


def corner_spheres(radius: float = 0.2, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Spheres centred on the eight corners of the box [lo, hi]^3: inside the
    box they form the corner-inclusion arrangement of Sec. 3.3, with the same
    inclusion volume as one sphere of that radius."""
    c = [lo, hi]
    return np.array([[x, y, z, radius] for x in c for y in c for z in c], dtype=float)


def two_phase_conductivity(X, Y, Z, spheres: np.ndarray, k_matrix: float, k_incl: float) -> np.ndarray:
    """k = k_incl at points inside (inclusive) any sphere, else k_matrix.

    X, Y, Z are (nz, ny, nx) tensor-grid coordinates; each sphere is tested
    only on the sub-block of grid lines that its bounding box covers."""
    x, y, z = X[0, 0, :], Y[0, :, 0], Z[:, 0, 0]
    inside = np.zeros(X.shape, dtype=bool)

    def span(c, r, t):
        idx = np.nonzero((t >= c - r) & (t <= c + r))[0]
        return (idx.min(), idx.max() + 1) if idx.size else (0, 0)

    for cx, cy, cz, r in spheres:
        i0, i1 = span(cx, r, x)
        j0, j1 = span(cy, r, y)
        k0, k1 = span(cz, r, z)
        if i1 <= i0 or j1 <= j0 or k1 <= k0:
            continue
        d2 = ((x[i0:i1] - cx) ** 2)[None, None, :] + ((y[j0:j1] - cy) ** 2)[None, :, None] \
            + ((z[k0:k1] - cz) ** 2)[:, None, None]
        inside[k0:k1, j0:j1, i0:i1] |= d2 <= r * r
    return np.where(inside, k_incl, k_matrix).astype(float)


# ----------------------------------------------------------------------------
# lognormal conductivity from a Gaussian random field
# ----------------------------------------------------------------------------

def gaussian_rff(seed: int, n_features: int = 512, corr_len: float = 0.2, dim: int = 3):
    """Random Fourier features of a unit-variance Gaussian field with covariance
    exp(-|r|^2 / (2 corr_len^2)): frequencies ~ N(0, corr_len^-2 I), phases ~ U(0, 2 pi)."""
    g = rng(seed)
    omega = g.normal(0.0, 1.0 / corr_len, size=(n_features, dim))
    phase = g.uniform(0.0, 2 * math.pi, size=n_features)
    return omega, phase


def eval_rff(omega: np.ndarray, phase: np.ndarray, X, Y, Z) -> np.ndarray:
    """g(x) = sqrt(2/M) sum_m cos(omega_m . x + phase_m) on the grid."""
    M = len(phase)
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)[:, : omega.shape[1]]
    acc = np.zeros(pts.shape[0])
    for s in range(0, M, 64):
        arg = pts @ omega[s:s + 64].T + phase[s:s + 64]
        acc += np.cos(arg).sum(axis=1)
    return (math.sqrt(2.0 / M) * acc).reshape(X.shape)


def lognormal_conductivity(X, Y, Z, seed: int, sigma: float = 0.5, corr_len: float = 0.2,
                           n_features: int = 512) -> np.ndarray:
    """K0 = exp(sigma * g) with g the unit-variance Gaussian field above."""
    omega, phase = gaussian_rff(seed, n_features, corr_len)
    return np.exp(sigma * eval_rff(omega, phase, X, Y, Z))


def batch_sizes(seed: int = 1, count: int = 16, nmin: int = 33, nmax: int = 97) -> list[int]:
    """Uniform random points-per-axis for a batch of uneven instances."""
    return [int(v) for v in rng(seed).integers(nmin, nmax + 1, size=count)]
