"""Pins of the oracle's constant-coefficient preconditioner: M^{-1} r equals
the dense direct solve of the constant-K system on small grids for every
boundary pattern and dimension, and the preconditioned GMRES reproduces
direct solves of heterogeneous problems.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("bc", [list(t) for t in itertools.product([0, 1], repeat=6)][:-1:5])
def test_fdm_is_exact_inverse_of_constant_K_operator(bc):
    g = O.Grid((7, 6, 5), lo=(0, -1, 0), hi=(1, 1, 3), bc=bc)
    kref = 1.7
    M = O.FDMPreconditioner(g, kref)
    r = W.random_field(g.shape, 7)
    x = M(r)
    ref = O.solve_direct(np.full(g.shape, kref), r, g)
    assert np.allclose(x, ref, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("n,bc", [((9,), [1, 0, 0, 0, 0, 0]), ((9, 7), [1, 1, 0, 1, 0, 0]),
                                  ((9, 7), [0, 1, 1, 1, 0, 0])])
def test_fdm_lower_dimensions(n, bc):
    g = O.Grid(n, bc=bc)
    M = O.FDMPreconditioner(g, 0.5)
    r = W.random_field(g.shape, 8)
    ref = O.solve_direct(np.full(g.shape, 0.5), r, g)
    assert np.allclose(M(r), ref, atol=1e-10 * np.abs(ref).max())


def test_preconditioned_gmres_matches_direct_on_spheres():
    bc = [0, 0, 1, 1, 1, 1]
    g = O.Grid((13, 11, 12), bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 100.0)
    b = W.random_field(g.shape, 9)
    u, info = O.solve_preconditioned(K, b, g, rtol=1e-14)
    ud = O.solve_direct(K, b, g)
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-11
    assert info["iterations"] < 300


@pytest.mark.parametrize("n,bc", [((5, 4, 6), [0, 1, 1, 0, 2, 1]), ((5, 4, 6), [1, 0, 2, 2, 0, 1]),
                                  ((5, 4, 6), [2, 0, 1, 1, 1, 1]), ((7, 5), [1, 0, 2, 0, 0, 0]),
                                  ((9,), [2, 0, 0, 0, 0, 0])])
def test_fdm_transpose_is_dense_transpose(n, bc):
    """M^{-T} y from the transposed steps equals the transpose of the dense
    matrix of M^{-1} (built column by column), flux rows included."""
    g = O.Grid(n, bc=bc)
    M = O.FDMPreconditioner(g, 1.3)
    e = np.zeros(g.size)
    Md = np.zeros((g.size, g.size))
    for c in range(g.size):
        e[c] = 1.0
        Md[:, c] = M(e.reshape(g.shape)).ravel()
        e[c] = 0.0
    y = W.random_field(g.shape, 10)
    ref = Md.T @ y.ravel()
    assert np.abs(M.transpose(y).ravel() - ref).max() < 1e-13 * np.abs(ref).max()


def test_preconditioned_adjoint_solve_matches_direct():
    bc = [0, 0, 1, 1, 2, 1]
    g = O.Grid((13, 11, 12), bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 100.0)
    c = W.random_field(g.shape, 11)
    lam, info = O.adjoint_solve_preconditioned(K, c, g, rtol=1e-14)
    ref = O.adjoint_solve_direct(K, c, g)
    assert np.linalg.norm(lam - ref) / np.linalg.norm(ref) < 1e-11
