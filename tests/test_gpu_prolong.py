"""Parity of the CUDA modal prolongation (DCT-I, zero padding, inverse
DCT-I) with the oracle's barycentric interpolation, exactness on
polynomials, and the hierarchical solve (Alg. 4) against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_prolong_exact_for_polynomials_of_degree_N():
    import paper_2606_21410_b300 as P
    nc, nf = (9, 17, 33), (17, 33, 65)
    lo, hi = (0, -1, -2), (1, 1, 2)
    pc, pf = P.Plan(nc, lo, hi), P.Plan(nf, lo, hi)
    coeffs = {(8, 0, 0): 1.0, (3, 16, 0): -0.5, (0, 2, 32): 0.25, (8, 16, 32): 1e-3}
    Xc, Yc, Zc = pc.mesh()
    Xf, Yf, Zf = pf.mesh()
    uc = W.polynomial_3d(coeffs, Xc, Yc, Zc)[0]
    uf = W.polynomial_3d(coeffs, Xf, Yf, Zf)[0]
    got = P.prolong(pc, pf, _dev(uc)).cpu().numpy()
    assert np.abs(got - uf).max() < 1e-12 * np.abs(uf).max()
    # coarse nodes nest in the fine grid: injection returns the coarse field
    assert np.abs(got[::2, ::2, ::2] - uc).max() < 1e-13 * np.abs(uc).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nc", [(33, 33, 33), (65, 17, 9), (129, 5, 5)])
def test_prolong_matches_oracle_barycentric(nc, dtype):
    import paper_2606_21410_b300 as P
    nf = tuple(2 * (v - 1) + 1 for v in nc)
    gc, gf = O.Grid(nc), O.Grid(nf)
    pc, pf = P.Plan(nc), P.Plan(nf)
    u = W.random_field(gc.shape, 21)
    ref = O.prolong(u, gc, gf)
    got = P.prolong(pc, pf, _dev(u, dtype)).double().cpu().numpy()
    tol = 1e-12 if dtype == torch.float64 else 5e-6
    assert _rel(got, ref) < tol


def test_prolong_1d_2d_and_full_size_sampled():
    import paper_2606_21410_b300 as P
    for nc in ((33,), (17, 65)):
        nf = tuple(2 * (v - 1) + 1 for v in nc)
        gc, gf = O.Grid(nc), O.Grid(nf)
        u = W.random_field(gc.shape, 22)
        got = P.prolong(P.Plan(nc), P.Plan(nf), _dev(u)).cpu().numpy()
        assert _rel(got, O.prolong(u, gc, gf)) < 1e-12
    # 129^3 -> 257^3: sampled fine values against per-point barycentric sums
    gc = O.Grid((129,) * 3)
    Xc, Yc, Zc = gc.mesh()
    u = np.sin(3 * Xc + Yc) * np.exp(Zc) + 0.1 * W.random_field(gc.shape, 23)
    got = P.prolong(P.Plan((129,) * 3), P.Plan((257,) * 3), _dev(u)).cpu().numpy()
    Pm = O.barycentric_matrix(128, 256)
    rng = W.rng(24)
    for _ in range(50):
        k, j, i = (int(v) for v in rng.integers(0, 257, size=3))
        ref = np.einsum("a,b,c,abc->", Pm[k], Pm[j], Pm[i], u)
        assert abs(got[k, j, i] - ref) < 1e-12 * np.abs(u).max()


def test_hierarchy_spheres_matches_oracle():
    """Alg. 4 on the seeded sphere microstructure (contrast 100), 9^3 -> 17^3
    -> 33^3, mixed precision, against the oracle's own hierarchy (its
    barycentric prolongation and preconditioned GMRES, K and b sampled on
    its own grids): every level's solution and every level's refinement
    indicator e_ref."""
    import paper_2606_21410_b300 as P
    bc = [0, 0, 1, 1, 1, 1]
    sp = W.sphere_packing(0)
    xbc = lambda X, Y, Z: (X, (np.ones_like(X), 0 * X, 0 * X), 0 * X)
    plans, Ks, bs = [], [], []
    grids, Ko, bo = [], [], []
    for n in (9, 17, 33):
        p = P.Plan((n,) * 3, bc=bc)
        X, Y, Z = p.mesh()
        K = W.two_phase_conductivity(X, Y, Z, sp, 1.0, 100.0)
        faces = W.face_values(bc, p.nodes(0), p.nodes(1), p.nodes(2), xbc)
        b = p.rhs(_dev(np.zeros(p.shape)), [_dev(f) for f in faces])
        plans.append(p)
        Ks.append(_dev(K))
        bs.append(b)
        g = O.Grid((n,) * 3, bc=bc)
        Xo, Yo, Zo = g.mesh()
        grids.append(g)
        Ko.append(W.two_phase_conductivity(Xo, Yo, Zo, sp, 1.0, 100.0))
        bo.append(O.rhs(np.zeros(g.shape), W.face_values(bc, g.nodes(0), g.nodes(1), g.nodes(2), xbc), g))
    us, infos, eref = P.solve_hierarchy(plans, Ks, bs, mode=1, rtol=1e-12)
    uo, io, eref_o = O.solve_hierarchy(Ko, bo, grids, rtol=1e-13)
    for lvl in range(3):
        assert _rel(us[lvl].cpu().numpy(), uo[lvl]) < 1e-10, lvl
    assert eref[0] == 0.0 and eref_o[0] == 0.0
    for lvl in (1, 2):
        # e_ref differences of solutions that agree to 1e-10 relative
        assert abs(eref[lvl] - eref_o[lvl]) <= 1e-8 * eref_o[lvl], (lvl, eref[lvl], eref_o[lvl])
    assert eref[2] < 0.5


def test_repeated_fp64_hierarchies_on_the_same_plans():
    """Regression: the prolongation's intermediate arrays (after the x and y
    passes) must fit their scratch; an undersized scratch wrote past its end
    and broke later FP64 solves on the fine plan.  Two FP64 hierarchies at
    different tolerances on the same plans, then a solve on the fine plan,
    all converge and agree with a fresh plan."""
    import paper_2606_21410_b300 as P
    bc = [0, 0, 1, 1, 1, 1]
    plans = [P.Plan((n,) * 3, bc=bc) for n in (33, 65, 129)]
    pf = plans[-1]
    X, Y, Z = pf.mesh()
    K = _dev(W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 10.0))
    faces = W.face_values(bc, pf.nodes(0), pf.nodes(1), pf.nodes(2),
                          lambda X, Y, Z: (X, (np.ones_like(X), 0 * X, 0 * X), 0 * X))
    b = pf.rhs(_dev(np.zeros(pf.shape)), [_dev(f) for f in faces])
    for rtol in (1e-12, 1e-11):
        u, infos, _ = P.solve_hierarchy_fine(plans, K, b, mode=0, rtol=rtol)
        assert all(i["status"] == 0 for i in infos), infos
    u2, info = pf.solve(K, b, mode=0, rtol=1e-12)
    assert info["status"] == 0 and info["iterations"] < 200, info
    u3, _ = P.Plan((129,) * 3, bc=bc).solve(K, b, mode=0, rtol=1e-12)
    assert _rel(u2.cpu().numpy(), u3.cpu().numpy()) < 1e-10
