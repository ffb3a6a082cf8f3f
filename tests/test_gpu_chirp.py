"""The transform route for any N (Sec. 2.2: the DCT-I of a line as the DFT
of its even extension, here of length 2N that need not be a power of two,
evaluated by Bluestein's chirp-z convolution) against the FP64 oracle:
first derivatives and their transposes, the operator apply with every
boundary type, the adjoint apply, the Jacobian action, solves, and modal
prolongation N -> 2N (Sec. 2.3.3) with a two-level hierarchy, on axis sizes
whose n - 1 is not a power of two.  The axes above the dense route's
n <= 129 (n = 131, 201) have no other route.

Tolerances: relative L2 error against the oracle with uniform random
inputs.  The FP64 rounding of a line derivative grows with N on both
transform forms (derivatives of random data are dominated by the top modes;
measured on B300: power-of-two N = 256 4.2e-14, chirp N = 99 2.2e-14, i.e.
at most 1.0 N eps for a derivative and 1.7 N eps for an apply or adjoint
apply, eps = 2^-52), so the FP64 bounds are 5 N eps (derivatives) and
8 N eps (applies) with N the largest axis degree.  FP32: measured at most
5.9e-7 for applies and 2.4e-7 for derivatives, bound 1e-6."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -52
TRANSFORM = 0


def _tol(dtype, n, per_n):
    """FP64: per_n * N * eps with N the largest axis degree; FP32: 1e-6."""
    if dtype == torch.float32:
        return 1e-6
    return per_n * (max(n) - 1) * EPS64


def _plan(n, lo=(-1, -1, -1), hi=(1, 1, 1), bc=(0,) * 6, force=True):
    import paper_2606_21410_b300 as P
    p = P.Plan(n, lo, hi, bc)
    if force:
        for a in range(3):
            p.set_route(a, TRANSFORM)
    return p


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# (n, lo, hi): N = 12, 6, 200 / 2, 5, 99 / 129, 10, 4 (the last one a power of two)
DERIV_CASES = [
    ((13, 7, 201), (-1, 0, 0.5), (1, 2, 3.0)),
    ((3, 6, 100), (0, 0, 0), (1, 1, 1)),
    ((130, 11, 5), (-2, -1, 0), (2, 1, 0.25)),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", DERIV_CASES)
def test_chirp_deriv_and_transpose_match_oracle(case, dtype):
    n, lo, hi = case
    g = O.Grid(n, lo, hi)
    p = _plan(n, lo, hi)
    u = W.random_field(g.shape, 301)
    ud = _dev(u, dtype)
    for a in range(3):
        assert p.route(a) == TRANSFORM
        tol = _tol(dtype, n, 5)
        ref = O.grad(u, g, a)
        got = p.deriv(ud, a).double().cpu().numpy()
        assert _rel(got, ref) < tol, (a, _rel(got, ref))
        refT = np.moveaxis(np.tensordot(g.D(a).T, u, axes=([1], [2 - a])), 0, 2 - a)
        gotT = p.deriv(ud, a, transpose=True).double().cpu().numpy()
        assert _rel(gotT, refT) < tol, (a, "T", _rel(gotT, refT))


def test_chirp_deriv_is_exact_on_polynomials():
    """A degree-N polynomial is differentiated exactly by the collocation
    derivative, for every N the chirp form covers (N = 2 .. 256)."""
    for N in [2, 3, 5, 6, 7, 9, 15, 17, 31, 33, 63, 65, 100, 127, 129, 200, 255]:
        p = _plan((N + 1, 1, 1), force=False)
        p.set_route(0, TRANSFORM)
        x = p.nodes(0)
        rng = np.random.default_rng(N)
        c = rng.standard_normal(N + 1)
        f = np.polynomial.chebyshev.chebval(x, c)
        df = np.polynomial.chebyshev.chebval(x, np.polynomial.chebyshev.chebder(c))
        got = p.deriv(_dev(f[None, None, :]), 0).cpu().numpy()[0, 0]
        assert np.abs(got - df).max() <= 1e-13 * np.abs(df).max() * max(1, N / 16), (N, np.abs(got - df).max())


BC_PATTERNS = [[0, 0, 0, 0, 0, 0], [0, 1, 1, 0, 1, 1], [2, 0, 1, 2, 0, 2], [0, 2, 2, 2, 2, 2]]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("bc", BC_PATTERNS)
def test_chirp_apply_and_adjoint_match_oracle(bc, dtype):
    n = (21, 131, 6)
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    u = W.random_field(g.shape, 302)
    K = W.random_positive_field(g.shape, 303)
    tol = _tol(dtype, n, 8)
    ref = O.apply(u, K, g)
    got = p.apply(_dev(K, dtype), _dev(u, dtype)).double().cpu().numpy()
    assert _rel(got, ref) < tol, _rel(got, ref)
    own = O.owners(g)
    for kind in (0, 1, 2):
        mask = np.isin(own, [f for f in range(6) if bc[f] == kind])
        if mask.any():
            e = np.abs(got[mask] - ref[mask]).max() / np.abs(ref[mask]).max()
            if kind == 0 and dtype == torch.float64:
                assert e == 0.0, e  # Dirichlet rows copy u
            else:
                assert e < tol, (kind, e)
    refT = O.adjoint_apply(u, K, g)
    gotT = p.adjoint_apply(_dev(K, dtype), _dev(u, dtype)).double().cpu().numpy()
    assert _rel(gotT, refT) < tol, _rel(gotT, refT)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_chirp_jacobian_apply_matches_oracle(dtype):
    n, bc = (10, 19, 7), [0, 2, 2, 1, 0, 0]
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    K = W.random_positive_field(g.shape, 304)
    C = [W.random_field(g.shape, 305 + a) for a in range(3)]
    du = W.random_field(g.shape, 308)
    ref = O.linearized_apply(du, K, C, g)
    got = p.jacobian_apply(_dev(K, dtype), [_dev(c, dtype) for c in C], _dev(du, dtype)).double().cpu().numpy()
    assert _rel(got, ref) < _tol(dtype, n, 8), _rel(got, ref)


def test_chirp_route_agrees_with_dense_route():
    """Both routes evaluate the same collocation derivative."""
    n = (45, 23, 11)
    g = O.Grid(n)
    pt = _plan(n)
    pd = _plan(n, force=False)
    for a in range(3):
        pd.set_route(a, 1)
    u = _dev(W.random_field(g.shape, 309))
    K = _dev(W.random_positive_field(g.shape, 310))
    at = pt.apply(K, u).cpu().numpy()
    ad = pd.apply(K, u).cpu().numpy()
    assert _rel(at, ad) < _tol(torch.float64, n, 8), _rel(at, ad)


def test_default_routes_with_chirp_axes():
    """Without a forced route: power-of-two N takes the plain transform,
    other N up to n = 129 the dense route, larger ones the chirp transform."""
    p = _plan((201, 17, 12), force=False)
    assert [p.route(a) for a in range(3)] == [TRANSFORM, TRANSFORM, 1]


@pytest.mark.parametrize("mode", [0, 1])
def test_chirp_solve_matches_oracle(mode):
    """rtol 1e-11: with N = 130 and Neumann / flux faces the interior rows
    scale like N^4 = 3e8, and the attainable preconditioned residual in FP64
    is near 1e-12 (the oracle's own GMRES ends at 8e-13), so 1e-12 sits on
    the rounding floor.  The error bound is kappa(M^-1 A) ~ 10 (contrast 10)
    times rtol, with a factor 5 margin."""
    n, bc = (131, 5, 4), [0, 1, 2, 0, 1, 0]
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0, 0.2, 0.4, 0.2), 1.0, 10.0)
    b = W.random_field(g.shape, 311)
    ud = O.solve_direct(K, b, g)
    u, info = p.solve(_dev(K), _dev(b), mode=mode, rtol=1e-11)
    assert _rel(u.cpu().numpy(), ud) < 5e-10, info


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nc", [(7, 4, 13), (5, 7, 9), (101, 5, 4)])
def test_chirp_prolongation_matches_oracle(nc, dtype):
    """Coarse N = (6, 3, 12), (4, 6, 8) (plain and chirp axes mixed),
    (100, 4, 3); fine N = 2 N.  The oracle prolongs by barycentric
    interpolation of the coarse interpolant."""
    import paper_2606_21410_b300 as P
    nf = tuple(2 * (m - 1) + 1 for m in nc)
    lo, hi = (-1, 0, 0.5), (1, 2, 3.0)
    gc, gf = O.Grid(nc, lo, hi), O.Grid(nf, lo, hi)
    pc, pf = _plan(nc, lo, hi, force=False), _plan(nf, lo, hi, force=False)
    uc = W.random_field(gc.shape, 312)
    ref = O.prolong(uc, gc, gf)
    got = P.prolong(pc, pf, _dev(uc, dtype)).double().cpu().numpy()
    assert _rel(got, ref) < (1e-13 if dtype == torch.float64 else 1e-6), _rel(got, ref)
    # prolongation followed by injection is the identity (nested CGL grids)
    back = O.restrict_inject(got, gc, gf)
    assert _rel(back, uc) < (1e-13 if dtype == torch.float64 else 1e-6)


def test_prolongation_from_N2_is_rejected():
    import paper_2606_21410_b300 as P
    from paper_2606_21410_b300._lib import ChebError
    pc, pf = _plan((3, 5, 5), force=False), _plan((5, 9, 9), force=False)
    with pytest.raises(ChebError):
        P.prolong(pc, pf, torch.zeros(pc.shape, dtype=torch.float64, device="cuda"))


def test_chirp_hierarchy_matches_oracle():
    """Two-level hierarchy (Alg. 4) on chirp sizes, N = (12, 6, 6) -> (24, 12, 12):
    the fine solution equals the oracle's direct solve, and e_ref equals the
    oracle's relative difference of the fine solution and the prolonged
    coarse one."""
    import paper_2606_21410_b300 as P
    lo, hi = (0, 0, 0), (1, 1, 1)
    ns = [(13, 7, 7), (25, 13, 13)]
    plans, Ks, bs, grids = [], [], [], []
    for n in ns:
        g = O.Grid(n, lo, hi)
        X, Y, Z = g.mesh()
        K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(1, 0.08, 0.2, 0.2, 0.0, 1.0), 1.0, 10.0)
        plans.append(_plan(n, lo, hi, force=False))
        grids.append(g)
        Ks.append(K)
        bs.append(np.sin(np.pi * X) * Y * (1 - Z) + 1.0)
    us, infos, eref = P.solve_hierarchy(plans, [_dev(k) for k in Ks], [_dev(b) for b in bs], mode=1,
                                        rtol=1e-12)
    ud = [O.solve_direct(Ks[i], bs[i], grids[i]) for i in range(2)]
    for i in range(2):
        assert _rel(us[i].cpu().numpy(), ud[i]) < 1e-10, (i, infos[i])
    ref_eref = O.e_ref(ud[1], O.prolong(ud[0], grids[0], grids[1]))
    assert abs(eref[1] - ref_eref) <= 1e-8 * ref_eref + 1e-14, (eref, ref_eref)


@pytest.mark.parametrize("mode", [0, 1])
def test_chirp_adjoint_solve_and_gradient_match_oracle(mode):
    """Adjoint solve A^T lam = c and dJ/dK on an axis that only the chirp
    transform covers (n = 131), against the oracle's dense transpose solve
    (rtol 1e-11 as for the forward solve on this grid)."""
    n, bc = (131, 5, 4), [0, 1, 2, 0, 1, 0]
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0, 0.2, 0.4, 0.2), 1.0, 10.0)
    b = W.random_field(g.shape, 321)
    c = W.random_field(g.shape, 322)
    ud = O.solve_direct(K, b, g)
    lam_ref = O.adjoint_solve_direct(K, c, g)
    gK_ref = O.grad_K(ud, lam_ref, g)
    dK = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    lam, dK, info = p.adjoint_solve(_dev(K), _dev(c), u=_dev(ud), dJdK=dK, mode=mode, rtol=1e-11)
    assert _rel(lam.cpu().numpy(), lam_ref) < 5e-10, info
    assert _rel(dK.cpu().numpy(), gK_ref) < 5e-9


def test_chirp_hierarchy_from_fine_data_matches_oracle():
    """cheb_solve_hierarchy_fine on chirp sizes (N = (12, 6, 6) -> (24, 12, 12)):
    coarse K and b injected from the fine data, the fine solution equal to
    the oracle's direct solve."""
    import paper_2606_21410_b300 as P
    lo, hi = (0, 0, 0), (1, 1, 1)
    ns = [(13, 7, 7), (25, 13, 13)]
    plans = [_plan(n, lo, hi, force=False) for n in ns]
    g = O.Grid(ns[-1], lo, hi)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(1, 0.08, 0.2, 0.2, 0.0, 1.0), 1.0, 10.0)
    b = np.sin(np.pi * X) * Y * (1 - Z) + 1.0
    u, infos, eref = P.solve_hierarchy_fine(plans, _dev(K), _dev(b), mode=1, rtol=1e-12)
    assert all(i["status"] == 0 for i in infos), infos
    assert _rel(u.cpu().numpy(), O.solve_direct(K, b, g)) < 1e-10
