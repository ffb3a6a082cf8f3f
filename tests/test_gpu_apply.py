"""Parity of the CUDA line passes with the FP64 oracle: first derivatives
(transform and dense routes, FP64 and FP32, every axis, uneven sizes with
ragged tiles), their transposes, the operator apply with every boundary-type
pattern, the adjoint apply, and the right-hand side.

Tolerances: relative L2 error against the oracle's output, with uniform
random input fields.  Their derivatives are dominated by the top Chebyshev
modes, so the rounding of the line transforms stays at a few units of the
working precision relative to the output (measured on B300: FP64 at most
2.3e-15, FP32 at most 1.9e-7 for derivatives, applies and adjoint applies).
The bounds, 1e-14 (FP64) and 1e-6 (FP32), sit about five times above that.
Boundary rows are checked element-wise as well: Dirichlet rows are copies of
u (bit-exact in FP64), Neumann rows are one derivative and carry the same
relative error bound against the largest Neumann-row value."""
import itertools

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-14, torch.float32: 1e-6}


def _plan(n, lo=(-1, -1, -1), hi=(1, 1, 1), bc=(0,) * 6):
    import paper_2606_21410_b300 as P
    return P.Plan(n, lo, hi, bc)


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    ((17, 9, 33), (-1, 0, 0.5), (1, 2, 3.0)),
    ((65, 33, 9), (0, 0, 0), (1, 1, 1)),
    ((9, 17, 5), (-2, -1, 0), (2, 1, 0.25)),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", CASES)
def test_deriv_transform_route_matches_dense_D(case, dtype):
    n, lo, hi = case
    g = O.Grid(n, lo, hi)
    p = _plan(n, lo, hi)
    u = W.random_field(g.shape, 101)
    ud = _dev(u, dtype)
    for a in range(3):
        assert p.route(a) == 0
        ref = O.grad(u, g, a)
        got = p.deriv(ud, a).double().cpu().numpy()
        assert _rel(got, ref) < TOL[dtype], (a, _rel(got, ref))
        refT = np.moveaxis(np.tensordot(g.D(a).T, u, axes=([1], [2 - a])), 0, 2 - a)
        gotT = p.deriv(ud, a, transpose=True).double().cpu().numpy()
        assert _rel(gotT, refT) < TOL[dtype], (a, "T", _rel(gotT, refT))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_deriv_dense_route_any_size(dtype):
    n, lo, hi = (12, 7, 10), (0, -1, -1), (3, 1, 2)
    g = O.Grid(n, lo, hi)
    p = _plan(n, lo, hi)
    u = W.random_field(g.shape, 102)
    for a in range(3):
        assert p.route(a) == 1
        got = p.deriv(_dev(u, dtype), a).double().cpu().numpy()
        assert _rel(got, O.grad(u, g, a)) < TOL[dtype], (a, _rel(got, O.grad(u, g, a)))
        gotT = p.deriv(_dev(u, dtype), a, transpose=True).double().cpu().numpy()
        refT = np.moveaxis(np.tensordot(g.D(a).T, u, axes=([1], [2 - a])), 0, 2 - a)
        assert _rel(gotT, refT) < TOL[dtype], (a, "T", _rel(gotT, refT))


def test_dense_and_transform_routes_agree():
    n = (33, 17, 9)
    p = _plan(n)
    u = _dev(W.random_field((9, 17, 33), 103))
    K = _dev(W.random_positive_field((9, 17, 33), 104))
    a0 = p.apply(K, u).cpu().numpy()
    for a in range(3):
        p.set_route(a, 1)
    a1 = p.apply(K, u).cpu().numpy()
    assert _rel(a1, a0) < 1e-12


def test_deriv_exact_on_chebyshev_polynomials():
    """d/dx T_k = k U_{k-1} at every node, for every k <= N (FP64, 1-D)."""
    N = 64
    p = _plan((N + 1,))
    th = np.pi * np.arange(N + 1) / N
    for k in range(N + 1):
        Tk = np.cos(k * th)
        d = p.deriv(_dev(Tk), 0).cpu().numpy()
        ex = np.empty(N + 1)
        ex[1:-1] = k * np.sin(k * th[1:-1]) / np.sin(th[1:-1])
        ex[0], ex[-1] = k * k, (-1) ** (k + 1) * k * k
        assert np.abs(d - ex).max() < 1e-13 * max(1, k * k) * N


def _check_boundary_rows(got, ref, u, g, bc, dtype):
    """Dirichlet rows copy u (exactly in FP64); Neumann rows element-wise
    against the oracle relative to their largest value."""
    own = O.owners(g)
    dmask = np.isin(own, [f for f in range(2 * g.dim) if bc[f] == 0])
    if dtype == torch.float64:
        assert np.array_equal(got[dmask], u[dmask])
    else:
        assert np.array_equal(got[dmask], u.astype(np.float32).astype(np.float64)[dmask])
    nmask = np.isin(own, [f for f in range(2 * g.dim) if bc[f] == 1])
    if nmask.any():
        err = np.abs(got[nmask] - ref[nmask]).max() / np.abs(ref[nmask]).max()
        assert err < TOL[dtype], ("Neumann rows", err)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("bc", [list(t) for t in itertools.product([0, 1], repeat=6)][::7])
def test_apply_every_bc_pattern(bc, dtype):
    n, lo, hi = (17, 9, 33), (0, -1, 0), (1, 1, 2)
    g = O.Grid(n, lo, hi, bc)
    p = _plan(n, lo, hi, bc)
    u = W.random_field(g.shape, 201)
    K = W.random_positive_field(g.shape, 202)
    ref = O.apply(u, K, g)
    got = p.apply(_dev(K, dtype), _dev(u, dtype)).double().cpu().numpy()
    err = _rel(got, ref)
    assert err < TOL[dtype], err
    interior = O.owners(g) < 0
    assert np.abs(got[interior] - ref[interior]).max() / np.abs(ref[interior]).max() < TOL[dtype]
    _check_boundary_rows(got, ref, u, g, bc, dtype)


@pytest.mark.parametrize("dim,n", [(1, (33,)), (2, (17, 65)), (3, (5, 9, 3))])
def test_apply_lower_dimensions(dim, n):
    bc = [1, 0, 0, 1, 0, 0]
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    u = W.random_field(g.shape, 300 + dim)
    K = W.random_positive_field(g.shape, 310 + dim)
    ref = O.apply(u, K, g)
    got = p.apply(_dev(K), _dev(u)).cpu().numpy()
    assert _rel(got, ref) < TOL[torch.float64], _rel(got, ref)
    _check_boundary_rows(got, ref, u, g, bc, torch.float64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_adjoint_apply_matches_oracle_and_dot_product(dtype):
    bc = [1, 0, 1, 1, 0, 1]
    n, lo, hi = (17, 9, 33), (0, 0, 0), (1, 2, 1)
    g = O.Grid(n, lo, hi, bc)
    p = _plan(n, lo, hi, bc)
    lam = W.random_field(g.shape, 401)
    K = W.random_positive_field(g.shape, 402)
    ref = O.adjoint_apply(lam, K, g)
    got = p.adjoint_apply(_dev(K, dtype), _dev(lam, dtype)).double().cpu().numpy()
    assert _rel(got, ref) < TOL[dtype], _rel(got, ref)
    if dtype == torch.float64:
        x = W.random_field(g.shape, 403)
        Ax = p.apply(_dev(K), _dev(x)).cpu().numpy()
        lhs, rhs = (Ax * lam).sum(), (x * got).sum()
        assert abs(lhs - rhs) < 1e-12 * np.abs(Ax).sum() * np.abs(lam).max()


def test_rhs_boundary_rows():
    bc = [0, 1, 1, 0, 0, 1]
    n = (9, 17, 5)
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    f = W.random_field(g.shape, 501)
    shapes = [(5, 17), (5, 17), (5, 9), (5, 9), (17, 9), (17, 9)]
    faces = [W.random_field(s, 510 + i) for i, s in enumerate(shapes)]
    ref = O.rhs(f, faces, g)
    got = p.rhs(_dev(f), [_dev(x) for x in faces]).cpu().numpy()
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------- large sizes

def _line_apply_samples(u, K, g, pts):
    """(A u)_p at sample interior nodes p, from the oracle's dense D one line
    at a time (cheap at any size)."""
    out = []
    for (k, j, i) in pts:
        v = 0.0
        idx = {0: i, 1: j, 2: k}
        for a in g.axes:
            D = g.D(a)
            sl = [k, j, i]
            sl[2 - a] = slice(None)
            line_u = u[tuple(sl)]
            line_K = K[tuple(sl)]
            q = line_K * (D @ line_u)
            v -= D[idx[a]] @ q
        out.append(v)
    return np.array(out)


@pytest.mark.parametrize("nn", [129, 257])
def test_apply_full_size_sampled(nn):
    """At 129^3 and 257^3 (the solve sizes): the FP64 apply at sampled
    interior rows against the oracle's per-line dense evaluation, and the
    FP32 apply over the whole field against the FP64 apply, for a smooth
    field with noise and for a random field, on the two-phase medium."""
    bc = [0, 0, 1, 1, 1, 1]
    g = O.Grid((nn,) * 3, bc=bc)
    p = _plan((nn,) * 3, bc=bc)
    X, Y, Z = g.mesh()
    u = np.sin(2 * X + Y) * np.cos(3 * Z) + 0.01 * W.random_field(g.shape, 601)
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 10.0)
    rng = W.rng(602)
    pts = [tuple(int(v) for v in rng.integers(1, nn - 1, size=3)) for _ in range(200)]
    ref = _line_apply_samples(u, K, g, pts)
    got64 = p.apply(_dev(K), _dev(u)).cpu().numpy()
    vals = np.array([got64[k, j, i] for (k, j, i) in pts])
    err64 = np.abs(vals - ref).max() / np.abs(ref).max()
    assert err64 < 1e-12, err64
    # FP32 against FP64 over the whole field: smooth + noise (the output
    # is small against ||D||^2 ||u||, so the FP32 rounding shows, measured
    # 1.0e-5 at 257^3 with contrast 100) and random (measured 2.5e-7)
    got32 = p.apply(_dev(K, torch.float32), _dev(u, torch.float32)).double().cpu().numpy()
    e32 = _rel(got32, got64)
    assert e32 < 5e-5, e32
    ur = W.random_field(g.shape, 603)
    r64 = p.apply(_dev(K), _dev(ur)).cpu().numpy()
    r32 = p.apply(_dev(K, torch.float32), _dev(ur, torch.float32)).double().cpu().numpy()
    er = _rel(r32, r64)
    assert er < TOL[torch.float32], er


def test_autotuner_picks_a_route_and_caches(tmp_path):
    """The autotuner times every route an axis allows, each with line tiles
    of 8 and 16 lines (FP32 also the tensor-core route), records the (route,
    tile) decision, reuses it from the cache file, and the tuned plan still
    matches the oracle."""
    import paper_2606_21410_b300 as P
    cache = str(tmp_path / "routes.txt")
    n = (65, 33, 12)
    p = P.Plan(n)
    r = p.autotune(cache)
    assert r["fp64"][2] == "dense" and r["fp32"][2] == "dense"   # n = 12: dense only
    assert all(x in ("transform", "dense") for x in r["fp64"])
    assert all(x in ("transform", "dense", "tensor") for x in r["fp32"])
    lines = open(cache).read().splitlines()
    assert len(lines) == 6        # 65, 33 and 12 (dense with 8- or 16-line tiles), two precisions
    assert all(r[k][a] in (8, 16) for k in ("tile64", "tile32") for a in range(3))
    r2 = P.Plan(n).autotune(cache)
    assert r2 == r and len(open(cache).read().splitlines()) == 6
    g = O.Grid(n)
    u = W.random_field(g.shape, 71)
    K = W.random_positive_field(g.shape, 72)
    got = p.apply(_dev(K), _dev(u)).cpu().numpy()
    ref = O.apply(u, K, g)
    assert _rel(got, ref) < TOL[torch.float64], _rel(got, ref)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [(17, 9, 33), (12, 7, 10), (65, 33, 9)])
def test_line_tiles_of_8_and_16_agree_bitwise(n, dtype):
    """The line tile (8 or 16 lines per CTA) only changes which CTA computes a
    line, not the arithmetic of any line: the operator apply, its adjoint and
    the Jacobian action are bit-identical for both tiles, on the transform
    route (power-of-two N) and the dense route (other N), ragged tiles included."""
    import paper_2606_21410_b300 as P
    bc = [0, 1, 2, 1, 0, 2]
    p = _plan(n, bc=bc)
    u = _dev(W.random_field(p.shape, 701), dtype)
    K = _dev(W.random_positive_field(p.shape, 702), dtype)
    C = [_dev(W.random_field(p.shape, 703 + a), dtype) for a in range(3)]
    prec = P.FP64 if dtype == torch.float64 else P.FP32
    res = {}
    for lines in (16, 8):
        for a in range(3):
            p.set_tile(a, prec, lines)
            assert p.tile(a, prec) == lines
        res[lines] = [p.apply(K, u).cpu(), p.adjoint_apply(K, u).cpu(), p.jacobian_apply(K, C, u).cpu()]
    for x16, x8 in zip(res[16], res[8]):
        assert torch.equal(x16, x8)
