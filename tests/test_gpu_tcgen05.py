"""Parity of the FP32 fast-diagonalization preconditioner on the tcgen05
tensor-core contraction path (taken when every padded interior extent lies
in [32, 256] and each contraction has at least 128 lines) against the FP64
oracle preconditioner, against the mma.sync split-TF32 path of the same
library, and, for the transposed preconditioner, through the duality
<M^{-1} r, y> = <r, M^{-T} y> with the oracle's M^{-1}.

Shapes cover a ragged last K chunk (K = 36 = 32 + 4, K = 40), N tiles
padded to 16 rows (N = 36 -> 48), a ragged last 128-line tile
(M = 1440), two dimensions, and the 129^3 / 257^3 solve sizes.

Tolerance: the split-TF32 products carry FP32-level rounding (~2^-22 per
product), so the tensor-core path must match the oracle to 1e-4 relative
(as the FP32 path does at small sizes) and stay within a factor 4 (+1e-6)
of the mma.sync path's own error."""
import os

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.precond import FDMPreconditioner

pytestmark = pytest.mark.gpu

CASES = [((35, 34, 41), [0, 1, 1, 0, 0, 1]), ((66, 40, 33), [0] * 6), ((129, 129), [1, 0, 0, 1, 0, 0])]


def _plan(n, bc):
    import paper_2606_21410_b300 as P
    return P.Plan(n, (-1, -1, -1), (1, 1, 1), bc)


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _without_tcgen05(fn):
    """Run fn with the tcgen05 contraction disabled for plans set up inside."""
    os.environ["CHEB_FDM_NO_TCGEN05"] = "1"
    try:
        return fn()
    finally:
        del os.environ["CHEB_FDM_NO_TCGEN05"]


@pytest.mark.parametrize("n,bc", CASES)
def test_tcgen05_precond_matches_oracle_and_mma_path(n, bc):
    g = O.Grid(n, bc=bc)
    r = W.random_field(g.shape, 21)
    kref = 1.3
    ref = FDMPreconditioner(g, kref)(r)
    p = _plan(n, bc)
    got64 = p.precond_apply(_dev(r), kref).cpu().numpy()
    assert _rel(got64, ref) < 1e-10
    got_tc = p.precond_apply(_dev(r, torch.float32), kref).double().cpu().numpy()

    def legacy():
        q = _plan(n, bc)
        return q.precond_apply(_dev(r, torch.float32), kref).double().cpu().numpy()

    got_mma = _without_tcgen05(legacy)
    e_tc, e_mma = _rel(got_tc, ref), _rel(got_mma, ref)
    assert e_tc < 1e-4, (e_tc, e_mma)
    assert e_tc <= 4 * e_mma + 1e-6, (e_tc, e_mma)


@pytest.mark.parametrize("n,bc", CASES[:2])
def test_tcgen05_transposed_precond_by_duality(n, bc):
    g = O.Grid(n, bc=bc)
    kref = 0.8
    r = W.random_field(g.shape, 22)
    y = W.random_field(g.shape, 23)
    Mr = FDMPreconditioner(g, kref)(r)
    p = _plan(n, bc)
    lhs = float((Mr * y).sum())
    for dtype, tol in ((torch.float64, 1e-10), (torch.float32, 1e-4)):
        Mty = p.precond_apply_t(_dev(y, dtype), kref).double().cpu().numpy()
        rhs = float((r * Mty).sum())
        scale = np.linalg.norm(Mr) * np.linalg.norm(y)
        assert abs(lhs - rhs) < tol * scale, (dtype, lhs, rhs)


@pytest.mark.parametrize("nn", [129, 257])
def test_tcgen05_precond_full_size(nn):
    """At the solve sizes: FP32 (tensor-core path) against the FP64 path,
    and at 129^3 also against the oracle."""
    bc = [0, 0, 1, 1, 1, 1]
    n = (nn,) * 3
    g = O.Grid(n, bc=bc)
    r = W.random_field(g.shape, 24)
    p = _plan(n, bc)
    got64 = p.precond_apply(_dev(r), 2.0).cpu().numpy()
    got32 = p.precond_apply(_dev(r, torch.float32), 2.0).double().cpu().numpy()
    assert _rel(got32, got64) < 1e-4
    if nn == 129:
        ref = FDMPreconditioner(g, 2.0)(r)
        assert _rel(got64, ref) < 1e-10


# ------------------------------------------------ tensor-core route of the apply
#
# Tolerances of the split-TF32 route: relative L2 against the oracle with
# random inputs, measured 1.1e-6 .. 2.2e-6 on B300 (the three TF32 products
# carry about 2^-22 relative rounding each, accumulated over n terms in
# FP32); bound 1e-5.  Neumann rows element-wise against their largest value
# (measured up to 1.9e-6), same bound; Dirichlet rows exact copies of u.

TENSOR_TOL = 1e-5

TENSOR_CASES = [
    ((33, 40, 65), [0, 1, 1, 0, 0, 1]),   # ragged 128-line tiles, n = 40 off the transform sizes
    ((65, 33, 41), [1, 1, 0, 1, 1, 0]),   # Neumann-owned edges and corners
    ((41, 65, 33), [0] * 6),
    ((129, 129), [1, 0, 0, 1, 0, 0]),     # 2-D
    ((129, 257), [0, 1, 1, 0, 0, 0]),     # 257 points: 272 output columns in two MMA groups
]


@pytest.mark.parametrize("n,bc", TENSOR_CASES)
def test_tensor_route_apply_matches_oracle(n, bc):
    import paper_2606_21410_b300 as P
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc)
    for a in range(len(n)):
        p.set_route32(a, P.ROUTE_TENSOR)
        assert p.route32(a) == P.ROUTE_TENSOR
    u = W.random_field(g.shape, 31)
    K = W.random_positive_field(g.shape, 32)
    ref = O.apply(u, K, g)
    got = p.apply(_dev(K, torch.float32), _dev(u, torch.float32)).double().cpu().numpy()
    err = _rel(got, ref)
    assert err < TENSOR_TOL, err
    own = O.owners(g)
    dmask = np.isin(own, [f for f in range(2 * g.dim) if bc[f] == 0])
    assert np.array_equal(got[dmask], u.astype(np.float32).astype(np.float64)[dmask])
    nmask = np.isin(own, [f for f in range(2 * g.dim) if bc[f] == 1])
    if nmask.any():
        en = np.abs(got[nmask] - ref[nmask]).max() / np.abs(ref[nmask]).max()
        assert en < TENSOR_TOL, en


def test_tensor_route_unsupported_sizes_are_refused():
    import paper_2606_21410_b300 as P
    p = _plan((17, 33, 33), [0] * 6)
    with pytest.raises(P.ChebError):
        p.set_route32(0, P.ROUTE_TENSOR)      # n = 17 < 33
    q = _plan((65,), [0] * 6)
    with pytest.raises(P.ChebError):
        q.set_route32(0, P.ROUTE_TENSOR)      # 1-D: a single line


@pytest.mark.parametrize("nn", [129, 257])
def test_tensor_route_full_size_against_fp64(nn):
    """At the solve sizes, over the whole field: the tensor route against
    the FP64 transform-route apply (itself checked against the oracle at
    sampled rows in test_gpu_apply), on the two-phase medium at contrast
    100, for the bench's smooth-plus-noise field (measured 5.4e-6 at 257^3,
    6.0e-6 at 129^3) and a random field (measured 2.6e-6); and the FP32
    transform route beside it."""
    import paper_2606_21410_b300 as P
    bc = [0, 0, 1, 1, 1, 1]
    g = O.Grid((nn,) * 3, bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 100.0)
    pt = _plan((nn,) * 3, bc)
    pc = _plan((nn,) * 3, bc)
    for a in range(3):
        pc.set_route32(a, P.ROUTE_TENSOR)
    for u, tol in ((np.sin(2 * X + Y) * np.cos(3 * Z) + 0.01 * W.random_field(g.shape, 33), 3e-5),
                   (W.random_field(g.shape, 36), 1.5e-5)):
        a64 = pt.apply(_dev(K), _dev(u)).cpu().numpy()
        Kd, ud = _dev(K, torch.float32), _dev(u, torch.float32)
        a_tc = pc.apply(Kd, ud).double().cpu().numpy()
        a_tr = pt.apply(Kd, ud).double().cpu().numpy()
        e_tc, e_tr = _rel(a_tc, a64), _rel(a_tr, a64)
        assert e_tc < tol, (e_tc, e_tr)
        assert e_tr < 2 * tol, (e_tc, e_tr)


def test_tensor_route_mixed_solve_matches_fp64():
    """A mixed-precision solve whose FP32 applies run on the tensor route
    reaches the FP64 solution (the refinement is in FP64)."""
    import paper_2606_21410_b300 as P
    n = (65, 65, 65)
    bc = [0, 0, 1, 1, 0, 0]
    g = O.Grid(n, bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 10.0)
    b = W.random_field(g.shape, 35)
    p64 = _plan(n, bc)
    u64, i64 = p64.solve(_dev(K), _dev(b), mode=0, rtol=1e-12)
    pm = _plan(n, bc)
    for a in range(3):
        pm.set_route32(a, P.ROUTE_TENSOR)
    um, im = pm.solve(_dev(K), _dev(b), mode=1, rtol=1e-12)
    assert im["status"] == 0 and im["applies_fp32"] > 0
    assert _rel(um.cpu().numpy(), u64.cpu().numpy()) < 1e-9


def test_bounded_wait_gives_up_and_context_stays_usable():
    """Failure detection without a fault: a tensor-core CTA waits on a barrier
    that nothing completes, with a short limit (2^20 SM clocks, about half a
    millisecond); the wait gives up, the library reports CHEB_ERR_CUDA with
    the give-up message, the CTA has freed its tensor memory, and the next
    tensor-core preconditioner call runs and matches the oracle."""
    import paper_2606_21410_b300 as P
    lib = P.lib
    st = lib.cheb_selftest_bounded_wait(1 << 20)
    assert st == -2
    assert b"bounded pipeline wait gave up" in lib.cheb_last_error()
    # the error word was read and cleared: a second self-test reports again
    assert lib.cheb_selftest_bounded_wait(1 << 20) == -2
    n, bc = (35, 34, 41), [0, 1, 1, 0, 0, 1]
    g = O.Grid(n, bc=bc)
    r = W.random_field(g.shape, 25)
    ref = FDMPreconditioner(g, 1.1)(r)
    got = _plan(n, bc).precond_apply(_dev(r, torch.float32), 1.1).double().cpu().numpy()
    assert _rel(got, ref) < 1e-4


# ------------------------------------- preconditioner with TF32-rounded matrices
#
# CHEB_PMAT_TF32 (the default of the FP32 inner solves) contracts the field,
# split hi + lo, against the eigenvector matrices rounded to TF32 (10 fraction
# bits: relative entry error <= 2^-11), two products per step.  What must hold:
# it is a fixed linear map to FP32 accuracy (the Krylov relation of the inner
# LGMRES needs that, not the exact matrices); it differs from the FP32-matrix
# preconditioner (the rounding is real); its distance from the exact FDM
# inverse stays within the perturbation of six rounded matrices,
# 6 * 2^-11 * max cond(S_a) (measured 3.4e-4 .. 4.2e-4 with the oracle's own
# bases); and the mixed solves it preconditions reach the same solutions in
# about as many iterations.

def _cond_S(g):
    from oracle.precond import _axis_tables
    return max(np.linalg.cond(_axis_tables(g, a)["S"]) for a in g.axes)


@pytest.mark.parametrize("n,bc", CASES)
def test_tf32_matrix_precond_is_linear_and_close_to_exact(n, bc):
    import paper_2606_21410_b300 as P
    g = O.Grid(n, bc=bc)
    kref = 1.3
    r1 = W.random_field(g.shape, 26)
    r2 = W.random_field(g.shape, 27)
    ref = FDMPreconditioner(g, kref)(r1)
    p = _plan(n, bc)

    def tf(r):
        return p.precond_apply(_dev(r, torch.float32), kref, matrices=P.PMAT_TF32).double().cpu().numpy()

    z1, z2 = tf(r1), tf(r2)
    a, b = 0.75, -1.5
    z12 = tf(a * r1 + b * r2)
    lin = _rel(z12, a * z1 + b * z2)
    assert lin < 1e-5, lin
    zf = p.precond_apply(_dev(r1, torch.float32), kref, matrices=P.PMAT_FP32).double().cpu().numpy()
    assert _rel(zf, ref) < 1e-4
    d_mode = _rel(z1, zf)
    assert d_mode > 2e-5, d_mode            # the TF32 matrices are in use
    bound = 6 * 2.0 ** -11 * _cond_S(g)
    assert _rel(z1, ref) < bound, (_rel(z1, ref), bound)


def test_tf32_matrix_mixed_solves_match_oracle_and_fp32_matrices():
    """Mixed solves of a 65^3 two-phase problem (contrast 100) with either
    matrix precision reach the oracle's solution; iteration counts within
    10 %; a captured-graph solve of one precision is not replayed for the
    other (the graph key holds it)."""
    import paper_2606_21410_b300 as P
    n = (65, 65, 65)
    bc = [0, 0, 1, 1, 1, 1]
    g = O.Grid(n, bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 100.0)
    b = W.random_field(g.shape, 36)
    uo, io = O.solve_preconditioned(K, b, g, rtol=1e-12)
    p = _plan(n, bc)
    res = {}
    for pm in (P.PMAT_TF32, P.PMAT_FP32):
        u, info = p.solve(_dev(K), _dev(b), mode=1, rtol=1e-12, precond_matrices=pm)
        assert info["status"] == 0
        assert _rel(u.cpu().numpy(), uo) < 1e-9, (pm, _rel(u.cpu().numpy(), uo))
        res[pm] = (u.cpu().numpy(), info["iterations"])
    it_t, it_f = res[P.PMAT_TF32][1], res[P.PMAT_FP32][1]
    assert abs(it_t - it_f) <= max(3, 0.1 * it_f), (it_t, it_f)
    for pm in (P.PMAT_TF32, P.PMAT_FP32, P.PMAT_TF32):
        ug, _ = p.solve(_dev(K), _dev(b), mode=1, rtol=1e-12, precond_matrices=pm, use_graph=1)
        assert _rel(ug.cpu().numpy(), res[pm][0]) < 1e-11, pm


def test_precond_matrices_option_is_checked():
    import paper_2606_21410_b300 as P
    from paper_2606_21410_b300._lib import ChebError
    n, bc = (35, 34, 41), [0, 1, 1, 0, 0, 1]
    p = _plan(n, bc)
    r = _dev(W.random_field(p.shape, 28), torch.float32)
    with pytest.raises(ChebError):
        p.precond_apply(r, 1.0, matrices=7)
    with pytest.raises(ChebError):
        p.solve(_dev(np.ones(p.shape)), _dev(W.random_field(p.shape, 29)), precond_matrices=2)
