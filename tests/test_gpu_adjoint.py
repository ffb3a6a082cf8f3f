"""Parity of the discrete adjoint: the transposed preconditioner against the
dense inverse transpose, the adjoint solve against the oracle's dense
transposed solve and the adjoint identity <lam, b> = <c, u> with the
oracle's forward solution, dJ/dK against the oracle's dense-transpose
gradient and central finite differences, and the autograd wrapper
(including the mean flux through the x = +1 face of the sphere problem)."""
import itertools

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _plan(n, lo=(-1, -1, -1), hi=(1, 1, 1), bc=(0,) * 6):
    import paper_2606_21410_b300 as P
    return P.Plan(n, lo, hi, bc)


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("bc", [list(t) for t in itertools.product([0, 1], repeat=6)][:-1:5])
def test_transposed_precond_is_dense_inverse_transpose(bc):
    n, lo, hi = (9, 6, 7), (0, -1, 0), (1, 1, 3)
    g = O.Grid(n, lo, hi, bc)
    p = _plan(n, lo, hi, bc)
    y = W.random_field(g.shape, 41)
    A = O.assemble(np.full(g.shape, 1.3), g)
    ref = np.linalg.solve(A.T, y.ravel()).reshape(g.shape)
    got = p.precond_apply_t(_dev(y), 1.3).cpu().numpy()
    assert _rel(got, ref) < 1e-10
    got32 = p.precond_apply_t(_dev(y, torch.float32), 1.3).double().cpu().numpy()
    assert _rel(got32, ref) < 1e-4


@pytest.mark.parametrize("n,bc", [((17,), [1, 0, 0, 0, 0, 0]), ((9, 7), [1, 1, 0, 1, 0, 0]),
                                  ((7, 9), [0, 1, 1, 1, 0, 0])])
def test_transposed_precond_lower_dimensions(n, bc):
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    y = W.random_field(g.shape, 42)
    A = O.assemble(np.full(g.shape, 0.7), g)
    ref = np.linalg.solve(A.T, y.ravel()).reshape(g.shape)
    assert _rel(p.precond_apply_t(_dev(y), 0.7).cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("mode", [0, 1])
def test_adjoint_solve_and_gradient_vs_dense(mode):
    bc = [1, 0, 1, 1, 0, 1]
    n = (9, 8, 11)
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0, 0.2, 0.4, 0.2), 1.0, 10.0)
    b = W.random_field(g.shape, 43)
    c = W.random_field(g.shape, 44)
    u = O.solve_direct(K, b, g)
    lam_ref = O.adjoint_solve_direct(K, c, g)
    gK_ref = O.grad_K(u, lam_ref, g)
    dK = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    lam, dK, info = p.adjoint_solve(_dev(K), _dev(c), u=_dev(u), dJdK=dK, mode=mode, rtol=1e-12)
    assert _rel(lam.cpu().numpy(), lam_ref) < 1e-10, info
    assert _rel(dK.cpu().numpy(), gK_ref) < 1e-9


def test_adjoint_identity_at_33_against_oracle_forward():
    """<lam, b> = <c, A^{-1} b> with u from the oracle's solve (any size)."""
    bc = [0, 0, 1, 1, 1, 1]
    n = (33, 33, 33)
    g = O.Grid(n, bc=bc)
    p = _plan(n, bc=bc)
    X, Y, Z = g.mesh()
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, 100.0)
    b = W.random_field(g.shape, 45)
    c = W.random_field(g.shape, 46)
    uo, _ = O.solve_preconditioned(K, b, g, rtol=1e-13)
    lam, _, info = p.adjoint_solve(_dev(K), _dev(c), mode=1, rtol=1e-12)
    lhs = float((lam.cpu().numpy() * b).sum())
    rhs = float((c * uo).sum())
    assert abs(lhs - rhs) < 1e-9 * abs(rhs), (lhs, rhs, info)


def test_gradient_against_central_differences():
    """J = <c, u(K)>: the adjoint dJ/dK along a random direction and for the
    two phase conductivities against central differences of GPU solves."""
    bc = [0, 0, 1, 1, 1, 1]
    n = (17, 17, 17)
    p = _plan(n, bc=bc)
    X, Y, Z = p.mesh()
    sp = W.sphere_packing(0)
    inc = W.two_phase_conductivity(X, Y, Z, sp, 0.0, 1.0)
    K = 1.0 + 9.0 * inc
    b = _dev(W.random_field(p.shape, 47))
    c = _dev(W.random_field(p.shape, 48))

    def J(Kn):
        u, _ = p.solve(_dev(Kn), b, mode=0, rtol=1e-14)
        return float((c * u).sum())

    u, _ = p.solve(_dev(K), b, mode=0, rtol=1e-14)
    dK = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    p.adjoint_solve(_dev(K), c, u=u, dJdK=dK, mode=0, rtol=1e-14)
    g = dK.cpu().numpy()
    for direction in (W.random_field(p.shape, 49), inc, 1.0 - inc):
        h = 1e-4
        fd = (J(K + h * direction) - J(K - h * direction)) / (2 * h)
        ad = float((g * direction).sum())
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)


def test_autograd_mean_flux_gradient():
    """J = mean outward flux K d_x u on x = +1 (Clenshaw-Curtis weights on the
    face) of the sphere problem; torch autograd through ChebSolve/ChebDeriv
    against central differences in the inclusion conductivity."""
    import paper_2606_21410_b300 as P
    from paper_2606_21410_b300 import autograd as AG
    bc = [0, 0, 1, 1, 1, 1]
    n = (17, 17, 17)
    p = P.Plan(n, bc=bc)
    X, Y, Z = p.mesh()
    inc = _dev(W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 0.0, 1.0))
    faces = W.face_values(bc, p.nodes(0), p.nodes(1), p.nodes(2),
                          lambda X, Y, Z: (X, (np.ones_like(X), 0 * X, 0 * X), 0 * X))
    b = p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"), [_dev(f) for f in faces])
    wy = O.cc_weights(16)
    wface = _dev(np.outer(wy, wy) / 4.0)  # face area 4

    def objective(kinc):
        K = 1.0 + (kinc - 1.0) * inc
        u = AG.solve(p, K, b, mode=0, rtol=1e-14)
        flux = K * AG.deriv(p, u, 0)
        return (wface * flux[:, :, 0]).sum()   # x index 0 is the x = +1 face

    k = torch.tensor(10.0, dtype=torch.float64, device="cuda", requires_grad=True)
    Jv = objective(k)
    Jv.backward()
    h = 1e-4
    fd = (objective(torch.tensor(10.0 + h, dtype=torch.float64, device="cuda")).item()
          - objective(torch.tensor(10.0 - h, dtype=torch.float64, device="cuda")).item()) / (2 * h)
    assert abs(k.grad.item() - fd) <= 1e-6 * abs(fd), (k.grad.item(), fd)


def _two_phase(p_or_g, contrast, nodes):
    bc = [0, 0, 1, 1, 1, 1]
    X, Y, Z = W.mesh(*nodes)
    K = W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0, contrast)
    faces = W.face_values(bc, nodes[0], nodes[1], nodes[2],
                          lambda X, Y, Z: (X, (np.ones_like(X), 0 * X, 0 * X), 0 * X))
    return K, faces


def test_hierarchy_from_fine_data_equals_sampled_levels():
    """cheb_solve_hierarchy_fine recomputes the coarse K and b by injection
    (CGL grids nest); it must give the hierarchy of separately sampled
    levels: same fine solution, same e_ref."""
    import paper_2606_21410_b300 as P
    bc = [0, 0, 1, 1, 1, 1]
    plans, Ks, bs = [], [], []
    for n in (9, 17, 33):
        p = P.Plan((n,) * 3, bc=bc)
        K, faces = _two_phase(p, 100.0, [p.nodes(0), p.nodes(1), p.nodes(2)])
        plans.append(p)
        Ks.append(_dev(K))
        bs.append(p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"), [_dev(f) for f in faces]))
    us, _, eref = P.solve_hierarchy(plans, Ks, bs, mode=1, rtol=1e-12)
    plans2 = [P.Plan((n,) * 3, bc=bc) for n in (9, 17, 33)]
    uf, _, eref2 = P.solve_hierarchy_fine(plans2, Ks[-1], bs[-1], mode=1, rtol=1e-12)
    assert _rel(uf.cpu().numpy(), us[-1].cpu().numpy()) < 1e-12
    for a, b_ in zip(eref, eref2):
        assert abs(a - b_) <= 1e-9 * max(a, 1e-300)


def _mean_flux(p, K, u, wface):
    """J = mean of K d_x u over the x = +1 face (x index 0), Clenshaw-Curtis
    weights on the face nodes; -J is the outward heat flux."""
    from paper_2606_21410_b300 import autograd as AG
    return (wface * (K * AG.deriv(p, u, 0))[:, :, 0]).sum()


def test_hierarchical_gradient_129_by_central_differences():
    """The 129^3 two-phase configuration (contrast 10) solved by the
    hierarchy 33^3 -> 65^3 -> 129^3 from the fine data; J = mean flux on
    x = +1.  dJ/dk_incl by autograd (fine-level adjoint solve) against central
    differences of hierarchical solves, relative error <= 1e-6."""
    import paper_2606_21410_b300 as P
    from paper_2606_21410_b300 import autograd as AG
    bc = [0, 0, 1, 1, 1, 1]
    plans = [P.Plan((n,) * 3, bc=bc) for n in (33, 65, 129)]
    pf = plans[-1]
    chi, faces = _two_phase(pf, 1.0 + 1.0, [pf.nodes(0), pf.nodes(1), pf.nodes(2)])
    inc = _dev(chi - 1.0)                   # indicator of the inclusions
    b = pf.rhs(torch.zeros(pf.shape, dtype=torch.float64, device="cuda"), [_dev(f) for f in faces])
    w = O.cc_weights(128)
    wface = _dev(np.outer(w, w) / 4.0)

    def J(kinc):
        K = 1.0 + (kinc - 1.0) * inc
        u = AG.solve_hierarchy(plans, K, b, mode=1, rtol=1e-12)
        return _mean_flux(pf, K, u, wface)

    k = torch.tensor(10.0, dtype=torch.float64, device="cuda", requires_grad=True)
    Jv = J(k)
    Jv.backward()
    h = 1e-3
    with torch.no_grad():
        fd = (J(torch.tensor(10.0 + h, dtype=torch.float64, device="cuda")).item()
              - J(torch.tensor(10.0 - h, dtype=torch.float64, device="cuda")).item()) / (2 * h)
    assert abs(k.grad.item() - fd) <= 1e-6 * abs(fd), (k.grad.item(), fd)


def test_adjoint_and_gradient_33_against_oracle_transposed_gmres():
    """The C3 geometry at 33^3 (contrast 10), J = <c, u>: lambda from the GPU
    adjoint solve against the oracle's transposed-preconditioned GMRES, and
    dJ/dK against the oracle's gradient formula with the oracle's own u and
    lambda."""
    bc = [0, 0, 1, 1, 1, 1]
    n = (33, 33, 33)
    g = O.Grid(n, bc=bc)
    Ko, faces_o = _two_phase(g, 10.0, [g.nodes(0), g.nodes(1), g.nodes(2)])
    bo = O.rhs(np.zeros(g.shape), faces_o, g)
    c = W.random_field(g.shape, 231)
    uo, _ = O.solve_preconditioned(Ko, bo, g, rtol=1e-13)
    lo, io = O.adjoint_solve_preconditioned(Ko, c, g, rtol=1e-13)
    gK_o = O.grad_K(uo, lo, g)
    p = _plan(n, bc=bc)
    Kp, faces_p = _two_phase(p, 10.0, [p.nodes(0), p.nodes(1), p.nodes(2)])
    b = p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"), [_dev(f) for f in faces_p])
    u, _ = p.solve(_dev(Kp), b, mode=0, rtol=1e-13)
    dK = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    lam, dK, info = p.adjoint_solve(_dev(Kp), _dev(c), u=u, dJdK=dK, mode=0, rtol=1e-13)
    assert _rel(lam.cpu().numpy(), lo) < 1e-9, (info, io["iterations"])
    assert _rel(dK.cpu().numpy(), gK_o) < 1e-8
