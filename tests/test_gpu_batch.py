"""Picard iteration and batched solves: the GPU Picard fixed point against
the oracle's Picard iteration (uneven sizes exercising both line-derivative
routes), batched solves against single solves and the oracle, and a batch
of the configuration's uneven lognormal instances.  Batches run in both
iteration modes: LOCKSTEP (all instances in one iteration stream, batched
line passes over an (instance, tile) work list, per-instance converged
mask, one captured graph per Arnoldi step) and CONCURRENT (one solver per
instance)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

BC4 = [0, 0, 1, 1, 0, 1]   # Dirichlet on x = +-1 and z = -1, Neumann on y = +-1 and z = +1


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _instance(n, seed):
    import paper_2606_21410_b300 as P
    p = P.Plan(n, bc=BC4)
    X, Y, Z = p.mesh()
    K0 = W.lognormal_conductivity(X, Y, Z, seed=seed)
    faces = W.face_values(BC4, p.nodes(0), p.nodes(1), p.nodes(2),
                          lambda X, Y, Z: (X, (np.ones_like(X), 0 * X, 0 * X), 0 * X))
    b = p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"), [_dev(f) for f in faces])
    return p, K0, b


LOCKSTEP, CONCURRENT = 1, 2


@pytest.mark.parametrize("mode", [0, 1])
def test_picard_matches_oracle(mode):
    n = (13, 9, 11)
    p, K0, b = _instance(n, 1)
    assert [p.route(a) for a in range(3)] == [1, 0, 1]
    # plain Picard settles into a 2-cycle (~5e-3) on these lognormal fields;
    # relaxation 0.5 converges (in the oracle as well)
    u, info, its, d = p.picard_solve(_dev(K0), b, beta=0.5, tol=1e-12, maxit=100, omega=0.5, mode=mode,
                                     rtol=1e-13)
    g = O.Grid(n, bc=BC4)
    uo, io = O.picard_solve(K0, b.cpu().numpy(), g, tol=1e-13, maxit=100, omega=0.5)
    assert d <= 1e-12 and its > 3
    assert _rel(u.cpu().numpy(), uo) < 1e-9, (its, io["iterations"])
    # the returned u is a fixed point: A(K(u)) u = b
    K = O.picard_conductivity(K0, u.cpu().numpy(), g)
    r = O.apply(u.cpu().numpy(), K, g) - b.cpu().numpy()
    assert np.linalg.norm(O.FDMPreconditioner(g, O.geometric_mean(K))(r)) < 1e-9 * np.abs(u.cpu().numpy()).max()


@pytest.mark.parametrize("batch_mode", [LOCKSTEP, CONCURRENT])
def test_batched_solve_matches_single_solves(batch_mode):
    """Both iteration modes against single solves (rtol 1e-12 everywhere:
    solutions agree to 1e-10, the bound of kappa(M^-1 A) ~ 10-100 times the
    tolerance) and the oracle's direct solve."""
    import paper_2606_21410_b300 as P
    sizes = [(17, 17, 17), (13, 21, 9), (33, 9, 17), (9, 9, 9)]
    items = [_instance(n, 10 + i) for i, n in enumerate(sizes)]
    plans = [it[0] for it in items]
    K = [_dev(it[1]) for it in items]
    b = [it[2] for it in items]
    ub, infos = P.solve_batched(plans, K, b, mode=1, rtol=1e-12, batch_mode=batch_mode)
    for i, (p, Ki, bi) in enumerate(zip(plans, K, b)):
        us, _ = p.solve(Ki, bi, mode=1, rtol=1e-12)
        assert _rel(ub[i].cpu().numpy(), us.cpu().numpy()) < 1e-10
        assert infos[i]["status"] == 0
    if batch_mode == LOCKSTEP:
        assert all(i["graph_captures"] > 0 for i in infos)
    g = O.Grid(sizes[3], bc=BC4)
    ud = O.solve_direct(K[3].cpu().numpy(), b[3].cpu().numpy(), g)
    assert _rel(ub[3].cpu().numpy(), ud) < 1e-10


def test_picard_batch_of_uneven_lognormal_instances():
    """The batched configuration's shape: uneven sizes drawn from U{33..97}
    (seed 1), lognormal K0 (sigma 0.5, correlation length 0.2), Picard with
    beta = 0.5; here the first 4 instances (63^3 .. 94^3: the preconditioner
    takes its tcgen05 route, so lockstep runs the batched lift, face and
    boundary-line steps), in both iteration modes, each instance against its
    single-instance Picard solve."""
    import paper_2606_21410_b300 as P
    sizes = W.batch_sizes(1)[:4]
    items = [_instance((n, n, n), 100 + i) for i, n in enumerate(sizes)]
    plans = [it[0] for it in items]
    K0 = [_dev(it[1]) for it in items]
    b = [it[2] for it in items]
    single = []
    for i, p in enumerate(plans):
        us, _, its1, _ = p.picard_solve(K0[i], b[i], beta=0.5, tol=1e-9, maxit=60, omega=0.5, mode=1,
                                        rtol=1e-12)
        single.append(us.cpu().numpy())
    for bm in (LOCKSTEP, CONCURRENT):
        u, infos, its = P.picard_batched(plans, K0, b, beta=0.5, tol=1e-9, maxit=60, omega=0.5, mode=1,
                                         rtol=1e-12, use_graph=1, batch_mode=bm)
        for i in range(len(plans)):
            assert infos[i]["status"] == 0, (bm, sizes[i], infos[i], its[i])
            assert _rel(u[i].cpu().numpy(), single[i]) < 1e-9, (bm, sizes[i])
        if bm == LOCKSTEP:
            assert infos[0]["graph_captures"] > 0


@pytest.mark.parametrize("batch_mode", [LOCKSTEP, CONCURRENT])
def test_picard_batch_each_instance_matches_oracle(batch_mode):
    """A batch of small uneven instances (both line routes, lognormal K0,
    K = K0 (1 + 0.5 |grad u|^2)) solved by cheb_picard_batched in both
    iteration modes: every instance against the oracle's relaxed Picard
    iteration."""
    import paper_2606_21410_b300 as P
    sizes = [(9, 9, 9), (11, 11, 11), (13, 9, 11), (9, 13, 7)]
    items = [_instance(n, 300 + i) for i, n in enumerate(sizes)]
    plans = [it[0] for it in items]
    K0 = [_dev(it[1]) for it in items]
    b = [it[2] for it in items]
    u, infos, its = P.picard_batched(plans, K0, b, beta=0.5, tol=1e-12, maxit=100, omega=0.5, mode=1,
                                     rtol=1e-13, batch_mode=batch_mode)
    for i, n in enumerate(sizes):
        assert infos[i]["status"] == 0, (n, infos[i], its[i])
        g = O.Grid(n, bc=BC4)
        X, Y, Z = g.mesh()
        K0o = W.lognormal_conductivity(X, Y, Z, seed=300 + i)
        faces = W.face_values(BC4, g.nodes(0), g.nodes(1), g.nodes(2),
                              lambda X, Y, Z: (X, (np.ones_like(X), 0 * X, 0 * X), 0 * X))
        bo = O.rhs(np.zeros(g.shape), faces, g)
        uo, io = O.picard_solve(K0o, bo, g, tol=1e-13, maxit=100, omega=0.5)
        assert _rel(u[i].cpu().numpy(), uo) < 1e-9, (n, its[i], io["iterations"])


@pytest.mark.parametrize("mode", [0, 1])
def test_lockstep_converged_mask_and_uneven_instances(mode):
    """Instances that need very different work in one lockstep batch: a
    zero right-hand side (u = 0 without an iteration), a constant K (the
    preconditioner is the exact inverse: a step or two), lognormal fields of
    uneven and non-power-of-two sizes, two boundary sets.  Each leaves the
    iteration when it converges (per-instance iteration counts), and each
    solution equals the concurrent mode's and, for the small ones, the
    oracle's direct solve."""
    import paper_2606_21410_b300 as P
    # (33, 33, 33): the preconditioner's tcgen05 route, batched lift / face / line steps
    sizes = [(17, 17, 17), (25, 12, 7), (9, 9, 9), (33, 19, 11), (13, 13, 13), (11, 11, 11), (33, 33, 33)]
    items = [_instance(n, 500 + i) for i, n in enumerate(sizes)]
    plans = [it[0] for it in items]
    K = [_dev(it[1]) for it in items]
    b = [it[2].clone() for it in items]
    b[2].zero_()                           # zero right-hand side
    K[4] = torch.full_like(K[4], 2.5)      # constant conductivity
    bc5 = [0, 0, 0, 0, 0, 0]
    p5 = P.Plan(sizes[5], bc=bc5)
    plans[5] = p5
    b[5] = _dev(W.random_field(p5.shape, 77))
    # flux faces (their preconditioner rescales the flux data first)
    bc6 = [0, 2, 2, 2, 0, 2]
    p6 = P.Plan((15, 10, 12), bc=bc6)
    sizes.append((15, 10, 12))
    plans.append(p6)
    K.append(_dev(W.random_positive_field(p6.shape, 78)))
    b.append(_dev(W.random_field(p6.shape, 79)))
    kw = dict(mode=mode, rtol=1e-12)
    ul, il = P.solve_batched(plans, K, b, batch_mode=LOCKSTEP, **kw)
    uc, ic = P.solve_batched(plans, K, b, batch_mode=CONCURRENT, **kw)
    for i in range(len(plans)):
        assert il[i]["status"] == 0, (i, il[i])
        if i == 2:
            assert float(ul[i].abs().max()) == 0.0 and il[i]["iterations"] == 0
            continue
        assert _rel(ul[i].cpu().numpy(), uc[i].cpu().numpy()) < 1e-10, (i, il[i], ic[i])
    its = [il[i]["iterations"] for i in range(len(plans))]
    assert its[4] <= 3 and min(its[0], its[1], its[3]) > 3 * max(its[4], 1), its
    # one step graph per (step, Krylov-direction count, augmentation slot),
    # whichever instances are still iterating: at most 4 x (30 + 3 + 1)
    assert 0 < il[0]["graph_captures"] <= 4 * 34, il[0]["graph_captures"]
    for i in (2, 5):
        g = O.Grid(sizes[i], bc=plans[i].bc)
        ud = O.solve_direct(K[i].cpu().numpy(), b[i].cpu().numpy(), g)
        assert np.allclose(ul[i].cpu().numpy(), ud, rtol=0, atol=1e-10 * max(1.0, np.abs(ud).max()))


def test_lockstep_batch_needs_supported_plans():
    """LOCKSTEP needs the dense route on every axis (n <= 129): forced on a
    batch holding a 131-point axis it is refused; AUTO runs that batch in
    the concurrent mode."""
    import paper_2606_21410_b300 as P
    from paper_2606_21410_b300._lib import ChebError
    sizes = [(9, 9, 9), (131, 5, 5)]
    items = [_instance(n, 600 + i) for i, n in enumerate(sizes)]
    plans = [it[0] for it in items]
    K = [_dev(it[1]) for it in items]
    b = [it[2] for it in items]
    with pytest.raises(ChebError):
        P.solve_batched(plans, K, b, mode=1, rtol=1e-10, batch_mode=LOCKSTEP)
    u, infos = P.solve_batched(plans, K, b, mode=1, rtol=1e-10)
    assert all(i["status"] == 0 and i["graph_captures"] == 0 for i in infos)


def test_auto_batch_mode_follows_instance_count_and_size():
    """AUTO runs lockstep for many small instances (captured step graphs)
    and one solver per instance for a few large ones (no captures)."""
    import paper_2606_21410_b300 as P
    small = [_instance((9, 9, 9), 800 + i) for i in range(40)]
    u, infos = P.solve_batched([it[0] for it in small], [_dev(it[1]) for it in small], [it[2] for it in small],
                               mode=1, rtol=1e-10)
    assert all(i["status"] == 0 for i in infos) and infos[0]["graph_captures"] > 0
    big = [_instance((65, 65, 65), 900 + i) for i in range(2)]
    u, infos = P.solve_batched([it[0] for it in big], [_dev(it[1]) for it in big], [it[2] for it in big],
                               mode=1, rtol=1e-10)
    assert all(i["status"] == 0 for i in infos) and infos[0]["graph_captures"] == 0
