"""Homogenised response of the unit-cell study (Sec. 3.3): the volume-averaged
flux by Clenshaw-Curtis quadrature against the oracle, the effective
conductivity K_num of a centred sphere against the oracle's and against
Maxwell's estimate, and the contrast sweep k_i/k_m in [1e-4, 1e4].

Setting: (0,1)^3, u = -1 on x = 0, u = +1 on x = 1, zero normal derivative
elsewhere, f = 0, so G = 2 g / L_x = 2 and K_num = <K d_x u> / G."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

BC = [0, 0, 1, 1, 1, 1]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def _xfaces(X, Y, Z):
    return np.where(X > 0.5, 1.0, -1.0) * np.ones_like(X), (0 * X, 0 * X, 0 * X), 0 * X


@pytest.mark.parametrize("n,lo,hi", [((17, 9, 33), (0, -1, 0.5), (1, 2, 1.5)),
                                     ((65, 33), (0, 0), (2, 1)), ((33,), (-1,), (3,))])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_flux_average_matches_oracle(n, lo, hi, axis):
    import paper_2606_21410_b300 as P
    g = O.Grid(n, lo, hi)
    if axis >= g.dim:
        pytest.skip("axis not active")
    p = P.Plan(n, lo, hi)
    u = W.random_field(g.shape, 90 + axis)
    K = W.random_positive_field(g.shape, 95)
    ref = O.volume_average(K * O.grad(u, g, axis), g)
    got = p.flux_average(_dev(K), _dev(u), axis)
    assert abs(got - ref) <= 1e-13 * max(1.0, np.abs(K * O.grad(u, g, axis)).mean()), (got, ref)


def _cell(n, contrast, spheres, nodes):
    X, Y, Z = W.mesh(*nodes)
    K = W.two_phase_conductivity(X, Y, Z, spheres, 1.0, contrast)
    faces = W.face_values(BC, nodes[0], nodes[1], nodes[2], _xfaces)
    return K, faces


@pytest.mark.parametrize("contrast", [1e-4, 1e-2, 10.0, 1e2, 1e4])
def test_contrast_sweep_matches_oracle_33(contrast):
    """Centred sphere of radius 0.2 (phi = 0.0335) at 33^3: K_num and the
    solution against the oracle's preconditioned GMRES at every contrast.
    The solves stop at a preconditioned residual of 1e-12; the solution can
    differ by up to the conditioning of M^{-1} A times that, which grows with
    the contrast, so the solution bound is 1e-7 and K_num's 1e-8."""
    import paper_2606_21410_b300 as P
    n = (33, 33, 33)
    g = O.Grid(n, (0, 0, 0), (1, 1, 1), BC)
    Ko, faces_o = _cell(33, contrast, W.single_sphere(), [g.nodes(0), g.nodes(1), g.nodes(2)])
    uo, io = O.solve_preconditioned(Ko, O.rhs(np.zeros(g.shape), faces_o, g), g, rtol=1e-12,
                                    maxiter=5000)
    k_or = O.effective_conductivity(uo, Ko, g, G=2.0)
    p = P.Plan(n, (0, 0, 0), (1, 1, 1), BC)
    Kp, faces_p = _cell(33, contrast, W.single_sphere(), [p.nodes(0), p.nodes(1), p.nodes(2)])
    b = p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"), [_dev(f) for f in faces_p])
    u, info = p.solve(_dev(Kp), b, mode=1, rtol=1e-12, maxiter=20000, inner_maxiter=4000,
                      max_refinements=60)
    k_gpu = p.flux_average(_dev(Kp), u, 0) / 2.0
    assert abs(k_gpu - k_or) <= 1e-8 * k_or, (k_gpu, k_or, info["iterations"], io["iterations"])
    err = np.linalg.norm(u.cpu().numpy() - uo) / np.linalg.norm(uo)
    assert err <= 1e-7, (err, info)


@pytest.mark.parametrize("n", [33, 65])
def test_centred_sphere_maxwell_and_oracle(n):
    """The centred sphere at contrast 10: K_num against the oracle's K_num
    on the same grid (1e-9), and at 33^3 against Maxwell's dilute estimate to
    below 1e-3, the agreement the paper reports.  (At 65^3 the nodal sampling
    of the jump moves K_num 2.7e-3 away from Maxwell: the sampled inclusion's
    volume fraction alone changes by -5.5 % at N = 32 and +0.6 % at N = 64,
    so the check against Maxwell stays at the resolution where the paper's
    statement holds.)"""
    import paper_2606_21410_b300 as P
    g = O.Grid((n,) * 3, (0, 0, 0), (1, 1, 1), BC)
    Ko, faces_o = _cell(n, 10.0, W.single_sphere(), [g.nodes(0), g.nodes(1), g.nodes(2)])
    uo, _ = O.solve_preconditioned(Ko, O.rhs(np.zeros(g.shape), faces_o, g), g, rtol=1e-12)
    k_or = O.effective_conductivity(uo, Ko, g, G=2.0)
    p = P.Plan((n,) * 3, (0, 0, 0), (1, 1, 1), BC)
    K, faces = _cell(n, 10.0, W.single_sphere(), [p.nodes(0), p.nodes(1), p.nodes(2)])
    b = p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"), [_dev(f) for f in faces])
    Kd = _dev(K)
    u, info = p.solve(Kd, b, mode=1, rtol=1e-12)
    k_num = p.flux_average(Kd, u, 0) / 2.0
    assert abs(k_num - k_or) <= 1e-9 * k_or, (k_num, k_or)
    if n == 33:
        k_max = O.maxwell_estimate(1.0, 10.0, 4.0 / 3.0 * math.pi * 0.2 ** 3)
        assert abs(k_num - k_max) / k_max < 1e-3, (k_num, k_max)
