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
