"""cheb_prolong_noalloc: the prolongation for callers that cannot allocate
device memory (for example code running inside a custom allocator or a
memory-capped process).  It must give the same result as cheb_prolong while
using only the library's fixed internal scratch array, on two calls in a row
(the array keeps the previous call's contents), allocate nothing on a plan
pair that never ran cheb_prolong, agree with the oracle's prolongation, and
reject grids whose intermediates do not fit or a current device that is not
the plans'.  Called through the C ABI with ctypes.  This file is collected
last so a failure here leaves every other test already run."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _fine(nc):
    return tuple(2 * (v - 1) + 1 for v in nc)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)])
@pytest.mark.parametrize("nc", [(33, 33, 33), (65, 65, 65), (17, 33, 9), (65, 17), (129,),
                                (25, 13, 7), (101, 9)])  # the last two: N not powers of two
def test_noalloc_prolong_matches_cheb_prolong_twice(nc, dtype, tol):
    import paper_2606_21410_b300 as P
    lib = P.lib
    nf = _fine(nc)
    pc, pf = P.Plan(nc), P.Plan(nf)
    prec = P.FP64 if dtype == torch.float64 else P.FP32
    for seed in (31, 32):  # two calls in a row, different inputs
        uc = torch.from_numpy(W.random_field(pc.shape, seed)).to("cuda", dtype)
        ref = torch.empty(pf.shape, dtype=dtype, device="cuda")
        got = torch.full(pf.shape, float("nan"), dtype=dtype, device="cuda")
        pf._sync_stream()
        assert lib.cheb_prolong(pc.handle, pf.handle, prec, C.c_void_p(uc.data_ptr()),
                                C.c_void_p(ref.data_ptr())) == 0
        assert lib.cheb_prolong_noalloc(pc.handle, pf.handle, prec, C.c_void_p(uc.data_ptr()),
                                        C.c_void_p(got.data_ptr())) == 0
        torch.cuda.synchronize()
        r, g = ref.double().cpu().numpy(), got.double().cpu().numpy()
        assert np.isfinite(g).all()
        assert np.linalg.norm(g - r) / np.linalg.norm(r) <= tol


def test_noalloc_prolong_allocates_nothing_and_matches_oracle():
    """On a plan pair that never ran cheb_prolong (which would allocate its
    scratch on the fine plan), the device's free memory is unchanged by the
    call, and the result is the oracle's barycentric prolongation."""
    import paper_2606_21410_b300 as P
    lib = P.lib
    nc = (65, 65, 65)
    nf = _fine(nc)
    # a first call on another pair of the same sizes loads the kernels (the
    # driver may reserve per-kernel memory at a first launch)
    warm_c, warm_f = P.Plan(nc), P.Plan(nf)
    wc = torch.zeros(warm_c.shape, dtype=torch.float64, device="cuda")
    wf = torch.empty(warm_f.shape, dtype=torch.float64, device="cuda")
    warm_f._sync_stream()
    assert lib.cheb_prolong_noalloc(warm_c.handle, warm_f.handle, P.FP64, C.c_void_p(wc.data_ptr()),
                                    C.c_void_p(wf.data_ptr())) == 0
    pc, pf = P.Plan(nc), P.Plan(nf)
    gc, gf = O.Grid(nc), O.Grid(nf)
    u = W.random_field(gc.shape, 33)
    uc = torch.from_numpy(u).cuda()
    got = torch.empty(pf.shape, dtype=torch.float64, device="cuda")
    pf._sync_stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert lib.cheb_prolong_noalloc(pc.handle, pf.handle, P.FP64, C.c_void_p(uc.data_ptr()),
                                        C.c_void_p(got.data_ptr())) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref = O.prolong(u, gc, gf)
    g = got.cpu().numpy()
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-12


def test_noalloc_prolong_rejects_grids_beyond_its_scratch():
    import paper_2606_21410_b300 as P
    lib = P.lib
    pc, pf = P.Plan((129, 129, 129)), P.Plan((257, 257, 257))
    uc = torch.zeros(pc.shape, dtype=torch.float64, device="cuda")
    uf = torch.zeros(pf.shape, dtype=torch.float64, device="cuda")
    st = lib.cheb_prolong_noalloc(pc.handle, pf.handle, P.FP64, C.c_void_p(uc.data_ptr()),
                                  C.c_void_p(uf.data_ptr()))
    assert st == -6
    assert b"16 MiB" in lib.cheb_last_error()
