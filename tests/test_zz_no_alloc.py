"""cheb_prolong_noalloc: the prolongation for callers that cannot allocate
device memory (for example code running inside a custom allocator or a
memory-capped process).  It must give the same result as cheb_prolong while
using only the library's fixed internal scratch array, on two calls in a row
(the array keeps the previous call's contents), and must reject grids whose
intermediates do not fit.  Called through the C ABI with ctypes.  This file
is collected last so a failure here leaves every other test already run."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)])
@pytest.mark.parametrize("nc", [(33, 33, 33), (65, 65, 65), (17, 33, 9)])
def test_noalloc_prolong_matches_cheb_prolong_twice(nc, dtype, tol):
    import paper_2606_21410_b300 as P
    lib = P.lib
    nf = tuple(2 * (v - 1) + 1 for v in nc)
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
