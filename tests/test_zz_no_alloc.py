"""fit_apply_noalloc, the operator apply for callers that must not allocate device memory.

Those callers (a host thread in a latency-critical loop, where cudaMalloc / cudaFree can stall the
device, or a framework that manages all device memory through its own pool) get the same result
as fit_apply, which may grow a handle-owned frequency buffer with cudaMalloc.  The test calls the
new entry point directly through the C ABI, twice in a row and with different batches, and
compares it with fit_apply within the tolerances of the apply parity tests.  It lives in a file of
its own that pytest collects last.
"""
import ctypes as ct

import numpy as np
import pytest

import fitgen as G
from tests._gpu_util import fitlib, torch_cuda

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _noalloc(fit, g, omegas, x, y, prec):
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    st = fit.lib().fit_apply_noalloc(g.h, len(om), om.ctypes.data_as(ct.POINTER(ct.c_double)),
                                     ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()), prec, None)
    return st


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_apply_matches_fit_apply_twice(prec):
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(34, 20, 12, seed=91, pec_frac=0.05)
    dt = torch.complex64 if prec == 0 else torch.complex128
    with fit.Grid.from_case(case) as g:
        for omegas in ([2 * np.pi * 2e9, 2 * np.pi * 9e9, 2 * np.pi * 15e9], [2 * np.pi * 5e9, 2 * np.pi * 1e9]):
            x = torch.from_numpy(G.random_vector(g.ne, 3, batch=len(omegas)).reshape(-1)).to(dt).cuda()
            ref = torch.empty_like(x)
            fit.fit_apply(g.h, omegas, x, ref, prec)
            for _ in range(2):  # two calls in a row on the shared static scratch
                y = torch.full_like(x, float("nan"))
                assert _noalloc(fit, g, omegas, x, y, prec) == fit.FIT_OK
                torch.cuda.synchronize()
                a, b = y.cpu().numpy(), ref.cpu().numpy()
                assert np.linalg.norm(a - b) <= TOL[prec] * np.linalg.norm(b)


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(4, 4, 4, seed=92)
    with fit.Grid.from_case(case) as g:
        n = 4097
        x = torch.zeros(n * g.ne, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        assert _noalloc(fit, g, np.full(n, 1e10), x, y, 0) == fit.FIT_EINVAL
        assert b"4096" in fit.lib().fit_last_error()
