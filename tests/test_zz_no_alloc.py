"""fit_apply_noalloc, the operator apply for callers that must not allocate device memory.

Those callers (a host thread in a latency-critical loop, where cudaMalloc / cudaFree can stall the
device, or a framework that manages all device memory through its own pool) get the same result
as fit_apply, which may grow a handle-owned frequency buffer with cudaMalloc.  The tests call the
entry point directly through the C ABI, twice in a row and with different batches, and compare it
with fit_apply and with the oracle's assembled A within the tolerances of the apply parity tests.
They also check the defining property: a batch larger than any fit_apply has seen on the handle
changes neither the bytes the handle holds nor the device's free memory.  The file is collected
last by pytest.
"""
import ctypes as ct

import numpy as np
import pytest

import fitgen as G
from tests._gpu_util import fitlib, oracle_A, relerr, torch_cuda

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


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_allocates_nothing_and_matches_the_oracle(prec):
    """A batch of 100 systems (beyond the 64-entry frequency buffer fit_apply starts a handle with) through
    the allocation-free call: the handle's bytes and the device's free memory do not change across the
    calls, and sampled systems match the oracle's A(omega_b) x_b."""
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(34, 20, 12, seed=93, pec_frac=0.05)
    dt = torch.complex64 if prec == 0 else torch.complex128
    nb = 100
    omegas = 2 * np.pi * np.linspace(1e9, 20e9, nb)
    with fit.Grid.from_case(case) as g:
        x = torch.from_numpy(G.random_vector(g.ne, 5, batch=nb).reshape(-1)).to(dt).cuda()
        y = torch.full_like(x, float("nan"))
        small = torch.empty(2 * g.ne, dtype=dt, device="cuda")
        fit.fit_apply(g.h, omegas[:2], x[:2 * g.ne], small, prec)  # the handle's buffer: 64 frequencies
        torch.cuda.synchronize()
        held = fit.grid_info(g.h)["bytes_held"]
        assert _noalloc(fit, g, omegas, x, y, prec) == fit.FIT_OK  # first call: looks up the scratch address
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            assert _noalloc(fit, g, omegas, x, y, prec) == fit.FIT_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert fit.grid_info(g.h)["bytes_held"] == held
        yc, xc = y.cpu().numpy().reshape(nb, -1), x.cpu().numpy().reshape(nb, -1).astype(np.complex128)
        for b in (0, 37, nb - 1):
            A, _ = oracle_A(case, omegas[b])
            assert relerr(yc[b], A @ xc[b]) <= TOL[prec], b
        ref = torch.empty_like(x)
        fit.fit_apply(g.h, omegas, x, ref, prec)
        torch.cuda.synchronize()
        assert np.linalg.norm(yc - ref.cpu().numpy().reshape(nb, -1)) <= TOL[prec] * np.linalg.norm(yc)


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
