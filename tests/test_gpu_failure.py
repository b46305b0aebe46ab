"""Failure detection on the GPU without a fault: the grid's abort word (pinned host memory that the
kernels read) and the device error word that fit_sync and fit_solve report.

Every failure here is made on the host: the abort word is set while work is queued or running, and
the kernels' bounded waits and the solver's loop tests return an error status that the host reads.
Nothing traps, faults or hangs; the grid is used again afterwards to show the context is intact."""
import ctypes as ct
import threading
import time

import numpy as np
import pytest

import fitgen as G
from tests._gpu_util import fitlib, oracle_A, relerr, torch_cuda

pytestmark = pytest.mark.gpu


def _pinned_omegas(torch, omegas):
    """Frequencies in pinned host memory, so that staging them never waits on the stream."""
    t = torch.tensor(omegas, dtype=torch.float64).pin_memory()
    return t, ct.cast(ct.c_void_p(t.data_ptr()), ct.POINTER(ct.c_double))


def test_abort_word_refuses_new_work():
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(16, 12, 8, seed=31)
    w = 2 * np.pi * 3e9
    with fit.Grid.from_case(case) as g:
        x = torch.from_numpy(G.random_vector(g.ne, 1)).to(torch.complex64).cuda()
        y = torch.full_like(x, float("nan"))
        fit.fit_set_abort(g.h, 1)
        with pytest.raises(fit.FitError) as e:
            g.apply([w], x, y, fit.FIT_C64)
        assert e.value.status == fit.FIT_ETIMEOUT and "abort" in str(e.value)
        b = torch.zeros(g.ne, dtype=torch.complex128, device="cuda")
        b[100] = 1.0
        xs = torch.zeros_like(b)
        st, _ = g.solve([w], b, xs, 1e-8)
        assert st == fit.FIT_ETIMEOUT
        torch.cuda.synchronize()
        assert torch.isnan(y).all()  # nothing was enqueued
        fit.fit_set_abort(g.h, 0)
        g.apply([w], x, y, fit.FIT_C64)
        assert fit.fit_sync(g.h) == fit.FIT_OK
        A, _ = oracle_A(case, w)
        assert relerr(y.cpu().numpy(), A @ x.cpu().numpy().astype(np.complex128)) <= 1e-5


@pytest.mark.parametrize("kernel", ["ws", "cta"])
def test_abort_stops_a_queued_fused_apply(kernel, monkeypatch):
    """The apply is enqueued behind a 100 ms spin, the abort word is set while it waits, and the fused
    kernel leaves without writing anything; fit_sync reports FIT_ETIMEOUT once and the next apply is
    correct."""
    torch = torch_cuda()
    fit = fitlib()
    # variant 21: warp-specialised, even split; variant 5: CTA-synchronous, balanced z-chunks
    monkeypatch.setenv("FIT_APPLY_KERNEL", "fused:21" if kernel == "ws" else "fused:5")
    case = G.small_random(64, 40, 24, seed=32, pec_frac=0.05)
    w = 2 * np.pi * 5e9
    with fit.Grid.from_case(case) as g:
        L = fit.lib()
        om_t, om = _pinned_omegas(torch, [w])
        x = torch.from_numpy(G.random_vector(g.ne, 2)).to(torch.complex64).cuda()
        ref = torch.empty_like(x)
        stream = torch.cuda.current_stream()
        sp = ct.c_void_p(stream.cuda_stream)
        assert L.fit_apply(g.h, 1, om, ct.c_void_p(x.data_ptr()), ct.c_void_p(ref.data_ptr()), 0, sp) == 0
        assert fit.fit_sync(g.h) == fit.FIT_OK
        y = torch.full_like(x, float("nan"))
        torch.cuda._sleep(int(2e8))  # about 100 ms at 2 GHz
        assert L.fit_apply(g.h, 1, om, ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()), 0, sp) == 0
        fit.fit_set_abort(g.h, 1)
        t0 = time.time()
        st = fit.fit_sync(g.h)
        assert st == fit.FIT_ETIMEOUT, fit.status_str(st)
        assert time.time() - t0 < 5.0
        assert b"abort" in L.fit_last_error()
        assert torch.isnan(y).all()
        fit.fit_set_abort(g.h, 0)
        assert fit.fit_sync(g.h) == fit.FIT_OK  # the error word was cleared by the first report
        assert L.fit_apply(g.h, 1, om, ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()), 0, sp) == 0
        assert fit.fit_sync(g.h) == fit.FIT_OK
        assert torch.equal(y, ref)
        del om_t


def test_abort_ends_a_running_solve():
    """A complex128 COCG solve of the 128^3 layered workload to 1e-12 runs for many seconds; another host
    thread sets the abort word after 2 s and the solve returns FIT_ETIMEOUT promptly with its report
    filled and x holding a finite iterate.  The grid then solves a small system normally."""
    torch = torch_cuda()
    fit = fitlib()
    case = G.layered_blocks()
    w = 2 * np.pi * float(case["freqs"][0])
    with fit.Grid.from_case(case) as g:
        b = (-1j * w) * torch.from_numpy(G.source_vector(case)).cuda()
        x = torch.zeros_like(b)
        # a short solve first, so that the apply kernels are tuned before the timed one starts
        st, _ = g.solve([w], b, x, 1e-12, method=fit.FIT_COCG, precision=fit.FIT_SOLVE_C128,
                        precond=fit.FIT_PC_JACOBI, max_iter=20, max_outer=1)
        assert st == fit.FIT_NOT_CONVERGED
        x.zero_()
        out = {}

        def run():
            out["st"], out["rep"] = g.solve([w], b, x, 1e-12, method=fit.FIT_COCG, precision=fit.FIT_SOLVE_C128,
                                            precond=fit.FIT_PC_JACOBI, max_iter=10_000_000, max_outer=1000)
            out["t"] = time.time()

        th = threading.Thread(target=run)
        th.start()
        time.sleep(2.0)
        assert th.is_alive(), "the solve ended before the abort"
        fit.fit_set_abort(g.h, 1)
        t_abort = time.time()
        th.join(timeout=60)
        assert not th.is_alive()
        fit.fit_set_abort(g.h, 0)
        assert out["st"] == fit.FIT_ETIMEOUT, fit.status_str(out["st"])
        assert out["t"] - t_abort < 5.0
        rep = out["rep"][0]
        # the refinement step length never lets the true residual grow past its start (relres 1)
        assert rep["iterations"] > 0 and 0 < rep["relres"] <= 1.0
        assert torch.isfinite(torch.view_as_real(x)).all()
        assert fit.fit_sync(g.h) == fit.FIT_OK
    small = G.small_random(12, 8, 8, seed=33)
    A, mask = oracle_A(small, w)
    bb = G.random_vector(A.shape[0], 4) * (1 - mask)
    with fit.Grid.from_case(small) as g2:
        bt = torch.from_numpy(bb).cuda()
        xt = torch.zeros_like(bt)
        st, _ = g2.solve([w], bt, xt, 1e-10, method=fit.FIT_COCG, precond=fit.FIT_PC_JACOBI)
        assert st == fit.FIT_OK
        assert relerr(A @ xt.cpu().numpy(), bb) <= 1e-10
