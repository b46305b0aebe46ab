"""GPU parity of the fused operator apply y = A(w) x against the oracle's assembled A (Eq. e2):
relative error <= 1e-12 in complex128 and <= 1e-5 in complex64, element by element on grids that
span several tiles with ragged tails, batched, with PEC cells; sampled rows at the full sizes of
the benchmark workloads."""
import numpy as np
import pytest

import fitgen as G
from tests._gpu_util import fitlib, oracle_A, oracle_matrices, rand_vec, relerr, torch_cuda

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}  # FIT_C64, FIT_C128


def _apply(fit, torch, g, omegas, xs, prec):
    dt = torch.complex64 if prec == fit.FIT_C64 else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(xs)).to(dt).cuda().reshape(-1)
    y = torch.empty_like(x)
    fit.fit_apply(g.h, omegas, x, y, prec)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128).reshape(len(omegas), -1)


@pytest.fixture(params=["auto", "generic", "fused:0"])
def kernel(request, monkeypatch):
    """Runs a test with the autotuned kernel, and with the generic / first fused kernel forced."""
    if request.param != "auto":
        monkeypatch.setenv("FIT_APPLY_KERNEL", request.param)
    return request.param


def _check_case(case, omegas, prec, use_matrices=False, seed=0):
    torch = torch_cuda()
    fit = fitlib()
    ne = 3 * case["nx"] * case["ny"] * case["nz"]
    g = fit.Grid(case["nx"], case["ny"], case["nz"], case["dx"], case["dy"], case["dz"])
    try:
        if use_matrices:
            me, mk, mn, mask = oracle_matrices(case)
            fit.fit_set_material_matrices(g.h, me, mk, mn, mask)
        else:
            fit.fit_set_materials(g.h, case["eps_r"], case["sigma"], case["inv_mu_r"], case["pec"])
        xs = rand_vec(ne, seed, batch=len(omegas))
        if prec == fit.FIT_C64:
            xs = xs.astype(np.complex64).astype(np.complex128)
        ys = _apply(fit, torch, g, omegas, xs, prec)
        for b, w in enumerate(omegas):
            A, mask = oracle_A(case, w)
            yo = A @ xs[b]
            err = relerr(ys[b], yo)
            assert err <= TOL[prec], (case["name"], b, err)
            # element-wise: every entry within tol of the largest entry
            assert np.max(np.abs(ys[b] - yo)) <= 4 * TOL[prec] * np.max(np.abs(yo))
            assert np.array_equal(ys[b][mask != 0], xs[b][mask != 0].astype(ys.dtype)) or prec == fit.FIT_C64
    finally:
        g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_cavity16(prec, kernel):
    _check_case(G.cavity(16), [2 * np.pi * 5e9], prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(37, 21, 19), (34, 21, 19), (66, 9, 5), (48, 40, 3), (33, 40, 3)])
def test_apply_random_ragged_batched(prec, shape, kernel):
    case = G.small_random(*shape, seed=sum(shape), pec_frac=0.08)
    _check_case(case, [2 * np.pi * 1e9, 2 * np.pi * 7.5e9, 2 * np.pi * 20e9], prec, seed=1)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_with_loaded_matrices(prec, kernel):
    case = G.small_random(20, 18, 11, seed=77, pec_frac=0.1)
    _check_case(case, [2 * np.pi * 3e9, 2 * np.pi * 9e9], prec, use_matrices=True, seed=2)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 1), (2, 1, 7), (3, 3, 1), (2, 2, 2)])
def test_apply_degenerate_shapes(shape, kernel):
    case = G.small_random(*shape, seed=5, pec_frac=0.0)
    _check_case(case, [2 * np.pi * 2e9], 1)
    _check_case(case, [2 * np.pi * 2e9], 0)


def _sampled_rows(case, omega, prec, nsample=200, seed=3):
    """Full-size workload: the GPU applies to the whole vector; the oracle computes sampled rows
    one by one from the definition of C (no full assembly)."""
    from oracle import fit as F
    torch = torch_cuda()
    fit = fitlib()
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    ne = 3 * nx * ny * nz
    g = fit.Grid.from_case(case)
    try:
        rng = np.random.default_rng(seed)
        dt = torch.complex64 if prec == 0 else torch.complex128
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        x = torch.randn(ne, dtype=dt, device="cuda", generator=gen)
        y = torch.empty_like(x)
        fit.fit_apply(g.h, [omega], x, y, prec)
        torch.cuda.synchronize()
        me, mk, mn, mask = oracle_matrices(case)
        rows = np.unique(np.concatenate([rng.choice(ne, nsample, replace=False),
                                         np.arange(0, 12), np.arange(ne - 12, ne)]))
        R = F.system_rows(omega, nx, ny, nz, rows, me, mk, mn, mask)
        cols = np.unique(R.indices)
        xs = x[torch.from_numpy(cols).cuda()].cpu().numpy().astype(np.complex128)
        xfull = np.zeros(ne, np.complex128)
        xfull[cols] = xs
        yo = R @ xfull
        yg = y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
        err = relerr(yg, yo)
        assert err <= TOL[prec], (case["name"], err)
    finally:
        g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_sampled_layered128(prec, kernel):
    case = G.layered_blocks()
    _sampled_rows(case, 2 * np.pi * case["freqs"][0], prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_sampled_stripline96(prec, kernel):
    case = G.stripline()
    _sampled_rows(case, 2 * np.pi * case["freqs"][-1], prec)


def test_apply_sampled_package256_c64(kernel):
    case = G.package()
    _sampled_rows(case, 2 * np.pi * case["freqs"][3], 0, nsample=300)


@pytest.mark.parametrize("prec", [0, 1])
def test_every_fused_variant(prec, monkeypatch):
    """Each launch shape the autotuner may pick, forced in turn, on a ragged grid: one system (where
    the warp-specialised kernel splits the (column, plane) pairs evenly over the CTAs, so ranges
    start and end inside columns) and a batch of two (tiles of whole z-chunks)."""
    fit = fitlib()
    case = G.small_random(70, 27, 37, seed=8, pec_frac=0.07)
    for k in range(fit.fit_apply_variant_count(prec)):
        monkeypatch.setenv("FIT_APPLY_KERNEL", f"fused:{k}")
        _check_case(case, [2 * np.pi * 5e9], prec, seed=100 + k)
        _check_case(case, [2 * np.pi * 2e9, 2 * np.pi * 11e9], prec, seed=k)


def test_autotuner_records_a_choice():
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(64, 32, 40, seed=9)
    with fit.Grid.from_case(case) as g:
        x = torch.randn(g.ne, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        assert fit.fit_apply_tuned(g.h, 0, 1)["choice"] == -2
        g.apply([1e10], x, y, 0)
        t = fit.fit_apply_tuned(g.h, 0, 1)
        assert t["choice"] >= -1 and t["tx"] == 32 and t["ws"] in (0, 1)
        assert (t["stages"] > 0) == (t["choice"] >= 0) and t["pf"] >= 0
