"""GPU symmetrised form (Eq. e2s / Eq. e2tt) against the oracle.

* fit_apply_sym: every output element against the oracle's assembled A_s(w) x' (complex128 to 1e-12 of
  the output norm; complex64 to 1e-5, the single-precision bound of the 13-term rows).
* FIT_PC_EPS: the change of variable e' = M_eps^{1/2} e as a split diagonal preconditioner.  Solves reach
  the oracle's direct solution; complex128 COCG takes the same number of iterations as the oracle's COCG
  with the M_eps^{-1} preconditioner (the same recurrence and stop test) up to rounding."""
import numpy as np
import pytest

import fitgen as G
from tests._gpu_util import fitlib, oracle_A, oracle_matrices, relerr, torch_cuda

pytestmark = pytest.mark.gpu


def _sym(case, w):
    from oracle import fit as F
    from oracle import symmetric as S
    me, mk, mn, mask = oracle_matrices(case)
    return S.symmetrised_matrix(w, F.curl(case["nx"], case["ny"], case["nz"]), me, mk, mn, mask), me, mask


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)])
@pytest.mark.parametrize("dims,pec", [((37, 11, 6), 0.1), ((8, 9, 5), 0.0)])
def test_apply_sym_matches_oracle(prec, tol, dims, pec):
    torch = torch_cuda()
    fit = fitlib()
    nx, ny, nz = dims
    case = G.small_random(nx, ny, nz, seed=17, pec_frac=pec)
    ne = 3 * nx * ny * nz
    ws = 2 * np.pi * np.array([0.9e9, 6e9])
    x = G.random_vector(ne, 5, batch=2)
    dt = torch.complex128 if prec == 1 else torch.complex64
    with fit.Grid.from_case(case) as g:
        xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to(dt).cuda()
        yd = torch.empty_like(xd)
        fit.fit_apply_sym(g.h, ws, xd, yd, prec)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().astype(np.complex128).reshape(2, ne)
    xin = x if prec == 1 else x.astype(np.complex64).astype(np.complex128)  # what the kernel was given
    for b, w in enumerate(ws):
        As, _, mask = _sym(case, w)
        want = As @ xin[b]
        assert relerr(y[b], want) <= tol, (b, relerr(y[b], want))
        assert np.array_equal(y[b][mask != 0], xin[b][mask != 0])  # identity rows, bit for bit


def test_apply_sym_is_scaled_apply():
    """A_s x' = D A (D x'): the symmetrised apply against the unsymmetrised fused apply of D x'."""
    torch = torch_cuda()
    fit = fitlib()
    from oracle import symmetric as S
    case = G.small_random(40, 16, 9, seed=2, pec_frac=0.05)
    ne = 3 * 40 * 16 * 9
    me, mk, mn, mask = oracle_matrices(case)
    d = S.eps_scaling(me, mask)
    w = 2 * np.pi * 2.5e9
    x = G.random_vector(ne, 8)
    with fit.Grid.from_case(case) as g:
        xs = torch.from_numpy(x).cuda()
        ys = torch.empty_like(xs)
        fit.fit_apply_sym(g.h, [w], xs, ys, fit.FIT_C128)
        xd = torch.from_numpy(np.where(mask != 0, 0, d * x)).cuda()
        yd = torch.empty_like(xd)
        g.apply([w], xd, yd, fit.FIT_C128)
        torch.cuda.synchronize()
        got, via = ys.cpu().numpy(), yd.cpu().numpy()
    free = mask == 0
    assert relerr(got[free], d[free] * via[free]) <= 1e-12


@pytest.mark.parametrize("method,precision", [(2, 0), (2, 1), (0, 1), (1, 1)])
def test_eps_preconditioned_solve(method, precision):
    from oracle import fit as F
    from oracle import krylov as K
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(20, 18, 11, seed=31, pec_frac=0.05)
    w = 2 * np.pi * 4e9
    A, mask = oracle_A(case, w)
    ne = A.shape[0]
    b = F.rhs_from_current(w, G.random_vector(ne, 3), mask)
    with fit.Grid.from_case(case) as g:
        bd = torch.from_numpy(b).cuda()
        xd = torch.zeros_like(bd)
        st, rep = g.solve([w], bd, xd, 1e-10, method=method, precision=precision, precond=fit.FIT_PC_EPS,
                          max_iter=40000, max_outer=1000)
        torch.cuda.synchronize()
        x = xd.cpu().numpy()
    assert st == 0 and rep[0]["status"] == 0, rep
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    xo = K.sparse_solve(A, b)
    assert relerr(x, xo) <= 1e-6


def test_cocg_eps_iterations_match_oracle():
    """Lossless graded grid: complex128 COCG with FIT_PC_EPS against the oracle's COCG with the M_eps^-1
    diagonal, i.e. COCG on the symmetrised system."""
    from oracle import fit as F
    from oracle import krylov as K
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(14, 12, 10, seed=6, pec_frac=0.05, lossy=False)
    w = 2 * np.pi * 1e9
    A, mask = oracle_A(case, w)
    me, _, _, _ = oracle_matrices(case)
    ne = A.shape[0]
    b = F.rhs_from_current(w, G.random_vector(ne, 4), mask)
    dinv = np.where(mask != 0, 1.0, 1.0 / np.where(mask != 0, 1.0, me))
    _, it_o, rr_o, st_o = K.cocg(A, b, tol=1e-9, maxiter=20000, dinv=dinv)
    assert st_o == 0
    with fit.Grid.from_case(case) as g:
        bd = torch.from_numpy(b).cuda()
        xd = torch.zeros_like(bd)
        st, rep = g.solve([w], bd, xd, 1e-9, method=fit.FIT_COCG, precision=fit.FIT_SOLVE_C128,
                          precond=fit.FIT_PC_EPS, max_iter=20000)
    assert st == 0, rep
    assert abs(rep[0]["iterations"] - it_o) <= max(5, 0.1 * it_o), (rep[0]["iterations"], it_o)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("workload", ["layered128", "stripline96"])
def test_apply_sym_sampled_full_size(prec, workload):
    """The full-size workloads: the GPU applies A_s to the whole vector; the oracle forms sampled rows of
    D A D one by one (rows of A from the definition of C, scaled by D = M_eps^-1/2; masked rows are the
    identity)."""
    from oracle import fit as F
    from oracle import symmetric as S
    torch = torch_cuda()
    fit = fitlib()
    case = G.layered_blocks() if workload == "layered128" else G.stripline()
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    ne = 3 * nx * ny * nz
    w = 2 * np.pi * float(case["freqs"][0])
    dt = torch.complex64 if prec == 0 else torch.complex128
    with fit.Grid.from_case(case) as g:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(11)
        x = torch.randn(ne, dtype=dt, device="cuda", generator=gen)
        y = torch.empty_like(x)
        fit.fit_apply_sym(g.h, [w], x, y, prec)
        torch.cuda.synchronize()
        me, mk, mn, mask = oracle_matrices(case)
        d = S.eps_scaling(me, mask)
        rng = np.random.default_rng(5)
        rows = np.unique(np.concatenate([rng.choice(ne, 200, replace=False), np.arange(12), np.arange(ne - 12, ne)]))
        R = F.system_rows(w, nx, ny, nz, rows, me, mk, mn, mask).tocoo()
        vals = R.data * d[rows[R.row]] * d[R.col]
        vals = np.where(mask[rows[R.row]] != 0, R.data, vals)  # identity rows stay 1
        cols = np.unique(R.col)
        xs = np.zeros(ne, np.complex128)
        xs[cols] = x[torch.from_numpy(cols).cuda()].cpu().numpy().astype(np.complex128)
        want = np.zeros(len(rows), np.complex128)
        np.add.at(want, R.row, vals * xs[R.col])
        got = y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
    assert relerr(got, want) <= (1e-5 if prec == 0 else 1e-12), relerr(got, want)


def test_material_ranges_are_checked_on_the_host():
    """Out-of-range materials are refused before any device work: a non-positive eps_r in
    fit_set_materials, and a zero M_eps on an unmasked edge for the symmetrised form (whose D divides
    by it) after fit_set_material_matrices; the unsymmetrised apply still accepts those matrices."""
    torch = torch_cuda()
    fit = fitlib()
    case = G.small_random(6, 5, 4, seed=3)
    with fit.Grid(6, 5, 4, case["dx"], case["dy"], case["dz"]) as g:
        bad = case["eps_r"].copy()
        bad[1, 2, 3] = 0.0
        with pytest.raises(fit.FitError):
            fit.fit_set_materials(g.h, bad, case["sigma"], case["inv_mu_r"], case["pec"])
        neg = case["sigma"].copy()
        neg[0, 0, 0] = -1.0
        with pytest.raises(fit.FitError):
            fit.fit_set_materials(g.h, case["eps_r"], neg, case["inv_mu_r"], case["pec"])
        me, mk, mn, mask = oracle_matrices(case)
        free = np.flatnonzero(mask == 0)
        me = me.copy()
        me[free[7]] = 0.0
        fit.fit_set_material_matrices(g.h, me, mk, mn, mask)
        ne = 3 * 6 * 5 * 4
        x = torch.zeros(ne, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        fit.fit_apply(g.h, [1e9], x, y, fit.FIT_C128)
        with pytest.raises(fit.FitError):
            fit.fit_apply_sym(g.h, [1e9], x, y, fit.FIT_C128)
        with pytest.raises(fit.FitError):
            g.solve([1e9], x, y, 1e-8, precond=fit.FIT_PC_EPS)
