"""Pins of the symmetrised (Eq. e2s) and factored (Eq. e2tt) forms in the oracle.

What fixes them, independently of the formulas:
* the vacuum PEC cube: the symmetrised operator is an ordinary eigenproblem whose spectrum is the
  closed-form discrete cavity spectrum (a wrong power of M_eps, a missing M_nu or a mask slip fails it);
* a graded, layered, lossless grid: its spectrum equals scipy's generalised eigenvalues of the pencil
  (K, M_eps) of the unsymmetrised system (a library routine);
* a lossy grid with PEC cells: e = D e' maps the symmetrised solution onto the unsymmetrised one
  (fails on a wrong right-hand-side scaling, sign of w^2 or loss term);
* the factored product cal_A^T cal_A and the scaled curl-curl matrix are the same operator;
* COCG on the symmetrised system and COCG on Eq. e2 with the diagonal preconditioner M_eps^{-1} take
  the same iterates (e_k = D e'_k), the reading the GPU path relies on."""
import numpy as np
import pytest
import scipy.linalg as sla

import fitgen as G
from oracle import fit as F
from oracle import krylov as K
from oracle import symmetric as S


def _mats(case):
    me, mk, mn, mask = F.material_diagonals(case["dx"], case["dy"], case["dz"], case["eps_r"], case["sigma"],
                                            case["inv_mu_r"], case["pec"])
    return F.curl(case["nx"], case["ny"], case["nz"]), me, mk, mn, mask


@pytest.mark.parametrize("n", [5, 6])
def test_vacuum_cube_spectrum_is_the_closed_form(n):
    h = 1e-3
    case = G.cavity(n, h=h)
    C, me, mk, mn, mask = _mats(case)
    free = np.flatnonzero(mask == 0)
    a = S.factor(C, me, mn, mask)
    core = (a.T @ a).toarray()[np.ix_(free, free)]
    lam = np.sort(np.linalg.eigvalsh(core))
    want = F.cavity_eigenvalues(n, h)
    assert lam.shape == want.shape
    assert np.allclose(lam, want, rtol=1e-10, atol=1e-10 * want.max())


def test_layered_spectrum_is_the_generalised_one():
    case = G.small_random(5, 4, 4, seed=8, lossy=False)
    C, me, mk, mn, mask = _mats(case)
    free = np.flatnonzero(mask == 0)
    As = S.symmetrised_matrix(0.0, C, me, mk, mn, mask).toarray()[np.ix_(free, free)]
    assert np.abs(As.imag).max() == 0 and np.abs(As - As.T).max() <= 1e-12 * np.abs(As).max()
    lam = np.sort(np.linalg.eigvalsh(As.real))
    Kc = F.curlcurl(C, mn, mask).toarray()[np.ix_(free, free)]
    gen = np.sort(sla.eigh(Kc, np.diag(me[free]), eigvals_only=True))
    assert np.allclose(lam, gen, rtol=1e-9, atol=1e-9 * gen.max())
    assert lam.min() >= -1e-9 * lam.max()  # cal_A^T cal_A is positive semidefinite


def test_factored_equals_scaled_curlcurl():
    case = G.small_random(6, 5, 4, seed=12, pec_frac=0.15)
    C, me, mk, mn, mask = _mats(case)
    w = 2 * np.pi * 3e9
    a = S.symmetrised_matrix(w, C, me, mk, mn, mask)
    b = S.factored_matrix(w, C, me, mk, mn, mask)
    assert abs(a - b).max() <= 1e-12 * abs(a).max()
    assert abs(a - a.T).max() <= 1e-12 * abs(a).max()  # complex symmetric


@pytest.mark.parametrize("seed,pec", [(3, 0.0), (4, 0.2)])
def test_solution_maps_back_to_the_unsymmetrised_one(seed, pec):
    case = G.small_random(7, 6, 5, seed=seed, pec_frac=pec)
    C, me, mk, mn, mask = _mats(case)
    w = 2 * np.pi * 2e9
    j = G.random_vector(len(mask), seed + 50)
    A = F.system_matrix(w, C, me, mk, mn, mask)
    e = K.sparse_solve(A, F.rhs_from_current(w, j, mask))
    As = S.symmetrised_matrix(w, C, me, mk, mn, mask)
    es = K.sparse_solve(As, S.symmetrised_rhs(w, j, me, mask))
    assert np.allclose(S.voltages(es, me, mask), e, rtol=0, atol=1e-9 * np.abs(e).max())


@pytest.mark.parametrize("lossy", [False, True])
def test_cocg_iterates_equal_eps_preconditioned_cocg(lossy):
    case = G.small_random(6, 5, 5, seed=21, pec_frac=0.1, lossy=lossy)
    C, me, mk, mn, mask = _mats(case)
    w = 2 * np.pi * 1.5e9
    j = G.random_vector(len(mask), 9)
    A = F.system_matrix(w, C, me, mk, mn, mask)
    As = S.symmetrised_matrix(w, C, me, mk, mn, mask)
    b = F.rhs_from_current(w, j, mask)
    bs = S.symmetrised_rhs(w, j, me, mask)
    dinv = np.where(mask != 0, 1.0, 1.0 / np.where(mask != 0, 1.0, me))
    # equal in exact arithmetic; rounding differences grow with the iteration count (the lossless
    # system's condition number is ~1e23), so the first 10 iterates are compared
    for k in (2, 5, 10):
        xs, _, _, _ = K.cocg(As, bs, tol=0.0, maxiter=k)
        x, _, _, _ = K.cocg(A, b, tol=0.0, maxiter=k, dinv=dinv)
        assert np.allclose(S.voltages(xs, me, mask), x, rtol=0, atol=1e-11 * np.abs(x).max()), k
