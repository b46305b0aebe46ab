"""Pins of the oracle's solvers: dense LU on a 4^3 grid = sparse direct = BiCGStab = GMRES = COCG, and
manufactured solutions b = A e* recovered within kappa * tol (Sec. IV solvers; Eq. e2)."""
import numpy as np
import pytest

import fitgen as G
from oracle import fit as F
from oracle import krylov as K


def _system(case, f):
    me, mk, mn, mask = F.material_diagonals(case["dx"], case["dy"], case["dz"], case["eps_r"], case["sigma"],
                                            case["inv_mu_r"], case["pec"])
    A = F.system_matrix(2 * np.pi * f, F.curl(case["nx"], case["ny"], case["nz"]), me, mk, mn, mask)
    return A, mask


@pytest.mark.parametrize("lossy", [True, False])
def test_direct_and_krylov_agree_on_4cubed(lossy):
    c = G.small_random(4, 4, 4, seed=5, lossy=lossy)
    A, mask = _system(c, 2e9)
    b = G.random_vector(A.shape[0], seed=6) * (1 - mask)
    x_dense = K.dense_solve(A, b)
    x_sparse = K.sparse_solve(A, b)
    assert np.linalg.norm(x_dense - x_sparse) <= 1e-12 * np.linalg.norm(x_dense)
    xb, it, rr, st = K.bicgstab(A, b, tol=1e-12, maxiter=5000)
    assert st == 0 and rr <= 1e-12
    xg, it, rr, st = K.fgmres(A, b, tol=1e-12, restart=40, maxiter=5000)
    assert st == 0 and rr <= 1e-12
    cond = np.linalg.cond(A.toarray())
    for x in (xb, xg):
        assert np.linalg.norm(x - x_dense) <= 10 * cond * 1e-12 * np.linalg.norm(x_dense)


@pytest.mark.parametrize("kind", ["random", "smooth"])
def test_manufactured_solution(kind):
    c = G.small_random(6, 5, 6, seed=12, pec_frac=0.05)
    A, mask = _system(c, 3e9)
    n = A.shape[0]
    if kind == "random":
        xs = G.random_vector(n, seed=13)
    else:
        cell = np.arange(n) // 3
        i, j, k = cell % 6, (cell // 6) % 5, cell // 30
        xs = np.sin(np.pi * (i + 0.5) / 6) * np.sin(np.pi * (j + 0.5) / 5) * np.sin(np.pi * (k + 0.5) / 6) + 0j
    xs = xs * (1 - mask)
    b = A @ xs
    x, it, rr, st = K.bicgstab(A, b, tol=1e-12, maxiter=20000)
    assert st == 0
    cond = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - xs) <= cond * 1e-12 * np.linalg.norm(xs) * 10
    x2 = K.sparse_solve(A, b)
    assert np.linalg.norm(x2 - xs) <= 1e-9 * np.linalg.norm(xs)


def test_cavity16_bicgstab_vs_sparse_direct():
    """The cavity workload: 16^3 PEC vacuum cube, 5 GHz, unit current on the centre z-edge."""
    c = G.cavity(16)
    A, mask = _system(c, c["freqs"][0])
    b = F.rhs_from_current(2 * np.pi * c["freqs"][0], G.source_vector(c), mask)
    x_d = K.sparse_solve(A, b)
    assert K.relres(A, x_d, b) < 1e-12
    x, it, rr, st = K.bicgstab(A, b, tol=1e-10, maxiter=20000)
    assert st == 0 and rr <= 1e-10
    assert np.linalg.norm(x - x_d) <= 1e-6 * np.linalg.norm(x_d)
    assert np.all(x[mask != 0] == 0)


def test_cocg_is_cg_on_real_spd():
    """On a real symmetric positive definite matrix the unconjugated form equals the inner product,
    so COCG must be CG: it matches the dense solution, and with 6 distinct eigenvalues (a
    block-diagonal matrix built from them) it terminates within 6 steps up to rounding."""
    import scipy.sparse as sp
    rng = np.random.default_rng(3)
    lam = np.array([0.5, 1.0, 2.0, 3.5, 7.0, 11.0])
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    A = sp.csr_matrix(Q @ np.diag(np.repeat(lam, 10)) @ Q.T)
    b = rng.standard_normal(60) + 0j
    x, it, rr, st = K.cocg(A, b, tol=1e-12, maxiter=100)
    assert st == 0 and it <= 7, (it, rr)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-10, atol=0)


@pytest.mark.parametrize("precond", [False, True])
def test_cocg_on_complex_symmetric_4cubed(precond):
    """The lossy 4^3 FIT system is complex symmetric (A^T = A, not Hermitian): COCG, with or without
    the Jacobi diagonal, reaches the dense solution; a conjugated CG on it does not."""
    c = G.small_random(4, 4, 4, seed=5, lossy=True)
    A, mask = _system(c, 2e9)
    assert abs(A - A.T).max() == 0 and abs(A - A.conj().T).max() > 0
    b = G.random_vector(A.shape[0], seed=6) * (1 - mask)
    x_dense = K.dense_solve(A, b)
    dinv = 1.0 / A.diagonal() if precond else None
    x, it, rr, st = K.cocg(A, b, tol=1e-12, maxiter=5000, dinv=dinv)
    assert st == 0 and rr <= 1e-12
    cond = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - x_dense) <= 10 * cond * 1e-12 * np.linalg.norm(x_dense)
    # the Hermitian CG recurrence (conjugated dots) on this non-Hermitian A stalls far above tol
    xr = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = np.vdot(r, r)
    for _ in range(3 * A.shape[0]):
        q = A @ p
        a = rho / np.vdot(p, q)
        xr, r = xr + a * p, r - a * q
        rho2 = np.vdot(r, r)
        p, rho = r + (rho2 / rho) * p, rho2
    assert K.relres(A, xr, b) > 1e-6


def test_cocr_is_minimal_residual_on_real_spd():
    """On a real SPD matrix COCR is the conjugate residual method, which minimises ||b - A x||_2 over
    the Krylov space: its k-th iterate must equal GMRES(k)'s (a different algorithm, Arnoldi +
    least squares) at every k, its residual norms must not increase, and with 6 distinct eigenvalues
    it terminates within 6 steps up to rounding."""
    import scipy.sparse as sp
    rng = np.random.default_rng(4)
    lam = np.array([0.5, 1.0, 2.0, 3.5, 7.0, 11.0])
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    A = sp.csr_matrix(Q @ np.diag(np.repeat(lam, 10)) @ Q.T)
    b = rng.standard_normal(60) + 0j
    prev = np.inf
    for k in range(1, 6):
        xc, _, _, _ = K.cocr(A, b, tol=0.0, maxiter=k)
        xg, _, _, _ = K.fgmres(A, b, tol=0.0, restart=k, maxiter=k)
        assert np.allclose(xc, xg, rtol=0, atol=1e-10 * np.linalg.norm(xg)), k
        rk = np.linalg.norm(b - A @ xc)
        assert rk <= prev * (1 + 1e-12)
        prev = rk
    x, it, rr, st = K.cocr(A, b, tol=1e-12, maxiter=100)
    assert st == 0 and it <= 7, (it, rr)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-10, atol=0)


@pytest.mark.parametrize("precond", [False, True])
def test_cocr_on_complex_symmetric_4cubed(precond):
    """COCR, with or without the Jacobi diagonal, reaches the dense solution of the lossy 4^3 system."""
    c = G.small_random(4, 4, 4, seed=5, lossy=True)
    A, mask = _system(c, 2e9)
    b = G.random_vector(A.shape[0], seed=6) * (1 - mask)
    x_dense = K.dense_solve(A, b)
    dinv = 1.0 / A.diagonal() if precond else None
    x, it, rr, st = K.cocr(A, b, tol=1e-12, maxiter=5000, dinv=dinv)
    assert st == 0 and rr <= 1e-12
    cond = np.linalg.cond(A.toarray())
    assert np.linalg.norm(x - x_dense) <= 10 * cond * 1e-12 * np.linalg.norm(x_dense)


def test_preconditioned_cocr_is_cocr_on_the_scaled_system():
    """COCR with a diagonal M takes the iterates of plain COCR on M^{1/2} A M^{1/2} (x = M^{1/2} x^)."""
    c = G.small_random(5, 4, 4, seed=9, lossy=True, pec_frac=0.1)
    A, mask = _system(c, 1.5e9)
    b = G.random_vector(A.shape[0], seed=2) * (1 - mask)
    dinv = np.abs(1.0 / A.diagonal())  # a positive diagonal, so that M^{1/2} is real
    s = np.sqrt(dinv)
    import scipy.sparse as sp
    As = (sp.diags(s) @ A @ sp.diags(s)).tocsr()
    for k in (2, 5, 10):
        xh, _, _, _ = K.cocr(As, s * b, tol=0.0, maxiter=k)
        x, _, _, _ = K.cocr(A, b, tol=0.0, maxiter=k, dinv=dinv)
        assert np.allclose(s * xh, x, rtol=0, atol=1e-10 * np.abs(x).max()), k
