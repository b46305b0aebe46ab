"""Pins of the oracle's system operator A(w) = C^T M_nu C - w^2 M_eps + j w M_kappa (Eq. e2):
complex symmetry, 13 nonzeros per interior line (Sec. II), the curl-curl null space, the exact
discrete spectrum of a uniform PEC cavity and its O(h^2) convergence to the analytic cavity
resonances (Sec. IV), and the sampled-row path used at full sizes."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse.linalg as spla

import fitgen as G
from oracle import fit as F


def _mats(case):
    return F.material_diagonals(case["dx"], case["dy"], case["dz"], case["eps_r"], case["sigma"],
                                case["inv_mu_r"], case["pec"])


def test_A_is_complex_symmetric_with_13_nonzeros():
    c = G.small_random(6, 5, 7, seed=4, pec_frac=0.1)
    me, mk, mn, mask = _mats(c)
    A = F.system_matrix(2 * np.pi * 3e9, F.curl(6, 5, 7), me, mk, mn, mask)
    assert abs(A - A.T).max() == 0
    nnz = np.diff(A.indptr)
    assert nnz.max() == 13
    assert np.all(A[np.nonzero(mask)[0]].toarray() == np.eye(A.shape[0])[np.nonzero(mask)[0]])
    assert np.all(A[:, np.nonzero(mask)[0]].toarray() == np.eye(A.shape[0])[:, np.nonzero(mask)[0]])


def test_interior_row_has_13_nonzeros():
    n = 6
    c = G.cavity(n)
    me, mk, mn, mask = _mats(c)
    A = F.system_matrix(2 * np.pi * 1e9, F.curl(n, n, n), me, mk, mn, mask)
    row = 3 * (2 + n * (3 + n * 3)) + 0  # x-edge well inside the box
    assert A[row].count_nonzero() == 13


@pytest.mark.parametrize("n", [4, 6, 8])
def test_curlcurl_is_psd_with_gradient_null_space(n):
    c = G.cavity(n)
    me, mk, mn, mask = _mats(c)
    K = F.curlcurl(F.curl(n, n, n), mn, mask)
    free = np.nonzero(mask == 0)[0]
    ev = np.linalg.eigvalsh(K[free][:, free].toarray())
    scale = ev.max()
    assert ev.min() > -1e-12 * scale
    assert int((ev < 1e-9 * scale).sum()) == (n - 1) ** 3


@pytest.mark.parametrize("n", [6, 8])
def test_cavity_full_spectrum_matches_discrete_closed_form(n):
    h = 1e-3
    c = G.cavity(n, h)
    me, mk, mn, mask = _mats(c)
    K = F.curlcurl(F.curl(n, n, n), mn, mask)
    free = np.nonzero(mask == 0)[0]
    ev = sl.eigh(K[free][:, free].toarray(), np.diag(me[free]), eigvals_only=True)
    cf = F.cavity_eigenvalues(n, h)
    assert len(ev) == len(cf) == 3 * n * (n - 1) ** 2
    assert np.max(np.abs(np.sort(ev) - cf)) <= 1e-12 * cf.max()


def _lowest_modes(n, h, k=5):
    c = G.cavity(n, h)
    me, mk, mn, mask = _mats(c)
    K = F.curlcurl(F.curl(n, n, n), mn, mask)
    free = np.nonzero(mask == 0)[0]
    Kf = K[free][:, free].tocsc()
    Mf = np.asarray(me[free])
    # Eq. e2s: the symmetric form M^-1/2 K M^-1/2 has the same eigenvalues
    import scipy.sparse as sp
    d = sp.diags(1.0 / np.sqrt(Mf))
    As = (d @ Kf @ d).tocsc()
    lam1 = (2 * F.C0 / h) ** 2 * 2 * np.sin(np.pi / (2 * n)) ** 2
    # shift-invert Lanczos near the lowest mode; the (n-1)^3-fold zero eigenvalue (gradients) is
    # filtered out, and extra Ritz vectors keep the degenerate modes from being missed
    ev = spla.eigsh(As, k=k + 8, sigma=1.2 * lam1, which="LM", ncv=60, return_eigenvectors=False)
    ev = np.sort(ev[ev > 1e-6 * lam1])
    return ev[:k]


def test_cavity16_lowest_modes_tight():
    """16^3 PEC cube (the cavity workload): lowest modes are (1,1,0) x3 and (1,1,1) x2."""
    n, h = 16, 1e-3
    ev = _lowest_modes(n, h, k=5)
    s1 = np.sin(np.pi / (2 * n)) ** 2
    want = (2 * F.C0 / h) ** 2 * np.array([2 * s1] * 3 + [3 * s1] * 2)
    assert np.allclose(ev, want, rtol=1e-10)
    f110 = np.sqrt(ev[0]) / (2 * np.pi)
    assert f110 > 5e9  # 5 GHz lies below the first resonance of the 16 mm cube
    assert f110 == pytest.approx(F.cavity_frequency(16e-3, 16e-3, 16e-3, 1, 1, 0), rel=5e-3)


def test_cavity_converges_to_analytic_at_second_order():
    a = 16e-3
    errs = []
    for n in (4, 8, 16):
        ev = _lowest_modes(n, a / n, k=3)
        f = np.sqrt(ev[0]) / (2 * np.pi)
        errs.append(abs(f - F.cavity_frequency(a, a, a, 1, 1, 0)) / F.cavity_frequency(a, a, a, 1, 1, 0))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2


def test_sampled_rows_equal_assembled_rows():
    c = G.small_random(5, 6, 4, seed=9, pec_frac=0.15)
    me, mk, mn, mask = _mats(c)
    w = 2 * np.pi * 7e9
    A = F.system_matrix(w, F.curl(5, 6, 4), me, mk, mn, mask)
    rows = np.random.default_rng(0).choice(A.shape[0], 40, replace=False)
    Ar = F.system_rows(w, 5, 6, 4, rows, me, mk, mn, mask)
    assert abs(Ar - A[rows]).max() <= 1e-15 * abs(A).max()


def test_jacobi_diagonal_is_diag_of_A():
    c = G.small_random(4, 4, 5, seed=11, pec_frac=0.1)
    me, mk, mn, mask = _mats(c)
    w = 2 * np.pi * 4e9
    A = F.system_matrix(w, F.curl(4, 4, 5), me, mk, mn, mask)
    d = F.jacobi_diagonal(w, 4, 4, 5, me, mk, mn, mask)
    assert np.allclose(d, A.diagonal(), rtol=1e-14, atol=0)


def test_A_is_singular_exactly_at_a_cavity_resonance():
    """A(w) of the vacuum PEC cube (restricted to unmasked edges) is singular when w^2 is an eigenvalue
    of the closed-form discrete spectrum and regular halfway between two of them: this fixes the sign
    and the scale of the -w^2 M_eps term against the curl-curl part independently of the solvers."""
    n, h = 4, 1e-3
    c = G.cavity(n, h)
    me, mk, mn, mask = _mats(c)
    free = np.nonzero(mask == 0)[0]
    lam = np.unique(np.round(F.cavity_eigenvalues(n, h)[F.cavity_eigenvalues(n, h) > 0], -6))
    for w2, singular in ((lam[0], True), (0.5 * (lam[0] + lam[1]), False)):
        A = F.system_matrix(np.sqrt(w2), F.curl(n, n, n), me, mk, mn, mask).toarray()[np.ix_(free, free)]
        smin = np.linalg.svd(A, compute_uv=False).min() / np.abs(A).max()
        assert (smin < 1e-8) == singular, (w2, smin)


def test_a_current_source_delivers_power_into_a_lossy_grid():
    """Time-harmonic convention of Eq. e2 (b = -j w j): the power a current source delivers to a passive
    lossy medium, -Re(e^T conj(j)) / 2, is positive.  A sign slip in the right-hand side or in the loss
    term makes it negative."""
    c = G.small_random(6, 5, 5, seed=23, pec_frac=0.05)
    me, mk, mn, mask = _mats(c)
    w = 2 * np.pi * 2e9
    A = F.system_matrix(w, F.curl(6, 5, 5), me, mk, mn, mask)
    for seed in (1, 2, 3):
        j = G.random_vector(A.shape[0], seed) * (1 - mask)
        e = spla.spsolve(A.tocsc(), F.rhs_from_current(w, j, mask))
        p = -0.5 * np.real(e @ np.conj(j))
        assert p > 0, (seed, p)
