"""Pins of the oracle's material matrices (Sec. II, Eq. Material) and PEC edge mask: hand-computed
entries on a non-uniform 2x2x2 grid (tests/golden/materials_2x2x2.txt), closed forms for a
homogeneous medium and a two-layer interface, and a loop-by-loop restatement."""
import os

import numpy as np
import pytest

import fitgen as G
from oracle import fit as F

GOLD = os.path.join(os.path.dirname(__file__), "golden", "materials_2x2x2.txt")


def _golden_case():
    nx = ny = nz = 2
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    eps = (1 + i + 2 * j + 4 * k).astype(np.float64)
    return dict(dx=np.array([1e-3, 2e-3]), dy=np.array([1e-3, 3e-3]), dz=np.array([2e-3, 1e-3]),
                eps_r=eps, sigma=10.0 * eps, inv_mu_r=1.0 / (1.0 + i))


def test_golden_2x2x2_entries():
    c = _golden_case()
    m_eps, m_kap, m_nu, mask = F.material_diagonals(c["dx"], c["dy"], c["dz"], c["eps_r"], c["sigma"], c["inv_mu_r"])
    n_checked = 0
    with open(GOLD) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, i, j, k, w, val = line.split()
            idx = 3 * (int(i) + 2 * (int(j) + 2 * int(k))) + int(w)
            got = {"eps": m_eps[idx] / F.EPS0, "kap": m_kap[idx], "nu": m_nu[idx] * F.MU0}[kind]
            assert got == pytest.approx(float(val), rel=1e-13), line
            n_checked += 1
    assert n_checked == 11


def test_homogeneous_uniform_closed_form():
    n, h, er, mur, sig = 5, 0.7e-3, 3.3, 2.0, 0.4
    one = np.ones((n, n, n))
    m_eps, m_kap, m_nu, mask = F.material_diagonals(np.full(n, h), np.full(n, h), np.full(n, h),
                                                    er * one, sig * one, one / mur)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    inner = ((i > 0) & (j > 0) & (k > 0)).ravel()
    for w in range(3):
        assert np.allclose(m_eps.reshape(-1, 3)[inner, w], F.EPS0 * er * h, rtol=1e-14)
        assert np.allclose(m_kap.reshape(-1, 3)[inner, w], sig * h, rtol=1e-14)
        assert np.allclose(m_nu.reshape(-1, 3)[inner, w], 1.0 / (F.MU0 * mur * h), rtol=1e-14)


def test_two_layer_interface_is_arithmetic_mean():
    """An x-edge lying on a z-interface between eps1 (below) and eps2 (above) sees (eps1+eps2)/2;
    a z-facet crossed by the dual edge through both layers sees the length-weighted 1/mu."""
    n, h = 4, 1e-3
    eps = np.ones((n, n, n))
    eps[:2] = 2.0
    eps[2:] = 6.0
    imu = np.ones((n, n, n))
    imu[2:] = 0.25
    m_eps, _, m_nu, _ = F.material_diagonals(np.full(n, h), np.full(n, h), np.full(n, h), eps, 0 * eps, imu)
    idx = 3 * (1 + n * (1 + n * 2))  # x-edge of cell (1,1,2): z-node 2 is the interface
    assert m_eps[idx] == pytest.approx(F.EPS0 * 4.0 * h, rel=1e-14)
    assert m_nu[idx + 2] == pytest.approx((0.5 * h * 1.0 + 0.5 * h * 0.25) / (F.MU0 * h * h), rel=1e-14)


@pytest.mark.parametrize("seed,shape,pec_frac", [(1, (3, 4, 5), 0.0), (2, (4, 3, 3), 0.3), (3, (2, 5, 2), 0.5)])
def test_vectorised_equals_loops(seed, shape, pec_frac):
    c = G.small_random(*shape, seed=seed, pec_frac=pec_frac)
    a = F.material_diagonals(c["dx"], c["dy"], c["dz"], c["eps_r"], c["sigma"], c["inv_mu_r"], c["pec"])
    b = F.material_diagonals_loops(c["dx"], c["dy"], c["dz"], c["eps_r"], c["sigma"], c["inv_mu_r"], c["pec"])
    for u, v in zip(a[:3], b[:3]):
        assert np.allclose(u, v, rtol=1e-14, atol=0)
    assert np.array_equal(a[3], b[3])


@pytest.mark.parametrize("n", [2, 3, 16])
def test_mask_counts_of_empty_cavity(n):
    """Free edges of an empty PEC box: 3 n (n-1)^2 (10800 for n = 16)."""
    mask = F.edge_mask(n, n, n)
    assert int((mask == 0).sum()) == 3 * n * (n - 1) ** 2


def test_pec_cell_masks_its_twelve_edges():
    n = 5
    pec = np.zeros((n, n, n), np.uint8)
    pec[2, 2, 2] = 1
    m = F.edge_mask(n, n, n, pec).reshape(n, n, n, 3) - F.edge_mask(n, n, n).reshape(n, n, n, 3)
    got = {(int(k), int(j), int(i), int(w)) for k, j, i, w in zip(*np.nonzero(m))}
    want = set()
    for a in (0, 1):
        for b in (0, 1):
            want |= {(2 + b, 2 + a, 2, 0), (2 + b, 2, 2 + a, 1), (2, 2 + b, 2 + a, 2)}
    assert got == want and len(want) == 12
