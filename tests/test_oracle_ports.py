"""Pins of the oracle's port post-processing (Sec. IV: impressed port currents, probe voltages summed
along edges, Z parameters, S parameters with Z0 = 50 Ohm).  What fixes the conventions here is
physics the discrete system must obey, not a restatement of the formulas:
reciprocity (Z = Z^T, since A = A^T), a lossless box has purely reactive Z and unitary S, a lossy
structure is passive, and the sign of the reactance: a floating patch over ground is a capacitor
(a frequency-independent C, bracketed by plate estimates) and a filament shorted through the walls an
inductor."""
import numpy as np
import pytest

import fitgen as G
from oracle import fit as F
from oracle import ports as PT

EPS0 = F.EPS0


def _box(nx, ny, nz, h=1e-3):
    eps, sig, imu, pec = G._empty(nx, ny, nz)
    return dict(name="box", nx=nx, ny=ny, nz=nz, dx=np.full(nx, h), dy=np.full(ny, h), dz=np.full(nz, h),
                eps_r=eps, sigma=sig, inv_mu_r=imu, pec=pec)


def _A(case, w):
    me, mk, mn, mask = F.material_diagonals(case["dx"], case["dy"], case["dz"], case["eps_r"], case["sigma"],
                                            case["inv_mu_r"], case["pec"])
    return F.system_matrix(w, F.curl(case["nx"], case["ny"], case["nz"]), me, mk, mn, mask).tocsr(), mask


def _zcol(case, i, j, k0, k1):
    """The z-edges of the cells (i, j, k0 .. k1-1), oriented +z: a port from node k0 to node k1."""
    nx, ny = case["nx"], case["ny"]
    return [3 * (i + nx * (j + ny * k)) + 2 for k in range(k0, k1)], [1.0] * (k1 - k0)


def test_floating_patch_is_a_capacitor():
    """A 6x6-cell PEC patch 3 cells above the ground wall of a 12x12x8 vacuum box, fed by a port from
    the ground to the patch.  At low frequency Z is a pure negative reactance with C = -1/(w Im Z)
    the same at 10 and 20 MHz (Z ~ 1/w).  C lies between the bottom-face parallel-plate value
    eps0 A / d and 3 x eps0 (whole patch surface) / (smallest gap to a wall)."""
    c = _box(12, 12, 8)
    c["pec"][3, 3:9, 3:9] = 1  # patch: one cell thick at k = 3, cells (3..8, 3..8)
    caps = []
    for f in (1e7, 2e7):
        w = 2 * np.pi * f
        A, mask = _A(c, w)
        Z = PT.z_matrix(A, w, [_zcol(c, 6, 6, 0, 3)], mask)[0, 0]
        assert abs(Z.real) <= 1e-9 * abs(Z)
        assert Z.imag < 0
        caps.append(-1.0 / (w * Z.imag))
    assert caps[1] == pytest.approx(caps[0], rel=1e-3)
    c_pp = EPS0 * (6e-3) ** 2 / 3e-3
    c_hi = 3 * EPS0 * (2 * 36e-6 + 4 * 6e-6) / 3e-3
    assert c_pp < caps[0] < c_hi, (caps[0], c_pp, c_hi)


def test_shorted_filament_is_an_inductor():
    """A port running from the ground wall to the lid of a closed vacuum box: the current returns
    through the walls, so at low frequency the port is a lossless inductance, L = Im Z / w the same
    at 10 and 20 MHz."""
    c = _box(10, 10, 6)
    ind = []
    for f in (1e7, 2e7):
        w = 2 * np.pi * f
        A, mask = _A(c, w)
        Z = PT.z_matrix(A, w, [_zcol(c, 5, 5, 0, 6)], mask)[0, 0]
        assert abs(Z.real) <= 1e-9 * abs(Z)
        assert Z.imag > 0
        ind.append(Z.imag / w)
    assert ind[1] == pytest.approx(ind[0], rel=1e-3)


def _three_port_lossy():
    c = G.small_random(8, 7, 6, seed=11, pec_frac=0.0)
    ports = [_zcol(c, 2, 2, 1, 4), _zcol(c, 5, 4, 2, 5), ([3 * (3 + 8 * (3 + 7 * 2)) + 0], [-1.0])]
    return c, ports


def test_reciprocity_and_passivity_lossy():
    c, ports = _three_port_lossy()
    w = 2 * np.pi * 3e9
    A, mask = _A(c, w)
    Z = PT.z_matrix(A, w, ports, mask)
    assert np.allclose(Z, Z.T, rtol=1e-9, atol=0), Z  # reciprocity: A is symmetric
    herm = 0.5 * (Z + Z.conj().T)
    assert np.min(np.linalg.eigvalsh(herm)) >= -1e-9 * np.abs(Z).max()  # delivered power >= 0
    S = PT.z_to_s(Z)
    assert np.linalg.norm(S, 2) <= 1 + 1e-9  # a passive network does not amplify


def test_lossless_box_has_reactive_z_and_unitary_s():
    c = _box(9, 8, 7)
    ports = [_zcol(c, 3, 3, 1, 4), _zcol(c, 6, 5, 2, 6)]
    w = 2 * np.pi * 2e9
    A, mask = _A(c, w)
    Z = PT.z_matrix(A, w, ports, mask)
    assert np.abs(Z.real).max() <= 1e-9 * np.abs(Z).max()
    S = PT.z_to_s(Z)
    assert np.allclose(S.conj().T @ S, np.eye(2), atol=1e-9)


def test_z_to_s_special_cases():
    one = np.eye(3)
    assert np.allclose(PT.z_to_s(50.0 * one), 0)                       # matched loads reflect nothing
    assert np.allclose(PT.z_to_s(1e12 * one), one, atol=1e-9)         # open circuits reflect fully
    assert np.allclose(PT.z_to_s(1e-12 * one), -one, atol=1e-9)       # short circuits invert
    z = 30.0 - 20.0j
    assert PT.z_to_s(np.array([[z]]))[0, 0] == pytest.approx((z - 50) / (z + 50))  # one-port formula


def test_probe_voltage_and_port_rhs_conventions():
    ne = 30
    x = np.arange(ne) * (1 + 2j)
    assert PT.probe_voltage(x, [4, 7], [1.0, -1.0]) == -(x[4] - x[7])
    mask = np.zeros(ne)
    mask[7] = 1
    b = PT.port_rhs(2.0, ne, [4, 7], [1.0, -1.0], mask, current=3.0)
    assert b[4] == -2j * 3.0 and b[7] == 0 and np.count_nonzero(b) == 1


def test_z_is_j_omega_s_ainv_s():
    """From b = -j w I s and V = -sum s x: Z_ij = j w s_i^T A^-1 s_j over unmasked edges.  The oracle's
    z_matrix (sparse LU solves, probe sums, division by I) against that closed form evaluated with a dense
    inverse, on a lossy grid with PEC cells, ports of mixed orientation, a shared edge and a masked edge."""
    c = G.small_random(6, 5, 4, seed=19, pec_frac=0.1)
    w = 2 * np.pi * 2.5e9
    A, mask = _A(c, w)
    nx, ny = c["nx"], c["ny"]
    e1 = [3 * (2 + nx * (2 + ny * k)) + 2 for k in (1, 2)]
    ports = [(e1, [1.0, 1.0]),
             ([e1[1], 3 * (3 + nx * (1 + ny * 2)) + 0], [-1.0, 1.0]),
             ([3 * (0 + nx * (2 + ny * 1)) + 1, 3 * (4 + nx * (3 + ny * 1)) + 1], [1.0, -1.0])]  # first is masked
    assert mask[ports[2][0][0]] == 1
    Z = PT.z_matrix(A, w, ports, mask, current=0.3)
    ainv = np.linalg.inv(A.toarray())
    S = np.zeros((A.shape[0], len(ports)))
    for q, (e, s) in enumerate(ports):
        for ee, ss in zip(e, s):
            S[ee, q] += ss * (1 - mask[ee])
    want = 1j * w * S.T @ ainv @ S
    assert np.allclose(Z, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())


def test_all_pins_in_one_right_hand_side_is_superposition():
    """Driving every port at once (one port made of all the pins' edges, the single-run excitation Sec. IV
    mentions) gives, by linearity, an impedance equal to the sum of all entries of the individual
    ports' Z matrix."""
    c, ports = _three_port_lossy()
    w = 2 * np.pi * 2e9
    A, mask = _A(c, w)
    Z = PT.z_matrix(A, w, ports, mask)
    edges = [e for p in ports for e in p[0]]
    signs = [s for p in ports for s in p[1]]
    assert len(set(edges)) == len(edges)  # disjoint pins
    Zc = PT.z_matrix(A, w, [(edges, signs)], mask)[0, 0]
    assert Zc == pytest.approx(Z.sum(), rel=1e-10)
