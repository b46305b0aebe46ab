"""Planted mistakes in the oracle, on the CPU: a mutated copy of an oracle module (one plausible slip
each: a wrong power or sign, a dropped factor, a conjugated bilinear form, a mask ignored) must fail at
least one of the pins that guard that module.  The mutants live only inside this test; the oracle
itself is untouched."""
import os
import types

import pytest

import tests.test_oracle_materials as TM
import tests.test_oracle_operator as TO
import tests.test_oracle_ports as TP
import tests.test_oracle_solvers as TK
import tests.test_oracle_symmetric as TS
import tests.test_oracle_topology as TT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mutant(name, old, new):
    path = os.path.join(ROOT, "oracle", name + ".py")
    with open(path) as fh:
        src = fh.read()
    assert src.count(old) == 1, (name, old)
    mod = types.ModuleType("oracle." + name)
    mod.__package__ = "oracle"
    mod.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    return mod


# Each group names the test-module globals through which its pins reach the oracle module (they are
# replaced by the mutant) and the pins themselves.
FIT_USERS = [(TT, "F"), (TM, "F"), (TO, "F"), (TK, "F"), (TP, "F"), (TS, "F")]
FIT_PINS = [
    lambda: TT.test_curl_of_gradient_and_divergence_of_curl_vanish((5, 4, 3)),
    lambda: TT.test_row_formulas_equal_block_kronecker_form((3, 4, 5)),
    TT.test_curl_nonzeros_per_line_and_fig_spy_grid,
    TT.test_interleaved_ordering_of_a_single_edge,
    TM.test_golden_2x2x2_entries,
    TM.test_homogeneous_uniform_closed_form,
    TM.test_two_layer_interface_is_arithmetic_mean,
    lambda: TM.test_mask_counts_of_empty_cavity(3),
    TM.test_pec_cell_masks_its_twelve_edges,
    TO.test_A_is_complex_symmetric_with_13_nonzeros,
    TO.test_interior_row_has_13_nonzeros,
    lambda: TO.test_curlcurl_is_psd_with_gradient_null_space(4),
    lambda: TO.test_cavity_full_spectrum_matches_discrete_closed_form(6),
    TO.test_sampled_rows_equal_assembled_rows,
    TO.test_jacobi_diagonal_is_diag_of_A,
    TO.test_A_is_singular_exactly_at_a_cavity_resonance,
    TO.test_a_current_source_delivers_power_into_a_lossy_grid,
    TP.test_reciprocity_and_passivity_lossy,
]
KRYLOV_USERS = [(TK, "K"), (TS, "K")]
KRYLOV_PINS = [
    lambda: TK.test_direct_and_krylov_agree_on_4cubed(True),
    lambda: TK.test_direct_and_krylov_agree_on_4cubed(False),
    lambda: TK.test_manufactured_solution("random"),
    TK.test_cocg_is_cg_on_real_spd,
    lambda: TK.test_cocg_on_complex_symmetric_4cubed(True),
    lambda: TS.test_cocg_iterates_equal_eps_preconditioned_cocg(True),
]
COCR_USERS = [(TK, "K")]
COCR_PINS = [
    TK.test_cocr_is_minimal_residual_on_real_spd,
    lambda: TK.test_cocr_on_complex_symmetric_4cubed(False),
    lambda: TK.test_cocr_on_complex_symmetric_4cubed(True),
    TK.test_preconditioned_cocr_is_cocr_on_the_scaled_system,
]
SYMMETRIC_USERS = [(TS, "S")]
SYMMETRIC_PINS = [
    lambda: TS.test_vacuum_cube_spectrum_is_the_closed_form(5),
    TS.test_layered_spectrum_is_the_generalised_one,
    TS.test_factored_equals_scaled_curlcurl,
    lambda: TS.test_solution_maps_back_to_the_unsymmetrised_one(4, 0.2),
    lambda: TS.test_cocg_iterates_equal_eps_preconditioned_cocg(True),
]
PORT_USERS = [(TP, "PT")]
PORT_PINS = [
    TP.test_floating_patch_is_a_capacitor,
    TP.test_shorted_filament_is_an_inductor,
    TP.test_reciprocity_and_passivity_lossy,
    TP.test_lossless_box_has_reactive_z_and_unitary_s,
    TP.test_z_to_s_special_cases,
    TP.test_probe_voltage_and_port_rhs_conventions,
    TP.test_z_is_j_omega_s_ainv_s,
]

FIT = ("fit", FIT_USERS, FIT_PINS)
KRY = ("krylov", KRYLOV_USERS, KRYLOV_PINS)
COCR = ("krylov", COCR_USERS, COCR_PINS)
SYM = ("symmetric", SYMMETRIC_USERS, SYMMETRIC_PINS)
PORTS = ("ports", PORT_USERS, PORT_PINS)

PLANTS = [
    # operator, right-hand side, topology and material matrices (Eq. e2, Eq. CP, Eq. Material)
    (FIT, "diag = free * (-(omega ** 2) * np.asarray(m_eps)", "diag = free * ((omega ** 2) * np.asarray(m_eps)"),
    (FIT, "+ 1j * omega * np.asarray(m_kap)) + mask", "- 1j * omega * np.asarray(m_kap)) + mask"),
    (FIT, "b = -1j * omega * np.asarray(j_current, dtype=np.complex128)",
     "b = 1j * omega * np.asarray(j_current, dtype=np.complex128)"),
    (FIT, "cp = (C.astype(np.float64) @ p).tocsr()", "cp = C.astype(np.float64).tocsr()"),
    (FIT, "a = 0.25 * _len(dy, j + dj) * _len(dz, k + dk)", "a = 0.5 * _len(dy, j + dj) * _len(dz, k + dk)"),
    (FIT, "m_nu[..., 0] += 0.5 * _len(dx, i + di)", "m_nu[..., 0] += 1.0 * _len(dx, i + di)"),
    (FIT, "m_kap[..., 0] /= dx[i]", "m_kap[..., 0] *= dx[i]"),
    (FIT, "m[..., 0] = (j == 0) | (k == 0)", "m[..., 0] = (j == 0)"),
    (FIT, "[[None, -pz, py], [pz, None, -px], [-py, px, None]]", "[[None, pz, py], [pz, None, -px], [-py, px, None]]"),
    (FIT, "main = -np.ones(n, dtype=np.int64)", "main = np.ones(n, dtype=np.int64)"),
    (FIT, "d = col_sq - omega ** 2 * np.asarray(m_eps)", "d = col_sq + omega ** 2 * np.asarray(m_eps)"),
    # COCG, BiCGStab, FGMRES (Sec. IV solvers)
    (KRY, "rho = r @ z  # unconjugated", "rho = np.vdot(r, z)  # unconjugated"),
    (KRY, "x = x + alpha * p + omega * s", "x = x + alpha * p - omega * s"),
    (KRY, "H[i, jj] = np.vdot(V[i], w)", "H[i, jj] = V[i] @ w"),
    # COCR (Sec. IV "cr")
    (COCR, "        rho_new = z @ w\n", "        rho_new = np.vdot(z, w)\n"),
    (COCR, "        sig = q @ m(q)\n", "        sig = q @ q\n"),
    (COCR, "        p = z + beta * p\n        q = w + beta * q\n", "        p = r + beta * p\n        q = w + beta * q\n"),
    # symmetrised form (Eq. e2s / Eq. e2tt)
    (SYM, "1.0 / np.sqrt(m_eps[free])", "np.sqrt(m_eps[free])"),
    (SYM, "np.asarray(m_kap, dtype=np.float64)[free] / np.asarray(m_eps, dtype=np.float64)[free]",
     "np.asarray(m_kap, dtype=np.float64)[free]"),
    (SYM, "-(omega ** 2) + 1j", "(omega ** 2) + 1j"),
    (SYM, "return eps_scaling(m_eps, mask) * F.rhs_from_current", "return F.rhs_from_current"),
    (SYM, "r = sp.diags(np.sqrt(np.asarray(m_nu, dtype=np.float64)))", "r = sp.diags(np.asarray(m_nu, dtype=np.float64))"),
    # ports (Sec. IV)
    (PORTS, "    return -np.sum(np.asarray(signs", "    return np.sum(np.asarray(signs"),
    (PORTS, "Z[ip, jp] = probe_voltage(x, ei, si) / current", "Z[ip, jp] = probe_voltage(x, ei, si)"),
    (PORTS, "current) * (1 - np.asarray(mask))", "current)"),
    (PORTS, "return (Z - z0 * one) @ np.linalg.inv(Z + z0 * one)", "return (Z + z0 * one) @ np.linalg.inv(Z - z0 * one)"),
]


def _install(monkeypatch, group, old, new):
    name, users, pins = group
    mutant = _mutant(name, old, new)
    for tmod, attr in users:
        monkeypatch.setattr(tmod, attr, mutant)
    return pins


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # a mutant may divide by zero or overflow
@pytest.mark.parametrize("group,old,new", PLANTS, ids=[f"{p[0][0]}-{i}" for i, p in enumerate(PLANTS)])
def test_planted_mistake_fails_a_pin(monkeypatch, group, old, new):
    failed = 0
    for pin in _install(monkeypatch, group, old, new):
        try:
            pin()
        except Exception:  # an assertion, or the mutant breaking a computation outright
            failed += 1
    assert failed >= 1, f"no pin caught the planted mistake {old!r} -> {new!r}"


@pytest.mark.parametrize("group,anchor", [
    (FIT, "main = -np.ones(n, dtype=np.int64)"),
    (KRY, "rho = r @ z  # unconjugated"),
    (COCR, "        sig = q @ m(q)\n"),
    (SYM, "1.0 / np.sqrt(m_eps[free])"),
    (PORTS, "    return -np.sum(np.asarray(signs"),
], ids=["fit", "krylov", "cocr", "symmetric", "ports"])
def test_unchanged_copy_passes_every_pin(monkeypatch, group, anchor):
    """Control: a copy loaded the same way but left unchanged passes all the pins, so a failure above
    comes from the planted mistake and not from the loading."""
    for pin in _install(monkeypatch, group, anchor, anchor):
        pin()
