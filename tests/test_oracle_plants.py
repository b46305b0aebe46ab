"""Planted mistakes in the oracle, on the CPU: a mutated copy of an oracle module (one plausible slip
each: a wrong power or sign, a dropped factor, a conjugated bilinear form, a mask ignored) must fail at
least one of the pins that guard that module.  The mutants live only inside this test; the oracle
itself is untouched."""
import os
import types

import pytest

import tests.test_oracle_ports as TP
import tests.test_oracle_solvers as TK
import tests.test_oracle_symmetric as TS

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


# each pin runs with the module global it reads (S, PT or K) replaced by the mutant
SYMMETRIC_PINS = [
    lambda: TS.test_vacuum_cube_spectrum_is_the_closed_form(5),
    TS.test_layered_spectrum_is_the_generalised_one,
    TS.test_factored_equals_scaled_curlcurl,
    lambda: TS.test_solution_maps_back_to_the_unsymmetrised_one(4, 0.2),
    lambda: TS.test_cocg_iterates_equal_eps_preconditioned_cocg(True),
]
PORT_PINS = [
    TP.test_floating_patch_is_a_capacitor,
    TP.test_shorted_filament_is_an_inductor,
    TP.test_reciprocity_and_passivity_lossy,
    TP.test_lossless_box_has_reactive_z_and_unitary_s,
    TP.test_z_to_s_special_cases,
    TP.test_probe_voltage_and_port_rhs_conventions,
    TP.test_z_is_j_omega_s_ainv_s,
]
COCR_PINS = [
    TK.test_cocr_is_minimal_residual_on_real_spd,
    lambda: TK.test_cocr_on_complex_symmetric_4cubed(False),
    lambda: TK.test_cocr_on_complex_symmetric_4cubed(True),
    TK.test_preconditioned_cocr_is_cocr_on_the_scaled_system,
]

PLANTS = [
    # symmetrised form (Eq. e2s / Eq. e2tt)
    ("symmetric", TS, "S", SYMMETRIC_PINS, "1.0 / np.sqrt(m_eps[free])", "np.sqrt(m_eps[free])"),
    ("symmetric", TS, "S", SYMMETRIC_PINS,
     "np.asarray(m_kap, dtype=np.float64)[free] / np.asarray(m_eps, dtype=np.float64)[free]",
     "np.asarray(m_kap, dtype=np.float64)[free]"),
    ("symmetric", TS, "S", SYMMETRIC_PINS, "-(omega ** 2) + 1j", "(omega ** 2) + 1j"),
    ("symmetric", TS, "S", SYMMETRIC_PINS, "return eps_scaling(m_eps, mask) * F.rhs_from_current",
     "return F.rhs_from_current"),
    ("symmetric", TS, "S", SYMMETRIC_PINS, "r = sp.diags(np.sqrt(np.asarray(m_nu, dtype=np.float64)))",
     "r = sp.diags(np.asarray(m_nu, dtype=np.float64))"),
    # ports (Sec. IV)
    ("ports", TP, "PT", PORT_PINS, "    return -np.sum(np.asarray(signs", "    return np.sum(np.asarray(signs"),
    ("ports", TP, "PT", PORT_PINS, "Z[ip, jp] = probe_voltage(x, ei, si) / current",
     "Z[ip, jp] = probe_voltage(x, ei, si)"),
    ("ports", TP, "PT", PORT_PINS, "current) * (1 - np.asarray(mask))", "current)"),
    ("ports", TP, "PT", PORT_PINS, "return (Z - z0 * one) @ np.linalg.inv(Z + z0 * one)",
     "return (Z + z0 * one) @ np.linalg.inv(Z - z0 * one)"),
    # COCR (Sec. IV "cr")
    ("krylov", TK, "K", COCR_PINS, "        rho_new = z @ w\n", "        rho_new = np.vdot(z, w)\n"),
    ("krylov", TK, "K", COCR_PINS, "        sig = q @ m(q)\n", "        sig = q @ q\n"),
    ("krylov", TK, "K", COCR_PINS, "        p = z + beta * p\n        q = w + beta * q\n",
     "        p = r + beta * p\n        q = w + beta * q\n"),
]


@pytest.mark.parametrize("name,tmod,attr,pins,old,new", PLANTS,
                         ids=[f"{p[0]}-{i}" for i, p in enumerate(PLANTS)])
def test_planted_mistake_fails_a_pin(monkeypatch, name, tmod, attr, pins, old, new):
    monkeypatch.setattr(tmod, attr, _mutant(name, old, new))
    failed = 0
    for pin in pins:
        try:
            pin()
        except Exception:  # an assertion, or the mutant breaking a computation outright
            failed += 1
    assert failed >= 1, f"no pin caught the planted mistake {old!r} -> {new!r}"


@pytest.mark.parametrize("name,tmod,attr,pins,anchor", [
    ("symmetric", TS, "S", SYMMETRIC_PINS, "1.0 / np.sqrt(m_eps[free])"),
    ("ports", TP, "PT", PORT_PINS, "    return -np.sum(np.asarray(signs"),
    ("krylov", TK, "K", COCR_PINS, "        sig = q @ m(q)\n"),
])
def test_unchanged_copy_passes_every_pin(monkeypatch, name, tmod, attr, pins, anchor):
    """Control: a copy loaded the same way but left unchanged passes all the pins, so a failure above
    comes from the planted mistake and not from the loading."""
    monkeypatch.setattr(tmod, attr, _mutant(name, anchor, anchor))
    for pin in pins:
        pin()
