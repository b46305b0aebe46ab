"""The C-ABI library builds, loads and exports every entry point that include/*.h declares; host
argument checks that need no GPU return FIT_EINVAL without touching the device."""
import ctypes as ct
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fit_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_1705_08849_gb300 import build, fit
    build.build()
    return fit.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert {"fit_grid_create", "fit_set_materials", "fit_apply", "fit_solve"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_status_strings(L):
    from paper_1705_08849_gb300 import fit
    for code, name in [(0, "FIT_OK"), (-1, "FIT_EINVAL"), (-5, "FIT_EBUDGET"), (2, "FIT_BREAKDOWN")]:
        assert fit.status_str(code) == name


def test_host_argument_checks_without_gpu(L):
    from paper_1705_08849_gb300 import fit
    h = ct.c_void_p()
    d = (ct.c_double * 4)(1e-3, 1e-3, 1e-3, 1e-3)
    assert L.fit_grid_create(0, 4, 4, d, d, d, 0x3F, ct.byref(h)) == fit.FIT_EINVAL
    assert L.fit_grid_create(4, 4, 4, d, d, d, 0x01, ct.byref(h)) == fit.FIT_EINVAL
    bad = (ct.c_double * 4)(1e-3, -1e-3, 1e-3, 1e-3)
    assert L.fit_grid_create(4, 4, 4, bad, d, d, 0x3F, ct.byref(h)) == fit.FIT_EINVAL
    assert b"dx" in L.fit_last_error()
    assert L.fit_apply(None, 1, None, None, None, 0, None) == fit.FIT_EINVAL
    o = fit.fit_solve_opts_default()
    assert o.restart == 30 and o.inner_tol == 1e-4 and o.precision == fit.FIT_SOLVE_MIXED


def test_library_has_no_oracle_dependency():
    """The product package never imports the oracle (the two share no code)."""
    for f in glob.glob(os.path.join(ROOT, "paper_1705_08849_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            assert "oracle" not in re.findall(r"(?:import|from)\s+(\w+)", src), f


def test_port_entry_points_reject_bad_arguments(L):
    from paper_1705_08849_gb300 import fit
    assert L.fit_port_rhs(None, 1, None, 0, None, None, 1.0, None, None) == fit.FIT_EINVAL
    assert L.fit_probe_voltages(None, 1, None, 1, None, None, None, None, None) == fit.FIT_EINVAL
    assert L.fit_z_parameters(None, 1, None, 1, None, None, None, 1.0, 1e-8, None, None, None) == fit.FIT_EINVAL
    z = (ct.c_double * 2)(1.0, 0.0)
    s = (ct.c_double * 2)()
    assert L.fit_z_to_s(1, z, 0.0, s) == fit.FIT_EINVAL  # z0 must be > 0
    zs = (ct.c_double * 2)(-50.0, 0.0)  # Z + z0 1 = 0
    assert L.fit_z_to_s(1, zs, 50.0, s) == fit.FIT_EINVAL
    assert b"singular" in L.fit_last_error()


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_z_to_s_matches_the_oracle(L, P):
    """fit_z_to_s is host code: the same S as the oracle's (Z - z0 1)(Z + z0 1)^-1 on random complex
    impedances, including ones that need row pivoting (a zero leading entry of Z + z0 1)."""
    import numpy as np
    from oracle import ports as PT
    from paper_1705_08849_gb300 import fit
    rng = np.random.default_rng(100 + P)
    Z = 80 * (rng.standard_normal((P, P)) + 1j * rng.standard_normal((P, P)))
    if P > 1:
        Z[0, 0] = -50.0  # Z + z0 1 has a zero pivot in its first column: rows must be exchanged
    S = fit.fit_z_to_s(Z, 50.0)
    want = PT.z_to_s(Z, 50.0)
    assert np.allclose(S, want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))


def test_header_compiles_as_c99_and_links(L, tmp_path):
    """include/fit.h is a plain C header: a C99 program that includes it builds with -Wall -Werror, links
    against the library and calls its host-only entry points (no GPU needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = tmp_path / "use_fit.c"
    src.write_text(r'''
#include <stdio.h>
#include "fit.h"
int main(void) {
  double z[2] = {30.0, -20.0}, s[2] = {0.0, 0.0};
  int choice = 0;
  fit_solve_opts o;
  fit_solve_opts_default(&o);
  if (fit_z_to_s(1, z, 50.0, s) != FIT_OK) return 1;
  if (fit_tuning_lookup("/nonexistent/fit-tune.txt", "dev", 1, 2, 2, 2, FIT_C64, 1, &choice) != FIT_OK) return 2;
  if (fit_grid_create(0, 1, 1, NULL, NULL, NULL, FIT_BC_PEC_ALL, NULL) != FIT_EINVAL) return 3;
  printf("%s %d %.12f %.12f %d %d\n", fit_status_str(FIT_EINVAL), choice, s[0], s[1], o.restart, o.method);
  return 0;
}
''')
    libdir = os.path.join(ROOT, "paper_1705_08849_gb300")
    exe = tmp_path / "use_fit"
    cuda_lib = "/usr/local/cuda/lib64"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lfitgb300", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=":".join(p for p in (libdir, cuda_lib, os.environ.get("LD_LIBRARY_PATH", ""))
                                                     if p))
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    name, choice, sr, si, restart, method = r.stdout.split()
    w = (30 - 20j - 50) / (30 - 20j + 50)
    assert name == "FIT_EINVAL" and int(choice) == -2 and int(restart) == 30
    assert abs(float(sr) - w.real) < 1e-12 and abs(float(si) - w.imag) < 1e-12
