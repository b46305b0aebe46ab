"""Helpers shared by the GPU tests: build/load the library, move cases to the oracle and back."""
import numpy as np
import pytest

import fitgen as G


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def fitlib():
    """The built FIT library binding (build on first use).  Raises if the build fails."""
    from paper_1705_08849_gb300 import build, fit
    build.build()
    fit.lib()
    return fit


def oracle_matrices(case):
    from oracle import fit as F
    return F.material_diagonals(case["dx"], case["dy"], case["dz"], case["eps_r"], case["sigma"],
                                case["inv_mu_r"], case["pec"])


def oracle_A(case, omega):
    from oracle import fit as F
    me, mk, mn, mask = oracle_matrices(case)
    return F.system_matrix(omega, F.curl(case["nx"], case["ny"], case["nz"]), me, mk, mn, mask), mask


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def rand_vec(n, seed, batch=None):
    return G.random_vector(n, seed, batch=batch)
