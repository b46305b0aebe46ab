"""Oracle of the symmetrised and factored forms of the FIT system -- TEST INFRASTRUCTURE (see
``oracle/__init__.py``).

Sec. II symmetrises the curl-curl system of Eq. e2 with the change of variable e' = M_eps^{1/2} e
(Eq. e2s); Sec. III writes the same operator as a product of shell operators (Eq. e2t) and, with
cal_A = M_mu^{-1/2} C M_eps^{-1/2}, as cal_A^T cal_A (Eq. e2tt).  With s = j w and the conductivity
term of the unsymmetrised system carried along (it becomes the diagonal j w M_kappa / M_eps):

    A_s(w) e' = (D C^T M_nu C D - w^2 I + j w D M_kappa D) e' = -j w D j,    D = M_eps^{-1/2},

on the unmasked edges; masked edges keep identity rows and columns as in Eq. e2 (D is taken as 0 there
inside the curl term, which is the same projection the unsymmetrised operator uses).  The voltages are
recovered as e = D e' (the "u = M_eps^{-1/2} e'" of Sec. IV).  Two constructions are given: the
diagonal scaling of the assembled curl-curl matrix, and the factored product cal_A^T cal_A.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fit as F


def eps_scaling(m_eps, mask):
    """D = M_eps^{-1/2} on unmasked edges, 0 on masked edges (a vector)."""
    m_eps = np.asarray(m_eps, dtype=np.float64)
    free = np.asarray(mask) == 0
    d = np.zeros_like(m_eps)
    d[free] = 1.0 / np.sqrt(m_eps[free])
    return d


def factor(C, m_eps, m_nu, mask) -> sp.csr_matrix:
    """cal_A = M_mu^{-1/2} C M_eps^{-1/2} (Eq. e2tt), facets x edges; masked edge columns are zero."""
    r = sp.diags(np.sqrt(np.asarray(m_nu, dtype=np.float64)))
    return (r @ C.astype(np.float64) @ sp.diags(eps_scaling(m_eps, mask))).tocsr()


def _finish(core, omega, m_eps, m_kap, mask):
    """core (the curl-curl part on unmasked edges) - w^2 I + j w M_kappa / M_eps; masked: identity."""
    mask = np.asarray(mask, dtype=np.int64)
    free = mask == 0
    ratio = np.zeros(len(mask))
    ratio[free] = np.asarray(m_kap, dtype=np.float64)[free] / np.asarray(m_eps, dtype=np.float64)[free]
    diag = np.where(free, -(omega ** 2) + 1j * omega * ratio, 1.0 + 0j)
    return (core.astype(np.complex128) + sp.diags(diag)).tocsr()


def symmetrised_matrix(omega, C, m_eps, m_kap, m_nu, mask) -> sp.csr_matrix:
    """A_s(w) = D (P C^T M_nu C P) D - w^2 I + j w M_kappa / M_eps on unmasked edges (Eq. e2s)."""
    d = sp.diags(eps_scaling(m_eps, mask))
    return _finish(d @ F.curlcurl(C, m_nu, mask) @ d, omega, m_eps, m_kap, mask)


def factored_matrix(omega, C, m_eps, m_kap, m_nu, mask) -> sp.csr_matrix:
    """The same operator as cal_A^T cal_A - w^2 I + j w M_kappa / M_eps (Eq. e2tt)."""
    a = factor(C, m_eps, m_nu, mask)
    return _finish(a.T @ a, omega, m_eps, m_kap, mask)


def symmetrised_rhs(omega, j_current, m_eps, mask):
    """b' = -j w D j (right-hand side of Eq. e2s); zero on masked edges."""
    return eps_scaling(m_eps, mask) * F.rhs_from_current(omega, j_current, mask)


def voltages(e_sym, m_eps, mask):
    """e = D e' on unmasked edges; masked edges keep the value of e' (0 for a consistent solve)."""
    d = eps_scaling(m_eps, mask)
    return np.where(np.asarray(mask) != 0, e_sym, d * e_sym)
