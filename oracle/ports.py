"""Oracle of the port post-processing -- TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Sec. IV excites the structures with time-harmonic currents impressed on the edges of input ports
and reads the voltages along the edges of probes (summed), from which impedance (Z) parameters
follow, and S parameters with a source impedance Z0 = 50 Ohm.  Written out plainly:

* a port (or probe) is a list of edges with orientations s_k = +1 / -1 relative to the port's
  reference direction;
* exciting port j with current I puts edge currents I * s_k on its edges; the right-hand side is
  b = -j w j (Eq. e2), zero on masked edges;
* the voltage of port i is V_i = - sum_k s_k e_k: the edge voltages summed against the current's
  direction, so that the power a source delivers, Re(V conj(I)) / 2, is >= 0 for a passive load;
* Z_ij = V_i / I_j with port j excited alone; S = (Z - Z0 1)(Z + Z0 1)^{-1}.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def port_current(ne, edges, signs, current=1.0):
    """The edge-current vector j of a port excited with ``current`` amperes."""
    j = np.zeros(ne, dtype=np.complex128)
    np.add.at(j, np.asarray(edges, dtype=np.int64), current * np.asarray(signs, dtype=np.float64))
    return j


def port_rhs(w, ne, edges, signs, mask, current=1.0):
    """b = -j w j for a port's current pattern, zero on masked edges (Eq. e2)."""
    return (-1j * w) * port_current(ne, edges, signs, current) * (1 - np.asarray(mask))


def probe_voltage(x, edges, signs):
    """V = - sum_k s_k x[edge_k] (complex volts)."""
    x = np.asarray(x)
    return -np.sum(np.asarray(signs, dtype=np.float64) * x[np.asarray(edges, dtype=np.int64)])


def z_matrix(A, w, ports, mask, current=1.0):
    """P x P impedance matrix: column j from one sparse direct solve with port j excited by ``current``."""
    ne = A.shape[0]
    lu = spla.splu(A.tocsc())
    P = len(ports)
    Z = np.zeros((P, P), dtype=np.complex128)
    for jp, (ej, sj) in enumerate(ports):
        x = lu.solve(port_rhs(w, ne, ej, sj, mask, current))
        for ip, (ei, si) in enumerate(ports):
            Z[ip, jp] = probe_voltage(x, ei, si) / current
    return Z


def z_to_s(Z, z0=50.0):
    """S = (Z - z0 1)(Z + z0 1)^{-1}."""
    Z = np.asarray(Z, dtype=np.complex128)
    one = np.eye(Z.shape[0])
    return (Z - z0 * one) @ np.linalg.inv(Z + z0 * one)
