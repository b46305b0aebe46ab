"""Oracle for the FIT grid operators, material matrices and the system A(w).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): only tests, the smoke entry and bench.py's
CPU legs may use it.  Everything here is float64 / complex128 scipy/numpy, written as the plain
definition from the paper, with no blocking, fusion or reordering.

Conventions (readings of the paper where it is silent):
  * cells (i, j, k), 0 <= i < nx etc.; linear cell index c = i + nx*(j + ny*k);
  * cell c owns the x-, y- and z-edge leaving its low node (i, j, k) and the x-, y- and z-facet
    of the primal grid through that node; unknown index = 3*c + w, w in {x, y, z} = {0, 1, 2}
    (the cell-by-cell ordering of Eq. e12Nxyz);
  * entities with node index nx (ny, nz) are not stored: they are identically zero, which is the
    truncation of the forward difference P_w at the high end (Eq. CP) and PEC on the high walls;
  * edges tangential to a low wall (x-edges with j == 0 or k == 0, ...) and all 12 edges of a
    PEC cell are "masked": their rows and columns of A are replaced by the identity (PEC, Sec. II).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Physical constants (reading: mu0 exact-by-definition value, c exact, eps0 = 1/(mu0 c^2)).
MU0 = 4.0e-7 * np.pi
C0 = 299792458.0
EPS0 = 1.0 / (MU0 * C0 * C0)


# ----------------------------------------------------------------------------------------------
# Topology: forward differences, curl, gradient, divergence (Sec. II, Eq. CP)
# ----------------------------------------------------------------------------------------------

def forward_difference(n: int) -> sp.csr_matrix:
    """D_n: (D u)_m = u_{m+1} - u_m, the +1 at m = n-1 falls off the grid (Eq. CP: P_w has
    two entries, +1 and -1, per line; the last line keeps only the -1)."""
    main = -np.ones(n, dtype=np.int64)
    upper = np.ones(max(n - 1, 0), dtype=np.int64)
    return sp.diags([main, upper], [0, 1], shape=(n, n), format="csr", dtype=np.int64)


def partial_differences(nx: int, ny: int, nz: int):
    """P_x, P_y, P_z on the N_p = nx*ny*nz node (= cell) index space, i fastest (Eq. CP)."""
    ix = sp.identity(nx, dtype=np.int64, format="csr")
    iy = sp.identity(ny, dtype=np.int64, format="csr")
    iz = sp.identity(nz, dtype=np.int64, format="csr")
    px = sp.kron(iz, sp.kron(iy, forward_difference(nx)), format="csr")
    py = sp.kron(iz, sp.kron(forward_difference(ny), ix), format="csr")
    pz = sp.kron(forward_difference(nz), sp.kron(iy, ix), format="csr")
    for p in (px, py, pz):
        p.eliminate_zeros()  # kron may store structural zeros; keep only the +-1 entries
    return px, py, pz


def interleave_permutation(ncell: int) -> sp.csr_matrix:
    """Pi with (Pi v)[3c + w] = v[w*ncell + c]: classical (all x, all y, all z) ordering to the
    cell-by-cell ordering of Eq. e12Nxyz."""
    rows = (3 * np.arange(ncell)[None, :] + np.arange(3)[:, None]).ravel()
    cols = (np.arange(3)[:, None] * ncell + np.arange(ncell)[None, :]).ravel()
    data = np.ones(3 * ncell, dtype=np.int64)
    return sp.csr_matrix((data, (rows, cols)), shape=(3 * ncell, 3 * ncell))


def curl_classical(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """C in the classical block ordering, Eq. CP: [[0, -Pz, Py], [Pz, 0, -Px], [-Py, Px, 0]]."""
    px, py, pz = partial_differences(nx, ny, nz)
    return sp.bmat([[None, -pz, py], [pz, None, -px], [-py, px, None]], format="csr")


def curl(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """Primal curl C (faces x edges) in the Eq. e12Nxyz interleaved ordering of rows and columns."""
    pi = interleave_permutation(nx * ny * nz)
    return (pi @ curl_classical(nx, ny, nz) @ pi.T).tocsr()


def gradient(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """Primal gradient G (edges x nodes): (G phi) on the w-edge of cell c = P_w phi (interleaved)."""
    px, py, pz = partial_differences(nx, ny, nz)
    pi = interleave_permutation(nx * ny * nz)
    return (pi @ sp.vstack([px, py, pz], format="csr")).tocsr()


def divergence(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """Primal divergence S (cells x faces): S = [Px, Py, Pz] acting on interleaved facet fluxes."""
    px, py, pz = partial_differences(nx, ny, nz)
    pi = interleave_permutation(nx * ny * nz)
    return (sp.hstack([px, py, pz], format="csr") @ pi.T).tocsr()


def curl_rows_direct(nx: int, ny: int, nz: int, faces) -> sp.csr_matrix:
    """Rows of C for the given facet indices, written out per component from Eq. CP with
    P_w u(n) = u(n+1) - u(n) (terms whose node index reaches nx/ny/nz are dropped):

        b_x(i,j,k) = e_y(i,j,k) - e_y(i,j,k+1) + e_z(i,j+1,k) - e_z(i,j,k)      (-Pz e_y + Py e_z)
        b_y(i,j,k) = e_z(i,j,k) - e_z(i+1,j,k) + e_x(i,j,k+1) - e_x(i,j,k)      ( Pz e_x - Px e_z)
        b_z(i,j,k) = e_x(i,j,k) - e_x(i,j+1,k) + e_y(i+1,j,k) - e_y(i,j,k)      (-Py e_x + Px e_y)

    Used for sampled rows on grids too large to assemble C whole.  Returned as a
    len(faces) x 3N sparse matrix."""
    faces = np.asarray(faces, dtype=np.int64)
    n3 = 3 * nx * ny * nz

    def e(i, j, k, w):
        return 3 * (i + nx * (j + ny * k)) + w

    rows, cols, vals = [], [], []
    for r, f in enumerate(faces):
        c, w = divmod(int(f), 3)
        i = c % nx
        j = (c // nx) % ny
        k = c // (nx * ny)
        if w == 0:
            terms = [((i, j, k, 1), +1), ((i, j, k + 1, 1), -1), ((i, j + 1, k, 2), +1), ((i, j, k, 2), -1)]
        elif w == 1:
            terms = [((i, j, k, 2), +1), ((i + 1, j, k, 2), -1), ((i, j, k + 1, 0), +1), ((i, j, k, 0), -1)]
        else:
            terms = [((i, j, k, 0), +1), ((i, j + 1, k, 0), -1), ((i + 1, j, k, 1), +1), ((i, j, k, 1), -1)]
        for (a, b, cc, ww), s in terms:
            if a < nx and b < ny and cc < nz:
                rows.append(r)
                cols.append(e(a, b, cc, ww))
                vals.append(s)
    return sp.csr_matrix((np.array(vals, dtype=np.int64), (rows, cols)), shape=(len(faces), n3))


# ----------------------------------------------------------------------------------------------
# Material matrices (Sec. II, Eq. Material) and the PEC edge mask
# ----------------------------------------------------------------------------------------------

def _cell(a, i, j, k):
    """a[k, j, i] or 0 outside the grid (cells beyond a wall do not contribute)."""
    nz, ny, nx = a.shape
    out = np.zeros(np.broadcast(i, j, k).shape, dtype=np.float64)
    ok = (i >= 0) & (i < nx) & (j >= 0) & (j < ny) & (k >= 0) & (k < nz)
    ii, jj, kk = np.broadcast_arrays(i, j, k)
    out[ok] = a[kk[ok], jj[ok], ii[ok]]
    return out


def _len(d, i):
    """d[i] or 0 outside the grid (a half cell beyond a wall has no extent)."""
    out = np.zeros(np.shape(i), dtype=np.float64)
    ok = (i >= 0) & (i < len(d))
    out[ok] = np.asarray(d, dtype=np.float64)[np.asarray(i)[ok]]
    return out


def material_diagonals(dx, dy, dz, eps_r, sigma, inv_mu_r, pec=None):
    """Diagonals of M_eps, M_kappa (edge-based) and M_nu = M_mu^{-1} (facet-based) plus the edge mask.

    Eq. Material: M_eps holds eps averaged over the dual facet crossed by each primal edge,
    M_mu^{-1} holds 1/mu averaged along the dual edge crossing each primal facet, both times the
    grid metric.  Reading: for the w-edge of cell (i, j, k) the dual facet is made of
    the four quarter facets in the (up to) four cells sharing the edge,

        M_eps  = eps0 * sum_cells eps_r(c) a_c / L,      a_c = (h_u(c)/2) (h_v(c)/2),  L = h_w(i)
        M_kap  =        sum_cells sigma(c) a_c / L,

    and for the w-facet of cell (i, j, k) the dual edge is made of the half cells on both sides,

        M_nu   = sum_{halves} (h_w/2) * inv_mu_r(c) / mu0 / A,          A = h_u(j) h_v(k).

    Cells outside the grid contribute nothing (half cells at walls).  Arrays eps_r, sigma,
    inv_mu_r, pec are indexed [k, j, i].  Returns (m_eps, m_kap, m_nu, mask) as length-3N arrays
    in the interleaved ordering; mask is uint8 (1 = PEC / boundary edge).
    """
    eps_r = np.asarray(eps_r, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    inv_mu_r = np.asarray(inv_mu_r, dtype=np.float64)
    nz, ny, nx = eps_r.shape
    dx = np.asarray(dx, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    dz = np.asarray(dz, dtype=np.float64)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    m_eps = np.zeros((nz, ny, nx, 3))
    m_kap = np.zeros((nz, ny, nx, 3))
    m_nu = np.zeros((nz, ny, nx, 3))

    # x-edge of (i,j,k): cells (i, j-1|j, k-1|k); quarter areas (dy/2)(dz/2); length dx[i]
    for dj in (-1, 0):
        for dk in (-1, 0):
            a = 0.25 * _len(dy, j + dj) * _len(dz, k + dk)
            m_eps[..., 0] += _cell(eps_r, i, j + dj, k + dk) * a
            m_kap[..., 0] += _cell(sigma, i, j + dj, k + dk) * a
    m_eps[..., 0] *= EPS0 / dx[i]
    m_kap[..., 0] /= dx[i]
    # y-edge of (i,j,k): cells (i-1|i, j, k-1|k); quarter areas (dx/2)(dz/2); length dy[j]
    for di in (-1, 0):
        for dk in (-1, 0):
            a = 0.25 * _len(dx, i + di) * _len(dz, k + dk)
            m_eps[..., 1] += _cell(eps_r, i + di, j, k + dk) * a
            m_kap[..., 1] += _cell(sigma, i + di, j, k + dk) * a
    m_eps[..., 1] *= EPS0 / dy[j]
    m_kap[..., 1] /= dy[j]
    # z-edge of (i,j,k): cells (i-1|i, j-1|j, k); quarter areas (dx/2)(dy/2); length dz[k]
    for di in (-1, 0):
        for dj in (-1, 0):
            a = 0.25 * _len(dx, i + di) * _len(dy, j + dj)
            m_eps[..., 2] += _cell(eps_r, i + di, j + dj, k) * a
            m_kap[..., 2] += _cell(sigma, i + di, j + dj, k) * a
    m_eps[..., 2] *= EPS0 / dz[k]
    m_kap[..., 2] /= dz[k]

    # facets: x-facet of (i,j,k) is crossed by the dual x-edge through cells (i-1, j, k), (i, j, k)
    for di in (-1, 0):
        m_nu[..., 0] += 0.5 * _len(dx, i + di) * _cell(inv_mu_r, i + di, j, k)
    m_nu[..., 0] /= MU0 * dy[j] * dz[k]
    for dj in (-1, 0):
        m_nu[..., 1] += 0.5 * _len(dy, j + dj) * _cell(inv_mu_r, i, j + dj, k)
    m_nu[..., 1] /= MU0 * dx[i] * dz[k]
    for dk in (-1, 0):
        m_nu[..., 2] += 0.5 * _len(dz, k + dk) * _cell(inv_mu_r, i, j, k + dk)
    m_nu[..., 2] /= MU0 * dx[i] * dy[j]

    mask = edge_mask(nx, ny, nz, pec)
    return m_eps.ravel(), m_kap.ravel(), m_nu.ravel(), mask


def edge_mask(nx, ny, nz, pec=None):
    """1 on edges where E_tan = 0 is enforced (Sec. II, PEC): edges lying in a low wall plane and
    every one of the 12 edges of a PEC cell.  (High-wall edges are not stored at all.)"""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = np.zeros((nz, ny, nx, 3), dtype=np.uint8)
    m[..., 0] = (j == 0) | (k == 0)
    m[..., 1] = (i == 0) | (k == 0)
    m[..., 2] = (i == 0) | (j == 0)
    if pec is not None:
        pec = np.asarray(pec).astype(bool)
        kk, jj, ii = np.nonzero(pec)
        for a in (0, 1):
            for b in (0, 1):
                # x-edges of the cell: (i, j+a, k+b); y-edges: (i+a, j, k+b); z-edges: (i+a, j+b, k)
                ok = (jj + a < ny) & (kk + b < nz)
                m[kk[ok] + b, jj[ok] + a, ii[ok], 0] = 1
                ok = (ii + a < nx) & (kk + b < nz)
                m[kk[ok] + b, jj[ok], ii[ok] + a, 1] = 1
                ok = (ii + a < nx) & (jj + b < ny)
                m[kk[ok], jj[ok] + b, ii[ok] + a, 2] = 1
    return m.ravel()


def material_diagonals_loops(dx, dy, dz, eps_r, sigma, inv_mu_r, pec=None):
    """Same quantities as ``material_diagonals`` by explicit per-entity Python loops (small grids
    only).  It builds each dual facet / dual edge from its pieces one by one."""
    nz, ny, nx = np.shape(eps_r)
    n = nx * ny * nz
    m_eps = np.zeros(3 * n)
    m_kap = np.zeros(3 * n)
    m_nu = np.zeros(3 * n)
    h = (list(map(float, dx)), list(map(float, dy)), list(map(float, dz)))
    size = (nx, ny, nz)

    def inside(c):
        return all(0 <= c[a] < size[a] for a in range(3))

    for kk in range(nz):
        for jj in range(ny):
            for ii in range(nx):
                c = ii + nx * (jj + ny * kk)
                node = (ii, jj, kk)
                for w in range(3):
                    u, v = [a for a in range(3) if a != w]
                    # edge: the 4 cells that share it differ from (i,j,k) by -1/0 along u and v
                    se = sk = 0.0
                    for du in (-1, 0):
                        for dv in (-1, 0):
                            cell = list(node)
                            cell[u] += du
                            cell[v] += dv
                            if inside(cell):
                                area = 0.5 * h[u][cell[u]] * 0.5 * h[v][cell[v]]
                                se += float(eps_r[cell[2]][cell[1]][cell[0]]) * area
                                sk += float(sigma[cell[2]][cell[1]][cell[0]]) * area
                    m_eps[3 * c + w] = EPS0 * se / h[w][node[w]]
                    m_kap[3 * c + w] = sk / h[w][node[w]]
                    # facet: dual edge through the cells at -1 and 0 along w
                    sn = 0.0
                    for dw in (-1, 0):
                        cell = list(node)
                        cell[w] += dw
                        if inside(cell):
                            sn += 0.5 * h[w][cell[w]] * float(inv_mu_r[cell[2]][cell[1]][cell[0]]) / MU0
                    m_nu[3 * c + w] = sn / (h[u][node[u]] * h[v][node[v]])
    return m_eps, m_kap, m_nu, edge_mask(nx, ny, nz, pec)


# ----------------------------------------------------------------------------------------------
# The system matrix A(w) (Eq. e2 with s = j w, plus the conductivity term) and its RHS
# ----------------------------------------------------------------------------------------------

def curlcurl(C, m_nu, mask) -> sp.csr_matrix:
    """K = P C^T M_nu C P with P the projection onto unmasked edges (real, symmetric PSD)."""
    p = sp.diags((1 - np.asarray(mask, dtype=np.int64)).astype(np.float64))
    cp = (C.astype(np.float64) @ p).tocsr()
    return (cp.T @ sp.diags(np.asarray(m_nu, dtype=np.float64)) @ cp).tocsr()


def system_matrix(omega, C, m_eps, m_kap, m_nu, mask) -> sp.csr_matrix:
    """A(w) = C^T M_nu C - w^2 M_eps + j w M_kappa on the unmasked edges; masked rows and columns
    are the identity (PEC folded into the operator, Sec. II).  Complex symmetric (A = A^T)."""
    mask = np.asarray(mask, dtype=np.int64)
    free = (1 - mask).astype(np.float64)
    k = curlcurl(C, m_nu, mask).astype(np.complex128)
    diag = free * (-(omega ** 2) * np.asarray(m_eps) + 1j * omega * np.asarray(m_kap)) + mask
    return (k + sp.diags(diag.astype(np.complex128))).tocsr()


def system_rows(omega, nx, ny, nz, rows, m_eps, m_kap, m_nu, mask) -> sp.csr_matrix:
    """Selected rows of A(w) without assembling C whole: for each requested edge e,
    A[e, :] = sum_f C[f, e] nu_f C[f, :] P + diagonal, with C[f, :] from ``curl_rows_direct``.
    Used to check sampled outputs on grids too large for ``system_matrix``."""
    rows = np.asarray(rows, dtype=np.int64)
    mask = np.asarray(mask, dtype=np.int64)
    n3 = 3 * nx * ny * nz
    out = sp.lil_matrix((len(rows), n3), dtype=np.complex128)
    for r, e in enumerate(rows):
        if mask[e]:
            out[r, e] = 1.0
            continue
        c, w = divmod(int(e), 3)
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        # facets whose boundary contains edge e: from Eq. CP, the w-edge of (i,j,k) appears in
        # the two other-component facets of cell (i,j,k) and of the cells one step back.
        cand = []
        for f_w in range(3):
            if f_w == w:
                continue
            for back in range(3):
                if back == f_w:
                    continue
                for d in (0, 1):
                    cc = [i, j, k]
                    cc[back] -= d
                    if min(cc) >= 0:
                        cand.append(3 * (cc[0] + nx * (cc[1] + ny * cc[2])) + f_w)
        cand = sorted(set(cand))
        crow = curl_rows_direct(nx, ny, nz, cand).tocsr()
        acc = {}
        for t, f in enumerate(cand):
            lo, hi = crow.indptr[t], crow.indptr[t + 1]
            cols, vals = crow.indices[lo:hi], crow.data[lo:hi]
            ce = vals[cols == e]
            if len(ce) == 0:
                continue
            for cidx, v in zip(cols, vals):
                if mask[cidx]:
                    continue
                acc[int(cidx)] = acc.get(int(cidx), 0.0) + float(ce[0]) * m_nu[f] * float(v)
        acc[int(e)] = acc.get(int(e), 0.0) + (-(omega ** 2) * m_eps[e] + 1j * omega * m_kap[e])
        for cidx, v in acc.items():
            out[r, cidx] = v
    return out.tocsr()


def rhs_from_current(omega, j_current, mask=None):
    """b = -s j = -j w j (Eq. e2 right-hand side).  Masked rows get b = 0."""
    b = -1j * omega * np.asarray(j_current, dtype=np.complex128)
    if mask is not None:
        b = np.where(np.asarray(mask) != 0, 0.0, b)
    return b


def cavity_eigenvalues(n: int, h: float):
    """Closed-form omega^2 of the uniform n^3 PEC cube (spacing h, vacuum) on the staggered grid:
    omega^2 = (2 c / h)^2 [sin^2(m pi/2n) + sin^2(q pi/2n) + sin^2(p pi/2n)],  m, q, p in 0..n-1,
    at most one index zero; multiplicity 2 if all indices >= 1, else 1.  Plus (n-1)^3 zeros
    (discrete gradients of the interior nodes).  Returns the sorted multiset."""
    s = np.sin(np.arange(n) * np.pi / (2 * n)) ** 2
    vals = []
    for m in range(n):
        for q in range(n):
            for p in range(n):
                zeros = (m == 0) + (q == 0) + (p == 0)
                if zeros > 1:
                    continue
                lam = (2 * C0 / h) ** 2 * (s[m] + s[q] + s[p])
                vals += [lam] * (2 if zeros == 0 else 1)
    vals += [0.0] * (n - 1) ** 3
    return np.sort(np.array(vals))


def cavity_frequency(a, b, d, m, q, p):
    """Continuum PEC rectangular-cavity resonance f_mqp = (c/2) sqrt((m/a)^2 + (q/b)^2 + (p/d)^2)."""
    return 0.5 * C0 * np.sqrt((m / a) ** 2 + (q / b) ** 2 + (p / d) ** 2)


def jacobi_diagonal(omega, nx, ny, nz, m_eps, m_kap, m_nu, mask):
    """diag(A(w)): for an unmasked edge, sum over the facets f containing it of M_nu[f] C[f,e]^2
    minus w^2 M_eps plus j w M_kappa (the column-sum-of-squares construction of Eq. Precond applied
    to the unsymmetrised operator).  Masked edges: 1."""
    C = curl(nx, ny, nz).astype(np.float64)
    col_sq = np.asarray(C.multiply(C).T @ np.asarray(m_nu, dtype=np.float64)).ravel()
    d = col_sq - omega ** 2 * np.asarray(m_eps) + 1j * omega * np.asarray(m_kap)
    return np.where(np.asarray(mask) != 0, 1.0 + 0j, d)
