"""Seeded synthetic inputs for the FIT operator and its solves.

This module is shared by the oracle, the tests and the benchmark.  It holds NONE of the
method's arithmetic (no curl, no material averaging, no masking): it only draws grids, per-cell
material fields and source currents with numpy ``Generator(PCG64(seed))``.

A case is a dict with
  nx, ny, nz          grid size in cells
  dx, dy, dz          float64 cell widths [m] per axis (length nx, ny, nz)
  eps_r, sigma, inv_mu_r   float32 arrays [nz, ny, nx]: relative permittivity, conductivity
                      [S/m], relative inverse permeability, per cell
  pec                 uint8 [nz, ny, nx], 1 = perfect electric conductor cell
  freqs               float64 array of frequencies [Hz]
  src_cells, src_comp int64 arrays: the source edges as (cell index, component 0/1/2)
  src_current         complex128 currents [A] on those edges
  name, seed          provenance

The geometries follow the recipes of the workloads described in the paper's Sec. IV family of
problems (layered dielectric stacks, strips, traces, vias), scaled to the sizes the benchmark
and tests use; the exact recipe of each is written in its docstring.
"""
from __future__ import annotations

import numpy as np

MU0 = 4.0e-7 * np.pi
C0 = 299792458.0
ETA0 = MU0 * C0


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _empty(nx, ny, nz):
    return (np.ones((nz, ny, nx), np.float32), np.zeros((nz, ny, nx), np.float32),
            np.ones((nz, ny, nx), np.float32), np.zeros((nz, ny, nx), np.uint8))


def absorber_sigma(nx, ny, nz, thickness_cells, h_mean, depth_cells=8, R=1e-6, m=2):
    """Graded-conductivity absorbing layer next to all six walls: at cell-centre depth d (0 = the
    innermost layer cell, depth_cells-1 = the cell touching the wall)
    sigma(d) = sigma_max ((d + 1/2)/depth)^m,  sigma_max = -(m+1) ln R / (2 eta0 L),
    L = thickness_cells * h_mean.  Returns float64 [nz, ny, nx] (0 in the interior)."""
    L = thickness_cells * h_mean
    smax = -(m + 1) * np.log(R) / (2.0 * ETA0 * L)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dist = np.minimum.reduce([i, nx - 1 - i, j, ny - 1 - j, k, nz - 1 - k])
    d = depth_cells - 1 - dist
    s = np.where(d >= 0, smax * ((d + 0.5) / depth_cells) ** m, 0.0)
    return s


def cavity(n=16, h=1e-3, freq=5e9):
    """Config 'cavity16': PEC-walled vacuum cube of n^3 uniform cells, one unit current on the
    z-edge owned by the centre cell (n/2, n/2, n/2)."""
    eps, sig, imu, pec = _empty(n, n, n)
    c = n // 2
    return dict(name=f"cavity{n}", seed=None, nx=n, ny=n, nz=n,
                dx=np.full(n, h), dy=np.full(n, h), dz=np.full(n, h),
                eps_r=eps, sigma=sig, inv_mu_r=imu, pec=pec, freqs=np.array([freq]),
                src_cells=np.array([c + n * (c + n * c)]), src_comp=np.array([2]),
                src_current=np.array([1.0 + 0j]))


def layered_blocks(n=128, seed=2, nlayers=8, nblocks=20, freq=3e9, nsrc=64, absorber=8,
                   eps_choices=(1.0, 2.2, 3.5, 4.4, 9.8), sigma_block=5.8e7, hlim=(0.8e-3, 1.2e-3)):
    """Config 'layered128' (and the U-Net family at other n): non-uniform n^3 grid, cell widths
    i.i.d. U[0.8, 1.2] mm per axis; eps_r piecewise constant in ``nlayers`` z-layers drawn from
    {1.0, 2.2, 3.5, 4.4, 9.8}; ``nblocks`` axis-aligned conductor blocks (sigma = 5.8e7 S/m) with
    side lengths U{4..16} cells (scaled by n/128, at least 2) placed uniformly inside the
    non-absorbing interior; an ``absorber``-cell graded-conductivity layer next to the PEC walls;
    ``nsrc`` distinct source edges drawn uniformly among the edges of interior cells, currents
    CN(0, 1) A."""
    rng = _rng(seed)
    dx = rng.uniform(hlim[0], hlim[1], n)
    dy = rng.uniform(hlim[0], hlim[1], n)
    dz = rng.uniform(hlim[0], hlim[1], n)
    eps, sig, imu, pec = _empty(n, n, n)
    layer_eps = rng.choice(np.array(eps_choices), size=nlayers)
    lz = n // nlayers
    for l in range(nlayers):
        eps[l * lz:(l + 1) * lz] = layer_eps[l]
    sig64 = absorber_sigma(n, n, n, absorber, 0.5 * (hlim[0] + hlim[1]))
    lo, hi = absorber, n - absorber
    smin, smax = max(2, (4 * n) // 128), max(3, (16 * n) // 128)
    for _ in range(nblocks):
        side = rng.integers(smin, smax + 1, size=3)
        start = [rng.integers(lo, hi - side[a] + 1) for a in range(3)]
        sig64[start[2]:start[2] + side[2], start[1]:start[1] + side[1], start[0]:start[0] + side[0]] = sigma_block
    sig[:] = sig64.astype(np.float32)
    inner = np.arange(lo, hi)
    ni = len(inner)
    pick = rng.choice(ni * ni * ni * 3, size=nsrc, replace=False)
    comp = pick % 3
    cid = pick // 3
    ii, jj, kk = inner[cid % ni], inner[(cid // ni) % ni], inner[cid // (ni * ni)]
    cur = (rng.standard_normal(nsrc) + 1j * rng.standard_normal(nsrc)) / np.sqrt(2.0)
    return dict(name=f"layered{n}", seed=seed, nx=n, ny=n, nz=n, dx=dx, dy=dy, dz=dz,
                eps_r=eps, sigma=sig, inv_mu_r=imu, pec=pec, freqs=np.array([freq]),
                src_cells=(ii + n * (jj + n * kk)).astype(np.int64), src_comp=comp.astype(np.int64),
                src_current=cur)


def stripline(n=96, h=0.5e-3, nfreq=64, fmin=1e9, fmax=20e9, seed=3):
    """Config 'stripline96': uniform n^3 grid (0.5 mm); 4 z-layers of n/4 cells with
    eps_r = 3.0, 4.4, 3.0, 4.4; 1-cell PEC ground slabs at k = 0 and k = n-1; two 1-cell-thick
    PEC strips 6 cells wide, centred in y, spanning x in [8, n-8), at mid-height of layers 2 and 3
    (k = 36 and k = 60 for n = 96); port = the z-edge column at node (9, n/2) from k = 1 to the
    cell below the lower strip, 1 A on each edge; ``nfreq`` frequencies linspace(fmin, fmax).
    No random draws (the seed is recorded only)."""
    eps, sig, imu, pec = _empty(n, n, n)
    lz = n // 4
    for l, e in enumerate((3.0, 4.4, 3.0, 4.4)):
        eps[l * lz:(l + 1) * lz] = e
    pec[0] = 1
    pec[n - 1] = 1
    yc = n // 2
    k1, k2 = lz + lz // 2, 2 * lz + lz // 2
    for k in (k1, k2):
        pec[k, yc - 3:yc + 3, 8:n - 8] = 1
    ks = np.arange(1, k1)
    cells = 9 + n * (yc + n * ks)
    return dict(name=f"stripline{n}", seed=seed, nx=n, ny=n, nz=n,
                dx=np.full(n, h), dy=np.full(n, h), dz=np.full(n, h),
                eps_r=eps, sigma=sig, inv_mu_r=imu, pec=pec,
                freqs=np.linspace(fmin, fmax, nfreq),
                src_cells=cells.astype(np.int64), src_comp=np.full(len(ks), 2, np.int64),
                src_current=np.ones(len(ks), np.complex128))


def package(nx=256, ny=256, nz=192, h=0.1e-3, seed=5, nlayers=6, ntraces=400, nvias=200,
            nfreq=8, fmin=1e9, fmax=40e9, absorber=8):
    """Config 'package256': uniform nx x ny x nz grid (0.1 mm); ``nlayers`` z-layers of nz/nlayers
    cells with eps_r i.i.d. from {3.5, 4.4, 11.9}; ``ntraces`` PEC traces spread evenly over the
    layers' top cell planes, 2 cells wide, 1 cell thick, length U{16..128} cells, along x or y with
    probability 1/2, inside the non-absorbing interior; ``nvias`` z-directed 1x1-cell PEC vias
    spanning one layer, each at a random cell of a random trace; an ``absorber``-cell graded layer;
    port = the z-edge directly below the first cell of trace 0, 1 A."""
    rng = _rng(seed)
    eps, sig, imu, pec = _empty(nx, ny, nz)
    lz = nz // nlayers
    layer_eps = rng.choice(np.array([3.5, 4.4, 11.9]), size=nlayers)
    for l in range(nlayers):
        eps[l * lz:(l + 1) * lz] = layer_eps[l]
    sig[:] = absorber_sigma(nx, ny, nz, absorber, h).astype(np.float32)
    lo = absorber
    traces = []
    for t in range(ntraces):
        layer = t % nlayers
        ktop = layer * lz + lz - 1
        length = int(rng.integers(16, 129))
        along_x = bool(rng.integers(0, 2))
        if along_x:
            x0 = int(rng.integers(lo, nx - lo - length + 1))
            y0 = int(rng.integers(lo, ny - lo - 2 + 1))
            pec[ktop, y0:y0 + 2, x0:x0 + length] = 1
            cells = [(x0 + a, y0) for a in range(length)]
        else:
            x0 = int(rng.integers(lo, nx - lo - 2 + 1))
            y0 = int(rng.integers(lo, ny - lo - length + 1))
            pec[ktop, y0:y0 + length, x0:x0 + 2] = 1
            cells = [(x0, y0 + a) for a in range(length)]
        traces.append((layer, ktop, cells))
    for _ in range(nvias):
        layer, ktop, cells = traces[int(rng.integers(0, ntraces))]
        ci, cj = cells[int(rng.integers(0, len(cells)))]
        pec[layer * lz:ktop + 1, cj, ci] = 1
    layer0, ktop0, cells0 = traces[0]
    pi, pj = cells0[0]
    port_k = ktop0 - 1
    return dict(name=f"package{nx}", seed=seed, nx=nx, ny=ny, nz=nz,
                dx=np.full(nx, h), dy=np.full(ny, h), dz=np.full(nz, h),
                eps_r=eps, sigma=sig, inv_mu_r=imu, pec=pec,
                freqs=np.linspace(fmin, fmax, nfreq),
                src_cells=np.array([pi + nx * (pj + ny * port_k)], np.int64),
                src_comp=np.array([2], np.int64), src_current=np.array([1.0 + 0j]))


def random_vector(n, seed, dtype=np.complex128, batch=None):
    """Seeded complex Gaussian test vector(s) CN(0, 1) of length n (shape [batch, n] if batch)."""
    rng = _rng(seed)
    shape = (n,) if batch is None else (batch, n)
    v = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    return v.astype(dtype)


def small_random(nx, ny, nz, seed, pec_frac=0.0, lossy=True, hlim=(0.5e-3, 1.5e-3)):
    """A small random case for element-by-element parity: random widths, eps_r in [1, 10],
    sigma in [0, 5] S/m (or 0), inv_mu_r in [0.5, 1.5], a fraction of PEC cells."""
    rng = _rng(seed)
    dx = rng.uniform(*hlim, nx)
    dy = rng.uniform(*hlim, ny)
    dz = rng.uniform(*hlim, nz)
    eps = rng.uniform(1.0, 10.0, (nz, ny, nx)).astype(np.float32)
    sig = (rng.uniform(0.0, 5.0, (nz, ny, nx)) if lossy else np.zeros((nz, ny, nx))).astype(np.float32)
    imu = rng.uniform(0.5, 1.5, (nz, ny, nx)).astype(np.float32)
    pec = (rng.uniform(0.0, 1.0, (nz, ny, nx)) < pec_frac).astype(np.uint8)
    return dict(name=f"random{nx}x{ny}x{nz}", seed=seed, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
                eps_r=eps, sigma=sig, inv_mu_r=imu, pec=pec, freqs=np.array([2e9]),
                src_cells=np.array([0]), src_comp=np.array([0]), src_current=np.array([1.0 + 0j]))


def source_vector(case):
    """The impressed current vector j (complex128, length 3N, interleaved cell-by-cell) of a case:
    a scatter of the drawn currents onto their edges (index 3*cell + component)."""
    n3 = 3 * case["nx"] * case["ny"] * case["nz"]
    j = np.zeros(n3, np.complex128)
    np.add.at(j, 3 * case["src_cells"] + case["src_comp"], case["src_current"])
    return j


CASES = {
    "cavity16": cavity,
    "layered128": layered_blocks,
    "stripline96": stripline,
    "package256": package,
}
