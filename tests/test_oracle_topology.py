"""Pins of the oracle's grid topology (Sec. II, Eq. CP, Eq. e12Nxyz) against facts the paper and
discrete exterior calculus fix: S C = 0, C G = 0 exactly, two nonzeros of +-1 per line of P_w,
four per line of C, and the unknown counts n_e = 3 Nx Ny Nz of every grid in Sec. IV."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fit as F

GRIDS = [(1, 1, 1), (2, 3, 4), (5, 4, 3), (15, 10, 10), (7, 1, 5)]


@pytest.mark.parametrize("g", GRIDS)
def test_curl_of_gradient_and_divergence_of_curl_vanish(g):
    C, G, S = F.curl(*g), F.gradient(*g), F.divergence(*g)
    assert C.dtype.kind == "i" and G.dtype.kind == "i"
    assert (C @ G).count_nonzero() == 0
    assert (S @ C).count_nonzero() == 0


@pytest.mark.parametrize("g", GRIDS)
def test_partial_difference_lines(g):
    for P in F.partial_differences(*g):
        P = P.tocsr()
        nnz = np.diff(P.indptr)
        assert set(np.unique(P.data)) <= {-1, 1}
        assert nnz.max() <= 2
        # exactly one line in every pencil keeps only the -1 (the truncated last node)
        assert (P @ np.ones(P.shape[1])).min() >= -1


def test_curl_nonzeros_per_line_and_fig_spy_grid():
    nx, ny, nz = 15, 10, 10  # the grid of the paper's sparsity figure
    C = F.curl(nx, ny, nz)
    assert C.shape == (4500, 4500)
    nnz = np.diff(C.indptr)
    assert nnz.max() == 4  # MatCreateMPIAIJ preallocation of 4 per row (Sec. III)
    assert set(np.unique(C.data)) <= {-1, 1}
    # facets away from the high walls have all four boundary edges
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    interior = ((i < nx - 1) & (j < ny - 1) & (k < nz - 1)).ravel()
    assert np.all(nnz.reshape(-1, 3)[interior] == 4)


@pytest.mark.parametrize("nxyz,ne", [((46, 73, 16), 161184), ((31, 77, 22), 157542),
                                     ((63, 45, 28), 238140), ((65, 65, 14), 177450)])
def test_unknown_counts_of_paper_grids(nxyz, ne):
    """Sec. IV states n_e for each structured mesh; 3 edges owned per cell reproduces all of them."""
    C = F.curl(*nxyz)
    assert C.shape[1] == ne


def test_unknown_counts_of_large_paper_grids():
    for (nx, ny, nz), ne in [((849, 608, 327), 506384352), ((497, 354, 193), 101868102)]:
        assert F.interleave_permutation(1).shape == (3, 3)
        assert 3 * nx * ny * nz == ne


@pytest.mark.parametrize("g", [(3, 4, 5), (6, 2, 3), (15, 10, 10)])
def test_row_formulas_equal_block_kronecker_form(g):
    """Two transcriptions of Eq. CP (block Kronecker + permutation, and per-component formulas)."""
    C = F.curl(*g)
    Cd = F.curl_rows_direct(*g, np.arange(C.shape[0]))
    assert abs(C - Cd).max() == 0


def test_interleaved_ordering_of_a_single_edge():
    """Eq. e12Nxyz: unknown 3c + w is component w of cell c; a unit y-voltage on the edge of cell
    (1,1,1) of a 3^3 grid has curl on exactly the x-facets (1,1,1) (+1) and (1,1,0) (-1) and the
    z-facets (1,1,1) (-1) and (0,1,1) (+1)."""
    nx = ny = nz = 3
    C = F.curl(nx, ny, nz).toarray()
    cell = lambda i, j, k: i + nx * (j + ny * k)
    col = C[:, 3 * cell(1, 1, 1) + 1]
    nz_rows = {int(r): int(col[r]) for r in np.nonzero(col)[0]}
    assert nz_rows == {3 * cell(1, 1, 1) + 0: +1, 3 * cell(1, 1, 0) + 0: -1,
                       3 * cell(1, 1, 1) + 2: -1, 3 * cell(0, 1, 1) + 2: +1}


def test_pins_catch_planted_block_mistakes():
    """The identity pins fail for plausible mistakes in C: a flipped sign or a swapped block."""
    px, py, pz = F.partial_differences(4, 3, 5)
    G = sp.vstack([px, py, pz])
    wrong_sign = sp.bmat([[None, pz, py], [pz, None, -px], [-py, px, None]])
    swapped = sp.bmat([[None, -py, pz], [pz, None, -px], [-py, px, None]])
    for Cw in (wrong_sign, swapped):
        assert (Cw @ G).count_nonzero() > 0
