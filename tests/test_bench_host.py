"""Host logic of bench.py that needs no GPU: the solve-kind syntax and the seeded port columns."""
import numpy as np
import pytest

import bench


class _Consts:
    FIT_BICGSTAB, FIT_FGMRES, FIT_COCG, FIT_COCR = 0, 1, 2, 3
    FIT_PC_NONE, FIT_PC_JACOBI, FIT_PC_UNET, FIT_PC_EPS = 0, 1, 2, 3
    FIT_SOLVE_C128, FIT_SOLVE_MIXED = 0, 1


@pytest.mark.parametrize("kind,want", [
    ("mixed", (1, 1, 1)),
    ("c128", (1, 0, 1)),
    ("cocg-mixed", (2, 1, 1)),
    ("cocr-c128+none", (3, 0, 0)),
    ("bicgstab-mixed+eps", (0, 1, 3)),
    ("fgmres-c128+jacobi", (1, 0, 1)),
    ("fgmres-mixed+unet", (1, 1, 2)),
    ("mixed+unet/3", (1, 1, 2)),
])
def test_parse_kind(kind, want):
    assert bench.valid_kind(kind)
    assert bench.parse_kind(_Consts, kind)[:3] == want


def test_learned_kinds_place_the_network():
    assert bench.parse_kind(_Consts, "fgmres-mixed+unet")[4] == 0  # once per restart cycle (the default)
    assert bench.parse_kind(_Consts, "fgmres-mixed+unet/3")[4] == 3  # steps j with (j + 1) % 3 == 0


@pytest.mark.parametrize("kind", ["cocg", "cocg-fp32", "gmres-mixed", "cocg-mixed+ilu", "none", "",
                                  "cocg-mixed+unet", "fgmres-c128+unet", "mixed+unet/1", "mixed+unet/x"])
def test_invalid_kinds_are_dropped(kind):
    assert not bench.valid_kind(kind)


def test_port_columns_are_seeded_distinct_and_in_range():
    case = dict(nx=128, ny=96, nz=40)
    a = bench.port_columns(case, 6)
    assert a == bench.port_columns(case, 6)  # seeded
    ne = 3 * 128 * 96 * 40
    heads = set()
    for edges, signs in a:
        assert len(edges) == 8 and signs == [1.0] * 8
        c = np.asarray(edges) // 3
        assert np.all(np.asarray(edges) % 3 == 2) and np.all((0 <= np.asarray(edges)) & (np.asarray(edges) < ne))
        i, j, k = c % 128, (c // 128) % 96, c // (128 * 96)
        assert len(set(i)) == 1 and len(set(j)) == 1 and list(k) == list(range(8))  # one column from z = 0
        assert 16 <= i[0] < 128 - 16 and 16 <= j[0] < 96 - 16
        heads.add((int(i[0]), int(j[0])))
    assert len(heads) == 6
    short = bench.port_columns(dict(nx=40, ny=40, nz=5), 2, margin=8)
    assert all(len(e) == 5 for e, _ in short)  # capped at the grid height


def test_learned_vs_plain_summary():
    solves = {
        "cocg-mixed": {"s_per_freq": 3.4, "status": "FIT_OK", "iterations": 21740, "method": "COCG"},
        "mixed": {"s_per_freq": 36.0, "status": "FIT_OK", "iterations": 42150, "method": "FGMRES"},
        "mixed+unet": {"s_per_freq": 30.0, "status": "FIT_OK", "iterations": 30000, "method": "FGMRES+U-Net"},
        "c128": {"s_per_freq": 270.0, "status": "FIT_NOT_CONVERGED", "iterations": 80000, "method": "FGMRES c128"},
    }
    out = bench.learned_vs_plain(solves)
    assert out["learned"]["s"] == 30.0 and out["without_network"]["s"] == 36.0
    assert [p["kind"] for p in out["plain_fp64"]] == ["c128"]  # cocg-c128 was not timed
    assert out["fastest_converged"]["method"] == "COCG"  # the unconverged solve is never the fastest
    assert bench.learned_vs_plain({})["learned"] is None
