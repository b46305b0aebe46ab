"""The autotuner's persistent cache (host code, no GPU): records round-trip, the last matching line wins,
other keys and other builds' variant tables are ignored, and malformed files do not break a lookup."""
import pytest


@pytest.fixture(scope="module")
def fit():
    from paper_1705_08849_gb300 import build, fit
    build.build()
    fit.lib()
    return fit


KEY = dict(device="NVIDIA GB300", sm_count=152, nx=128, ny=128, nz=128)


def _look(fit, path, prec=0, nbatch=1, **over):
    k = dict(KEY, **over)
    return fit.fit_tuning_lookup(path, k["device"], k["sm_count"], k["nx"], k["ny"], k["nz"], prec, nbatch)


def _rec(fit, path, choice, prec=0, nbatch=1, **over):
    k = dict(KEY, **over)
    fit.fit_tuning_record(path, k["device"], k["sm_count"], k["nx"], k["ny"], k["nz"], prec, nbatch, choice)


def test_round_trip_and_last_line_wins(fit, tmp_path):
    p = str(tmp_path / "tune.txt")
    assert _look(fit, p) == -2  # no file yet
    _rec(fit, p, 21)
    assert _look(fit, p) == 21
    _rec(fit, p, -1)
    assert _look(fit, p) == -1  # the generic kernel is a valid choice
    _rec(fit, p, 4)
    assert _look(fit, p) == 4
    lines = open(p).read().splitlines()
    assert len(lines) == 3 and lines[0].startswith("fit-tune 1 NVIDIA_GB300 152 128 128 128 0 1 ")


def test_keys_do_not_mix(fit, tmp_path):
    p = str(tmp_path / "tune.txt")
    _rec(fit, p, 3, prec=0, nbatch=1)
    _rec(fit, p, 5, prec=1, nbatch=1)
    _rec(fit, p, 7, prec=0, nbatch=8)
    assert _look(fit, p, prec=0, nbatch=1) == 3
    assert _look(fit, p, prec=1, nbatch=1) == 5
    assert _look(fit, p, prec=0, nbatch=8) == 7
    assert _look(fit, p, nx=64) == -2
    assert _look(fit, p, sm_count=148) == -2
    assert _look(fit, p, device="NVIDIA B200") == -2


def test_other_builds_and_bad_lines_are_ignored(fit, tmp_path):
    p = tmp_path / "tune.txt"
    nvar = fit.fit_apply_variant_count(0)
    p.write_text("garbage\n"
                 "fit-tune 2 NVIDIA_GB300 152 128 128 128 0 1 %d 1\n"  # another format version
                 "fit-tune 1 NVIDIA_GB300 152 128 128 128 0 1 %d 2\n"  # another variant table
                 "fit-tune 1 NVIDIA_GB300 152 128 128 128 0 1 %d %d\n"  # choice out of range
                 "fit-tune 1 NVIDIA_GB300 152 128 128 128 0 1 %d 6\n"  # the valid one
                 "fit-tune 1 NVIDIA_GB300 152 128\n"  # truncated
                 % (nvar, nvar + 1, nvar, nvar, nvar))
    assert _look(fit, str(p)) == 6


def test_bad_arguments(fit, tmp_path):
    p = str(tmp_path / "tune.txt")
    nvar = fit.fit_apply_variant_count(0)
    for bad in (dict(choice=nvar), dict(choice=-2)):
        with pytest.raises(fit.FitError):
            _rec(fit, p, bad["choice"])
    with pytest.raises(fit.FitError):
        fit.fit_tuning_record(p, "d", 152, 0, 1, 1, 0, 1, 0)
    with pytest.raises(fit.FitError):
        fit.fit_tuning_record(str(tmp_path / "no" / "such" / "dir.txt"), "d", 152, 1, 1, 1, 0, 1, 0)
    assert fit.lib().fit_tuning_lookup(None, b"d", 1, 1, 1, 1, 0, 1, None) == fit.FIT_EINVAL
