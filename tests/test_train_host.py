"""Host logic of the learned preconditioner's training module that needs no GPU: the checkpoint format
(the committed network included), the seeded head start of a residual-angle stage, the evaluation's
method table and the harvest's frequency draw."""
import json

import numpy as np
import pytest

from paper_1705_08849_gb300 import train_unet as T


class _Net:
    """Stands in for fit.UNet: the flat FP32 parameters and their count."""

    def __init__(self, n):
        self.nparams = n
        self.p = np.zeros(n, np.float32)

    def get_params(self):
        return self.p.copy()

    def set_params(self, p):
        self.p = np.asarray(p, np.float32).copy()


def test_checkpoint_round_trip(tmp_path):
    net = _Net(1000)
    net.p = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    path = tmp_path / "w.fitw"
    T.save(net, str(path), {"pairs": 12})
    other = _Net(1000)
    head = T.load(other, str(path))
    assert head["format"] == T.FORMAT and head["record"] == {"pairs": 12}
    assert np.array_equal(other.p, net.p)
    with pytest.raises(ValueError):
        T.load(_Net(999), str(path))  # another parameter count is refused


def test_committed_checkpoint_is_the_network_of_the_record():
    """The committed weights load into a network of the library's parameter count (the oracle's layer
    table gives it) and carry the training record the evaluation quotes."""
    from oracle import unet as U
    with open(T.DEFAULT_WEIGHTS, "rb") as fh:
        head = json.loads(fh.readline().decode())
        p = np.frombuffer(fh.read(), dtype="<f4")
    assert head["format"] == T.FORMAT and head["nparams"] == U.param_count() == p.size
    assert np.all(np.isfinite(p)) and np.abs(p).max() > 0
    rec = head["record"]
    assert rec["n"] == 64 and rec["pairs"] > 15000 and rec["stages"][0]["loss"] == "error"
    assert rec["stages"][0]["validation_loss_final"] < rec["stages"][0]["validation_loss_initial"]


def test_seed_head_touches_only_the_head_weights():
    net = _Net(500)
    T.seed_head(net, 7)
    nz = np.nonzero(net.p)[0]
    assert nz.min() >= 500 - (6 * 16 + 6) and nz.max() < 500 - 6  # the 6 x 16 head weights, not its biases
    assert len(nz) == 96
    again = _Net(500)
    T.seed_head(again, 7)
    assert np.array_equal(again.p, net.p)  # seeded


def test_methods_name_valid_solver_settings():
    class _Fit:
        FIT_FGMRES, FIT_BICGSTAB, FIT_COCG = 1, 0, 2
        FIT_SOLVE_MIXED = 1
        FIT_PC_NONE, FIT_PC_JACOBI, FIT_PC_UNET = 0, 1, 2
    for name, spec in T.METHODS.items():
        vals = [getattr(_Fit, a) for a in spec[:3]]
        assert len(vals) == 3
        if "unet" in name:
            assert spec[0] == "FIT_FGMRES" and spec[2] == "FIT_PC_UNET"
        if len(spec) > 3:
            assert spec[3] >= 2


def test_harvest_frequencies_are_seeded_and_in_band():
    fs = [T._freq(s, 1e9, 10e9) for s in range(1000, 1050)]
    assert fs == [T._freq(s, 1e9, 10e9) for s in range(1000, 1050)]
    assert min(fs) >= 1e9 and max(fs) <= 10e9 and len(set(fs)) == 50
