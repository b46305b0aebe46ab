"""Pins of the U-Net oracle: the torch-based conv3 / transposed conv against per-voxel loops written
from the layer definitions (tap and kernel-index conventions), and its autograd gradient against
central finite differences of the FP64 loss."""
import numpy as np
import pytest
import torch

from oracle import unet as U


def test_conv3_matches_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 3))
    w = rng.standard_normal((27, 2, 3))
    b = rng.standard_normal(2)
    xt = torch.as_tensor(x).permute(3, 0, 1, 2)[None]
    y = U.conv3(xt, torch.as_tensor(w), torch.as_tensor(b), relu=False)[0].permute(1, 2, 3, 0).numpy()
    assert np.allclose(y, U.conv3_loops(x, w, b), rtol=1e-12, atol=1e-12)


def test_tconv_matches_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 2, 4))
    w = rng.standard_normal((8, 3, 4))
    b = rng.standard_normal(3)
    xt = torch.as_tensor(x).permute(3, 0, 1, 2)[None]
    y = U.tconv(xt, torch.as_tensor(w), torch.as_tensor(b))[0].permute(1, 2, 3, 0).numpy()
    assert np.allclose(y, U.tconv_loops(x, w, b), rtol=1e-12, atol=1e-12)


def test_param_count_matches_library():
    from paper_1705_08849_gb300 import build, fit
    build.build()
    assert fit.lib().fit_unet_param_count() == U.param_count()


def test_autograd_matches_finite_differences():
    rng = np.random.default_rng(2)
    flat = rng.standard_normal(U.param_count()) * 0.2
    x = rng.standard_normal((4, 4, 4, 16))
    t = rng.standard_normal((4, 4, 4, 6))
    loss, g = U.loss_and_grad(flat, x, t, bf16=False)
    h = 1e-6
    idx = rng.choice(len(flat), 12, replace=False)
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = U.loss_and_grad(fp, x, t, bf16=False)
        lm, _ = U.loss_and_grad(fm, x, t, bf16=False)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), (i, fd, g[i])
