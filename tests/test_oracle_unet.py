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


def test_conv3_dgrad_is_the_adjoint_of_conv3():
    """<conv3(x; W), g> = <x, dgrad(g; W)> for every x and g (the data gradient of a linear map is its
    adjoint); a dropped tap, a wrong tap sign or an untransposed W breaks it."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 4, 5, 3))
    w = rng.standard_normal((27, 2, 3))
    g = rng.standard_normal((3, 4, 5, 2))
    lhs = np.sum(U.conv3_loops(x, w, np.zeros(2)) * g)
    rhs = np.sum(x * U.conv3_dgrad_loops(g, w))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_conv3_wgrad_is_linear_in_the_weights():
    """<conv3(x; W', b'), g> = <W', dW> + <b', db> for every W', b' (the map is linear in the weights)."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 4, 5, 3))
    g = rng.standard_normal((3, 4, 5, 2))
    dw, db = U.conv3_wgrad_loops(x, g)
    for _ in range(3):
        w2 = rng.standard_normal((27, 2, 3))
        b2 = rng.standard_normal(2)
        lhs = np.sum(U.conv3_loops(x, w2, b2) * g)
        assert lhs == pytest.approx(np.sum(w2 * dw) + np.sum(b2 * db), rel=1e-12)


def test_conv3_gradients_match_autograd():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 3, 4, 3))
    w = rng.standard_normal((27, 2, 3))
    g = rng.standard_normal((2, 3, 4, 2))
    xt = torch.as_tensor(x).permute(3, 0, 1, 2)[None].clone().requires_grad_(True)
    wt = torch.as_tensor(w).clone().requires_grad_(True)
    bt = torch.zeros(2, dtype=torch.float64, requires_grad=True)
    y = U.conv3(xt, wt, bt, relu=False)
    (y * torch.as_tensor(g).permute(3, 0, 1, 2)[None]).sum().backward()
    dw, db = U.conv3_wgrad_loops(x, g)
    assert np.allclose(xt.grad[0].permute(1, 2, 3, 0).numpy(), U.conv3_dgrad_loops(g, w), rtol=1e-12, atol=1e-12)
    assert np.allclose(wt.grad.numpy(), dw, rtol=1e-12, atol=1e-12)
    assert np.allclose(bt.grad.numpy(), db, rtol=1e-12, atol=1e-12)


def test_tconv_gradients_are_adjoint_and_linear():
    rng = np.random.default_rng(6)
    x = rng.standard_normal((2, 3, 2, 4))
    w = rng.standard_normal((8, 3, 4))
    g = rng.standard_normal((4, 6, 4, 3))
    lhs = np.sum(U.tconv_loops(x, w, np.zeros(3)) * g)
    assert lhs == pytest.approx(np.sum(x * U.tconv_dgrad_loops(g, w)), rel=1e-12)
    dw, db = U.tconv_wgrad_loops(x, g)
    w2, b2 = rng.standard_normal((8, 3, 4)), rng.standard_normal(3)
    assert np.sum(U.tconv_loops(x, w2, b2) * g) == pytest.approx(np.sum(w2 * dw) + np.sum(b2 * db), rel=1e-12)


def test_head_gradients_are_adjoint_and_linear():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((50, 16))
    w = rng.standard_normal((6, 16))
    g = rng.standard_normal((50, 6))
    din, dw, db = U.head_bwd(x, g, w)
    assert np.sum(U.head_fwd(x, w, np.zeros(6)) * g) == pytest.approx(np.sum(x * din), rel=1e-12)
    w2, b2 = rng.standard_normal((6, 16)), rng.standard_normal(6)
    assert np.sum(U.head_fwd(x, w2, b2) * g) == pytest.approx(np.sum(w2 * dw) + np.sum(b2 * db), rel=1e-12)


def test_residual_angle_gradient_matches_finite_differences():
    """The oracle's residual-angle loss: its autograd gradient (through the sparse apply's adjoint) equals
    central finite differences in FP64, on a small complex symmetric A."""
    import scipy.sparse as sp
    rng = np.random.default_rng(8)
    n = 4
    ne = 3 * n ** 3
    M = sp.random(ne, ne, density=0.05, random_state=1) + 1j * sp.random(ne, ne, density=0.05, random_state=2)
    A = (M + M.T + 4 * sp.eye(ne)).tocsr()  # complex symmetric
    mask = (rng.random(ne) < 0.1).astype(np.uint8)
    flat = rng.standard_normal(U.param_count()) * 0.2
    x = rng.standard_normal((n, n, n, 16))
    # rounding to bf16 inside forward makes the loss piecewise constant in the conv weights; difference the
    # head (FP32, no rounding) instead
    _, g = U.residual_angle_loss_and_grad(flat, x, A, mask)
    head0 = U.param_count() - 6 * 16 - 6
    h = 1e-6
    for i in rng.choice(np.arange(head0, U.param_count()), 6, replace=False):
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = U.residual_angle_loss_and_grad(fp, x, A, mask)
        lm, _ = U.residual_angle_loss_and_grad(fm, x, A, mask)
        assert (lp - lm) / (2 * h) == pytest.approx(g[i], rel=1e-5, abs=1e-10), i
