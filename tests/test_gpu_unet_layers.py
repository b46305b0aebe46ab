"""Per-layer parity of the learned preconditioner's kernels against the oracle's per-voxel loops.

Each layer kernel of the network (3x3x3 convolution forward, data gradient and weight gradient for
every (cin, cout) shape the network has; the 2x2x2 transposed convolutions forward and backward; the
1x1x1 head forward and backward) is called alone through the C ABI on a ragged grid (partial tiles in
x, y and z) and compared with the oracle's loops on the same bf16-rounded inputs:
  - bf16 outputs: against the oracle's FP64 result rounded to bf16 the same way, relative error
    <= 1e-3 in the 2-norm, and every element within one bf16 ulp (the FP32 accumulation may round
    the other way at a rounding boundary);
  - FP32 outputs (weight gradients, head): relative error <= 1e-3 in the 2-norm and in the largest
    element.
The convolutions run on both tensor-core paths (mma.sync and tcgen05)."""
import numpy as np
import pytest

from tests._gpu_util import fitlib, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 32), (32, 16)]
GRID = (5, 9, 37)  # (nz, ny, nx): two x tiles (one partial), partial y and z chunks


@pytest.fixture(params=["mma", "tc"])
def conv_kernel(request, monkeypatch):
    monkeypatch.setenv("FIT_CONV", request.param)
    return request.param


def _bf16(torch, a):
    return torch.as_tensor(a).to(torch.bfloat16)


def _check_bf16(torch, got_bf16, want64):
    """got: bf16 torch tensor; want: FP64 numpy result of the oracle on the same rounded inputs."""
    want_r = torch.as_tensor(want64).to(torch.bfloat16).double().numpy()
    got = got_bf16.double().cpu().numpy().reshape(want_r.shape)
    rel = np.linalg.norm(got - want_r) / max(np.linalg.norm(want_r), 1e-30)
    assert rel <= 1e-3, rel
    ulp = np.abs(want_r) * 2.0 ** -7 + 1e-5 * np.abs(want_r).max()
    bad = np.abs(got - want_r) > ulp
    assert not bad.any(), (int(bad.sum()), np.abs(got - want_r).max())


def _check_f32(got, want64):
    got = np.asarray(got, dtype=np.float64).reshape(want64.shape)
    rel = np.linalg.norm(got - want64) / max(np.linalg.norm(want64), 1e-30)
    assert rel <= 1e-3, rel
    assert np.abs(got - want64).max() <= 1e-3 * np.abs(want64).max()


def _inputs(torch, seed, shape, c):
    rng = np.random.default_rng(seed)
    x = _bf16(torch, rng.standard_normal(shape + (c,)).astype(np.float32))
    return x, x.double().numpy()


@pytest.mark.parametrize("cin,cout", SHAPES)
def test_conv3_forward(cin, cout, conv_kernel):
    torch = torch_cuda()
    fit = fitlib()
    from oracle import unet as U
    nz, ny, nx = GRID
    rng = np.random.default_rng(cin * 100 + cout)
    xb, x64 = _inputs(torch, cin + cout, GRID, cin)
    w = (rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin))).astype(np.float32)
    b = (0.1 * rng.standard_normal(cout)).astype(np.float32)
    w64 = _bf16(torch, w).double().numpy()
    out = torch.empty(nz * ny * nx, cout, dtype=torch.bfloat16, device="cuda")
    fit.fit_unet_conv3(nx, ny, nz, cin, cout, xb.cuda(), torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda(), 1, out)
    torch.cuda.synchronize()
    want = np.maximum(U.conv3_loops(x64, w64, b.astype(np.float64)), 0.0)
    _check_bf16(torch, out.cpu(), want)


@pytest.mark.parametrize("cin,cout", SHAPES)
def test_conv3_dgrad(cin, cout, conv_kernel):
    torch = torch_cuda()
    fit = fitlib()
    from oracle import unet as U
    nz, ny, nx = GRID
    rng = np.random.default_rng(cin * 100 + cout + 1)
    gb, g64 = _inputs(torch, cin + cout + 7, GRID, cout)
    w = (rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin))).astype(np.float32)
    w64 = _bf16(torch, w).double().numpy()
    din = torch.empty(nz * ny * nx, cin, dtype=torch.bfloat16, device="cuda")
    fit.fit_unet_conv3_dgrad(nx, ny, nz, cin, cout, gb.cuda(), torch.from_numpy(w).cuda(), din)
    torch.cuda.synchronize()
    _check_bf16(torch, din.cpu(), U.conv3_dgrad_loops(g64, w64))


@pytest.mark.parametrize("cin,cout", SHAPES)
def test_conv3_wgrad(cin, cout):
    torch = torch_cuda()
    fit = fitlib()
    from oracle import unet as U
    nz, ny, nx = GRID
    xb, x64 = _inputs(torch, cin + cout + 11, GRID, cin)
    gb, g64 = _inputs(torch, cin + cout + 13, GRID, cout)
    dw = torch.full((27, cout, cin), float("nan"), device="cuda")
    db = torch.full((cout,), float("nan"), device="cuda")
    fit.fit_unet_conv3_wgrad(nx, ny, nz, cin, cout, xb.cuda(), gb.cuda(), dw, db)
    torch.cuda.synchronize()
    dwo, dbo = U.conv3_wgrad_loops(x64, g64)
    _check_f32(dw.cpu().numpy(), dwo)
    _check_f32(db.cpu().numpy(), dbo)


@pytest.mark.parametrize("cin,cout", [(64, 32), (32, 16)])
def test_tconv_forward_and_backward(cin, cout, conv_kernel):
    torch = torch_cuda()
    fit = fitlib()
    from oracle import unet as U
    mz, my, mx = 3, 5, 19  # the fine grid 6 x 10 x 38
    rng = np.random.default_rng(cin + cout)
    xb, x64 = _inputs(torch, cin * 3 + cout, (mz, my, mx), cin)
    w = (rng.standard_normal((8, cout, cin)) / np.sqrt(cin)).astype(np.float32)
    b = (0.1 * rng.standard_normal(cout)).astype(np.float32)
    wd, bd = torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty(8 * mz * my * mx, cout, dtype=torch.bfloat16, device="cuda")
    fit.fit_unet_tconv(mx, my, mz, cin, cout, xb.cuda(), wd, bd, out)
    torch.cuda.synchronize()
    w64 = _bf16(torch, w).double().numpy()  # the network multiplies with bf16 weights
    _check_bf16(torch, out.cpu(), U.tconv_loops(x64, w64, b.astype(np.float64)))
    gb, g64 = _inputs(torch, cin * 3 + cout + 1, (2 * mz, 2 * my, 2 * mx), cout)
    din = torch.empty(mz * my * mx, cin, dtype=torch.bfloat16, device="cuda")
    dw = torch.full((8, cout, cin), float("nan"), device="cuda")
    db = torch.full((cout,), float("nan"), device="cuda")
    fit.fit_unet_tconv_backward(mx, my, mz, cin, cout, xb.cuda(), gb.cuda(), wd, din, dw, db)
    torch.cuda.synchronize()
    _check_bf16(torch, din.cpu(), U.tconv_dgrad_loops(g64, w64))
    dwo, dbo = U.tconv_wgrad_loops(x64, g64)
    _check_f32(dw.cpu().numpy(), dwo)
    _check_f32(db.cpu().numpy(), dbo)


def test_head_forward_and_backward():
    torch = torch_cuda()
    fit = fitlib()
    from oracle import unet as U
    n = 4 * 9 * 37 + 5  # not a multiple of the block size
    rng = np.random.default_rng(99)
    xb = _bf16(torch, rng.standard_normal((n, 16)).astype(np.float32))
    x64 = xb.double().numpy()
    w = rng.standard_normal((6, 16)).astype(np.float32)
    b = rng.standard_normal(6).astype(np.float32)
    wd, bd = torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty(n, 6, device="cuda")
    fit.fit_unet_head(n, xb.cuda(), wd, bd, out)
    torch.cuda.synchronize()
    _check_f32(out.cpu().numpy(), U.head_fwd(x64, w.astype(np.float64), b.astype(np.float64)))
    g = rng.standard_normal((n, 6)).astype(np.float32)
    din = torch.empty(n, 16, dtype=torch.bfloat16, device="cuda")
    dw = torch.full((6, 16), float("nan"), device="cuda")
    db = torch.full((6,), float("nan"), device="cuda")
    fit.fit_unet_head_backward(n, xb.cuda(), torch.from_numpy(g).cuda(), wd, din, dw, db)
    torch.cuda.synchronize()
    dino, dwo, dbo = U.head_bwd(x64, g.astype(np.float64), w.astype(np.float64))
    _check_bf16(torch, din.cpu(), dino)
    _check_f32(dw.cpu().numpy(), dwo)
    _check_f32(db.cpu().numpy(), dbo)
