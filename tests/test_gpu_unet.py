"""GPU parity of the learned preconditioner's U-Net against the oracle (plain torch-CPU FP64 with
bf16 rounding where the GPU stores bf16): forward output, loss and every parameter gradient;
training reduces the loss; packing/unpacking; FGMRES with the network attached."""
import numpy as np
import pytest

import fitgen as G
from tests._gpu_util import fitlib, oracle_A, oracle_matrices, torch_cuda

pytestmark = pytest.mark.gpu


def _net_and_input(seed, shape, head_scale=0.5):
    torch = torch_cuda()
    fit = fitlib()
    from oracle import unet as U
    net = fit.UNet(seed=seed)
    p = net.get_params()
    # the library starts the head at zero; give it values so the output is non-trivial
    off = 0
    for name, (kind, ci, co) in zip(U.NAMES, U.LAYERS):
        nw = U._taps(kind) * ci * co
        if name == "head":
            p[off:off + nw] = np.random.default_rng(seed).standard_normal(nw).astype(np.float32) * head_scale
            p[off + nw:off + nw + co] = 0.1
        off += nw + co
    net.set_params(p)
    nz, ny, nx = shape
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    x = torch.randn(nz, ny, nx, 16, device="cuda", generator=gen).to(torch.bfloat16)
    return net, p, x


@pytest.fixture(params=["mma", "tc"])
def conv_kernel(request, monkeypatch):
    """Every network test runs with the mma.sync convolutions and with the tcgen05 ones."""
    monkeypatch.setenv("FIT_CONV", request.param)
    return request.param


@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 12, 16), (12, 8, 36)])
def test_forward_matches_oracle(shape, conv_kernel):
    torch = torch_cuda()
    from oracle import unet as U
    net, p, x = _net_and_input(11, shape)
    nz, ny, nx = shape
    y = torch.empty(nz, ny, nx, 6, device="cuda", dtype=torch.float32)
    net.forward(nx, ny, nz, x, y)
    torch.cuda.synchronize()
    yo = U.forward(U.unflatten(p), x.float().cpu().numpy(), bf16=True).numpy()
    yg = y.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
    assert rel <= 5e-3, rel


def test_gradients_match_oracle(conv_kernel):
    torch = torch_cuda()
    from oracle import unet as U
    shape = (8, 8, 12)
    net, p, x = _net_and_input(12, shape)
    nz, ny, nx = shape
    t = torch.randn(nz, ny, nx, 6, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    grad = torch.empty(net.nparams, device="cuda", dtype=torch.float32)
    loss = net.backward(nx, ny, nz, x, t, grad)
    torch.cuda.synchronize()
    lo, go = U.loss_and_grad(p, x.float().cpu().numpy(), t.cpu().numpy(), bf16=True)
    assert loss == pytest.approx(lo, rel=1e-2)
    gg = grad.cpu().numpy().astype(np.float64)
    off = 0
    for name, (kind, ci, co) in zip(U.NAMES, U.LAYERS):
        n = U._taps(kind) * ci * co + co
        a, b = gg[off:off + n], go[off:off + n]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= 5e-2, (name, rel)
        off += n


def test_training_reduces_loss(conv_kernel):
    torch = torch_cuda()
    shape = (8, 8, 8)
    net, p, x = _net_and_input(13, shape, head_scale=0.0)
    nz, ny, nx = shape
    t = torch.sin(torch.arange(nz * ny * nx * 6, device="cuda", dtype=torch.float32) * 0.01).reshape(nz, ny, nx, 6)
    losses = [net.train_step(nx, ny, nz, x, t, 3e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], losses[::10]


def test_pack_unpack_and_jacobi():
    torch = torch_cuda()
    fit = fitlib()
    from oracle import fit as F
    case = G.small_random(8, 12, 4, seed=21, pec_frac=0.1)
    with fit.Grid.from_case(case) as g:
        ne = g.ne
        r = torch.randn(ne, dtype=torch.complex64, device="cuda")
        x16 = torch.empty(ne // 3, 16, dtype=torch.bfloat16, device="cuda")
        fit.fit_unet_pack(g.h, r, 2.0, x16)
        torch.cuda.synchronize()
        rr = torch.view_as_real(r).reshape(-1, 6).cpu()
        assert torch.equal(x16[:, :6].cpu(), (2.0 * rr).to(torch.bfloat16))
        assert torch.count_nonzero(x16[:, 10:]).item() == 0
        assert x16[:, 6].float().cpu().numpy() == pytest.approx(case["eps_r"].ravel() / 10, rel=1e-2)
        y6 = torch.randn(ne // 3, 6, device="cuda")
        z = torch.empty(ne, dtype=torch.complex64, device="cuda")
        fit.fit_unet_unpack(g.h, y6, 0.5, z)
        torch.cuda.synchronize()
        mask = F.edge_mask(8, 12, 4, case["pec"])
        zz = torch.view_as_complex(0.5 * y6.cpu().reshape(-1, 3, 2)).reshape(-1).numpy() * (1 - mask)
        assert np.allclose(z.cpu().numpy(), zz)
        # Jacobi: y = diag(A)^-1 x against the oracle's diagonal
        w = 2 * np.pi * 3e9
        me, mk, mn, msk = oracle_matrices(case)
        d = F.jacobi_diagonal(w, 8, 12, 4, me, mk, mn, msk)
        xv = torch.from_numpy(G.random_vector(ne, 3)).cuda()
        yv = torch.empty_like(xv)
        fit.fit_jacobi(g.h, [w], xv, yv, fit.FIT_C128)
        torch.cuda.synchronize()
        assert np.allclose(yv.cpu().numpy(), xv.cpu().numpy() / d, rtol=1e-12)


def test_fgmres_with_attached_unet():
    """FGMRES(20) with the learned preconditioner (an untrained network gives plain Jacobi) reaches
    the tolerance under the oracle's residual."""
    torch = torch_cuda()
    fit = fitlib()
    from oracle import fit as F
    case = G.small_random(16, 16, 12, seed=22, pec_frac=0.05)
    net = fit.UNet(seed=1)
    w = 2 * np.pi * 4e9
    A, mask = oracle_A(case, w)
    b = G.random_vector(A.shape[0], 7) * (1 - mask)
    with fit.Grid.from_case(case) as g:
        fit.fit_set_preconditioner(g.h, net)
        bt = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bt)
        st, rep = g.solve([w], bt, x, 1e-8, method=1, restart=20, precond=fit.FIT_PC_UNET, max_outer=2000,
                          max_iter=40000)
        torch.cuda.synchronize()
    rr = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert st == 0 and rr <= 1e-8, (rr, rep)
