"""Oracle of the learned right preconditioner (a 3-level 3D U-Net) -- TEST INFRASTRUCTURE.

Plain PyTorch CPU float64 ops (conv3d, avg_pool3d, conv_transpose3d) and autograd for the
gradients.  With ``bf16=True`` it rounds to bfloat16 exactly where the GPU network stores bf16
(conv inputs/outputs, pooled and upsampled activations, the 3x3x3 and transposed-conv weights: the
network keeps BF16 weights and activations with FP32 accumulation), so GPU and oracle can be
compared on the same rounded values; with ``bf16=False`` it is the exact FP64 network (used for the
finite-difference pins).

Network (same flat parameter layout as the library): per layer W then b, layers
c1a c1b | c2a c2b | c3a c3b | t2 c2c c2d | t1 c1c c1d | head, with
  conv3 W[tap][co][ci], tap = dz*9 + dy*3 + dx  (out[v] = sum in[v + (dx-1, dy-1, dz-1)] W)
  tconv W[k][co][ci],   k = x%2 + 2 (y%2) + 4 (z%2)  (2x2x2, stride 2)
  head  W[o][c]         (1x1x1, 16 -> 6)
Tensors are NDHWC numpy/torch arrays [nz, ny, nx, C] at the interface.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn

LAYERS = [("conv3", 16, 16), ("conv3", 16, 16), ("conv3", 16, 32), ("conv3", 32, 32), ("conv3", 32, 64),
          ("conv3", 64, 64), ("tconv", 64, 32), ("conv3", 64, 32), ("conv3", 32, 32), ("tconv", 32, 16),
          ("conv3", 32, 16), ("conv3", 16, 16), ("head", 16, 6)]
NAMES = ["c1a", "c1b", "c2a", "c2b", "c3a", "c3b", "t2", "c2c", "c2d", "t1", "c1c", "c1d", "head"]


def _taps(kind):
    return {"conv3": 27, "tconv": 8, "head": 1}[kind]


def param_count():
    return sum(_taps(k) * ci * co + co for k, ci, co in LAYERS)


def unflatten(flat):
    """flat float vector -> {name: (W tensor in library layout, b tensor)} as float64 torch tensors."""
    flat = torch.as_tensor(np.asarray(flat), dtype=torch.float64)
    out, off = {}, 0
    for name, (kind, ci, co) in zip(NAMES, LAYERS):
        nw = _taps(kind) * ci * co
        w = flat[off:off + nw].reshape(_taps(kind), co, ci) if kind != "head" else flat[off:off + nw].reshape(co, ci)
        off += nw
        b = flat[off:off + co]
        off += co
        out[name] = (w, b)
    assert off == flat.numel()
    return out


def _bf(t, on):
    return t.to(torch.bfloat16).to(torch.float64) if on else t


def conv3(x, w, b, relu=True):
    """x: [1, ci, nz, ny, nx]; w: [27, co, ci] (library layout) -> torch conv3d weight [co, ci, kz, ky, kx]."""
    co, ci = w.shape[1], w.shape[2]
    wt = w.reshape(3, 3, 3, co, ci).permute(3, 4, 0, 1, 2)
    y = Fn.conv3d(x, wt, b, padding=1)
    return torch.relu(y) if relu else y


def tconv(x, w, b):
    """x: [1, ci, Z, Y, X]; w: [8, co, ci] with k = kx + 2 ky + 4 kz -> weight [ci, co, kz, ky, kx]."""
    co, ci = w.shape[1], w.shape[2]
    wt = w.reshape(2, 2, 2, co, ci).permute(4, 3, 0, 1, 2)
    return Fn.conv_transpose3d(x, wt, b, stride=2)


def forward(params, x_ndhwc, bf16=True):
    """Network output [nz, ny, nx, 6] (float64 torch tensor) for an input [nz, ny, nx, 16]."""
    x = torch.as_tensor(np.asarray(x_ndhwc, dtype=np.float64)).permute(3, 0, 1, 2)[None]
    r = lambda t: _bf(t, bf16)
    W = {k: (r(w) if LAYERS[NAMES.index(k)][0] in ("conv3", "tconv") else w, b) for k, (w, b) in params.items()}
    x0 = r(x)
    a1a = r(conv3(x0, *W["c1a"]))
    s1 = r(conv3(a1a, *W["c1b"]))
    p1 = r(Fn.avg_pool3d(s1, 2))
    a2a = r(conv3(p1, *W["c2a"]))
    s2 = r(conv3(a2a, *W["c2b"]))
    p2 = r(Fn.avg_pool3d(s2, 2))
    a3a = r(conv3(p2, *W["c3a"]))
    b3 = r(conv3(a3a, *W["c3b"]))
    u2 = r(tconv(b3, *W["t2"]))
    a2c = r(conv3(torch.cat([s2, u2], 1), *W["c2c"]))
    b2 = r(conv3(a2c, *W["c2d"]))
    u1 = r(tconv(b2, *W["t1"]))
    a1c = r(conv3(torch.cat([s1, u1], 1), *W["c1c"]))
    b1 = r(conv3(a1c, *W["c1d"]))
    wh, bh = W["head"]
    y = Fn.conv3d(b1, wh[:, :, None, None, None], bh)
    return y[0].permute(1, 2, 3, 0)


def loss_and_grad(flat, x_ndhwc, target_ndhwc, bf16=True):
    """L = ||U(x) - t||^2 / ||t||^2 and dL/dflat (float64) by autograd through ``forward``."""
    p = torch.as_tensor(np.asarray(flat, dtype=np.float64)).clone().requires_grad_(True)
    y = forward(unflatten_t(p), x_ndhwc, bf16=bf16)
    t = torch.as_tensor(np.asarray(target_ndhwc, dtype=np.float64))
    loss = ((y - t) ** 2).sum() / (t ** 2).sum()
    loss.backward()
    return float(loss.detach()), p.grad.numpy()


def unflatten_t(p):
    """``unflatten`` for a torch tensor that requires grad (keeps the graph)."""
    out, off = {}, 0
    for name, (kind, ci, co) in zip(NAMES, LAYERS):
        nw = _taps(kind) * ci * co
        w = p[off:off + nw].reshape(_taps(kind), co, ci) if kind != "head" else p[off:off + nw].reshape(co, ci)
        off += nw
        out[name] = (w, p[off:off + co])
        off += co
    return out


def conv3_loops(x, w, b):
    """Per-voxel loops of out[z,y,x,co] = b[co] + sum_{dz,dy,dx,ci} in[z+dz-1, y+dy-1, x+dx-1, ci] W[tap][co][ci]
    (zero outside), NDHWC numpy in and out; tiny shapes only."""
    nz, ny, nx, ci = x.shape
    co = w.shape[1]
    out = np.zeros((nz, ny, nx, co))
    for z in range(nz):
        for y in range(ny):
            for xx in range(nx):
                acc = np.array(b, dtype=np.float64).copy()
                for tap in range(27):
                    dz, dy, dx = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
                    zs, ys, xs = z + dz, y + dy, xx + dx
                    if 0 <= zs < nz and 0 <= ys < ny and 0 <= xs < nx:
                        acc += w[tap] @ x[zs, ys, xs]
                out[z, y, xx] = acc
    return out


def tconv_loops(x, w, b):
    """Per-voxel loops of out[z,y,x,co] = b[co] + sum_ci in[z//2, y//2, x//2, ci] W[k][co][ci]."""
    Z, Y, X, ci = x.shape
    co = w.shape[1]
    out = np.zeros((2 * Z, 2 * Y, 2 * X, co))
    for z in range(2 * Z):
        for y in range(2 * Y):
            for xx in range(2 * X):
                k = (xx % 2) + 2 * (y % 2) + 4 * (z % 2)
                out[z, y, xx] = np.asarray(b) + w[k] @ x[z // 2, y // 2, xx // 2]
    return out


def conv3_dgrad_loops(dout, w):
    """Data gradient of ``conv3_loops`` for the loss sum(out * dout): per input voxel u,
    din[u] = sum over taps with v = u - off(tap) inside the grid of W[tap]^T dout[v]
    (NDHWC numpy in and out; tiny shapes only)."""
    nz, ny, nx, co = dout.shape
    ci = w.shape[2]
    din = np.zeros((nz, ny, nx, ci))
    for z in range(nz):
        for y in range(ny):
            for xx in range(nx):
                acc = np.zeros(ci)
                for tap in range(27):
                    dz, dy, dx = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
                    zs, ys, xs = z - dz, y - dy, xx - dx
                    if 0 <= zs < nz and 0 <= ys < ny and 0 <= xs < nx:
                        acc += w[tap].T @ dout[zs, ys, xs]
                din[z, y, xx] = acc
    return din


def conv3_wgrad_loops(x, dout):
    """Weight and bias gradients of ``conv3_loops`` for the loss sum(out * dout):
    dW[tap][co][ci] = sum_v dout[v][co] x[v + off(tap)][ci] (inside the grid), db[co] = sum_v dout[v][co]."""
    nz, ny, nx, ci = x.shape
    co = dout.shape[3]
    dw = np.zeros((27, co, ci))
    for z in range(nz):
        for y in range(ny):
            for xx in range(nx):
                for tap in range(27):
                    dz, dy, dx = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
                    zs, ys, xs = z + dz, y + dy, xx + dx
                    if 0 <= zs < nz and 0 <= ys < ny and 0 <= xs < nx:
                        dw[tap] += np.outer(dout[z, y, xx], x[zs, ys, xs])
    return dw, dout.reshape(-1, co).sum(axis=0)


def tconv_dgrad_loops(dout, w):
    """Data gradient of ``tconv_loops``: din[V] = sum_k W[k]^T dout[child(V, k)], child(V, k) = 2V + (kx, ky, kz)."""
    Z2, Y2, X2, co = dout.shape
    ci = w.shape[2]
    din = np.zeros((Z2 // 2, Y2 // 2, X2 // 2, ci))
    for z in range(Z2):
        for y in range(Y2):
            for xx in range(X2):
                k = (xx % 2) + 2 * (y % 2) + 4 * (z % 2)
                din[z // 2, y // 2, xx // 2] += w[k].T @ dout[z, y, xx]
    return din


def tconv_wgrad_loops(x, dout):
    """Weight and bias gradients of ``tconv_loops``: dW[k] = sum_V outer(dout[child(V, k)], x[V]), db = sum dout."""
    Z2, Y2, X2, co = dout.shape
    ci = x.shape[3]
    dw = np.zeros((8, co, ci))
    for z in range(Z2):
        for y in range(Y2):
            for xx in range(X2):
                k = (xx % 2) + 2 * (y % 2) + 4 * (z % 2)
                dw[k] += np.outer(dout[z, y, xx], x[z // 2, y // 2, xx // 2])
    return dw, dout.reshape(-1, co).sum(axis=0)


def head_fwd(x, w, b):
    """1x1x1 head: out[v][o] = b[o] + sum_c x[v][c] W[o][c] (x [N, C] numpy)."""
    return x @ w.T + b


def head_bwd(x, dout, w):
    """Gradients of ``head_fwd`` for the loss sum(out * dout): (din, dW, db)."""
    return dout @ w, dout.T @ x, dout.sum(axis=0)


class _SparseApply(torch.autograd.Function):
    """w = A z for a complex symmetric scipy sparse A (A^T = A), with the adjoint A^H = conj(A) in the
    backward pass: d conj(z) = A^H d conj(w)."""

    @staticmethod
    def forward(ctx, z, A):
        ctx.A = A
        return torch.as_tensor(A @ z.detach().numpy())

    @staticmethod
    def backward(ctx, gw):
        return torch.as_tensor(ctx.A.conj() @ gw.numpy()), None


def residual_angle_loss_and_grad(flat, x_ndhwc, A_in, mask):
    """The residual-angle loss of the network for one input and its gradient by autograd: r = the complex
    vector of the input's first six channels (zero on masked edges), z = U(x) as a complex vector (zero on
    masked edges), w = A_in z, L = 1 - |<w, r>|^2 / (||w||^2 ||r||^2).  bf16 rounding as in ``forward``.
    Returns (L, dL/dflat)."""
    p = torch.as_tensor(np.asarray(flat, dtype=np.float64)).clone().requires_grad_(True)
    y = forward(unflatten_t(p), x_ndhwc, bf16=True)
    keep = torch.as_tensor(1.0 - np.asarray(mask, dtype=np.float64))
    z = torch.complex(y[..., 0::2], y[..., 1::2]).reshape(-1) * keep
    xb = torch.as_tensor(np.asarray(x_ndhwc, dtype=np.float64)).to(torch.bfloat16).to(torch.float64)
    r = torch.complex(xb[..., 0:6:2], xb[..., 1:6:2]).reshape(-1) * keep
    w = _SparseApply.apply(z, A_in)
    c = torch.sum(torch.conj(w) * r)
    loss = 1.0 - (c.abs() ** 2) / (torch.sum(w.abs() ** 2) * torch.sum(r.abs() ** 2))
    loss.backward()
    return float(loss.detach()), p.grad.numpy()
