"""Training of the learned right preconditioner (3D U-Net) on residual -> correction pairs.

    python -m paper_1705_08849_gb300.train_unet --out weights.bin [--geometries 12] [--steps 3000]

Pairs come from plain solves: for seeded 64^3 geometries of the layered / conductor-block family
(fitgen.layered_blocks) at frequencies drawn in 1-10 GHz, fit_solve (complex64 FGMRES(30) + Jacobi
inside FP64 refinement, tol 1e-7) records the iterate x_k every few refinement steps.  With x* the
converged solution:
    r_k = b - A x_k,   e_k = x* - x_k,   input = r_k / rms(r_k) (+ material channels),
    target = (e_k - D^-1 r_k) / (s rms(r_k))
so the network learns the part of A^-1 r that the Jacobi term D^-1 r misses, in the units of the
scaled complex64 operator (s = fit_coef_scale).  Training minimises ||U(in) - target||^2 / ||target||^2
with Adam on the GPU (the library's own forward and backward kernels).

Checkpoint format: one JSON header line (format, parameter count, training record), then the
parameters as little-endian float32.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FORMAT = "fit-unet-v1"


def save(net, path, record):
    p = net.get_params()
    with open(path, "wb") as fh:
        fh.write((json.dumps({"format": FORMAT, "nparams": int(p.size), "record": record}) + "\n").encode())
        fh.write(p.astype("<f4").tobytes())


def load(net, path):
    with open(path, "rb") as fh:
        head = json.loads(fh.readline().decode())
        if head.get("format") != FORMAT or head.get("nparams") != net.nparams:
            raise ValueError(f"{path}: not a {FORMAT} checkpoint for {net.nparams} parameters")
        p = np.frombuffer(fh.read(), dtype="<f4")
    net.set_params(p)
    return head


def harvest(seeds, n=64, every=6, slots=24, tol=1e-7, fmin=1e9, fmax=10e9, log=print):
    """Returns a list of (in16, target6) device tensors."""
    import torch

    import fitgen as G
    from . import fit
    samples = []
    for s in seeds:
        case = G.layered_blocks(n=n, seed=int(s))
        f = float(np.random.default_rng(int(s)).uniform(fmin, fmax))
        w = 2 * math.pi * f
        t0 = time.time()
        with fit.Grid.from_case(case) as g:
            ne, ncell = g.ne, g.ne // 3
            b = (-1j * w) * torch.from_numpy(G.source_vector(case)).cuda()
            x = torch.zeros_like(b)
            hist = torch.zeros(slots, ne, dtype=torch.complex128, device="cuda")
            st, rep = g.solve([w], b, x, tol, method=fit.FIT_FGMRES, restart=30, precond=fit.FIT_PC_JACOBI,
                              max_iter=200000, max_outer=20000, history=hist.data_ptr(), history_len=slots,
                              history_every=every)
            sc = fit.fit_coef_scale(g.h)
            ns = rep[0]["snapshots"]
            for k in range(ns):
                xk = hist[k]
                ax = torch.empty_like(xk)
                fit.fit_apply(g.h, [w], xk, ax, fit.FIT_C128)
                r = b - ax
                dr = torch.empty_like(r)
                fit.fit_jacobi(g.h, [w], r, dr, fit.FIT_C128)
                rms = float(torch.linalg.vector_norm(r)) / math.sqrt(ne)
                if not rms > 0:
                    continue
                in16 = torch.empty(ncell, 16, dtype=torch.bfloat16, device="cuda")
                t6 = torch.empty(ncell, 6, dtype=torch.float32, device="cuda")
                fit.fit_unet_pack(g.h, r.to(torch.complex64), 1.0 / rms, in16)
                fit.fit_unet_pack_target(g.h, (x - xk) - dr, 1.0 / (sc * rms), t6)
                samples.append((in16, t6))
            torch.cuda.synchronize()
        log(f"harvest seed {s}: f = {f / 1e9:.2f} GHz, {rep[0]['iterations']} iterations, relres "
            f"{rep[0]['relres']:.2e}, {ns} snapshots, {time.time() - t0:.1f} s")
    return samples


def train(net, samples, n, steps, lr=1e-3, lr_min=1e-4, seed=0, val=None, log=print):
    """Adam with a cosine learning rate; with validation pairs the parameters with the lowest
    validation loss seen at the checkpoints (every steps/10) are kept (early stopping)."""
    rng = np.random.default_rng(seed)
    hist = []
    best = (validate(net, val, n), net.get_params()) if val else None
    t0 = time.time()
    for it in range(steps):
        lr_t = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * it / max(1, steps)))
        x, t = samples[int(rng.integers(len(samples)))]
        loss = net.train_step(n, n, n, x, t, lr_t)
        hist.append(loss)
        if (it + 1) % max(1, steps // 10) == 0:
            msg = f"step {it + 1}: train loss (mean of last {steps // 10}) {np.mean(hist[-(steps // 10):]):.4f}"
            if val:
                v = validate(net, val, n)
                msg += f", validation {v:.4f}"
                if v < best[0]:
                    best = (v, net.get_params())
            log(msg + f", {time.time() - t0:.1f} s")
    if best is not None:
        net.set_params(best[1])
    return hist


def validate(net, samples, n):
    import torch
    losses = []
    for x, t in samples:
        losses.append(net.backward(n, n, n, x, t))
    torch.cuda.synchronize()
    return float(np.mean(losses))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--geometries", type=int, default=12)
    ap.add_argument("--validation", type=int, default=2)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1000)
    args = ap.parse_args(argv)
    from . import build, fit
    build.build()
    fit.lib()
    t0 = time.time()
    seeds = list(range(args.seed, args.seed + args.geometries + args.validation))
    samples = harvest(seeds[:args.geometries], n=args.n)
    val = harvest(seeds[args.geometries:], n=args.n) if args.validation else None
    t_h = time.time() - t0
    net = fit.UNet(seed=args.seed)
    v0 = validate(net, val, args.n) if val else None
    t1 = time.time()
    hist = train(net, samples, args.n, args.steps, lr=args.lr, val=val)
    t_t = time.time() - t1
    v1 = validate(net, val, args.n) if val else None
    record = {"geometries": seeds[:args.geometries], "validation_geometries": seeds[args.geometries:], "n": args.n,
              "pairs": len(samples), "validation_pairs": len(val) if val else 0, "steps": args.steps, "lr": args.lr,
              "harvest_s": t_h, "train_s": t_t, "final_train_loss": float(np.mean(hist[-max(1, args.steps // 10):])),
              "validation_loss_initial": v0, "validation_loss_final": v1}
    save(net, args.out, record)
    print(json.dumps(record), flush=True)


if __name__ == "__main__":
    main()
