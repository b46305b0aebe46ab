"""Training and evaluation of the learned right preconditioner (3D U-Net) on residual -> correction pairs.

    python -m paper_1705_08849_gb300.train_unet --out weights.fitw [--geometries 75] [--pairs 20000]
                                                [--epochs 3] [--eval-n 64]

Harvest.  For seeded n^3 geometries of the layered / conductor-block family (fitgen.layered_blocks, the
benchmark workload's material law) at frequencies drawn uniformly in 1-10 GHz, fit_solve (complex64
FGMRES(30) + Jacobi inside FP64 refinement, tol 1e-7) records the iterate x_k after every refinement step
(one FGMRES cycle each).  With x* the converged solution, evenly spaced snapshots become pairs built on
the device by fit_unet_training_pair:
    r_k = b - A x_k,   input = r_k / rms(r_k) (+ the geometry's material channels),
    target = e_k / rms(e_k),   e_k = x* - x_k   (A e_k = r_k)
so the network learns the direction of the error that remains after a residual r_k: the direction that
would finish the solve in one step.  Both sides have unit rms whatever the iterate, so the loss weighs
early and late iterates alike.  Pairs stay on the GPU as one bf16 shard per geometry
([pairs, cells, 12], 24 bytes per cell and pair: 6.3 MB per 64^3 pair, about 126 GB for 20 000 pairs,
inside the 288 GB of HBM), so training never waits on storage.

Training.  Adam (cosine learning rate) with the library's own forward and backward kernels, one pair per
step in a shuffled order, the parameters with the lowest validation loss (held-out geometries) kept.  Two
losses, run as stages in the order ``--loss`` lists them (default: error, then residual):
  - error: the error direction, ||U(in) - e^||^2 / ||e^||^2;
  - residual: the residual angle (fit_unet_train_step_residual): with z = U(in) and w = A z on the pair's
    own grid and frequency, L = 1 - |<w, r^>|^2 / (||w||^2 ||r^||^2), the part of the residual the
    network's direction cannot remove, which is what flexible GMRES gains from it.
A network that gets the error's direction to within 18% in the first norm still leaves a residual that A
amplifies (the high-frequency part of its error), so it does not help the solver by itself; the residual
angle measures the error in the norm the solver sees, and the first stage gives it a start with a
non-zero output (the angle has no gradient at z = 0).

Evaluation (``evaluate``).  FGMRES(30) with one direction from the network per restart cycle (z_1 =
U(v_0), v_0 the cycle's normalised true residual, the input the pairs are made of; the Jacobi direction
D^-1 v_j on every other step) against FGMRES(30) + Jacobi, plain FGMRES(30) and plain BiCGStab on unseen
geometries, each to a 1e-8 true residual: iterations, wall time, status.

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
# the checkpoint the benchmark's learned solve loads (trained by this module, see its record)
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_layered64.fitw")


def save(net, path, record):
    p = net.get_params()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
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


def _freq(seed, fmin, fmax):
    return float(np.random.default_rng(int(seed)).uniform(fmin, fmax))


def harvest(seeds, n=64, pairs_per_geometry=270, slots=2400, tol=1e-7, fmin=1e9, fmax=10e9, log=print):
    """One shard per geometry: dict(seed, f, omega, grid (the open fit.Grid, for the residual loss), base16
    [cells, 16] bf16, pairs [k, cells, 12] bf16) on the GPU."""
    import torch

    import fitgen as G
    from . import fit
    shards = []
    for s in seeds:
        case = G.layered_blocks(n=n, seed=int(s))
        f = _freq(s, fmin, fmax)
        w = 2 * math.pi * f
        t0 = time.time()
        g = fit.Grid.from_case(case)
        if True:  # the grid stays open: the residual loss applies the pair's own operator
            ne, ncell = g.ne, g.ne // 3
            b = (-1j * w) * torch.from_numpy(G.source_vector(case)).cuda()
            x = torch.zeros_like(b)
            hist = torch.zeros(slots, ne, dtype=torch.complex128, device="cuda")
            st, rep = g.solve([w], b, x, tol, method=fit.FIT_FGMRES, restart=30, precond=fit.FIT_PC_JACOBI,
                              max_iter=30 * slots, max_outer=slots, history=hist.data_ptr(), history_len=slots,
                              history_every=1)
            # x* must be the solution: a geometry whose solve did not converge gives no pairs; the last
            # snapshot is x* itself (no error left), so it is not a pair either
            ns = max(0, rep[0]["snapshots"] - 1) if st == fit.FIT_OK else 0
            pick = np.unique(np.linspace(0, ns - 1, min(ns, pairs_per_geometry)).round().astype(int)) if ns else []
            pairs = torch.empty(len(pick), ncell, 12, dtype=torch.bfloat16, device="cuda")
            for q, k in enumerate(pick):
                fit.fit_unet_training_pair(g.h, w, hist[int(k)], x, b, pairs[q])
            del hist
            base16 = torch.empty(ncell, 16, dtype=torch.bfloat16, device="cuda")
            fit.fit_unet_pack(g.h, torch.zeros(ne, dtype=torch.complex64, device="cuda"), 1.0, base16)
            torch.cuda.synchronize()
        if len(pick):
            shards.append(dict(seed=int(s), f=f, omega=w, grid=g, base16=base16, pairs=pairs))
        else:
            g.close()
        log(f"harvest seed {s}: f = {f / 1e9:.2f} GHz, {fit.status_str(st)}, {rep[0]['iterations']} iterations, "
            f"relres {rep[0]['relres']:.2e}, {rep[0]['snapshots']} snapshots -> {len(pick)} pairs, "
            f"{time.time() - t0:.1f} s")
    return shards


def _sample(fit, shard, k, in16, t6):
    fit.fit_unet_pair_sample(in16.shape[0], shard["pairs"][k], shard["base16"], in16, t6)


def train(net, shards, n, epochs, lr=5e-4, lr_min=2e-5, seed=0, val=None, checks=10, loss="residual", log=print):
    """Adam with a cosine learning rate over ``epochs`` passes of the pairs in a shuffled order; with
    validation shards the parameters with the lowest validation loss at the checkpoints are kept."""
    import torch

    from . import fit
    rng = np.random.default_rng(seed)
    index = [(si, k) for si, sh in enumerate(shards) for k in range(sh["pairs"].shape[0])]
    steps = max(1, int(epochs * len(index)))
    ncell = n * n * n
    in16 = torch.empty(ncell, 16, dtype=torch.bfloat16, device="cuda")
    t6 = torch.empty(ncell, 6, dtype=torch.float32, device="cuda")
    hist = []
    best = (validate(net, val, n, loss=loss), net.get_params()) if val else None
    t0 = time.time()
    order = []
    every = max(1, steps // checks)
    for it in range(steps):
        if not order:
            order = list(rng.permutation(len(index)))
        si, k = index[order.pop()]
        lr_t = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * it / steps))
        sh = shards[si]
        _sample(fit, sh, k, in16, t6)
        if loss == "residual":
            hist.append(net.train_step_residual(sh["grid"].h, sh["omega"], in16, lr_t))
        else:
            hist.append(net.train_step(n, n, n, in16, t6, lr_t))
        if (it + 1) % every == 0:
            msg = f"step {it + 1}/{steps}: train loss (mean of last {every}) {np.mean(hist[-every:]):.4f}"
            if val:
                v = validate(net, val, n, loss=loss)
                msg += f", validation {v:.4f}"
                if v < best[0]:
                    best = (v, net.get_params())
            log(msg + f", {time.time() - t0:.1f} s")
    if best is not None:
        net.set_params(best[1])
    return hist, steps


def validate(net, shards, n, per_shard=16, loss="residual"):
    """Mean loss over up to ``per_shard`` evenly spaced pairs of every validation shard."""
    import torch

    from . import fit
    ncell = n * n * n
    in16 = torch.empty(ncell, 16, dtype=torch.bfloat16, device="cuda")
    t6 = torch.empty(ncell, 6, dtype=torch.float32, device="cuda")
    losses = []
    for sh in shards:
        m = sh["pairs"].shape[0]
        for k in np.unique(np.linspace(0, m - 1, min(m, per_shard)).round().astype(int)):
            _sample(fit, sh, int(k), in16, t6)
            if loss == "residual":
                losses.append(net.residual_loss(sh["grid"].h, sh["omega"], in16))
            else:
                losses.append(net.backward(n, n, n, in16, t6))
    torch.cuda.synchronize()
    return float(np.mean(losses))


METHODS = {  # label: (fit_solve method, precision, preconditioner[, pc_every])
    "fgmres30+unet": ("FIT_FGMRES", "FIT_SOLVE_MIXED", "FIT_PC_UNET"),
    "fgmres30+unet/3": ("FIT_FGMRES", "FIT_SOLVE_MIXED", "FIT_PC_UNET", 3),
    "fgmres30+jacobi": ("FIT_FGMRES", "FIT_SOLVE_MIXED", "FIT_PC_JACOBI"),
    "fgmres30": ("FIT_FGMRES", "FIT_SOLVE_MIXED", "FIT_PC_NONE"),
    "bicgstab": ("FIT_BICGSTAB", "FIT_SOLVE_MIXED", "FIT_PC_NONE"),
    "bicgstab+jacobi": ("FIT_BICGSTAB", "FIT_SOLVE_MIXED", "FIT_PC_JACOBI"),
    "cocg+jacobi": ("FIT_COCG", "FIT_SOLVE_MIXED", "FIT_PC_JACOBI"),
}


def evaluate(net, seeds, freqs, n=128, methods=tuple(METHODS), tol=1e-8, max_iter=60000, log=print):
    """Solve b = -j w j on each unseen geometry and frequency with each method; returns a list of records
    (seed, f, method, iterations, seconds, relres, status)."""
    import torch

    import fitgen as G
    from . import fit
    out = []
    for s in seeds:
        case = G.layered_blocks(n=n, seed=int(s))
        with fit.Grid.from_case(case) as g:
            fit.fit_set_preconditioner(g.h, net)
            j = torch.from_numpy(G.source_vector(case)).cuda()
            for f in freqs:
                w = 2 * math.pi * f
                b = (-1j * w) * j
                for mname in methods:
                    spec = METHODS[mname]
                    meth, prec, pc = (getattr(fit, a) for a in spec[:3])
                    every = spec[3] if len(spec) > 3 else 0
                    x = torch.zeros_like(b)
                    torch.cuda.synchronize()
                    t0 = time.time()
                    st, rep = g.solve([w], b, x, tol, method=meth, precision=prec, restart=30, precond=pc,
                                      max_iter=max_iter, max_outer=max_iter, pc_every=every)
                    torch.cuda.synchronize()
                    r = dict(seed=int(s), f=f, method=mname, iterations=rep[0]["iterations"],
                             seconds=time.time() - t0, relres=rep[0]["relres"], status=fit.status_str(rep[0]["status"]))
                    out.append(r)
                    log(json.dumps(r))
    return out


def seed_head(net, seed, scale=0.1):
    """Give the 1x1x1 head (the last 6 x 16 weights and 6 biases of the flat parameters) a small seeded
    He-normal start.  The library starts it at zero, so that an untrained network adds nothing to the
    preconditioner; the residual angle has no gradient at a zero output, so a residual-angle stage
    that starts from scratch starts from here."""
    p = net.get_params()
    rng = np.random.default_rng(seed)
    p[-(6 * 16 + 6):-6] = (scale * np.sqrt(2.0 / 16) * rng.standard_normal(6 * 16)).astype(p.dtype)
    net.set_params(p)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--geometries", type=int, default=75)
    ap.add_argument("--validation", type=int, default=3)
    ap.add_argument("--pairs", type=int, default=20000, help="training pairs in all (spread over the geometries)")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--epochs", type=float, default=3.0)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--loss", default="error,residual",
                    help="comma list of training stages, each 'error' or 'residual', run in order with --epochs "
                         "epochs each (default: the error direction first, then the residual angle)")
    ap.add_argument("--init", default="", help="checkpoint to start from (default: the library's seeded start)")
    ap.add_argument("--eval-n", type=int, default=0, help="grid of an evaluation on unseen geometries (0: none)")
    ap.add_argument("--eval-seeds", default="5000")
    ap.add_argument("--eval-freqs", default="1e9,4e9,7e9,10e9")
    ap.add_argument("--eval-methods", default=",".join(METHODS))
    ap.add_argument("--eval-max-iter", type=int, default=60000)
    args = ap.parse_args(argv)
    from . import build, fit
    build.build()
    fit.lib()
    t0 = time.time()
    seeds = list(range(args.seed, args.seed + args.geometries + args.validation))
    per = max(1, args.pairs // max(1, args.geometries))
    shards = harvest(seeds[:args.geometries], n=args.n, pairs_per_geometry=per)
    val = harvest(seeds[args.geometries:], n=args.n, pairs_per_geometry=32) if args.validation else None
    t_h = time.time() - t0
    npairs = sum(sh["pairs"].shape[0] for sh in shards)
    net = fit.UNet(seed=args.seed)
    if args.init:
        load(net, args.init)
    stages = [v for v in args.loss.split(",") if v]
    if any(v not in ("error", "residual") for v in stages):
        raise SystemExit(f"--loss: unknown stage in {args.loss!r}")
    if stages and stages[0] == "residual" and not args.init:
        seed_head(net, args.seed)
    t1 = time.time()
    record_stages, steps = [], 0
    for loss in stages:
        v0 = validate(net, val, args.n, loss=loss) if val else None
        hist, k = train(net, shards, args.n, args.epochs, lr=args.lr, val=val, loss=loss)
        steps += k
        record_stages.append({"loss": loss, "steps": k, "final_train_loss": float(np.mean(hist[-max(1, k // 10):])),
                              "validation_loss_initial": v0,
                              "validation_loss_final": validate(net, val, args.n, loss=loss) if val else None})
        print(json.dumps(record_stages[-1]), flush=True)
    t_t = time.time() - t1
    record = {"geometries": [seeds[0], seeds[args.geometries - 1]], "validation_geometries": seeds[args.geometries:],
              "n": args.n, "pairs": npairs, "pairs_per_geometry": per, "epochs": args.epochs, "steps": steps,
              "stages": record_stages, "init": os.path.basename(args.init) if args.init else None,
              "lr": args.lr, "harvest_s": t_h, "train_s": t_t}
    save(net, args.out, record)
    print(json.dumps(record), flush=True)
    for sh in shards + (val or []):
        sh["grid"].close()
    del shards, val
    if args.eval_n:
        res = evaluate(net, [int(v) for v in args.eval_seeds.split(",")], [float(v) for v in args.eval_freqs.split(",")],
                       n=args.eval_n, methods=args.eval_methods.split(","), max_iter=args.eval_max_iter)
        print(json.dumps({"evaluation": res}), flush=True)


if __name__ == "__main__":
    main()
