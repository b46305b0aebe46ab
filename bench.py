#!/usr/bin/env python
"""Benchmark of the matrix-free FIT operator apply (and the Krylov solve built on it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fit|reference] [--workload NAME]

One step = one fused operator apply y = A(w) x (the kernel every Krylov iteration repeats) over the
whole synthetic workload, complex64 vectors with FP32 coefficients.  The timed region holds
exactly K steps; between steps the L2 is flushed (a 512 MiB buffer is written, then a second one
is read, so no dirty line of the flush is written back inside a timed apply), and each apply is
timed with CUDA events on the stream it is launched on.  ``value`` = unknowns per second (GDoF/s)
over all ranks; ``e2e`` is the same metric through the C ABI with pinned host buffers, the
host->device copy of x and the device->host copy of y inside the timed region.

``--impl reference`` times the CPU oracle (scipy CSR sparse matrix-vector product of the
explicitly assembled A, single-threaded) on a bounded z-slab sample of the same workload.
Under torchrun (N > 1) every rank runs an independent replica (frequencies / right-hand sides
are independent units: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_DOF_C64 = 28.0   # read x 8 + write y 8 + M_nu, M_eps, M_kappa 3 x 4 (compulsory, per unknown)
# learned preconditioner network: (voxel level, Cin, Cout) of the 3x3x3 convs (level l has (n/2^l)^3
# voxels), the 2x2x2 transposed convs (one tap per output voxel) and the 1x1x1 head
UNET_CONV3 = [(0, 16, 16), (0, 16, 16), (1, 16, 32), (1, 32, 32), (2, 32, 64), (2, 64, 64), (1, 64, 32), (1, 32, 32),
              (0, 32, 16), (0, 16, 16)]
UNET_TCONV = [(1, 64, 32), (0, 32, 16)]
UNET_HEAD = (0, 16, 6)


def unet_flops(nx, ny, nz):
    """Multiply-add flops (2 per MAC) of one network application on an nx x ny x nz grid."""
    v = lambda lvl: (nx >> lvl) * (ny >> lvl) * (nz >> lvl)
    f = sum(2 * 27 * ci * co * v(l) for l, ci, co in UNET_CONV3)
    f += sum(2 * ci * co * v(l) for l, ci, co in UNET_TCONV)
    l, ci, co = UNET_HEAD
    return f + 2 * ci * co * v(l)
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# DRAM traffic per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch forced with
# FIT_APPLY_KERNEL after three warm-up steps of this bench) of the launch shapes the autotuner picks
# on the 128^3 layered workload, one system, complex64; key (warp-specialised, TY, TZ, stages,
# L2 prefetch).  A shape not in the table reports null.
TRAFFIC_LAYERED128_C64 = {(1, 8, -1, 4, 0): 167_289_344, (1, 8, -1, 4, 2): 168_340_480}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of this launch shape on this workload "
                  "(the apply's ncu summary under profiles/), not measured in this run")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def _workload(name):
    import fitgen as G
    if name == "layered128":
        return G.layered_blocks()
    if name == "stripline96":
        return G.stripline()
    if name == "package256":
        return G.package()
    if name == "cavity16":
        return G.cavity()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"fit_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [t.strip() for t in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_oracle_apply(case, target_s=10.0, nz_sample=16, reps_max=1000):
    """Time the oracle's CSR SpMV of the assembled A on the first nz_sample z-planes of the case."""
    from oracle import fit as F
    nx, ny = case["nx"], case["ny"]
    nz = min(nz_sample, case["nz"])
    sl = slice(0, nz)
    me, mk, mn, mask = F.material_diagonals(case["dx"], case["dy"], case["dz"][:nz], case["eps_r"][sl],
                                            case["sigma"][sl], case["inv_mu_r"][sl], case["pec"][sl])
    w = 2 * np.pi * float(case["freqs"][0])
    A = F.system_matrix(w, F.curl(nx, ny, nz), me, mk, mn, mask)
    x = np.random.default_rng(0).standard_normal(A.shape[0]) + 0j
    A @ x
    times = []
    t_start = time.perf_counter()
    while (time.perf_counter() - t_start) < target_s and len(times) < reps_max:
        t0 = time.perf_counter()
        A @ x
        times.append(time.perf_counter() - t0)
    ne = A.shape[0]
    return dict(ne=ne, times=times, sample=f"{nx}x{ny}x{nz} z-slab of {case['name']} ({ne} unknowns), "
                                            f"{len(times)} CSR SpMVs of the assembled A")


def run_reference(args, rank):
    if rank != 0:
        return
    case = _workload(args.workload)
    budget_s = min(60.0, max(5.0, 0.5 * (args.steps + args.warmup)))
    # W warm-up and K timed steps; each step is one SpMV of the bounded sample
    rr = cpu_oracle_apply(case, target_s=budget_s, reps_max=args.steps + args.warmup)
    ne = rr["ne"]
    ts = rr["times"][args.warmup:] or rr["times"]
    total = sum(ts)
    val = ne * len(ts) / total / 1e9
    line = {"impl": "reference", "metric": "GDoF/s operator apply", "value": val, "unit": "GDoF/s",
            "n_gpus": args.gpus, "steps": len(ts), "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": args.workload, "sample": rr["sample"]},
            "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": 1, "kind": "oracle", "sample": rr["sample"]},
            "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def parse_kind(fit, kind):
    """"[method-]precision[+pc]": method fgmres (FGMRES(30), the default), cocg, cocr or bicgstab; precision
    "mixed" (complex64 inner solve inside FP64 refinement) or "c128"; pc jacobi (the Eq. Precond
    diagonal, the default), eps (M_eps^-1: the symmetrised form's change of variable, Eq. e2s), none, or
    unet (the learned preconditioner from the committed checkpoint: one direction from the network per
    restart cycle, at its last step, the Jacobi term on the other steps; FGMRES mixed only) / unet/K (the
    network's direction on the steps j with (j + 1) % K == 0).
    Returns (method, precision, precond, label, pc_every)."""
    base, _, pcname = kind.partition("+")
    pcname = pcname or "jacobi"
    mname, _, pname = base.rpartition("-")
    mname = mname or "fgmres"
    method = {"fgmres": fit.FIT_FGMRES, "cocg": fit.FIT_COCG, "cocr": fit.FIT_COCR, "bicgstab": fit.FIT_BICGSTAB}[mname]
    every = 0
    if pcname.startswith("unet/"):
        pcname, every = "unet", int(pcname[5:])
    pc = {"jacobi": fit.FIT_PC_JACOBI, "eps": fit.FIT_PC_EPS, "none": fit.FIT_PC_NONE, "unet": fit.FIT_PC_UNET}[pcname]
    prec = fit.FIT_SOLVE_MIXED if pname == "mixed" else fit.FIT_SOLVE_C128
    label = {"fgmres": "FGMRES(30)", "cocg": "COCG", "cocr": "COCR", "bicgstab": "BiCGStab"}[mname] + \
        {"jacobi": "+Jacobi", "eps": "+M_eps^-1", "none": "", "unet": "+U-Net+Jacobi"}[pcname] + \
        (f"(network every {every} steps)" if every else "") + \
        (" complex64+FP64 refinement" if pname == "mixed" else " complex128")
    return method, prec, pc, label, every


def valid_kind(kind):
    base, _, pcname = kind.partition("+")
    mname, _, pname = base.rpartition("-")
    unet_k = re.fullmatch(r"unet/([2-9]|[1-9][0-9]+)", pcname) is not None
    ok = pname in ("mixed", "c128") and mname in ("", "fgmres", "cocg", "cocr", "bicgstab") and \
        (pcname in ("", "jacobi", "eps", "none", "unet") or unet_k)
    return ok and (not pcname.startswith("unet") or (mname in ("", "fgmres") and pname == "mixed"))


def time_solves(fit, torch, case, kinds, max_iter, use_graph=1):
    """Seconds per frequency to a 1e-8 true residual, one system at the workload's first frequency,
    for each kind of ``parse_kind``.  Inputs are resident on the device; the timed region is the
    fit_solve call."""
    import fitgen as G
    w = 2 * np.pi * float(case["freqs"][0])
    j = torch.from_numpy(G.source_vector(case)).cuda()
    out = {}
    net = None
    with fit.Grid.from_case(case) as g:
        b = (-1j * w) * j  # b = -j w j (masked source edges carry no current in these workloads)
        for kind in kinds:
            method, prec, pc, label, every = parse_kind(fit, kind)
            extra = {}
            if pc == fit.FIT_PC_UNET and net is None:
                from paper_1705_08849_gb300 import train_unet
                net = fit.UNet(seed=0)
                head = train_unet.load(net, train_unet.DEFAULT_WEIGHTS)
                fit.fit_set_preconditioner(g.h, net)
                extra["weights"] = os.path.relpath(train_unet.DEFAULT_WEIGHTS, ROOT)
                extra["trained_on"] = {k: head["record"].get(k) for k in ("n", "pairs", "geometries", "epochs")}
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, rep = g.solve([w], b, x, 1e-8, precision=prec, method=method, restart=30,
                              precond=pc, max_iter=max_iter, max_outer=max_iter, use_graph=use_graph, pc_every=every)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[kind] = {"s_per_freq": dt, "iterations": rep[0]["iterations"], "outer": rep[0]["outer"],
                         "relres": rep[0]["relres"], "status": fit.status_str(rep[0]["status"]),
                         "method": label, "tol": 1e-8, **extra}
    if net is not None:
        net.close()
    return out


def learned_vs_plain(solves):
    """The solve half of the headline: seconds per frequency of the learned, mixed-precision FGMRES(30)
    against the plain complex128 solves and the same mixed FGMRES without the network, with every
    solve's status (a solve that did not reach 1e-8 is reported, not compared)."""
    def leg(k):
        r = solves.get(k)
        return None if r is None else {"kind": k, "s": r["s_per_freq"], "status": r["status"],
                                       "iterations": r["iterations"]}
    out = {"learned": leg("mixed+unet"), "plain_fp64": [v for v in (leg("c128"), leg("cocg-c128")) if v],
           "without_network": leg("mixed"), "fastest_mixed": leg("cocg-mixed")}
    ok = [r for r in solves.values() if r["status"] == "FIT_OK"]
    if ok:
        best = min(ok, key=lambda r: r["s_per_freq"])
        out["fastest_converged"] = {"method": best["method"], "s": best["s_per_freq"]}
    return out


def time_sweep(fit, torch, case, nfreq, kind, max_iter, band=None, seq_kind=None, budget_gb=0.0, restart=30,
               seq_max_iter=None):
    """A wide-band sweep: nfreq of the workload's frequencies (evenly picked, or evenly spaced over
    ``band``), b_f = -j w_f j, solved to a 1e-8 true residual, once as one batch (one graph launch per
    admitted batch: with an HBM budget, fit_solve halves the batch until its workspace fits) with
    ``kind``, and once as nfreq sequential single-frequency solves with ``seq_kind`` (default: the same
    kind).  Wall time of fit_solve; per-frequency status, iterations and true relative residual."""
    import fitgen as G
    if band:  # nfreq frequencies evenly spaced over [fmin, fmax]
        sel = np.linspace(band[0], band[1], max(1, nfreq))
    else:
        fr = np.asarray(case["freqs"], dtype=np.float64)
        sel = fr[np.unique(np.linspace(0, len(fr) - 1, max(1, min(nfreq, len(fr)))).round().astype(int))]
    ws = 2 * np.pi * sel
    seq_kind = seq_kind or kind
    j = torch.from_numpy(G.source_vector(case)).cuda()
    ne = j.numel()
    b = torch.stack([(-1j * w) * j for w in ws]).reshape(-1)

    def opts_of(k, cap):
        method, prec, pc, _, every = parse_kind(fit, k)
        return dict(precision=prec, method=method, restart=restart, precond=pc, max_iter=cap, max_outer=cap,
                    pc_every=every), pc

    out = {"frequencies_hz": sel.tolist(), "method": kind, "sequential_method": seq_kind, "restart": restart,
           "max_iter": max_iter}
    net = None
    with fit.Grid.from_case(case) as g:
        if budget_gb > 0:
            fit.fit_set_hbm_budget(g.h, int(budget_gb * 1e9))
            out["hbm_budget_gb"] = budget_gb
        for k in {kind, seq_kind}:
            if parse_kind(fit, k)[2] == fit.FIT_PC_UNET and net is None:
                from paper_1705_08849_gb300 import train_unet
                net = fit.UNet(seed=0)
                train_unet.load(net, train_unet.DEFAULT_WEIGHTS)
                fit.fit_set_preconditioner(g.h, net)
        o, _ = opts_of(kind, max_iter)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, rep = g.solve(ws, b, x, 1e-8, batch=0, **o)
        torch.cuda.synchronize()
        # systems solved in the same admitted batch share their batch's wall time
        groups = sorted({round(r["seconds"], 6) for r in rep})
        out["batched"] = {"s": time.perf_counter() - t0, "statuses": [fit.status_str(r["status"]) for r in rep],
                          "iterations": [r["iterations"] for r in rep], "relres": [r["relres"] for r in rep],
                          "admitted_batches": len(groups), "converged": sum(r["status"] == 0 for r in rep)}
        del x
        o, _ = opts_of(seq_kind, seq_max_iter or max_iter)
        seq_t, seq_rep = 0.0, []
        for f, w in enumerate(ws):
            xf = torch.zeros(ne, dtype=b.dtype, device="cuda")
            bf = b[f * ne:(f + 1) * ne].contiguous()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, rep1 = g.solve([w], bf, xf, 1e-8, **o)
            torch.cuda.synchronize()
            seq_t += time.perf_counter() - t0
            seq_rep.append(rep1[0])
        out["sequential"] = {"s": seq_t, "statuses": [fit.status_str(r["status"]) for r in seq_rep],
                             "iterations": [r["iterations"] for r in seq_rep], "relres": [r["relres"] for r in seq_rep],
                             "converged": sum(r["status"] == 0 for r in seq_rep)}
    if net is not None:
        net.close()
    return out


def port_columns(case, nport, seed=77, height=8, margin=16):
    """nport seeded z-edge columns (ports from the ground wall z = 0 up ``height`` edges) at distinct
    (i, j) positions at least ``margin`` cells from the side walls, orientation +z."""
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    rng = np.random.default_rng(seed)
    picks = set()
    while len(picks) < nport:
        picks.add((int(rng.integers(margin, nx - margin)), int(rng.integers(margin, ny - margin))))
    top = min(nz, height)
    return [([3 * (i + nx * (j + ny * k)) + 2 for k in range(top)], [1.0] * top) for i, j in sorted(picks)]


def time_ports(fit, torch, case, nport, nfreq, kind, max_iter, batch):
    """Multi-port Z/S extraction: nport z-edge column ports, each excited alone with 1 A at nfreq of
    the workload's frequencies, every system solved to 1e-8 (Jacobi preconditioner) inside one
    fit_z_parameters call (right-hand sides, solves, probe sums and Z all on the device); wall time
    of that call, then S = (Z - 50)(Z + 50)^-1 per frequency."""
    fr = np.asarray(case["freqs"], dtype=np.float64)
    sel = fr[np.unique(np.linspace(0, len(fr) - 1, max(1, min(nfreq, len(fr)))).round().astype(int))]
    ws = 2 * np.pi * sel
    method, prec, pc, _, _ = parse_kind(fit, kind)
    ports = port_columns(case, nport)
    with fit.Grid.from_case(case) as g:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, Z, rep = fit.fit_z_parameters(g.h, ws, ports, 1e-8, method=method, precision=prec, restart=30,
                                          precond=pc, max_iter=max_iter, max_outer=max_iter, batch=batch)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    zmax = float(np.abs(Z).max())
    recip = float(max(np.abs(Z[f] - Z[f].T).max() for f in range(len(ws))) / zmax) if zmax > 0 else 0.0
    smax = float(max(np.linalg.norm(fit.fit_z_to_s(Z[f]), 2) for f in range(len(ws))))
    nsys = len(ports) * len(ws)
    return {"metric": "Z-parameter extraction s per (port, frequency) system to 1e-8", "unit": "s",
            "value": dt / nsys, "systems": nsys, "ports": len(ports), "edges_per_port": len(ports[0][0]),
            "frequencies_hz": sel.tolist(), "method": kind, "batch": batch, "s_total": dt,
            "status": fit.status_str(st), "iterations": [r["iterations"] for r in rep],
            "relres_max": float(max(r["relres"] for r in rep)), "reciprocity_rel": recip, "max_norm_S": smax,
            "Z_ohm_first_freq": [[[float(z.real), float(z.imag)] for z in row] for row in Z[0]]}


def time_unet(fit, torch, case, steps, warmup):
    """One application of the learned preconditioner's network (bf16 NDHWC input of 16 channels ->
    6 FP32 channels) on the workload's grid, CUDA-event timed after warm-up; flops from the layer
    table, against the BF16 tensor peak."""
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    net = fit.UNet(seed=1)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    xin = torch.randn(nz, ny, nx, 16, device="cuda", generator=gen).to(torch.bfloat16)
    yout = torch.empty(nz, ny, nx, 6, device="cuda", dtype=torch.float32)
    for _ in range(max(3, warmup)):
        net.forward(nx, ny, nz, xin, yout)
    torch.cuda.synchronize()
    n = max(5, min(steps, 200))
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in evs:
        a.record(stream)
        net.forward(nx, ny, nz, xin, yout)
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.median([a.elapsed_time(b) for a, b in evs])
    flops = unet_flops(nx, ny, nz)
    peaks, kind = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    net.close()
    return {"metric": "learned preconditioner application", "unit": "ms", "value": ms, "higher_is_better": False,
            "workload": case["name"], "grid": [nx, ny, nz], "steps": n, "gflop": flops / 1e9,
            "roofline": {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (ms * 1e-3) / 1e12 / peak, "peak_kind": f"{kind} bf16 burst"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fit", choices=["fit", "reference"])
    ap.add_argument("--workload", default="layered128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=1, help="systems (frequencies) per apply in the apply mode")
    ap.add_argument("--nfreq", type=int, default=8, help="frequencies of the sweep mode")
    ap.add_argument("--band", default="", help="sweep mode: fmin,fmax in Hz (default: the workload's own frequencies)")
    ap.add_argument("--ports", type=int, default=4, help="ports of the ports mode (z-edge columns)")
    ap.add_argument("--mode", default="apply", choices=["apply", "solve", "unet", "sweep", "ports"],
                    help="apply: the operator-apply metric (default); solve: only the solve measurement")
    ap.add_argument("--solve", default="cocg-mixed,mixed,mixed+unet,cocg-c128,c128",
                    help="comma list of solves to time, each [method-]precision[+pc] with method fgmres (default), "
                         "cocg, cocr or bicgstab, precision mixed or c128, pc jacobi (default), eps, none or unet "
                         "(FGMRES mixed: the committed network's direction once per restart cycle; unet/K: on the "
                         "steps j with (j + 1) %% K == 0); none for no solve.  The default times the fastest mixed solve, "
                         "FGMRES(30) mixed without and with the learned network, and the plain complex128 COCG "
                         "and FGMRES(30)")
    ap.add_argument("--max-iter", type=int, default=80000, help="Krylov iteration cap of the timed solves")
    ap.add_argument("--hbm-budget-gb", type=float, default=0.0, help="sweep mode: the handle's HBM budget (0: none)")
    ap.add_argument("--restart", type=int, default=30, help="FGMRES restart length of the sweep mode")
    ap.add_argument("--seq-max-iter", type=int, default=0, help="sweep mode: iteration cap of the sequential solves "
                    "(0: --max-iter)")
    ap.add_argument("--e2e-chunks", type=int, default=1, help="end-to-end leg: each host<->device copy is split into "
                    "this many pieces on as many streams (several copy engines per direction)")
    ap.add_argument("--graph", type=int, default=1, help="1: the solve runs as one CUDA graph; 0: host-driven loop "
                    "(for per-kernel profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    from paper_1705_08849_gb300 import build, fit
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    fit.lib()

    case = _workload(args.workload)
    kinds = [k for k in args.solve.split(",") if valid_kind(k)]
    if args.mode == "sweep":
        if rank == 0:
            kind = kinds[0] if kinds else "cocg-mixed"
            seq = kinds[1] if len(kinds) > 1 else None
            print(json.dumps({"metric": "wide-band sweep s to 1e-8", "unit": "s", "workload": args.workload,
                              "sweep": time_sweep(fit, torch, case, args.nfreq, kind, args.max_iter,
                                                  [float(v) for v in args.band.split(",")] if args.band else None,
                                                  seq_kind=seq, budget_gb=args.hbm_budget_gb, restart=args.restart,
                                                  seq_max_iter=args.seq_max_iter or None)}),
                  flush=True)
        return
    if args.mode == "ports":
        if rank == 0:
            kind = "cocg-mixed" if "cocg-mixed" in kinds else (kinds[0] if kinds else "cocg-mixed")
            print(json.dumps({"workload": args.workload, **time_ports(fit, torch, case, args.ports, args.nfreq, kind,
                                                                     args.max_iter, max(1, args.batch))}),
                  flush=True)
        return
    if args.mode == "unet":
        if rank == 0:
            print(json.dumps(time_unet(fit, torch, case, args.steps, args.warmup)), flush=True)
        return
    if args.mode == "solve":
        res = time_solves(fit, torch, case, kinds, args.max_iter, args.graph)
        if rank == 0:
            print(json.dumps({"metric": "solve s/freq to 1e-8", "unit": "s", "workload": args.workload,
                              "solves": res}), flush=True)
        return
    ne = 3 * case["nx"] * case["ny"] * case["nz"]
    B = max(1, args.batch)
    w0 = 2 * np.pi * float(case["freqs"][0])
    w = [w0 * (1.0 + 0.5 * b / B) for b in range(B)]  # B frequencies from f0 to 1.5 f0
    g = fit.Grid.from_case(case)
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234 + rank)
    x = torch.randn(B * ne, dtype=torch.complex64, device="cuda", generator=gen)
    y = torch.empty_like(x)
    flush_w = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(128 << 20, dtype=torch.float32, device="cuda")

    def flush():
        flush_w.zero_()
        flush_r.sum()

    # the timed loop calls the C ABI directly with its arguments marshalled once, so that nothing
    # but the launch itself runs on the host between a step's two events
    import ctypes as ct
    L = fit.lib()
    om_arr = (ct.c_double * B)(*w)
    apply_args = (g.h, B, om_arr, ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()), fit.FIT_C64,
                  ct.c_void_p(stream.cuda_stream))

    def apply_once():
        st = L.fit_apply(*apply_args)
        if st != fit.FIT_OK:
            raise fit.FitError(st, "fit_apply: " + L.fit_last_error().decode())

    for _ in range(args.warmup):
        flush()
        apply_once()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # The device is held by a short spin kernel while the host enqueues the timed steps, so that the
    # GPU never waits on the host inside a step (a host hiccup would otherwise land between a
    # step's start event and its apply and be timed as apply time).
    spin_s = min(0.05, 0.004 + 2e-4 * args.steps)
    with ClockSampler(local) as clk:
        torch.cuda._sleep(int(spin_s * 2.0e9))
        for k in range(args.steps):
            flush()
            evs[k][0].record(stream)
            apply_once()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(times_ms)
    srt = sorted(times_ms)
    step_stats = {"min_ms": srt[0], "median_ms": statistics.median(times_ms), "mean_ms": total_ms / len(times_ms),
                  "p90_ms": srt[min(len(srt) - 1, int(0.9 * len(srt)))], "max_ms": srt[-1],
                  "max_step": int(np.argmax(times_ms)), "host_prequeue_spin_ms": 1e3 * spin_s}
    from paper_1705_08849_gb300 import replicas
    total_ms = replicas.max_over_ranks(total_ms)  # the job's time is the slowest replica's
    ms_step = total_ms / args.steps
    value = world * B * ne * args.steps / (total_ms * 1e-3) / 1e9

    # End to end through the C ABI with pinned host buffers: every step copies its input host -> device,
    # applies, and copies the result device -> host.  Steps are pipelined over three streams (copy in,
    # apply, copy out) with two device buffers each, so that the input copy of step k+1 and the output
    # copy of step k-1 overlap the apply of step k; the timed region runs from before the first input
    # copy to after the last output copy.
    xh = x.cpu().pin_memory()
    yh = [torch.empty_like(xh).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    yd = [torch.empty_like(x) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    nch = max(1, args.e2e_chunks)
    c_in = [torch.cuda.Stream() for _ in range(nch)]   # copy-in pieces, one stream each
    c_out = [torch.cuda.Stream() for _ in range(nch)]  # copy-out pieces
    bounds = [(B * ne * q) // nch for q in range(nch + 1)]
    ev_ci = [torch.cuda.Event() for _ in range(nch)]
    ev_co = [torch.cuda.Event() for _ in range(nch)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_ap = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e2e_args = [(g.h, B, om_arr, ct.c_void_p(xd[q].data_ptr()), ct.c_void_p(yd[q].data_ptr()), fit.FIT_C64,
                 ct.c_void_p(stream.cuda_stream)) for q in range(2)]

    def e2e_steps(n):
        for k in range(n):
            q = k % 2
            if k >= 2:
                s_in.wait_event(ev_ap[q])    # the apply of step k-2 has read xd[q]
            for c in range(nch):             # the input copy in pieces on parallel streams
                c_in[c].wait_stream(s_in)
                with torch.cuda.stream(c_in[c]):
                    xd[q][bounds[c]:bounds[c + 1]].copy_(xh[bounds[c]:bounds[c + 1]], non_blocking=True)
                ev_ci[c].record(c_in[c])
                s_in.wait_event(ev_ci[c])
            ev_in[q].record(s_in)
            stream.wait_event(ev_in[q])
            if k >= 2:
                stream.wait_event(ev_out[q])  # the output copy of step k-2 has read yd[q]
            st = L.fit_apply(*e2e_args[q])
            if st != fit.FIT_OK:
                raise fit.FitError(st, "fit_apply: " + L.fit_last_error().decode())
            ev_ap[q].record(stream)
            s_out.wait_event(ev_ap[q])
            for c in range(nch):
                c_out[c].wait_stream(s_out)
                with torch.cuda.stream(c_out[c]):
                    yh[q][bounds[c]:bounds[c + 1]].copy_(yd[q][bounds[c]:bounds[c + 1]], non_blocking=True)
                ev_co[c].record(c_out[c])
                s_out.wait_event(ev_co[c])
            ev_out[q].record(s_out)

    k_e2e = max(10, min(args.steps, 200))
    e2e_steps(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s_in):
        torch.cuda._sleep(int(min(0.05, 0.004 + 1e-3 * k_e2e) * 2.0e9))
    e0.record(s_in)
    e2e_steps(k_e2e)
    e1.record(s_out)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / k_e2e
    e2e_val = world * B * ne / (e2e_ms * 1e-3) / 1e9

    tuned = fit.fit_apply_tuned(g.h, fit.FIT_C64, B)
    peaks, kind = _peaks()
    # per unknown: x and y move once per system, the coefficients once per launch (shared by B systems)
    bytes_per_dof = 16.0 + (BYTES_PER_DOF_C64 - 16.0) / B
    achieved = bytes_per_dof * B * ne / (ms_step * 1e-3) / 1e9
    sig = (tuned["ws"], tuned["ty"], tuned["tz"], tuned["stages"], tuned["pf"])
    traffic = TRAFFIC_LAYERED128_C64.get(sig) if (args.workload == "layered128" and B == 1 and tuned["choice"] >= 0) else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_kind": kind, "traffic": traffic, "traffic_unit": "B per launch",
            "traffic_source": TRAFFIC_SOURCE if traffic is not None else "no capture of this launch shape",
            "bytes_per_dof": bytes_per_dof,
            "kernel": (("ws_apply_kernel" if tuned["ws"] else "fused_apply_kernel") if tuned["choice"] >= 0
                       else "apply_generic_kernel")}

    line = {"metric": "GDoF/s operator apply", "value": value, "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": args.workload, "grid": [case["nx"], case["ny"], case["nz"]], "unknowns": ne,
                       "batch": B, "omega_hz": float(case["freqs"][0]), "l2": "flushed between timed applies (512 MiB write "
                       "then 512 MiB read)", "parallelism": f"replicas{world}",
                       "autotuned_tile": [tuned["tx"], tuned["ty"], tuned["tz"]], "ring_stages": tuned["stages"],
                       "l2_prefetch_planes": tuned["pf"],
                       "kernel_choice": tuned["choice"]},
            "roofline": roof, "clocks": clk.summary(), "step_stats": step_stats,
            "e2e": {"value": e2e_val, "unit": "GDoF/s", "h2d_bytes_per_step": 8 * B * ne, "d2h_bytes_per_step": 8 * B * ne,
                    "copy_pieces": nch, "pipelined": "copy in / apply / copy out on separate streams, 2 buffers"},
            "gpu_launches": args.steps}

    g.close()
    if kinds and world == 1:  # the solve leg runs at N = 1 only: under torchrun it would hold every GPU
        line["solve"] = time_solves(fit, torch, case, kinds, args.max_iter)
        line["learned_vs_plain"] = learned_vs_plain(line["solve"])
    if rank == 0 and not args.no_cpu_baseline:
        r = cpu_oracle_apply(case, target_s=10.0)
        cv = r["ne"] * len(r["times"]) / sum(r["times"]) / 1e9
        line["cpu_baseline"] = {"value": cv, "unit": "GDoF/s", "cores": 1, "kind": "oracle", "sample": r["sample"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
