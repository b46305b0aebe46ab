"""Thin Python binding of the C ABI in include/fit.h (ctypes; argument marshalling only).

Every numerical step runs in the CUDA library ``libfitgb300.so``; this module only checks
argument shapes/dtypes, passes pointers and raises on error statuses.  Vectors are torch CUDA
tensors (complex64 for FIT_C64, complex128 for FIT_C128) in the cell-by-cell ordering of the
paper's Eq. e12Nxyz; material inputs are numpy arrays.  If the library is missing this module
raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

FIT_OK, FIT_NOT_CONVERGED, FIT_BREAKDOWN = 0, 1, 2
FIT_EINVAL, FIT_ENOMEM, FIT_ECUDA, FIT_ETIMEOUT, FIT_EBUDGET, FIT_ENAN = -1, -2, -3, -4, -5, -6
FIT_C64, FIT_C128 = 0, 1
FIT_BC_PEC_ALL = 0x3F
FIT_BICGSTAB, FIT_FGMRES, FIT_COCG, FIT_COCR = 0, 1, 2, 3
FIT_SOLVE_C128, FIT_SOLVE_MIXED = 0, 1
FIT_PC_NONE, FIT_PC_JACOBI, FIT_PC_UNET, FIT_PC_EPS = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfitgb300.so")
_lib = None


class FitError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_str(status)}: {msg}")
        self.status = status


class fit_solve_opts(ct.Structure):
    _fields_ = [("method", ct.c_int), ("restart", ct.c_int), ("precision", ct.c_int), ("max_iter", ct.c_int),
                ("max_outer", ct.c_int), ("inner_tol", ct.c_double), ("batch", ct.c_int),
                ("use_graph", ct.c_int), ("precond", ct.c_int), ("stream", ct.c_void_p),
                ("history", ct.c_void_p), ("history_len", ct.c_int), ("history_every", ct.c_int),
                ("pc_every", ct.c_int)]


class fit_solve_report(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iterations", ct.c_int), ("outer", ct.c_int), ("relres", ct.c_double),
                ("seconds", ct.c_double), ("snapshots", ct.c_int)]


def lib():
    """Load libfitgb300.so (built by ``paper_1705_08849_gb300.build.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1705_08849_gb300.build.build() first")
        L = ct.CDLL(LIB_PATH)
        vp, i, d, u = ct.c_void_p, ct.c_int, ct.c_double, ct.c_uint
        pd = ct.POINTER(ct.c_double)
        pf = ct.POINTER(ct.c_float)
        pu8 = ct.POINTER(ct.c_ubyte)
        L.fit_grid_create.argtypes = [i, i, i, pd, pd, pd, u, ct.POINTER(vp)]
        L.fit_set_materials.argtypes = [vp, pf, pf, pf, pu8]
        L.fit_set_material_matrices.argtypes = [vp, pd, pd, pd, pu8]
        L.fit_apply.argtypes = [vp, i, pd, vp, vp, i, vp]
        L.fit_apply_sym.argtypes = [vp, i, pd, vp, vp, i, vp]
        L.fit_apply_sym.restype = ct.c_int
        L.fit_solve.argtypes = [vp, i, pd, vp, vp, d, ct.POINTER(fit_solve_opts), ct.POINTER(fit_solve_report)]
        L.fit_solve_opts_default.argtypes = [ct.POINTER(fit_solve_opts)]
        L.fit_solve_opts_default.restype = None
        L.fit_set_hbm_budget.argtypes = [vp, ct.c_size_t]
        L.fit_grid_info.argtypes = [vp, ct.POINTER(ct.c_longlong)]
        L.fit_grid_destroy.argtypes = [vp]
        L.fit_grid_destroy.restype = None
        L.fit_status_str.argtypes = [i]
        L.fit_status_str.restype = ct.c_char_p
        L.fit_apply_variant_count.argtypes = [i]
        L.fit_apply_variant_count.restype = ct.c_int
        L.fit_apply_tuned.argtypes = [vp, i, i, ct.POINTER(ct.c_int)]
        L.fit_apply_tuned.restype = ct.c_int
        L.fit_apply_noalloc.argtypes = [vp, i, pd, vp, vp, i, vp]
        L.fit_apply_noalloc.restype = ct.c_int
        L.fit_jacobi.argtypes = [vp, i, pd, vp, vp, i, vp]
        L.fit_jacobi.restype = ct.c_int
        L.fit_coef_scale.argtypes = [vp, ct.POINTER(ct.c_double)]
        L.fit_coef_scale.restype = ct.c_int
        pfl = ct.POINTER(ct.c_float)
        L.fit_unet_create.argtypes = [ct.c_ulonglong, ct.POINTER(vp)]
        L.fit_unet_destroy.argtypes = [vp]
        L.fit_unet_destroy.restype = None
        L.fit_unet_param_count.argtypes = []
        L.fit_unet_param_count.restype = ct.c_longlong
        L.fit_unet_get_params.argtypes = [vp, pfl, ct.c_longlong]
        L.fit_unet_set_params.argtypes = [vp, pfl, ct.c_longlong]
        L.fit_unet_forward.argtypes = [vp, i, i, i, vp, vp, vp]
        L.fit_unet_backward.argtypes = [vp, i, i, i, vp, vp, vp, ct.POINTER(ct.c_double), vp]
        L.fit_unet_train_step.argtypes = [vp, i, i, i, vp, vp, ct.c_float, ct.POINTER(ct.c_double), vp]
        L.fit_unet_pack.argtypes = [vp, vp, d, vp, vp]
        L.fit_unet_pack_target.argtypes = [vp, vp, d, vp, vp]
        L.fit_unet_unpack.argtypes = [vp, vp, d, vp, vp]
        L.fit_set_preconditioner.argtypes = [vp, i, vp]
        for name in ("fit_unet_create", "fit_unet_get_params", "fit_unet_set_params", "fit_unet_forward",
                     "fit_unet_backward", "fit_unet_train_step", "fit_unet_pack", "fit_unet_pack_target",
                     "fit_unet_unpack", "fit_set_preconditioner"):
            getattr(L, name).restype = ct.c_int
        L.fit_tuning_record.argtypes = [ct.c_char_p, ct.c_char_p, i, i, i, i, i, i, i]
        L.fit_tuning_record.restype = ct.c_int
        L.fit_tuning_lookup.argtypes = [ct.c_char_p, ct.c_char_p, i, i, i, i, i, i, ct.POINTER(ct.c_int)]
        L.fit_tuning_lookup.restype = ct.c_int
        pll = ct.POINTER(ct.c_longlong)
        pi = ct.POINTER(ct.c_int)
        L.fit_port_rhs.argtypes = [vp, i, pd, i, pll, pd, d, vp, vp]
        L.fit_probe_voltages.argtypes = [vp, i, vp, i, pi, pll, pd, pd, vp]
        L.fit_z_to_s.argtypes = [i, pd, d, pd]
        L.fit_z_parameters.argtypes = [vp, i, pd, i, pi, pll, pd, d, d, ct.POINTER(fit_solve_opts),
                                       pd, ct.POINTER(fit_solve_report)]
        for name in ("fit_port_rhs", "fit_probe_voltages", "fit_z_to_s", "fit_z_parameters"):
            getattr(L, name).restype = ct.c_int
        ll = ct.c_longlong
        L.fit_unet_conv3.argtypes = [i, i, i, i, i, vp, vp, vp, i, vp, vp]
        L.fit_unet_conv3_dgrad.argtypes = [i, i, i, i, i, vp, vp, vp, vp]
        L.fit_unet_conv3_wgrad.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp]
        L.fit_unet_tconv.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp]
        L.fit_unet_tconv_backward.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp, vp, vp]
        L.fit_unet_head.argtypes = [ll, vp, vp, vp, vp, vp]
        L.fit_unet_head_backward.argtypes = [ll, vp, vp, vp, vp, vp, vp, vp]
        for name in ("fit_unet_conv3", "fit_unet_conv3_dgrad", "fit_unet_conv3_wgrad", "fit_unet_tconv",
                     "fit_unet_tconv_backward", "fit_unet_head", "fit_unet_head_backward"):
            getattr(L, name).restype = ct.c_int
        L.fit_unet_training_pair.argtypes = [vp, d, vp, vp, vp, vp, ct.POINTER(ct.c_double), vp]
        L.fit_unet_training_pair.restype = ct.c_int
        L.fit_unet_pair_sample.argtypes = [ll, vp, vp, vp, vp, vp]
        L.fit_unet_pair_sample.restype = ct.c_int
        L.fit_unet_train_step_residual.argtypes = [vp, vp, d, vp, ct.c_float, ct.POINTER(ct.c_double), vp]
        L.fit_unet_train_step_residual.restype = ct.c_int
        L.fit_unet_residual_loss.argtypes = [vp, vp, d, vp, ct.POINTER(ct.c_double), vp]
        L.fit_unet_residual_loss.restype = ct.c_int
        L.fit_set_abort.argtypes = [vp, i]
        L.fit_set_abort.restype = ct.c_int
        L.fit_sync.argtypes = [vp, vp]
        L.fit_sync.restype = ct.c_int
        L.fit_last_error.argtypes = []
        L.fit_last_error.restype = ct.c_char_p
        for name in ("fit_grid_create", "fit_set_materials", "fit_set_material_matrices", "fit_apply", "fit_solve",
                     "fit_set_hbm_budget", "fit_grid_info"):
            getattr(L, name).restype = ct.c_int
        _lib = L
    return _lib


def status_str(s):
    try:
        return lib().fit_status_str(int(s)).decode()
    except Exception:
        return str(s)


def _check(st, what):
    if st < 0:
        raise FitError(st, f"{what}: {lib().fit_last_error().decode()}")
    return st


def _dptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ct.POINTER(np.ctypeslib.as_ctypes_type(dtype)))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)


def fit_grid_create(nx, ny, nz, dx, dy, dz, bc_flags=FIT_BC_PEC_ALL):
    """Create a grid handle on the current CUDA device; returns an opaque ctypes pointer."""
    h = ct.c_void_p()
    dx, pdx = _dptr(dx, np.float64)
    dy, pdy = _dptr(dy, np.float64)
    dz, pdz = _dptr(dz, np.float64)
    if len(dx) != nx or len(dy) != ny or len(dz) != nz:
        raise ValueError("cell-width arrays must have nx, ny, nz entries")
    _check(lib().fit_grid_create(nx, ny, nz, pdx, pdy, pdz, bc_flags, ct.byref(h)), "fit_grid_create")
    return h


def fit_set_materials(g, eps_r, sigma, inv_mu_r, pec=None):
    e, pe = _dptr(np.asarray(eps_r).ravel(), np.float32)
    s, ps = _dptr(np.asarray(sigma).ravel(), np.float32)
    m, pm = _dptr(np.asarray(inv_mu_r).ravel(), np.float32)
    if pec is not None:
        p, pp = _dptr(np.asarray(pec).ravel(), np.uint8)
    else:
        pp = None
    _check(lib().fit_set_materials(g, pe, ps, pm, pp), "fit_set_materials")


def fit_set_material_matrices(g, m_eps, m_kappa, m_nu, edge_mask=None):
    a, pa = _dptr(m_eps, np.float64)
    b, pb = _dptr(m_kappa, np.float64)
    c, pc = _dptr(m_nu, np.float64)
    if edge_mask is not None:
        d, pdm = _dptr(edge_mask, np.uint8)
    else:
        pdm = None
    _check(lib().fit_set_material_matrices(g, pa, pb, pc, pdm), "fit_set_material_matrices")


def grid_info(g):
    out = (ct.c_longlong * 6)()
    _check(lib().fit_grid_info(g, out), "fit_grid_info")
    return dict(nx=out[0], ny=out[1], nz=out[2], ne=out[3], bytes_held=out[4], budget=out[5])


def _check_vec(t, ne, nbatch, prec, name):
    import torch
    want = torch.complex64 if prec == FIT_C64 else torch.complex128
    if not (t.is_cuda and t.dtype == want and t.is_contiguous() and t.numel() == ne * nbatch):
        raise ValueError(f"{name} must be a contiguous CUDA {want} tensor of {nbatch} x {ne} values")


def fit_apply(g, omega, x, y, prec=FIT_C64, stream=None):
    """y_b = A(omega_b) x_b for the batch of len(omega) vectors (torch CUDA tensors)."""
    om, pom = _dptr(np.atleast_1d(np.asarray(omega, dtype=np.float64)), np.float64)
    ne = grid_info(g)["ne"]
    _check_vec(x, ne, len(om), prec, "x")
    _check_vec(y, ne, len(om), prec, "y")
    _check(lib().fit_apply(g, len(om), pom, ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()), prec,
                           _stream_ptr(stream)), "fit_apply")


def fit_apply_sym(g, omega, x, y, prec=FIT_C64, stream=None):
    """y'_b = A_s(omega_b) x'_b, the symmetrised operator M_eps^-1/2 A M_eps^-1/2 of Eq. e2s."""
    om, pom = _dptr(np.atleast_1d(np.asarray(omega, dtype=np.float64)), np.float64)
    ne = grid_info(g)["ne"]
    _check_vec(x, ne, len(om), prec, "x")
    _check_vec(y, ne, len(om), prec, "y")
    _check(lib().fit_apply_sym(g, len(om), pom, _ptr(x), _ptr(y), prec, _stream_ptr(stream)), "fit_apply_sym")


def fit_apply_noalloc(g, omega, x, y, prec=FIT_C64, stream=None):
    """fit_apply without device allocations (static frequency scratch of 4096 systems)."""
    om, pom = _dptr(np.atleast_1d(np.asarray(omega, dtype=np.float64)), np.float64)
    ne = grid_info(g)["ne"]
    _check_vec(x, ne, len(om), prec, "x")
    _check_vec(y, ne, len(om), prec, "y")
    _check(lib().fit_apply_noalloc(g, len(om), pom, ct.c_void_p(x.data_ptr()), ct.c_void_p(y.data_ptr()), prec,
                                   _stream_ptr(stream)), "fit_apply_noalloc")


def fit_solve_opts_default():
    o = fit_solve_opts()
    lib().fit_solve_opts_default(ct.byref(o))
    return o


def fit_solve(g, omega, rhs, x, tol, opts=None, **kw):
    """Solve A(omega_f) x_f = rhs_f (complex128 CUDA tensors); returns (status, list of report dicts).
    Keyword arguments override fields of the options struct."""
    om, pom = _dptr(np.atleast_1d(np.asarray(omega, dtype=np.float64)), np.float64)
    nf = len(om)
    ne = grid_info(g)["ne"]
    _check_vec(rhs, ne, nf, FIT_C128, "rhs")
    _check_vec(x, ne, nf, FIT_C128, "x")
    o = opts if opts is not None else fit_solve_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    if o.stream is None:
        o.stream = _stream_ptr(None).value
    reps = (fit_solve_report * nf)()
    st = lib().fit_solve(g, nf, pom, ct.c_void_p(rhs.data_ptr()), ct.c_void_p(x.data_ptr()), float(tol),
                         ct.byref(o), reps)
    # per-system outcomes, and an abort or a device timeout (the reports are filled), are returned
    if st not in (FIT_OK, FIT_NOT_CONVERGED, FIT_BREAKDOWN, FIT_ENAN, FIT_ETIMEOUT):
        _check(st, "fit_solve")
    return st, [dict(status=r.status, iterations=r.iterations, outer=r.outer, relres=r.relres, seconds=r.seconds,
                     snapshots=r.snapshots) for r in reps]


def fit_apply_variant_count(prec):
    return int(lib().fit_apply_variant_count(prec))


def fit_apply_tuned(g, prec, nbatch):
    """The autotuner's pick for (prec, nbatch): dict(choice, tx, ty, tz, stages, ws, pf); choice -1 =
    generic kernel, -2 = not tuned yet, k >= 0 = fused variant k; tz 0 = balanced at launch; ws 1 =
    the warp-specialised fused kernel; pf = L2 prefetch distance in planes."""
    out = (ct.c_int * 7)()
    _check(lib().fit_apply_tuned(g, prec, nbatch, out), "fit_apply_tuned")
    return dict(choice=out[0], tx=out[1], ty=out[2], tz=out[3], stages=out[4], ws=out[5], pf=out[6])


def fit_tuning_record(path, device, sm_count, nx, ny, nz, prec, nbatch, choice):
    """Append one autotuner result to a tuning-cache file (see fit_apply_tuned)."""
    _check(lib().fit_tuning_record(os.fsencode(path), device.encode(), sm_count, nx, ny, nz, prec, nbatch, choice),
           "fit_tuning_record")


def fit_tuning_lookup(path, device, sm_count, nx, ny, nz, prec, nbatch):
    """The recorded choice for this key (-1 generic, k >= 0 fused variant k), or -2 if none."""
    out = ct.c_int()
    _check(lib().fit_tuning_lookup(os.fsencode(path), device.encode(), sm_count, nx, ny, nz, prec, nbatch,
                                   ct.byref(out)), "fit_tuning_lookup")
    return out.value


def fit_jacobi(g, omega, x, y, prec=FIT_C128, stream=None):
    """y_b = diag(A(omega_b))^-1 x_b (the Jacobi preconditioner of Eq. Precond)."""
    om, pom = _dptr(np.atleast_1d(np.asarray(omega, dtype=np.float64)), np.float64)
    ne = grid_info(g)["ne"]
    _check_vec(x, ne, len(om), prec, "x")
    _check_vec(y, ne, len(om), prec, "y")
    _check(lib().fit_jacobi(g, len(om), pom, _ptr(x), _ptr(y), prec, _stream_ptr(stream)), "fit_jacobi")


def fit_coef_scale(g):
    out = ct.c_double()
    _check(lib().fit_coef_scale(g, ct.byref(out)), "fit_coef_scale")
    return out.value


def _ptr(t):
    return ct.c_void_p(t.data_ptr())


def _ports(ports):
    """[(edges, signs), ...] -> (n, off int32, edges int64, signs float64) in the CSR layout of the ABI."""
    off = np.zeros(len(ports) + 1, dtype=np.int32)
    es, ss = [], []
    for q, (e, sg) in enumerate(ports):
        e = np.asarray(e, dtype=np.int64).ravel()
        sg = np.asarray(sg, dtype=np.float64).ravel()
        if e.shape != sg.shape:
            raise ValueError(f"port {q}: {e.size} edges but {sg.size} signs")
        off[q + 1] = off[q] + e.size
        es.append(e)
        ss.append(sg)
    e = np.ascontiguousarray(np.concatenate(es) if es else np.zeros(0, np.int64))
    sg = np.ascontiguousarray(np.concatenate(ss) if ss else np.zeros(0, np.float64))
    return len(ports), off, e, sg


def fit_port_rhs(g, omega, edges, signs, b, current=1.0, stream=None):
    """b_f = -j omega_f (I s) on the port's unmasked edges (complex128 CUDA tensor of len(omega) x n_e)."""
    om, pom = _dptr(np.atleast_1d(np.asarray(omega, dtype=np.float64)), np.float64)
    e, pe = _dptr(np.asarray(edges, dtype=np.int64).ravel(), np.int64)
    sg, ps = _dptr(np.asarray(signs, dtype=np.float64).ravel(), np.float64)
    if e.size != sg.size:
        raise ValueError(f"{e.size} edges but {sg.size} signs")
    _check_vec(b, grid_info(g)["ne"], len(om), FIT_C128, "b")
    _check(lib().fit_port_rhs(g, len(om), pom, e.size, pe, ps, float(current), _ptr(b), _stream_ptr(stream)),
           "fit_port_rhs")


def fit_probe_voltages(g, x, probes, stream=None):
    """V[f, q] = - sum_k s_k x_f[edge_k] for probes [(edges, signs), ...]; x is a complex128 CUDA tensor of
    nsys x n_e values.  Returns a complex128 numpy array of shape (nsys, nprobe)."""
    ne = grid_info(g)["ne"]
    if x.numel() % ne:
        raise ValueError("x must hold whole vectors of n_e values")
    nsys = x.numel() // ne
    _check_vec(x, ne, nsys, FIT_C128, "x")
    n, off, e, sg = _ports(probes)
    V = np.zeros((nsys, n), dtype=np.complex128)
    pv = V.view(np.float64).ctypes.data_as(ct.POINTER(ct.c_double))
    _check(lib().fit_probe_voltages(g, nsys, _ptr(x), n, off.ctypes.data_as(ct.POINTER(ct.c_int)),
                                    e.ctypes.data_as(ct.POINTER(ct.c_longlong)),
                                    sg.ctypes.data_as(ct.POINTER(ct.c_double)), pv, _stream_ptr(stream)),
           "fit_probe_voltages")
    return V


def fit_z_to_s(Z, z0=50.0):
    """S = (Z - z0 1)(Z + z0 1)^-1 for a P x P complex matrix (numpy in and out)."""
    Zc = np.ascontiguousarray(Z, dtype=np.complex128)
    if Zc.ndim != 2 or Zc.shape[0] != Zc.shape[1]:
        raise ValueError("Z must be square")
    S = np.zeros_like(Zc)
    _check(lib().fit_z_to_s(Zc.shape[0], Zc.view(np.float64).ctypes.data_as(ct.POINTER(ct.c_double)), float(z0),
                            S.view(np.float64).ctypes.data_as(ct.POINTER(ct.c_double))), "fit_z_to_s")
    return S


def fit_z_parameters(g, omega, ports, tol, current=1.0, opts=None, **kw):
    """Impedance matrices of ``ports`` ([(edges, signs), ...]) at every frequency, all (port, frequency)
    systems solved as one batch.  Returns (status, Z of shape (nfreq, P, P) complex128, reports in system
    order port-major).  Keyword arguments override fields of the options struct."""
    om, pom = _dptr(np.atleast_1d(np.asarray(omega, dtype=np.float64)), np.float64)
    n, off, e, sg = _ports(ports)
    o = opts if opts is not None else fit_solve_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    if o.stream is None:
        o.stream = _stream_ptr(None).value
    Z = np.zeros((len(om), n, n), dtype=np.complex128)
    reps = (fit_solve_report * (n * len(om)))()
    st = lib().fit_z_parameters(g, len(om), pom, n, off.ctypes.data_as(ct.POINTER(ct.c_int)),
                                e.ctypes.data_as(ct.POINTER(ct.c_longlong)), sg.ctypes.data_as(ct.POINTER(ct.c_double)),
                                float(current), float(tol), ct.byref(o),
                                Z.view(np.float64).ctypes.data_as(ct.POINTER(ct.c_double)), reps)
    if st not in (FIT_OK, FIT_NOT_CONVERGED, FIT_BREAKDOWN, FIT_ENAN):
        _check(st, "fit_z_parameters")
    return st, Z, [dict(status=r.status, iterations=r.iterations, outer=r.outer, relres=r.relres,
                        seconds=r.seconds, snapshots=r.snapshots) for r in reps]


class UNet:
    """Owning wrapper of a fit_unet handle (the learned right preconditioner)."""

    def __init__(self, seed=0):
        self.h = ct.c_void_p()
        _check(lib().fit_unet_create(int(seed), ct.byref(self.h)), "fit_unet_create")
        self.nparams = int(lib().fit_unet_param_count())

    def get_params(self):
        out = np.empty(self.nparams, np.float32)
        _check(lib().fit_unet_get_params(self.h, out.ctypes.data_as(ct.POINTER(ct.c_float)), self.nparams),
               "fit_unet_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(lib().fit_unet_set_params(self.h, p.ctypes.data_as(ct.POINTER(ct.c_float)), self.nparams),
               "fit_unet_set_params")

    def forward(self, nx, ny, nz, in16, out6, stream=None):
        _check(lib().fit_unet_forward(self.h, nx, ny, nz, _ptr(in16), _ptr(out6), _stream_ptr(stream)),
               "fit_unet_forward")

    def backward(self, nx, ny, nz, in16, target6, grad=None, stream=None):
        loss = ct.c_double()
        _check(lib().fit_unet_backward(self.h, nx, ny, nz, _ptr(in16), _ptr(target6),
                                       _ptr(grad) if grad is not None else None, ct.byref(loss), _stream_ptr(stream)),
               "fit_unet_backward")
        return loss.value

    def train_step(self, nx, ny, nz, in16, target6, lr, stream=None):
        loss = ct.c_double()
        _check(lib().fit_unet_train_step(self.h, nx, ny, nz, _ptr(in16), _ptr(target6), float(lr), ct.byref(loss),
                                         _stream_ptr(stream)), "fit_unet_train_step")
        return loss.value

    def train_step_residual(self, g, omega, in16, lr, stream=None):
        """One Adam step on the residual-angle loss 1 - |<A z, r>|^2 / (||A z||^2 ||r||^2) on grid handle g."""
        loss = ct.c_double()
        _check(lib().fit_unet_train_step_residual(self.h, g, float(omega), _ptr(in16), float(lr), ct.byref(loss),
                                                  _stream_ptr(stream)), "fit_unet_train_step_residual")
        return loss.value

    def residual_loss(self, g, omega, in16, stream=None):
        loss = ct.c_double()
        _check(lib().fit_unet_residual_loss(self.h, g, float(omega), _ptr(in16), ct.byref(loss), _stream_ptr(stream)),
               "fit_unet_residual_loss")
        return loss.value

    def close(self):
        if self.h is not None:
            lib().fit_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fit_unet_pack(g, r, scale, out16, stream=None):
    _check(lib().fit_unet_pack(g, _ptr(r), float(scale), _ptr(out16), _stream_ptr(stream)), "fit_unet_pack")


def fit_unet_pack_target(g, e, scale, out6, stream=None):
    _check(lib().fit_unet_pack_target(g, _ptr(e), float(scale), _ptr(out6), _stream_ptr(stream)),
           "fit_unet_pack_target")


def fit_unet_unpack(g, y6, scale, z, stream=None):
    _check(lib().fit_unet_unpack(g, _ptr(y6), float(scale), _ptr(z), _stream_ptr(stream)), "fit_unet_unpack")


def _p(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def fit_unet_conv3(nx, ny, nz, cin, cout, x, w, bias, relu, out, stream=None):
    """One 3x3x3 conv layer: x bf16 [N, cin], w float32 [27, cout, cin], bias float32 [cout] or None."""
    _check(lib().fit_unet_conv3(nx, ny, nz, cin, cout, _p(x), _p(w), _p(bias), int(relu), _p(out),
                                _stream_ptr(stream)), "fit_unet_conv3")


def fit_unet_conv3_dgrad(nx, ny, nz, cin, cout, dout, w, din, stream=None):
    _check(lib().fit_unet_conv3_dgrad(nx, ny, nz, cin, cout, _p(dout), _p(w), _p(din), _stream_ptr(stream)),
           "fit_unet_conv3_dgrad")


def fit_unet_conv3_wgrad(nx, ny, nz, cin, cout, x, dout, dw, db=None, stream=None):
    _check(lib().fit_unet_conv3_wgrad(nx, ny, nz, cin, cout, _p(x), _p(dout), _p(dw), _p(db), _stream_ptr(stream)),
           "fit_unet_conv3_wgrad")


def fit_unet_tconv(mx, my, mz, cin, cout, x, w, b, out, stream=None):
    _check(lib().fit_unet_tconv(mx, my, mz, cin, cout, _p(x), _p(w), _p(b), _p(out), _stream_ptr(stream)),
           "fit_unet_tconv")


def fit_unet_tconv_backward(mx, my, mz, cin, cout, x, dout, w, din, dw, db, stream=None):
    _check(lib().fit_unet_tconv_backward(mx, my, mz, cin, cout, _p(x), _p(dout), _p(w), _p(din), _p(dw), _p(db),
                                         _stream_ptr(stream)), "fit_unet_tconv_backward")


def fit_unet_head(nvox, x, w, b, out, stream=None):
    _check(lib().fit_unet_head(int(nvox), _p(x), _p(w), _p(b), _p(out), _stream_ptr(stream)), "fit_unet_head")


def fit_unet_head_backward(nvox, x, dout, w, din, dw, db, stream=None):
    _check(lib().fit_unet_head_backward(int(nvox), _p(x), _p(dout), _p(w), _p(din), _p(dw), _p(db),
                                        _stream_ptr(stream)), "fit_unet_head_backward")


def fit_unet_training_pair(g, omega, xk, xstar, b, pair, stream=None):
    """Build one 12-channel bf16 training pair (residual / rms, Jacobi-missed correction) on the device from
    the iterate xk of a solve with solution xstar; returns rms(b - A xk)."""
    rms = ct.c_double()
    _check(lib().fit_unet_training_pair(g, float(omega), _p(xk), _p(xstar), _p(b), _p(pair), ct.byref(rms),
                                        _stream_ptr(stream)), "fit_unet_training_pair")
    return rms.value


def fit_unet_pair_sample(ncell, pair, base16, in16, target6, stream=None):
    _check(lib().fit_unet_pair_sample(int(ncell), _p(pair), _p(base16), _p(in16), _p(target6), _stream_ptr(stream)),
           "fit_unet_pair_sample")


def fit_set_preconditioner(g, net):
    _check(lib().fit_set_preconditioner(g, FIT_PC_UNET, net.h if net is not None else None),
           "fit_set_preconditioner")


def fit_set_abort(g, value):
    """Set (1) or clear (0) the grid's abort word: queued and running fused applies and solves on the
    grid stop at their next bounded wait or loop test and report FIT_ETIMEOUT."""
    _check(lib().fit_set_abort(g, int(value)), "fit_set_abort")


def fit_sync(g, stream=None):
    """Synchronise the stream and report (and clear) a device-side failure of this grid's kernels since
    the last check: returns the status (FIT_OK or FIT_ETIMEOUT) instead of raising for FIT_ETIMEOUT."""
    st = lib().fit_sync(g, _stream_ptr(stream))
    if st not in (FIT_OK, FIT_ETIMEOUT):
        _check(st, "fit_sync")
    return st


def fit_set_hbm_budget(g, nbytes):
    _check(lib().fit_set_hbm_budget(g, int(nbytes)), "fit_set_hbm_budget")


def fit_grid_destroy(g):
    lib().fit_grid_destroy(g)


class Grid:
    """Owning wrapper: ``with Grid.from_case(case) as g: ...`` (case dicts as drawn by ``fitgen``)."""

    def __init__(self, nx, ny, nz, dx, dy, dz):
        self.h = fit_grid_create(nx, ny, nz, dx, dy, dz)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.ne = 3 * nx * ny * nz

    @classmethod
    def from_case(cls, case):
        g = cls(case["nx"], case["ny"], case["nz"], case["dx"], case["dy"], case["dz"])
        fit_set_materials(g.h, case["eps_r"], case["sigma"], case["inv_mu_r"], case.get("pec"))
        return g

    def apply(self, omega, x, y, prec=FIT_C64, stream=None):
        fit_apply(self.h, omega, x, y, prec, stream)

    def solve(self, omega, rhs, x, tol, **kw):
        return fit_solve(self.h, omega, rhs, x, tol, **kw)

    def close(self):
        if self.h is not None:
            fit_grid_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
