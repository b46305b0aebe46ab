"""Oracle solvers for A(w) x = b: direct (dense LU, sparse LU) and textbook Krylov methods.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  complex128 throughout.  The Krylov methods
follow the short-listed solvers of Sec. IV (bcgs and the gmres family, Fig. Iterative) as
textbook algorithms: BiCGStab (van der Vorst 1992), restarted (F)GMRES (Saad 1993) with
modified Gram-Schmidt and Givens rotations, and COCG and COCR (the paper's "cg" and "cr" on a
complex symmetric A).  Conventions (readings): conjugated inner products
<u, v> = u^H v, x0 = 0, shadow residual r^ = r0, stop on the true relative residual
||b - A x|| / ||b|| (Sec. IV fixes only "a relative decrease of the residual norm").
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def dense_solve(A, b):
    """x = A^{-1} b by dense LU (numpy.linalg.solve); small systems only."""
    return np.linalg.solve(A.toarray(), b)


def sparse_solve(A, b):
    """x = A^{-1} b by sparse LU (SuperLU through scipy.sparse.linalg.spsolve)."""
    return spla.spsolve(A.tocsc(), b)


def relres(A, x, b):
    """||b - A x||_2 / ||b||_2 in complex128."""
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


def cocg(A, b, tol=1e-10, maxiter=10000, dinv=None):
    """Conjugate orthogonal CG (van der Vorst and Melissen 1990) for complex symmetric A = A^T: the
    CG recurrences with the unconjugated bilinear form (u, v) = u^T v, the reading of the "cg"
    solver of Sec. IV on the complex symmetric system of Eq. e2.  ``dinv`` (optional) is the
    diagonal of a symmetric preconditioner M = diag(dinv).  Per step:
        q = A p,  alpha = rho / (p, q),  x += alpha p,  r -= alpha q,
        z = M r,  rho' = (r, z),  beta = rho' / rho,  p = z + beta p.
    Returns (x, iterations, true relative residual, status), status 0 = converged, 1 = iteration
    cap, 2 = breakdown (|(p, q)| or |rho| < 1e-300)."""
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0:
        return x, 0, 0.0, 0
    m = (lambda v: v) if dinv is None else (lambda v: dinv * v)
    r = b.copy()
    z = m(r)
    p = z.copy()
    rho = r @ z  # unconjugated
    for it in range(1, maxiter + 1):
        q = A @ p
        pq = p @ q
        if abs(pq) < 1e-300 or abs(rho) < 1e-300:
            return x, it, relres(A, x, b), 2
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        if np.linalg.norm(r) <= tol * nb:
            rr = relres(A, x, b)
            if rr <= tol:
                return x, it, rr, 0
        z = m(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, maxiter, relres(A, x, b), 1


def cocr(A, b, tol=1e-10, maxiter=10000, dinv=None):
    """Conjugate orthogonal conjugate residual (Sogabe and Zhang 2007) for complex symmetric A = A^T:
    the conjugate-residual recurrences with the unconjugated bilinear form (u, v) = u^T v, the
    reading of the "cr" solver of Sec. IV.  ``dinv`` (optional) is the diagonal of a symmetric
    preconditioner M = diag(dinv); the recurrences are those of COCR on M^{1/2} A M^{1/2} written in
    the original variables.  Start: z = M r, w = A z, p = z, q = w, rho = (z, w).  Per step:
        alpha = rho / (q, M q),  x += alpha p,  r -= alpha q,  z = M r,  w = A z,
        rho' = (z, w),  beta = rho' / rho,  p = z + beta p,  q = w + beta q   (q = A p throughout).
    Returns (x, iterations, true relative residual, status), status 0 = converged, 1 = iteration
    cap, 2 = breakdown (|(q, M q)| or |rho| < 1e-300)."""
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0:
        return x, 0, 0.0, 0
    m = (lambda v: v) if dinv is None else (lambda v: dinv * v)
    r = b.copy()
    z = m(r)
    w = A @ z
    p = z.copy()
    q = w.copy()
    rho = z @ w  # unconjugated
    for it in range(1, maxiter + 1):
        sig = q @ m(q)
        if abs(sig) < 1e-300 or abs(rho) < 1e-300:
            return x, it, relres(A, x, b), 2
        alpha = rho / sig
        x = x + alpha * p
        r = r - alpha * q
        if np.linalg.norm(r) <= tol * nb:
            rr = relres(A, x, b)
            if rr <= tol:
                return x, it, rr, 0
        z = m(r)
        w = A @ z
        rho_new = z @ w
        beta = rho_new / rho
        p = z + beta * p
        q = w + beta * q
        rho = rho_new
    return x, maxiter, relres(A, x, b), 1


def bicgstab(A, b, tol=1e-10, maxiter=10000):
    """Unpreconditioned BiCGStab.  Returns (x, iterations, true relative residual, status) with
    status 0 = converged, 1 = iteration cap, 2 = breakdown (|rho| or |omega| < 1e-300)."""
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0:
        return x, 0, 0.0, 0
    r = b.copy()
    rhat = r.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho = alpha = omega = 1.0 + 0j
    for it in range(1, maxiter + 1):
        rho_new = np.vdot(rhat, r)
        if abs(rho_new) < 1e-300:
            return x, it, relres(A, x, b), 2
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A @ p
        alpha = rho_new / np.vdot(rhat, v)
        s = r - alpha * v
        t = A @ s
        tt = np.vdot(t, t).real
        omega = np.vdot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        if np.linalg.norm(r) <= tol * nb:
            rr = relres(A, x, b)
            if rr <= tol:
                return x, it, rr, 0
            r = b - A @ x  # residual drift: restart the recurrence from the true residual
        if abs(omega) < 1e-300:
            return x, it, relres(A, x, b), 2
    return x, maxiter, relres(A, x, b), 1


def fgmres(A, b, tol=1e-10, restart=30, maxiter=10000, precond=None, precond_step=False, history=None):
    """Restarted right-preconditioned FGMRES(m) with modified Gram-Schmidt and Givens rotations.
    ``precond`` maps a vector v_j to z_j = M(v_j) (identity when None, which is plain GMRES); with
    ``precond_step`` it is called as M(V, j) with the cycle's basis V (rows 0 .. j filled) and the
    Arnoldi step j, and returns z_j: the flexible method minimises the residual over x0 + span(z_0 ..
    z_j) whatever the z_j are, so the preconditioner may change from step to step.  ``history``, if a list,
    receives the true relative residual after every restart cycle.
    Returns (x, iterations, true relative residual, status)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0:
        return x, 0, 0.0, 0
    M = precond if precond is not None else (lambda v: v)
    total = 0
    while total < maxiter:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            return x, total, beta / nb, 0
        m = restart
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        jlast = 0
        for jj in range(m):
            Z[jj] = M(V, jj) if precond_step else M(V[jj])
            w = A @ Z[jj]
            for i in range(jj + 1):  # modified Gram-Schmidt
                H[i, jj] = np.vdot(V[i], w)
                w = w - H[i, jj] * V[i]
            H[jj + 1, jj] = np.linalg.norm(w)
            if H[jj + 1, jj] != 0:
                V[jj + 1] = w / H[jj + 1, jj]
            for i in range(jj):  # apply the earlier rotations to the new column
                hi = H[i, jj]
                H[i, jj] = np.conj(cs[i]) * hi + np.conj(sn[i]) * H[i + 1, jj]
                H[i + 1, jj] = -sn[i] * hi + cs[i] * H[i + 1, jj]
            a, c = H[jj, jj], H[jj + 1, jj]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[jj] = a / den if den != 0 else 1.0
            sn[jj] = c / den if den != 0 else 0.0
            H[jj, jj] = den
            H[jj + 1, jj] = 0.0
            g[jj + 1] = -sn[jj] * g[jj]
            g[jj] = np.conj(cs[jj]) * g[jj]
            total += 1
            jlast = jj + 1
            if abs(g[jj + 1]) <= tol * nb or total >= maxiter or H[jj, jj] == 0:
                break
        y = np.linalg.solve(np.triu(H[:jlast, :jlast]), g[:jlast])
        x = x + Z[:jlast].T @ y
        rr = relres(A, x, b)
        if history is not None:
            history.append(rr)
        if rr <= tol:
            return x, total, rr, 0
    return x, total, relres(A, x, b), 1
