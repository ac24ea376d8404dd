"""Oracle: right-preconditioned BiCGSTAB (Section II.B; van der Vorst's method, ref. [18]).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section II.B applies BiCGSTAB to A K2^{-1} (K2 x) = b with K1 = I: each outer
iteration solves y = K2^{-1} p and z = K2^{-1} s. The recurrences below follow
van der Vorst's algorithm in that right-preconditioned form, with the
Hermitian inner product <a, b> = a^H b. Because the preconditioner may be an
inexact inner solve, x is updated with the y and z actually computed.

Pinned by tests/test_oracle_solver.py against numpy.linalg.solve on small
dense systems and by the single-block exact-inverse invariant.
"""
import numpy as np

CONVERGED = 0
NOT_CONVERGED = 1
BREAKDOWN = 2


def bicgstab(apply_A, b, tol, maxit, apply_Kinv=None, x0=None):
    """Solve A x = b to ||r|| <= tol ||b||.

    Returns (x, info) with info = {status, iters (half-steps counted as 0.5),
    matvecs, rel_res (recursive residual at exit), history}.
    """
    Kinv = apply_Kinv if apply_Kinv is not None else (lambda v: v)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    info = {"status": CONVERGED, "iters": 0.0, "matvecs": 0, "rel_res": 0.0, "history": []}
    if bnorm == 0.0:
        return np.zeros_like(b), info
    r = b - apply_A(x) if x0 is not None else b.copy()
    if x0 is not None:
        info["matvecs"] += 1
    rel = np.linalg.norm(r) / bnorm
    info["rel_res"] = rel
    if rel <= tol:
        return x, info
    rhat = r.copy()
    rho_prev = alpha = omega = 1.0 + 0.0j
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = np.vdot(rhat, r)
        if rho == 0 or not np.isfinite(rho):
            info["status"] = BREAKDOWN
            break
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        y = Kinv(p)
        v = apply_A(y)
        info["matvecs"] += 1
        sigma = np.vdot(rhat, v)
        if sigma == 0 or not np.isfinite(sigma):
            info["status"] = BREAKDOWN
            break
        alpha = rho / sigma
        s = r - alpha * v
        srel = np.linalg.norm(s) / bnorm
        if srel <= tol:
            x = x + alpha * y
            info["iters"] = it - 0.5
            info["rel_res"] = srel
            info["history"].append(srel)
            return x, info
        z = Kinv(s)
        t = apply_A(z)
        info["matvecs"] += 1
        tt = np.vdot(t, t).real
        if tt == 0 or not np.isfinite(tt):
            info["status"] = BREAKDOWN
            break
        omega = np.vdot(t, s) / tt
        x = x + alpha * y + omega * z
        r = s - omega * t
        rho_prev = rho
        rel = np.linalg.norm(r) / bnorm
        info["iters"] = float(it)
        info["rel_res"] = rel
        info["history"].append(rel)
        if rel <= tol:
            return x, info
        if omega == 0:
            info["status"] = BREAKDOWN
            break
    else:
        info["status"] = NOT_CONVERGED
    return x, info
