"""Oracle: incident field, full solve and far field (Sections II-III).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

solve() is the paper's outer loop: BiCGSTAB on A E = E_inc (Eq. 4 discretised),
right-preconditioned with the block-diagonal K2 of Eq. 10 when requested.
far_field_rcs() gives the bistatic radar cross-section used in Section III's
Mie comparison (Figs. 1-2) from the polarisation sum of the solved field.

Pinned by tests/test_oracle_mie.py (RCS against the Mie series, error falling
with resolution) and tests/test_oracle_solver.py (energy balance, solver
against dense LU).
"""
import numpy as np

from .krylov import bicgstab
from .mvm import FFTOperator
from .precond import BlockPreconditioner


def voxel_positions(n, h):
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) * h - 0.5 * nx * h
    y = (np.arange(ny) + 0.5) * h - 0.5 * ny * h
    z = (np.arange(nz) + 0.5) * h - 0.5 * nz * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def plane_wave(n, h, k, khat, pol):
    """E_inc = p exp(-j k khat . r) at voxel centres (exp(+jwt) convention, after Eq. 1)."""
    X, Y, Z = voxel_positions(n, h)
    ph = np.exp(-1j * k * (khat[0] * X + khat[1] * Y + khat[2] * Z))
    return np.stack([pol[c] * ph for c in range(3)]).astype(complex)


def solve(eps_r, block_id, h, k, einc, tol=1e-6, use_precond=True,
          inner_tol=1e-2, inner_maxit=1000, maxit=1000, near=None, expand=0):
    """Solve A E = E_inc; returns (E, info) with the true residual added to info.
    near = (radius, q): cube-integrated near-neighbour kernel entries (green.cube_kernel).
    expand = e: expanded blocks (precond.find_blocks)."""
    A = FFTOperator(eps_r, h, k, near=near)
    Kinv = None
    if use_precond and np.any(block_id >= 0):
        Kinv = BlockPreconditioner(eps_r, block_id, h, k, inner_tol, inner_maxit, near=near, expand=expand)
    E, info = bicgstab(A.apply, einc, tol, maxit, apply_Kinv=Kinv)
    info["true_rel_res"] = np.linalg.norm(einc - A.apply(E)) / np.linalg.norm(einc)
    return E, info


def far_field_rcs(E, eps_r, h, k, rhat):
    """Bistatic RCS sigma(rhat) = k^4/(4 pi) |(I - rhat rhat) . sum_j chi_j E_j h^3 e^{jk rhat.r_j}|^2.

    Far-zone limit of E_s = k^2 int G chi E dv (Eq. 1 with J = jw eps0 chi E)."""
    nz, ny, nx = eps_r.shape
    X, Y, Z = voxel_positions((nx, ny, nz), h)
    chi = eps_r - 1.0
    rhat = np.atleast_2d(rhat)
    out = np.empty(rhat.shape[0])
    for i, u in enumerate(rhat):
        ph = np.exp(1j * k * (u[0] * X + u[1] * Y + u[2] * Z))
        P = np.array([np.sum(chi * E[c] * ph) for c in range(3)]) * h ** 3
        Pt = P - u * np.dot(u, P)
        out[i] = k ** 4 / (4 * np.pi) * np.real(np.vdot(Pt, Pt))
    return out


def absorbed_power(E, eps_r):
    """Power absorbed in the scatterer, proportional to sum -Im(eps_r) |E|^2 (exp(+jwt))."""
    return float(np.sum(-np.imag(eps_r)[None] * np.abs(E) ** 2))
