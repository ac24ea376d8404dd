"""Pins for oracle/krylov.py, oracle/precond.py and oracle/solve.py (Section II.B, Eq. 10)."""
import numpy as np
import pytest

from oracle import krylov, mvm, precond, solve
from paper_2501_13512_gb300 import inputs

K0 = 2 * np.pi
H = 0.05


def test_bicgstab_matches_dense_solve():
    eps_r, _, b = inputs.random_case((4, 4, 3), seed=21)
    A = mvm.dense_operator(eps_r, H, K0)
    xref = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    op = mvm.FFTOperator(eps_r, H, K0)
    x, info = krylov.bicgstab(op.apply, b, tol=1e-11, maxit=500)
    assert info["status"] == krylov.CONVERGED
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - xref) <= 10 * kappa * 1e-11 * np.linalg.norm(xref)
    r = np.linalg.norm(b - op(x)) / np.linalg.norm(b)
    assert r <= 1e-10


def test_bicgstab_initial_guess_matches_dense_solve():
    # x0 branch: r0 = b - A x0, stopping test still relative to ||b|| (van der Vorst's algorithm from
    # an arbitrary start); pinned against LU from three starts: a perturbed solution, a random vector,
    # and the exact solution (no iteration at all)
    eps_r, _, b = inputs.random_case((4, 3, 3), seed=23)
    A = mvm.dense_operator(eps_r, H, K0)
    xref = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    op = mvm.FFTOperator(eps_r, H, K0)
    rng = np.random.default_rng(5)
    kappa = np.linalg.cond(A)
    noise = rng.normal(size=b.shape) + 1j * rng.normal(size=b.shape)
    for x0 in (xref + 0.1 * noise, noise):
        x0_copy = x0.copy()
        x, info = krylov.bicgstab(op.apply, b, tol=1e-11, maxit=500, x0=x0)
        assert info["status"] == krylov.CONVERGED
        assert np.array_equal(x0, x0_copy)                # the start is not modified
        assert np.linalg.norm(x - xref) <= 10 * kappa * 1e-11 * np.linalg.norm(xref)
        assert np.linalg.norm(b.ravel() - A @ x.ravel()) <= 1e-10 * np.linalg.norm(b)
    x, info = krylov.bicgstab(op.apply, b, tol=1e-9, maxit=500, x0=xref)
    assert info["iters"] == 0 and info["matvecs"] == 1 and np.array_equal(x, xref)
    # a start closer to the solution takes fewer iterations than a cold start to the same tolerance
    _, cold = krylov.bicgstab(op.apply, b, tol=1e-8, maxit=500)
    _, warm = krylov.bicgstab(op.apply, b, tol=1e-8, maxit=500, x0=xref + 1e-4 * noise)
    assert warm["iters"] < cold["iters"]


def test_bicgstab_zero_rhs_and_identity():
    b = np.zeros((3, 2, 2, 2), complex)
    x, info = krylov.bicgstab(lambda v: v, b, 1e-6, 10)
    assert info["status"] == krylov.CONVERGED and not np.any(x)
    b = np.ones((3, 2, 2, 2), complex)
    x, info = krylov.bicgstab(lambda v: 2 * v, b, 1e-12, 10)
    assert info["iters"] == 0.5 and np.allclose(x, 0.5 * b, rtol=1e-15)


def test_block_inverse_matches_dense_lu():
    eps_r, bid, x = inputs.random_case((6, 5, 4), seed=3, block_grid=(3, 3, 2))
    P = precond.BlockPreconditioner(eps_r, bid, H, K0, inner_tol=1e-13, inner_maxit=400)
    y = P(x)
    A = mvm.dense_operator(eps_r, H, K0)
    fb = np.tile(bid.ravel(), 3)
    yref = x.ravel().copy()
    for blk in P.blocks:
        idx = np.nonzero(fb == blk.bid)[0]
        yref[idx] = np.linalg.solve(A[np.ix_(idx, idx)], x.ravel()[idx])
    assert np.linalg.norm(y.ravel() - yref) <= 1e-10 * np.linalg.norm(yref)


def test_inexact_block_inverse_within_inner_tolerance():
    eps_r, bid, x = inputs.random_case((6, 5, 4), seed=8, block_grid=(3, 5, 4))
    tol = 1e-2
    P = precond.BlockPreconditioner(eps_r, bid, H, K0, inner_tol=tol)
    y = P(x)
    A = mvm.dense_operator(eps_r, H, K0)
    fb = np.tile(bid.ravel(), 3)
    for blk in P.blocks:
        idx = np.nonzero(fb == blk.bid)[0]
        Ak = A[np.ix_(idx, idx)]
        res = np.linalg.norm(x.ravel()[idx] - Ak @ y.ravel()[idx]) / np.linalg.norm(x.ravel()[idx])
        assert res <= tol


def test_single_block_is_exact_inverse():
    # K2 = A when one block holds every voxel: the outer solve stops at its first half-step.
    eps_r, _, b = inputs.random_case((5, 4, 3), seed=9)
    bid = np.zeros(eps_r.shape, np.int32)
    E, info = solve.solve(eps_r, bid, H, K0, b, tol=1e-6, use_precond=True,
                          inner_tol=1e-12, inner_maxit=500)
    assert info["iters"] == 0.5
    assert info["true_rel_res"] <= 1e-6


def test_preconditioned_and_plain_agree():
    eps_r, bid, b = inputs.random_case((6, 6, 4), seed=13, block_grid=(3, 3, 4))
    E1, i1 = solve.solve(eps_r, bid, H, K0, b, tol=1e-10, use_precond=True, inner_tol=1e-2)
    E0, i0 = solve.solve(eps_r, bid, H, K0, b, tol=1e-10, use_precond=False)
    assert i1["true_rel_res"] <= 1e-9 and i0["true_rel_res"] <= 1e-9
    assert np.linalg.norm(E1 - E0) <= 1e-7 * np.linalg.norm(E0)


def test_absorbed_power_nonnegative():
    w = inputs.sphere(n=10, eps=3.0 - 0.5j, voxels_per_wl=20)
    ein = solve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    E, info = solve.solve(w.eps_r, w.block_id, w.h, w.k0, ein, tol=1e-8, use_precond=False)
    assert info["true_rel_res"] <= 1e-7
    assert solve.absorbed_power(E, w.eps_r) > 0


def test_optical_theorem_soft():
    # extinction (forward amplitude) ~ scattering + absorption; the discrete
    # system satisfies it only approximately, so this is a loose check.
    w = inputs.sphere(n=12, eps=2.25 - 0.2j, voxels_per_wl=24)
    k = w.k0
    ein = solve.plane_wave(w.n, w.h, k, w.khat, w.pol)
    E, _ = solve.solve(w.eps_r, w.block_id, w.h, k, ein, tol=1e-10, use_precond=False)
    X, Y, Z = solve.voxel_positions(w.n, w.h)
    chi = w.eps_r - 1
    P = np.array([np.sum(chi * E[c] * np.exp(1j * k * Z)) for c in range(3)]) * w.h ** 3
    # exp(+jwt): C_ext = -k Im(conj(E0) . P), P projected on the incident wave
    c_ext = -k * np.imag(P[0])
    th = np.linspace(0, np.pi, 121)
    ph = np.linspace(0, 2 * np.pi, 121, endpoint=False)
    T, F = np.meshgrid(th, ph, indexing="ij")
    rh = np.stack([np.sin(T) * np.cos(F), np.sin(T) * np.sin(F), np.cos(T)], -1).reshape(-1, 3)
    s = solve.far_field_rcs(E, w.eps_r, w.h, k, rh).reshape(T.shape) / (4 * np.pi)
    c_sca = np.sum(s * np.sin(T)) * (th[1] - th[0]) * (ph[1] - ph[0])
    c_abs = k * np.sum(-np.imag(w.eps_r) * np.sum(np.abs(E) ** 2, 0)) * w.h ** 3
    assert c_ext > 0
    assert abs(c_ext - (c_sca + c_abs)) <= 0.1 * c_ext


# ---------------------------------------------------------------- expanded blocks
def _dense_expanded(eps_r, bid, b, expand):
    """Restricted additive Schwarz by dense LU: each block solved on S_k+, its own voxels kept."""
    A = mvm.dense_operator(eps_r, H, K0)
    N = eps_r.size
    chi_nz = ((eps_r - 1.0) != 0).ravel()
    y = b.ravel().copy()
    for blk in precond.find_blocks(bid, expand, (eps_r - 1.0) != 0):
        sel = np.zeros(bid.shape, bool)
        sel[blk.slices] = blk.mask
        core = np.zeros(bid.shape, bool)
        core[blk.slices] = blk.core
        idx = np.nonzero(np.tile(sel.ravel(), 3))[0]
        xk = np.linalg.solve(A[np.ix_(idx, idx)], b.ravel()[idx])
        keep = np.tile(core.ravel(), 3)[idx]
        y[idx[keep]] = xk[keep]
        assert np.all(chi_nz[sel.ravel()] | core.ravel()[sel.ravel()])   # halo voxels are never air
    return y.reshape(b.shape)


@pytest.mark.parametrize("expand", [1, 2])
def test_expanded_blocks_match_dense_lu(expand):
    eps_r, bid, b = inputs.random_case((6, 5, 4), seed=33, block_grid=(3, 3, 2))
    P = precond.BlockPreconditioner(eps_r, bid, H, K0, inner_tol=1e-13, inner_maxit=500, expand=expand)
    yref = _dense_expanded(eps_r, bid, b, expand)
    assert np.linalg.norm(P(b) - yref) <= 1e-10 * np.linalg.norm(yref)
    # the expanded sets really grow, and the plain blocks are the expand = 0 case
    plain = precond.find_blocks(bid)
    grown = precond.find_blocks(bid, expand, (eps_r - 1.0) != 0)
    assert sum(g.mask.sum() for g in grown) > sum(p.mask.sum() for p in plain)
    assert all(np.array_equal(p.mask, p.core) for p in plain)
    assert all(g.core.sum() == p.mask.sum() for g, p in zip(grown, plain))


def test_expanded_blocks_reaching_every_voxel_are_exact_on_the_blocks():
    # every non-air voxel lies in some block; with an expansion that covers the grid each block solves
    # the closed system of all non-air voxels, so y equals A^-1 b on the blocks' voxels
    eps_r, bid, b = inputs.random_case((5, 4, 4), seed=34, block_grid=(3, 2, 2))
    A = mvm.dense_operator(eps_r, H, K0)
    x = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    P = precond.BlockPreconditioner(eps_r, bid, H, K0, inner_tol=1e-13, inner_maxit=800, expand=5)
    y = P(b)
    on = bid >= 0
    assert np.linalg.norm(y[:, on] - x[:, on]) <= 1e-10 * np.linalg.norm(x[:, on])
    assert np.array_equal(y[:, ~on], b[:, ~on])


def test_expanded_blocks_same_solution_fewer_outer_iterations():
    # the preconditioner changes the iterations, not the solution of A E = E_inc
    w = inputs.metasurface(cells=2, period=8, nz=6, seed=5, block_cells=1)
    ein = solve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    e0, i0 = solve.solve(w.eps_r, w.block_id, w.h, w.k0, ein, tol=1e-10, inner_tol=1e-2)
    e2, i2 = solve.solve(w.eps_r, w.block_id, w.h, w.k0, ein, tol=1e-10, inner_tol=1e-2, expand=2)
    assert np.linalg.norm(e2 - e0) <= 1e-8 * np.linalg.norm(e0)
    assert i2["iters"] <= i0["iters"]
