"""GPU parity: every step of the CUDA path, called through the C ABI, against the CPU oracle.

Tolerances (relative 2-norm over all entries):
  * complex128 MVM: 1e-12 (FP64 FFTs; observed ~1e-15);
  * complex64 MVM: 1e-5 (FP32 FFTs of length <= 512 per axis: a few units of
    2^-24 per butterfly stage, ~20 stages in forward + inverse);
  * preconditioner with tight inner tolerance (1e-12), complex128: 1e-9
    (both sides approximate the exact block inverse);
  * solves: relative field error vs the oracle solved to 1e-10.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import mvm as omvm
from oracle import precond as oprecond
from oracle import solve as osolve
from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu

K0 = 2 * np.pi
H = 0.05


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SHAPES = [(16, 16, 16), (5, 7, 3), (12, 20, 9), (1, 1, 1), (33, 4, 2), (2, 1, 40), (64, 48, 8)]


@pytest.mark.parametrize("n", SHAPES)
def test_matvec_c128(n):
    eps_r, _, x = inputs.random_case(n, seed=sum(n))
    g = vie.Grid(eps_r, H)
    sp = g.spectrum(K0)
    y = g.matvec(sp, dev(x))
    ref = omvm.FFTOperator(eps_r, H, K0)(x)
    assert rel(host(y), ref) <= 1e-12


@pytest.mark.parametrize("n", SHAPES)
def test_matvec_c64(n):
    eps_r, _, x = inputs.random_case(n, seed=sum(n) + 1)
    g = vie.Grid(eps_r, H)
    sp = g.spectrum(K0)
    y = g.matvec(sp, dev(x, torch.complex64))
    ref = omvm.FFTOperator(eps_r, H, K0)(x.astype(np.complex64).astype(np.complex128))
    assert rel(host(y), ref) <= 1e-5


def test_matvec_metasurface_full_size():
    # the 256x256x16 metasurface grid (padded FFT 512x512x32), both precisions
    w = inputs.metasurface()
    rng = np.random.default_rng(5)
    x = rng.normal(size=(3,) + w.eps_r.shape) + 1j * rng.normal(size=(3,) + w.eps_r.shape)
    ref = omvm.FFTOperator(w.eps_r, w.h, w.k0)(x)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    assert rel(host(g.matvec(sp, dev(x))), ref) <= 1e-12
    assert rel(host(g.matvec(sp, dev(x, torch.complex64))), ref) <= 1e-5


def test_matvec_rejects_aliasing_and_bad_precision():
    eps_r, _, x = inputs.random_case((4, 4, 4), seed=2)
    g = vie.Grid(eps_r, H)
    sp = g.spectrum(K0, vie.C128)
    xd = dev(x)
    lib = vie.load()
    rc = lib.vie_matvec(g.handle, sp.handle, vie.C128, xd.data_ptr(), xd.data_ptr(), None)
    assert rc == vie.VIE_EINVAL
    rc = lib.vie_matvec(g.handle, sp.handle, vie.C64, xd.data_ptr(), g.empty(vie.C64).data_ptr(), None)
    assert rc == vie.VIE_EINVAL


def test_plane_wave():
    n = (9, 6, 5)
    g = vie.Grid(np.ones(n[::-1], complex), H)
    khat = np.array([0.3, -0.5, 0.8])
    khat /= np.linalg.norm(khat)
    pol = np.array([1.0, 0.2j, -0.3 + 0.1j])
    ref = osolve.plane_wave(n, H, K0, khat, pol)
    assert rel(host(g.plane_wave(K0, khat, pol)), ref) <= 1e-13
    assert rel(host(g.plane_wave(K0, khat, pol, precision=vie.C64)), ref) <= 1e-6


INNER_PATHS = [vie.INNER_BATCHED, vie.INNER_PERSISTENT]


@pytest.mark.parametrize("inner", INNER_PATHS)
def test_precond_tight_matches_oracle(inner):
    eps_r, bid, b = inputs.random_case((12, 10, 8), seed=31, block_grid=(4, 5, 4))
    P = oprecond.BlockPreconditioner(eps_r, bid, H, K0, inner_tol=1e-12, inner_maxit=300)
    ref = P(b)
    g = vie.Grid(eps_r, H, bid, inner=inner)
    sp = g.spectrum(K0)
    y, st = g.precond(sp, dev(b), inner_tol=1e-12, inner_maxit=300)
    assert st["nblocks"] == len(P.blocks)
    assert st["not_converged"] == 0 and st["breakdowns"] == 0
    assert rel(host(y), ref) <= 1e-9


@pytest.mark.parametrize("inner", INNER_PATHS)
@pytest.mark.parametrize("precision", [vie.C128, vie.C64])
def test_precond_loose_meets_inner_tolerance(precision, inner):
    # uneven blocks (ragged at the grid edge) solved to 1e-2: each block's own residual meets it
    eps_r, bid, b = inputs.random_case((13, 11, 7), seed=17, block_grid=(5, 4, 7))
    g = vie.Grid(eps_r, H, bid, inner=inner)
    sp = g.spectrum(K0)
    dt = torch.complex128 if precision == vie.C128 else torch.complex64
    y, st = g.precond(sp, dev(b, dt), inner_tol=1e-2, inner_maxit=100)
    y = host(y)
    bb = b.astype(np.complex64).astype(np.complex128) if precision == vie.C64 else b
    for blk in oprecond.find_blocks(bid):
        sl = (slice(None),) + blk.slices
        op = omvm.FFTOperator(eps_r[blk.slices], H, K0, mask=blk.mask)
        bk = np.where(blk.mask[None], bb[sl], 0)
        xk = np.where(blk.mask[None], y[sl], 0)
        assert np.linalg.norm(bk - op(xk)) <= 1.01e-2 * np.linalg.norm(bk)
    air = bid < 0
    assert np.array_equal(y[:, air], bb[:, air])


@pytest.mark.parametrize("precision", [vie.C128, vie.C64])
def test_precond_paths_agree_on_metasurface_blocks(precision):
    # the two inner-solver paths run the same recurrences with different rounding
    # orders (2D plane FFTs vs pencil passes): results agree to the inner tolerance
    w = inputs.metasurface(cells=4, seed=3)
    rng = np.random.default_rng(2)
    b = rng.normal(size=(3,) + w.eps_r.shape) + 1j * rng.normal(size=(3,) + w.eps_r.shape)
    dt = torch.complex128 if precision == vie.C128 else torch.complex64
    itol = 1e-6 if precision == vie.C128 else 1e-4     # FP32 stalls near 1e-6
    out = []
    for inner in INNER_PATHS:
        g = vie.Grid.from_workload(w, inner=inner)
        sp = g.spectrum(w.k0)
        y, st = g.precond(sp, dev(b, dt), inner_tol=itol, inner_maxit=200)
        assert st["nblocks"] == 16 and st["not_converged"] == 0
        out.append((host(y), st))
    assert rel(out[1][0], out[0][0]) <= 10 * itol
    m0, m1 = out[0][1]["mean_iters"], out[1][1]["mean_iters"]
    assert abs(m0 - m1) <= max(1.0, 0.1 * m0)


def test_precond_without_blocks_is_identity():
    eps_r, _, b = inputs.random_case((6, 5, 4), seed=3)
    g = vie.Grid(eps_r, H)
    sp = g.spectrum(K0)
    y, st = g.precond(sp, dev(b))
    assert st["nblocks"] == 0
    assert np.array_equal(host(y), b)


def _sphere_case():
    w = inputs.sphere()
    ein = osolve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    ref, _ = osolve.solve(w.eps_r, w.block_id, w.h, w.k0, ein, tol=1e-10, use_precond=False)
    return w, ein, ref


def test_solve_sphere_plain_c128():
    w, ein, ref = _sphere_case()
    _, info = osolve.solve(w.eps_r, w.block_id, w.h, w.k0, ein, tol=1e-6, use_precond=False)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    e, st = g.solve(sp, dev(ein), outer_tol=1e-6, use_precond=False, mode=vie.MODE_PLAIN_C128)
    assert st["status"] == vie.VIE_OK
    assert st["true_rel_res"] <= 1e-6
    assert st["outer_iters"] == info["iters"]        # same recurrences in FP64
    assert rel(host(e), ref) <= 1e-5


def test_solve_sphere_mixed():
    w, ein, ref = _sphere_case()
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    e, st = g.solve(sp, dev(ein), outer_tol=1e-6, use_precond=False, mode=vie.MODE_MIXED)
    assert st["status"] == vie.VIE_OK
    assert st["true_rel_res"] <= 1e-6
    assert rel(host(e), ref) <= 1e-5


@pytest.mark.parametrize("mode", [vie.MODE_PLAIN_C128, vie.MODE_MIXED])
def test_solve_metasurface_crop_preconditioned(mode):
    w = inputs.metasurface(cells=3, seed=2)
    ein = osolve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    ref, _ = osolve.solve(w.eps_r, w.block_id, w.h, w.k0, ein, tol=1e-10, use_precond=True, inner_tol=1e-2)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    e, st = g.solve(sp, dev(ein), outer_tol=1e-6, inner_tol=1e-2, use_precond=True, mode=mode)
    assert st["status"] == vie.VIE_OK
    assert st["true_rel_res"] <= 1e-6
    e = host(e)
    A = omvm.FFTOperator(w.eps_r, w.h, w.k0)
    assert np.linalg.norm(ein - A(e)) <= 1.05e-6 * np.linalg.norm(ein)
    assert rel(e, ref) <= 1e-4
    assert st["precond_applies"] > 0 and st["inner_iters"] > 0


def test_solve_metasurface_full_size_mixed():
    # the full 256x256x16 metasurface, the benchmark's workload: FP64 residual checked by the oracle
    w = inputs.metasurface()
    ein = osolve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    e, st = g.solve(sp, dev(ein), outer_tol=1e-6, inner_tol=1e-2, use_precond=True, mode=vie.MODE_MIXED)
    assert st["status"] == vie.VIE_OK
    e = host(e)
    A = omvm.FFTOperator(w.eps_r, w.h, w.k0)
    r = np.linalg.norm(ein - A(e)) / np.linalg.norm(ein)
    assert r <= 1.05e-6
    assert abs(r - st["true_rel_res"]) <= 1e-3 * r


def test_solve_zero_rhs():
    eps_r, bid, _ = inputs.random_case((6, 5, 4), seed=3, block_grid=(3, 3, 2))
    g = vie.Grid(eps_r, H, bid)
    sp = g.spectrum(K0)
    z = torch.zeros((3, 4, 5, 6), dtype=torch.complex128, device="cuda")
    for mode in (vie.MODE_PLAIN_C128, vie.MODE_MIXED):
        e, st = g.solve(sp, z, mode=mode)
        assert st["status"] == vie.VIE_OK
        assert not np.any(host(e))


@pytest.mark.parametrize("mode", [vie.MODE_PLAIN_C128, vie.MODE_MIXED])
def test_solve_warm_start(mode):
    # E_0 = the converged field: no iteration; E_0 = a partial solve (in place): finishes to tolerance
    w = inputs.metasurface(cells=2, seed=4)
    ein = osolve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    A = omvm.FFTOperator(w.eps_r, w.h, w.k0)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    b = dev(ein)
    e_ref, st = g.solve(sp, b, outer_tol=1e-8, mode=vie.MODE_PLAIN_C128)
    assert st["status"] == vie.VIE_OK and st["elapsed_ms"] > 0
    e, st = g.solve(sp, b, outer_tol=1e-6, mode=mode, x0=e_ref)
    assert st["status"] == vie.VIE_OK and st["outer_iters"] == 0
    assert rel(host(e), host(e_ref)) <= 1e-12
    e, st0 = g.solve(sp, b, outer_tol=1e-6, mode=mode, outer_maxit=3, max_refinements=1)
    assert st0["status"] == vie.VIE_ENOTCONV
    e, st = g.solve(sp, b, e=e, outer_tol=1e-6, mode=mode, x0=e)
    assert st["status"] == vie.VIE_OK
    eh = host(e)
    r = np.linalg.norm(ein - A(eh)) / np.linalg.norm(ein)
    assert r <= 1.05e-6 and abs(r - st["true_rel_res"]) <= 1e-3 * r


def test_solve_rejects_overlapping_x0():
    eps_r, bid, x = inputs.random_case((6, 5, 4), seed=3, block_grid=(3, 3, 2))
    g = vie.Grid(eps_r, H, bid)
    sp = g.spectrum(K0)
    buf = torch.zeros((2,) + (3, 4, 5, 6), dtype=torch.complex128, device="cuda")
    b, e = dev(x), buf[0]
    lib = vie.load()
    o = vie.SolveOpts(1e-6, 1e-2, 10, 10, 1, vie.MODE_MIXED, 0, 0.0, b.data_ptr())
    st = vie.SolveStats()
    assert lib.vie_solve(g.handle, sp.handle, b.data_ptr(), e.data_ptr(), o, None, st) == vie.VIE_EINVAL


def test_precond_every_tuner_candidate_meets_inner_tolerance():
    # the first apply of a persistent grid warms up, the next ones run the tuner's candidates (blocks of
    # the slab MVM: 2, 1 and 4 CTAs per block with 4 kz planes per round, 2 CTAs with 2 planes, and the
    # register MVM on 2 CTAs; other blocks: 2, 4 and the split launch), the seventh the chosen one;
    # every block of every apply meets the inner tolerance
    w = inputs.metasurface(cells=4, seed=3)
    rng = np.random.default_rng(8)
    b = rng.normal(size=(3,) + w.eps_r.shape) + 1j * rng.normal(size=(3,) + w.eps_r.shape)
    g = vie.Grid.from_workload(w, inner=vie.INNER_PERSISTENT)
    sp = g.spectrum(w.k0)
    bb = b.astype(np.complex64).astype(np.complex128)
    blocks = oprecond.find_blocks(w.block_id)
    ops = [omvm.FFTOperator(w.eps_r[blk.slices], w.h, w.k0, mask=blk.mask) for blk in blocks]
    for apply in range(7):
        y, st = g.precond(sp, dev(b, torch.complex64), inner_tol=1e-2)
        assert st["nblocks"] == 16 and st["not_converged"] == 0 and st["breakdowns"] == 0
        y = host(y)
        for blk, op in zip(blocks, ops):
            sl = (slice(None),) + blk.slices
            bk = np.where(blk.mask[None], bb[sl], 0)
            xk = np.where(blk.mask[None], y[sl], 0)
            assert np.linalg.norm(bk - op(xk)) <= 1.01e-2 * np.linalg.norm(bk), (apply, blk.slices)
    assert g.info()["inner_cluster"][1] in (1, 2, 4, -1)


GOLDEN_MS = os.path.join(os.path.dirname(__file__), "golden", "metasurface_reference.json")

# Outer tolerance at which the solved field is within 1e-5 of the exact solution of the discretised
# system (the oracle solved to 1e-10), in both modes, on the metasurface crops below.
OUTER_TOL_FOR_1E5 = 1e-6


def _crop_reference(cells):
    p = os.path.join(os.path.dirname(__file__), "golden", f"metasurface_crop_{cells}x{cells}.npz")
    if not os.path.exists(p):
        pytest.skip(f"oracle reference {os.path.basename(p)} not recorded")
    z = np.load(p)
    return json.loads(str(z["meta"])), z["index"], z["value"]


@pytest.mark.parametrize("cells", [4, 8])
@pytest.mark.parametrize("mode", [vie.MODE_MIXED, vie.MODE_PLAIN_C128])
def test_metasurface_crop_field_within_1e5_of_tight_oracle(cells, mode):
    # 64x64x16 (4x4 pillars, every entry) and 128x128x16 (8x8 pillars, 65536 seeded entries): the
    # block-preconditioned solve at outer tolerance 1e-6 against the oracle's solve to 1e-10, element
    # by element over the stored entries (Section II.B; SURVEY's "several correct results" reading:
    # iterates agree only within tolerance, so the reference is solved far tighter than the solve)
    meta, idx, ref = _crop_reference(cells)
    assert meta["true_rel_res"] <= 1e-10
    w = inputs.metasurface(cells=cells, seed=0)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    e, st = g.solve(sp, g.plane_wave(w.k0, w.khat, w.pol), outer_tol=OUTER_TOL_FOR_1E5, inner_tol=w.inner_tol,
                    mode=mode)
    assert st["status"] == vie.VIE_OK and st["true_rel_res"] <= OUTER_TOL_FOR_1E5
    got = host(e.reshape(-1)[torch.from_numpy(idx).cuda()])
    err = rel(got, ref)
    print(f"crop {cells}x{cells} mode {mode}: outer {st['outer_iters']} res {st['true_rel_res']:.2e} "
          f"field err {err:.2e}")
    assert err <= 1e-5


@pytest.mark.skipif(not os.path.exists(GOLDEN_MS), reason="oracle full-size reference not recorded")
def test_metasurface_full_size_field_at_oracle_samples():
    # full 256x256x16 metasurface: the GPU field (mixed, solved to 1e-8) against the oracle's FP64
    # block-preconditioned solve (true residual 9.8e-7) at 4096 seeded voxel samples. Both solve the
    # same system; the difference is the oracle's own error (measured 2.4e-6 with the GPU at 4.5e-7).
    gd = json.load(open(GOLDEN_MS))
    if not gd["true_rel_res"] <= 1.05e-6:
        pytest.skip(f"the oracle's reference solve stopped at true residual {gd['true_rel_res']:.2e}")
    w = inputs.metasurface()
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    e, st = g.solve(sp, g.plane_wave(w.k0, w.khat, w.pol), outer_tol=1e-8, inner_tol=w.inner_tol,
                    mode=vie.MODE_MIXED)
    assert st["status"] == vie.VIE_OK
    idx = torch.tensor(gd["sample_index"], device="cuda")
    got = host(e.reshape(-1)[idx])
    ref = np.array(gd["sample_re"]) + 1j * np.array(gd["sample_im"])
    assert rel(got, ref) <= 1e-4
