"""Batched independent solves (vie_batch_*) against single solves and the oracle's operator.

Each instance is the unpreconditioned system of Eq. 4 with its own permittivity,
wavenumber and incident field. The batch result must match the per-instance
vie_solve result (mixed) to the solve tolerance scale, and its FP64 residual,
evaluated with the oracle's operator, must meet the tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import mvm as omvm
from oracle import solve as osolve
from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu


def _instances(n, count, seed0):
    ws = [inputs.blob(n=n, seed=seed0 + i, voxels_per_wl=20) for i in range(count)]
    k0s = [w.k0 * (1.0 + 0.05 * i) for i, w in enumerate(ws)]       # distinct wavenumbers
    eincs = [osolve.plane_wave(w.n, w.h, k, w.khat, w.pol) for w, k in zip(ws, k0s)]
    return ws, k0s, eincs


@pytest.mark.parametrize("n,count,persistent", [(12, 6, True), (16, 3, True), (48, 2, False)])
def test_batch_matches_single_solves(n, count, persistent):
    ws, k0s, eincs = _instances(n, count, seed0=10 * n)
    b = vie.Batch([w.eps_r for w in ws], ws[0].h)
    assert b.info()["persistent"] == persistent
    ein = torch.from_numpy(np.stack(eincs)).cuda()
    e, stats = b.solve(k0s, ein, outer_tol=1e-6)
    torch.cuda.synchronize()
    e = e.cpu().numpy()
    for i, (w, k, inc) in enumerate(zip(ws, k0s, eincs)):
        assert stats[i]["status"] == vie.VIE_OK
        A = omvm.FFTOperator(w.eps_r, w.h, k)
        res = np.linalg.norm(inc - A(e[i])) / np.linalg.norm(inc)
        assert res <= 1.05e-6, (i, res)
        assert abs(res - stats[i]["true_rel_res"]) <= 1e-2 * res + 1e-12
        g = vie.Grid(w.eps_r, w.h)
        sp = g.spectrum(k)
        e1, st1 = g.solve(sp, torch.from_numpy(inc).cuda(), outer_tol=1e-6, use_precond=False, mode=vie.MODE_MIXED)
        ref = e1.cpu().numpy()
        assert np.linalg.norm(e[i] - ref) <= 1e-5 * np.linalg.norm(ref)


def test_batch_identical_instances_agree_and_zero_rhs():
    w = inputs.blob(n=10, seed=3)
    b = vie.Batch([w.eps_r] * 4, w.h)
    inc = osolve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    ein = torch.from_numpy(np.stack([inc, inc, np.zeros_like(inc), inc])).cuda()
    e, stats = b.solve([w.k0] * 4, ein, outer_tol=1e-7)
    e = e.cpu().numpy()
    assert np.array_equal(e[0], e[1]) and np.array_equal(e[0], e[3])   # same work, same bits
    assert not np.any(e[2]) and stats[2]["status"] == vie.VIE_OK


def test_batches_of_several_sizes_share_launches():
    # vie_batch_solve_many: batches of 12^3, 16^3 and 24^3 instances at once, their corrections merged into
    # one persistent launch per refinement step; each instance's FP64 residual (oracle operator) meets the
    # tolerance and its field equals the batch solved alone up to rounding
    specs = [(12, 3), (16, 2), (24, 2)]
    jobs, alone, cases = [], [], []
    for n, count in specs:
        ws, k0s, eincs = _instances(n, count, seed0=7 * n)
        ein = torch.from_numpy(np.stack(eincs)).cuda()
        jobs.append({"batch": vie.Batch([w.eps_r for w in ws], ws[0].h), "k0s": k0s, "einc": ein, "outer_tol": 1e-6})
        alone.append(vie.Batch([w.eps_r for w in ws], ws[0].h))
        cases.append((ws, k0s, eincs))
    res, ms = vie.batch_solve_many(jobs)
    assert ms["launches"] >= 1 and ms["max_solves"] == 3
    for (e, stats), job, b1, (ws, k0s, eincs) in zip(res, jobs, alone, cases):
        e1, _ = b1.solve(k0s, job["einc"], outer_tol=1e-6)
        torch.cuda.synchronize()
        e, e1 = e.cpu().numpy(), e1.cpu().numpy()
        for i, (w, k, inc) in enumerate(zip(ws, k0s, eincs)):
            assert stats[i]["status"] == vie.VIE_OK
            res_i = np.linalg.norm(inc - omvm.FFTOperator(w.eps_r, w.h, k)(e[i])) / np.linalg.norm(inc)
            assert res_i <= 1.05e-6, (w.n, i, res_i)
            assert np.linalg.norm(e[i] - e1[i]) <= 1e-5 * np.linalg.norm(e1[i])
    with pytest.raises(vie.VieError):
        vie.batch_solve_many([jobs[0], dict(jobs[0])])             # a batch listed twice
