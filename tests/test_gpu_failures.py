"""Failure detection, exercised without any GPU fault.

Every failure is made on the host: a wait bound far below the solve time (the
library's host waits give up with VIE_ETIMEOUT while the device keeps working
normally), non-finite inputs, a device budget that refuses an allocation
(VIE_EBUSY), and an injected out-of-memory result of the allocation call
(VIE_ENOMEM, no device call made). After each failure the same process, grid
and stream must keep working.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import mvm as omvm
from oracle import solve as osolve
from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu

K0 = 2 * np.pi
H = 0.05


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _raw_solve(g, sp, ein, e, timeout_ms, mode=vie.MODE_MIXED):
    o = vie.SolveOpts(1e-6, 1e-2, 1000, 1000, 1, mode, 0, timeout_ms, None)
    st = vie.SolveStats()
    rc = vie.load().vie_solve(g.handle, sp.handle, ctypes.c_void_p(ein.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                              ctypes.byref(o), _stream(), ctypes.byref(st))
    return rc, st


def test_wait_timeout_returns_and_the_grid_keeps_working():
    w = inputs.metasurface(cells=8)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    ein = g.plane_wave(w.k0, w.khat, w.pol)
    e = g.empty()
    rc, _ = _raw_solve(g, sp, ein, e, 1e-3)            # 1 microsecond: the first host wait gives up
    assert rc == vie.VIE_ETIMEOUT, vie.last_error()
    assert "wait bound" in vie.last_error()
    torch.cuda.synchronize()                          # the abandoned work finishes normally
    e, st = g.solve(sp, ein)                          # same grid, same stream
    assert st["status"] == vie.VIE_OK and st["true_rel_res"] <= 1e-6
    ein_h = osolve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    A = omvm.FFTOperator(w.eps_r, w.h, w.k0)
    assert np.linalg.norm(ein_h - A(e.cpu().numpy())) <= 1.05e-6 * np.linalg.norm(ein_h)


def test_wait_timeout_in_a_batch():
    ws = [inputs.blob(n=16, seed=40 + i) for i in range(4)]
    b = vie.Batch([x.eps_r for x in ws], ws[0].h)
    g0 = vie.Grid(ws[0].eps_r, ws[0].h)
    ein = torch.stack([g0.plane_wave(x.k0, x.khat, x.pol) for x in ws])
    e = b.empty()
    o = vie.SolveOpts(1e-6, 0.0, 1000, 1, 0, vie.MODE_MIXED, 0, 1e-3, None)
    st = (vie.SolveStats * 4)()
    k = (ctypes.c_double * 4)(*[x.k0 for x in ws])
    rc = vie.load().vie_batch_solve(b.handle, k, ctypes.c_void_p(ein.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                    ctypes.byref(o), _stream(), st)
    assert rc == vie.VIE_ETIMEOUT, vie.last_error()
    torch.cuda.synchronize()
    _, sts = b.solve([x.k0 for x in ws], ein, e)
    assert all(s["status"] == vie.VIE_OK and s["true_rel_res"] <= 1e-6 for s in sts)


def test_non_finite_inputs_are_rejected():
    eps_r, bid, x = inputs.random_case((6, 5, 4), seed=3, block_grid=(3, 3, 2))
    for bad in (np.nan, np.inf, complex(1.0, np.nan)):
        e2 = eps_r.copy()
        e2[1, 2, 3] = bad
        with pytest.raises(vie.VieError) as ei:
            vie.Grid(e2, H, bid)
        assert ei.value.code == vie.VIE_EINVAL and "non-finite" in str(ei.value)
    g = vie.Grid(eps_r, H, bid)
    sp = g.spectrum(K0)
    xb = x.copy()
    xb[0, 1, 1, 1] = np.nan
    for mode in (vie.MODE_MIXED, vie.MODE_PLAIN_C128):
        rc, _ = _raw_solve(g, sp, torch.from_numpy(xb).cuda(), g.empty(), 0.0, mode)
        assert rc == vie.VIE_EINVAL and "non-finite" in vie.last_error()
    e, st = g.solve(sp, torch.from_numpy(x).cuda())   # the grid still solves a finite right-hand side
    assert st["status"] == vie.VIE_OK


def test_device_budget_refuses_with_ebusy_and_keeps_nothing():
    held0, budget0 = vie.device_usage()
    assert budget0 == 0
    w = inputs.metasurface(cells=2)
    try:
        vie.set_device_budget(held0 + 1024)             # far less than a grid needs
        with pytest.raises(vie.VieError) as ei:
            vie.Grid.from_workload(w)
        assert ei.value.code == vie.VIE_EBUSY and "admission refused" in str(ei.value)
        assert vie.device_usage()[0] == held0           # the refused grid freed what it took
        vie.set_device_budget(0)
        g = vie.Grid.from_workload(w)
        need = g.info()["device_bytes"]
        assert vie.device_usage()[0] == held0 + need
        # a budget that fits the grid but not its spectra: the spectrum call is refused
        vie.set_device_budget(held0 + need + 4096)
        with pytest.raises(vie.VieError) as ei:
            g.spectrum(w.k0)
        assert ei.value.code == vie.VIE_EBUSY
        assert vie.device_usage()[0] == held0 + need
        vie.set_device_budget(0)
        sp = g.spectrum(w.k0)
        e, st = g.solve(sp, g.plane_wave(w.k0, w.khat, w.pol))
        assert st["status"] == vie.VIE_OK
        sp.release()
        g.close()
        assert vie.device_usage()[0] == held0
    finally:
        vie.set_device_budget(0)


def test_injected_allocation_failure_gives_enomem():
    held0, _ = vie.device_usage()
    lib = vie.load()
    w = inputs.metasurface(cells=2)
    for after in (0, 3, 10):
        assert lib.vie_fault_inject_alloc(after) == vie.VIE_OK
        with pytest.raises(vie.VieError) as ei:
            vie.Grid.from_workload(w)
        assert ei.value.code == vie.VIE_ENOMEM and "cudaMalloc" in str(ei.value)
        assert vie.device_usage()[0] == held0
    g = vie.Grid.from_workload(w)                     # one failure per injection: this one succeeds
    assert lib.vie_fault_inject_alloc(0) == vie.VIE_OK
    with pytest.raises(vie.VieError) as ei:
        g.spectrum(w.k0)
    assert ei.value.code == vie.VIE_ENOMEM
    sp = g.spectrum(w.k0)
    _, st = g.solve(sp, g.plane_wave(w.k0, w.khat, w.pol))
    assert st["status"] == vie.VIE_OK
    assert lib.vie_fault_inject_alloc(-1) == vie.VIE_OK
