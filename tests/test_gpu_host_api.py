"""vie_solve_host: the solve from host buffers (E_inc copied in, E copied out inside the call) equals the
device-buffer solve, from pinned and from pageable memory, and rejects overlapping buffers."""
import numpy as np
import pytest
import torch

from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu


def test_solve_host_equals_the_device_solve():
    w = inputs.metasurface(cells=2, seed=4)
    g = vie.Grid.from_workload(w)
    sp = g.spectrum(w.k0)
    ein = g.plane_wave(w.k0, w.khat, w.pol)
    e_dev, st = g.solve(sp, ein, outer_tol=1e-8, inner_tol=1e-2)
    ref = e_dev.cpu().numpy()
    for pinned in (True, False):
        h_in = ein.cpu()
        h_out = torch.empty_like(h_in)
        if pinned:
            h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
        out, st_h = g.solve_host(sp, h_in, h_out, outer_tol=1e-8, inner_tol=1e-2)
        assert out is h_out and st_h["status"] == vie.VIE_OK and st_h["true_rel_res"] <= 1e-8
        assert np.linalg.norm(h_out.numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
    with pytest.raises(vie.VieError):
        g.solve_host(sp, h_in, h_in)                  # the same buffer in and out
    sp.release()
    g.close()
