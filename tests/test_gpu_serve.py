"""Serving on the GPU: a result is the same alone and in the mix (continuous batching)."""
import copy

import numpy as np
import pytest

from paper_2501_13512_gb300 import inputs, serve

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    ms5 = inputs.metasurface(cells=2, seed=5)                      # 32 x 32 x 16, 4 pillar blocks
    ms6 = inputs.metasurface(cells=2, seed=6)
    for key, w in (("ms5", ms5), ("ms6", ms6)):
        for lam_scale, th in ((1.0, 0.0), (1.1, 0.3)):
            khat = np.array([np.sin(th), 0.0, np.cos(th)])
            pol = np.array([np.cos(th), 0.0, -np.sin(th)], complex)
            out.append(serve.Request(structure=key, eps_r=w.eps_r, h=w.h, k0=w.k0 / lam_scale, khat=khat,
                                     pol=pol, block_id=w.block_id, outer_maxit=400))
    return out


def test_same_result_alone_and_in_the_mix():
    srv = serve.Server(budget_bytes=16 << 30, slots=4)
    try:
        reqs = _requests()
        alone = [srv.submit(copy.copy(r)).result(timeout=120) for r in reqs]     # one at a time
        futs = [srv.submit(copy.copy(r)) for r in reqs]                          # all overlapping
        mixed = [f.result(timeout=120) for f in futs]
        st = srv.latency_stats()
    finally:
        srv.close()
    for a, m in zip(alone, mixed):
        assert a.stats["status"] == 0 and m.stats["status"] == 0
        assert a.stats["true_rel_res"] <= 1e-6
        assert np.linalg.norm(m.field - a.field) <= 1e-12 * np.linalg.norm(a.field)
    assert st["requests"] == 8
    eng = srv.engine
    assert eng.hits["spectrum_miss"] == 4 and eng.hits["spectrum_hit"] >= 4   # one spectrum per (structure, k0)


def test_spectrum_serves_a_compatible_grid_only():
    from paper_2501_13512_gb300 import vie
    import torch
    w = inputs.metasurface(cells=2, seed=5)
    g1 = vie.Grid.from_workload(w)
    g2 = vie.Grid.from_workload(w)                      # same structure, second instance
    other = vie.Grid.from_workload(inputs.metasurface(cells=3, seed=6))   # another grid size
    sp = g1.spectrum(w.k0)
    x = g1.plane_wave(w.k0, w.khat, w.pol)
    y1 = g1.matvec(sp, x)
    y2 = g2.matvec(sp, x)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    g1.close()                                          # the spectrum outlives the grid it was made for
    assert torch.equal(g2.matvec(sp, x), y1)
    with pytest.raises(vie.VieError):
        other.matvec(sp, other.plane_wave(w.k0, w.khat, w.pol))     # shapes differ: rejected
