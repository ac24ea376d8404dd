"""The serving request stream (inputs.serving_draws / serving_geometry) and the stored oracle solves of its
sampled requests (tests/golden/serve_requests.npz): seeded, with the stated size mix and geometry."""
import json
import os

import numpy as np

from paper_2501_13512_gb300 import inputs, serve

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "serve_requests.npz")


def test_draws_are_seeded_and_follow_the_size_mix():
    a = inputs.serving_draws(2000, seed=4)
    b = inputs.serving_draws(2000, seed=4)
    assert [d["structure"] for d in a] == [d["structure"] for d in b]
    n = np.array([d["n"] for d in a])
    frac = [np.mean(n == s) for s in inputs.SERVING_SIZES]
    assert np.allclose(frac, inputs.SERVING_SIZE_WEIGHTS, atol=0.035)
    assert [d["kind"] for d in a[:4]] == ["metasurface", "solar_cell", "metasurface", "solar_cell"]
    lam = np.array([d["lambda_nm"] for d in a])
    assert lam.min() >= 400 and lam.max() <= 800 and np.all(lam % 10 == 0)
    for d in a[:50]:
        assert abs(np.linalg.norm(d["khat"]) - 1) < 1e-12 and abs(np.dot(d["khat"], d["pol"])) < 1e-12
        assert np.degrees(np.arcsin(d["khat"][0])) <= 30.0


def test_streams_of_both_modes_hold_the_same_problems():
    m = serve.make_stream(6, seed=2, mode=1)
    f = serve.make_stream(6, seed=2, mode=0)
    assert [r.structure for r in m] == [r.structure for r in f] and [r.k0 for r in m] == [r.k0 for r in f]
    assert {r.mode for r in m} == {1} and {r.mode for r in f} == {0}


def test_metasurface_tile_is_the_unit_cell_layer_in_a_cubic_box():
    for n in (32, 64):
        w = inputs.serving_geometry("metasurface", n, 0)
        assert w.n == (n, n, n)
        solid = np.nonzero(np.any(w.eps_r != 1.0, axis=(1, 2)))[0]
        z0 = (n - 16) // 2
        assert solid.min() == z0 and solid.max() == z0 + 15          # pillars 16 voxels tall
        assert w.block_id.max() + 1 == (n // 16) ** 2                  # one block per pillar
        assert np.all((w.block_id >= 0) == (w.eps_r != 1.0))


def test_solar_cell_tile_spheres_lie_inside_the_slab():
    for n in (32, 64):
        w = inputs.serving_geometry("solar_cell", n, 1)
        metal = w.eps_r.real < 0
        z = np.nonzero(np.any(metal, axis=(1, 2)))[0]
        z0, z1 = ((n - 40) // 2, (n - 40) // 2 + 40) if n >= 48 else (n // 5, n // 5 + (5 * n) // 8)
        assert z.min() >= z0 and z.max() < z1
        nsph = (n // min(32, n)) ** 2
        assert w.block_id.max() + 1 == nsph + 4


def test_golden_serving_references_match_their_draws():
    gd = np.load(GOLDEN)
    draws = inputs.serving_draws(4, 1, (32, 64), (0.4, 0.3))
    kinds = set()
    for i in range(3):
        meta = json.loads(str(gd[f"meta_{i}"]))
        d = draws[meta["request"]]
        assert (d["structure"], d["lambda_nm"], d["n"]) == (meta["structure"], meta["lambda_nm"], meta["n"])
        assert meta["status"] == 0 and meta["true_rel_res"] <= 1e-10
        idx, val = gd[f"index_{i}"], gd[f"value_{i}"]
        assert idx.size == 8192 and np.all(np.diff(idx) > 0) and idx.max() < 3 * d["n"] ** 3
        assert np.all(np.isfinite(val)) and 0 < np.linalg.norm(val) <= meta["field_norm"]
        kinds.add(d["kind"])
    assert kinds == {"metasurface", "solar_cell"}
