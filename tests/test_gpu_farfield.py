"""GPU far-field / bistatic RCS (vie_far_field_rcs) against the oracle, and the Mie validation
pipeline of Section III (Figs. 1-2) run end to end on the GPU: plane wave, solve, RCS."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import mie
from oracle import solve as osolve
from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sphere_rcs.json")


def _dirs(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[0] = [0.0, 0.0, 1.0]      # axis directions: separable phase factors equal to 1 on two axes
    d[1] = [1.0, 0.0, 0.0]
    return d


@pytest.mark.parametrize("shape", [(9, 7, 5), (1, 1, 1), (16, 16, 16), (33, 4, 20)])
def test_far_field_matches_oracle(shape):
    eps_r, _, x = inputs.random_case(shape, seed=sum(shape) + 5)
    k0, h = 2 * np.pi, 0.05
    g = vie.Grid(eps_r, h)
    dirs = _dirs(37, 1)
    got = g.far_field_rcs(k0, torch.from_numpy(x).cuda(), dirs)
    ref = osolve.far_field_rcs(x, eps_r, h, k0, dirs)
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-300)


def test_far_field_rejects_bad_directions():
    eps_r, _, x = inputs.random_case((4, 4, 4), seed=2)
    g = vie.Grid(eps_r, 0.05)
    with pytest.raises(vie.VieError):
        g.far_field_rcs(2 * np.pi, torch.from_numpy(x).cuda(), np.array([[1.0, 1.0, 0.0]]))


def _gpu_rcs_error(n, radius, eps, lambda0, theta):
    h = 2.0 * radius / n
    w = inputs.sphere_radius_voxels(n, radius, eps, h, lambda0=lambda0)
    g = vie.Grid(w.eps_r, w.h)
    sp = g.spectrum(w.k0)
    einc = g.plane_wave(w.k0, w.khat, w.pol)
    e, st = g.solve(sp, einc, outer_tol=1e-8, use_precond=False, mode=vie.MODE_PLAIN_C128, outer_maxit=3000)
    assert st["status"] == vie.VIE_OK and st["true_rel_res"] <= 1e-7
    rh = np.stack([np.sin(theta), 0 * theta, np.cos(theta)], 1)
    s = g.far_field_rcs(w.k0, e, rh)
    m = mie.rcs_eplane(eps, radius, w.k0, theta)
    return float(np.linalg.norm(s - m) / np.linalg.norm(m))


def test_paper_spheres_on_gpu_within_printed_error():
    # Figs. 1-2 configuration (radius 400 nm, 750 THz; eps_r 2.25 and the metal -1.05 - j5.62) at 20^3:
    # within twice the paper's printed relative L2 RCS errors against Mie
    gd = json.load(open(GOLDEN))
    th = np.linspace(0, np.pi, 181)
    for case in gd["cases"]:
        eps = complex(case["eps_r_re"], case["eps_r_im"])
        err = _gpu_rcs_error(20, gd["radius_nm"], eps, gd["lambda0_nm"], th)
        assert err <= 2.0 * case["paper_rel_l2_rcs_error"], (eps, err)
