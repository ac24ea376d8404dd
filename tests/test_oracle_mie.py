"""Pins for oracle/mie.py and the VIE oracle against the Mie series (Section III, Figs. 1-2)."""
import json
import os

import numpy as np
import pytest

from oracle import mie, solve
from paper_2501_13512_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sphere_rcs.json")


@pytest.mark.parametrize("m,x", [(1.5, 3.0), (1.33, 0.7), (2.0, 5.5), (3.5, 1.2)])
def test_lossless_extinction_equals_scattering(m, x):
    qext, qsca = mie.efficiencies(m, x)
    assert abs(qext - qsca) <= 1e-10 * qsca


@pytest.mark.parametrize("m", [1.5, 2.0 + 0.3j, 1.2 + 2.0j])
def test_rayleigh_limit(m):
    x = 1e-3
    _, qsca = mie.efficiencies(m, x)
    ray = 8.0 / 3.0 * x ** 4 * abs((m * m - 1) / (m * m + 2)) ** 2
    assert abs(qsca - ray) <= 1e-4 * ray


def test_forward_amplitudes_equal_and_index_one_is_transparent():
    S1, S2 = mie.amplitudes(1.7 + 0.1j, 2.3, np.array([0.0]))
    assert abs(S1[0] - S2[0]) <= 1e-13 * abs(S1[0])
    a, b = mie.coefficients(1.0 + 0j, 2.0)
    assert np.abs(a).max() < 1e-13 and np.abs(b).max() < 1e-13


def _rcs_error(n, radius, eps, lambda0, theta):
    h = 2.0 * radius / n
    w = inputs.sphere_radius_voxels(n, radius, eps, h, lambda0=lambda0)
    ein = solve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    E, info = solve.solve(w.eps_r, w.block_id, w.h, w.k0, ein, tol=1e-8, use_precond=False, maxit=3000)
    assert info["true_rel_res"] <= 1e-7
    rh = np.stack([np.sin(theta), 0 * theta, np.cos(theta)], 1)
    s = solve.far_field_rcs(E, w.eps_r, w.h, w.k0, rh)
    m = mie.rcs_eplane(eps, radius, w.k0, theta)
    return np.linalg.norm(s - m) / np.linalg.norm(m)


def test_vie_sphere_converges_to_mie():
    # 0.25 lambda0 sphere, eps_r 4: error falls with resolution
    th = np.linspace(0, np.pi, 91)
    errs = [_rcs_error(n, 0.25, 4.0, 1.0, th) for n in (12, 16, 24)]
    assert errs[1] < 0.10
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.slow
def test_paper_sphere_cases_within_printed_error():
    # Figs. 1-2 configuration at a 20^3 grid: within twice the paper's printed errors
    g = json.load(open(GOLDEN))
    th = np.linspace(0, np.pi, 181)
    for case in g["cases"]:
        eps = complex(case["eps_r_re"], case["eps_r_im"])
        err = _rcs_error(20, g["radius_nm"], eps, g["lambda0_nm"], th)
        assert err <= 2.0 * case["paper_rel_l2_rcs_error"], (eps, err)
