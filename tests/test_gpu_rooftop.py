"""GPU parity of the paper's rooftop / pulse discretisation (Section II.A, Eqs. 5-9; vie_rooftop_*) against
the oracle (oracle/rooftop.py), and the sphere's RCS against the Mie series in both discretisations (the
collocation operator of vie_matvec and the rooftop operator), as in Figs. 1-2."""
import numpy as np
import pytest
import torch

from oracle import krylov, mie
from oracle import rooftop as ort
from oracle import solve as osolve
from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu

K0 = 2 * np.pi
H = 0.05


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,seed", [((5, 4, 3), 61), ((4, 4, 4), 62), ((6, 3, 2), 63), ((1, 5, 4), 64),
                                    ((7, 5, 6), 65), ((16, 16, 16), 66)])
def test_rooftop_matvec_matches_oracle(n, seed):
    eps_r, _, x = inputs.random_case(n, seed=seed)
    op = ort.RooftopOperator(eps_r, H, K0)
    ref = op(x)
    g = vie.Grid(eps_r, H)
    r = vie.Rooftop(g, K0)
    y = r.matvec(dev(x)).cpu().numpy()
    assert rel(y, ref) <= 1e-12
    y64 = r.matvec(dev(x, torch.complex64)).cpu().numpy()
    assert rel(y64, ref) <= 1e-5
    assert not np.any(y[~op.act])                  # faces without a rooftop stay 0


def test_rooftop_incident_matches_oracle():
    eps_r, _, _ = inputs.random_case((6, 5, 4), seed=67)
    act = ort.active_faces(eps_r)
    khat, pol = np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.2j, 0.0])
    ref = ort.incident((6, 5, 4), H, K0, khat, pol, act)
    g = vie.Grid(eps_r, H)
    r = vie.Rooftop(g, K0)
    assert rel(r.incident(khat, pol).cpu().numpy(), ref) <= 1e-13


def _sphere(n, eps):
    radius = 0.25
    return inputs.sphere_radius_voxels(n, radius, eps, 2 * radius / n), radius


@pytest.mark.parametrize("eps", [4.0, 2.25])
def test_rooftop_sphere_solve_and_rcs(eps):
    w, radius = _sphere(16, eps)
    op = ort.RooftopOperator(w.eps_r, w.h, w.k0)
    b = ort.incident(w.n, w.h, w.k0, w.khat, w.pol, op.act)
    ref, info = krylov.bicgstab(op, b, 1e-10, 3000)
    g = vie.Grid.from_workload(w)
    r = vie.Rooftop(g, w.k0)
    bd = r.incident(w.khat, w.pol)
    x, st = r.solve(bd, tol=1e-8, maxit=3000)
    assert st["status"] == vie.VIE_OK and st["true_rel_res"] <= 1e-8
    xh = x.cpu().numpy()
    assert rel(xh, ref) <= 1e-6
    th = np.linspace(0, np.pi, 91)
    dirs = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    s_gpu = r.far_field_rcs(x, dirs)
    assert rel(s_gpu, ort.far_field_rcs(ref, w.n, w.h, w.k0, dirs)) <= 1e-5
    # both discretisations against the Mie series (the oracle's pins give the convergence in n)
    m = mie.rcs_eplane(eps, radius, w.k0, th)
    err_rooftop = rel(s_gpu, m)
    sp = g.spectrum(w.k0)
    e, st2 = g.solve(sp, g.plane_wave(w.k0, w.khat, w.pol), outer_tol=1e-8, use_precond=False,
                     mode=vie.MODE_PLAIN_C128)
    err_colloc = rel(g.far_field_rcs(w.k0, e, dirs), m)
    print(f"sphere eps {eps} 16^3: RCS error vs Mie rooftop {err_rooftop:.4f} collocation {err_colloc:.4f}")
    assert err_rooftop <= (0.035 if eps == 4.0 else 0.13)
    assert err_colloc <= 0.06


def test_rooftop_rejects_bad_arguments():
    eps_r, _, x = inputs.random_case((4, 4, 4), seed=68)
    g = vie.Grid(eps_r, H)
    with pytest.raises(vie.VieError):
        vie.Rooftop(g, -1.0)
    r = vie.Rooftop(g, K0, precision=vie.C128)
    with pytest.raises(vie.VieError):
        r.matvec(dev(x, torch.complex64))          # built without complex64 spectra
    xd = dev(x)
    with pytest.raises(vie.VieError):
        r.matvec(xd, xd)                           # overlapping
