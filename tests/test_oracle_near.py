"""Pins for the near-field variant of the oracle (cube-integrated kernel entries, oracle/green.py).

The paper gives no near-neighbour integration; the variant integrates k^2 G over the source voxel
for offsets with max |D| <= radius. Checked against: an adaptive cubature (scipy), convergence in
the quadrature order, the mean of a Helmholtz solution over a cube (Taylor: f(c)(1 - (kh)^2/24)
+ O(h^4)), per-axis parities, reciprocity, and FFT form == dense form with the variant's entries.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import green, mvm
from paper_2501_13512_gb300 import inputs

K0 = 2 * np.pi


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("d", [(1, 1, 0), (0, 1, 2)])
def test_cube_kernel_matches_adaptive_cubature(d):
    h = 0.05
    ref = green.cube_kernel(d, h, K0, 16)
    scale = max(abs(ref[n]) for n in green.COMPONENTS)
    for comp in ("xx", "xy", "yz"):
        for part in (np.real, np.imag):
            def f(z, y, x):
                return float(part(green.k2G_at(np.array(x), np.array(y), np.array(z), K0)[comp]))
            lo = [(c - 0.5) * h for c in d]
            hi = [(c + 0.5) * h for c in d]
            val, _ = integrate.tplquad(f, lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], epsabs=0, epsrel=1e-11)
            want = float(part(ref[comp]))
            assert abs(val - want) <= 1e-9 * scale, (comp, part.__name__)


def test_quadrature_order_converges():
    h = 0.05
    for d in [(1, 0, 0), (1, 1, 0), (1, 1, 1), (0, 2, 1)]:
        a = green.cube_kernel(d, h, K0, 16)
        b = green.cube_kernel(d, h, K0, 24)
        scale = max(abs(b[n]) for n in green.COMPONENTS)
        assert max(abs(a[n] - b[n]) for n in green.COMPONENTS) <= 1e-10 * scale


@pytest.mark.parametrize("d", [(6, 0, 0), (5, 3, 0), (4, 4, 4), (10, 0, 0)])
def test_cube_mean_of_helmholtz_solution(d):
    # each component of k^2 G solves (laplacian + k^2) f = 0 away from the origin, so its mean over
    # a cube of side h is f(c) (1 - (kh)^2 / 24) up to O(h^4): a dropped or wrong term breaks this
    kh = 0.3
    h = kh / K0
    cube = green.cube_kernel(d, h, K0, 12)
    mid = green.k2G_at(np.array(d[0] * h), np.array(d[1] * h), np.array(d[2] * h), K0)
    scale = max(abs(mid[n]) for n in green.COMPONENTS) * h ** 3
    corr = kh * kh / 24.0
    for n in green.COMPONENTS:
        pred = h ** 3 * mid[n] * (1.0 - corr)
        assert abs(cube[n] - pred) <= 0.05 * corr * scale, n
    # and the correction itself is visible (the test is not vacuous)
    assert max(abs(cube[n] - h ** 3 * mid[n]) for n in green.COMPONENTS) >= 0.5 * corr * scale


def test_near_entries_keep_the_parities():
    h = 0.05
    base = green.cube_kernel((1, 2, 1), h, K0, 10)
    for sx, sy, sz in [(-1, 1, 1), (1, -1, 1), (1, 1, -1), (-1, -1, -1)]:
        m = green.cube_kernel((sx, 2 * sy, sz), h, K0, 10)
        sign = {"xx": 1, "yy": 1, "zz": 1, "xy": sx * sy, "xz": sx * sz, "yz": sy * sz}
        for n in green.COMPONENTS:
            assert abs(m[n] - sign[n] * base[n]) <= 1e-12 * abs(base["xx"]), (n, sx, sy, sz)


@pytest.mark.parametrize("shape", [(5, 4, 3), (3, 3, 3)])
def test_fft_operator_equals_dense_with_near_terms(shape):
    eps_r, _, x = inputs.random_case(shape, seed=7)
    near = (1, 8)
    h = 0.05
    A = mvm.dense_operator(eps_r, h, K0, near=near)
    y_dense = (A @ x.reshape(-1)).reshape(x.shape)
    y_fft = mvm.FFTOperator(eps_r, h, K0, near=near)(x)
    assert np.linalg.norm(y_fft - y_dense) <= 1e-12 * np.linalg.norm(y_dense)
    G = mvm.dense_G((shape[0], shape[1], shape[2]), h, K0, near=near)
    assert np.abs(G - G.T).max() <= 1e-14 * np.abs(G).max()
    # the variant changes exactly the near entries
    G0 = mvm.dense_G((shape[0], shape[1], shape[2]), h, K0)
    assert np.abs(G - G0).max() > 1e-3 * np.abs(G0).max()
