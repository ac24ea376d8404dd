"""Pins for oracle/green.py (Section II.A, Eq. 1): the dyadic kernel and self term.

Each check ties the oracle to something other than its own formula: finite
differences of the scalar Green's function, the electrostatic limit, the
Helmholtz trace identity, tensor symmetries, and the Clausius-Mossotti field.
"""
import numpy as np
import pytest

from oracle import green
from oracle.mvm import dense_operator

pytestmark = pytest.mark.filterwarnings("ignore")

POINTS = [np.array(p) for p in ([0.3, -0.2, 0.45], [0.05, 0.0, 0.0], [0.0, 0.7, -0.1],
                                [-0.4, -0.4, 0.4], [1.3, 0.2, -0.9])]


def _hessian_fd(r, k, eps):
    def g(v):
        return green.scalar_green(np.linalg.norm(v), k)
    H = np.zeros((3, 3), complex)
    for a in range(3):
        for b in range(3):
            ea = np.eye(3)[a] * eps
            eb = np.eye(3)[b] * eps
            H[a, b] = (g(r + ea + eb) - g(r + ea - eb) - g(r - ea + eb) + g(r - ea - eb)) / (4 * eps * eps)
    return H


@pytest.mark.parametrize("k", [2 * np.pi, 7.5, 0.9])
@pytest.mark.parametrize("i", range(len(POINTS)))
def test_dyadic_matches_finite_differences(k, i):
    r = POINTS[i]
    eps = 1e-4 * np.linalg.norm(r)
    ref = k * k * green.scalar_green(np.linalg.norm(r), k) * np.eye(3) + _hessian_fd(r, k, eps)
    got = green.dyadic_k2(r, k)
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("i", range(len(POINTS)))
def test_static_limit(i):
    r = POINTS[i]
    k = 1e-7
    R = np.linalg.norm(r)
    u = r / R
    static = (3 * np.outer(u, u) - np.eye(3)) / (4 * np.pi * R ** 3)
    got = green.dyadic_k2(r, k)
    assert np.abs(got - static).max() <= 1e-9 * np.abs(static).max()


@pytest.mark.parametrize("i", range(len(POINTS)))
def test_trace_identity(i):
    # tr[(I + grad grad/k^2) g] = 3g + lap(g)/k^2 = 2g off the source (Helmholtz).
    r = POINTS[i]
    k = 5.0
    got = np.trace(green.dyadic_k2(r, k))
    ref = 2 * k * k * green.scalar_green(np.linalg.norm(r), k)
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_symmetry_and_parity():
    k, h = 2 * np.pi, 0.05
    d = np.arange(-4, 5)
    DZ, DY, DX = np.meshgrid(d, d, d, indexing="ij")
    K = green.kernel_components(DX, DY, DZ, h, k)
    # K(D) == K(-D)
    for c in green.COMPONENTS:
        assert np.allclose(K[c], K[c][::-1, ::-1, ::-1], rtol=0, atol=1e-15 * np.abs(K[c]).max())
    # per-axis parity: axis order in the arrays is (z, y, x)
    flips = {"x": (slice(None), slice(None), slice(None, None, -1)),
             "y": (slice(None), slice(None, None, -1), slice(None)),
             "z": (slice(None, None, -1), slice(None), slice(None))}
    for c in green.COMPONENTS:
        for ax, fl in flips.items():
            sign = -1.0 if c.count(ax) == 1 else 1.0
            assert np.allclose(K[c][fl], sign * K[c], rtol=0, atol=1e-15 * np.abs(K[c]).max()), (c, ax)
    # the vectorised form equals the 3x3 form entry by entry, and the tensor is symmetric
    for (dx, dy, dz) in [(1, 0, 0), (2, -3, 1), (0, 0, 0), (-4, 4, -2)]:
        M = green.kernel_entry((dx, dy, dz), h, k)
        assert np.allclose(M, M.T, rtol=0, atol=0)
        i = (dz + 4, dy + 4, dx + 4)
        for c, (p, q) in green.PAIRS.items():
            assert abs(K[c][i] - M[p, q]) <= 1e-14 * max(1.0, abs(M[p, q]))


def test_self_term_limits():
    # ka -> 0 gives the depolarisation -1/3 of a sphere
    assert abs(green.self_term(1e-9, 1.0) + 1.0 / 3.0) < 1e-15
    # small-ka expansion: (1 + jx) e^{-jx} = 1 + x^2/2 - j x^3/3 + O(x^4)
    for x in (1e-2, 3e-2, 1e-1):
        h = x / (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)
        s = green.self_term(h, 1.0)
        approx = -1.0 / 3.0 + x * x / 3.0 - 2j * x ** 3 / 9.0
        assert abs(s - approx) < 0.2 * x ** 4


@pytest.mark.parametrize("eps", [4.0, 2.25, 12.25, -1.05 - 5.62j])
def test_clausius_mossotti_single_voxel(eps):
    # One voxel in a static field: E = 3 E_inc / (eps_r + 2).
    eps_r = np.full((1, 1, 1), complex(eps))
    A = dense_operator(eps_r, h=1e-3, k=1e-4)
    E = np.linalg.solve(A, np.array([1.0, 0.0, 0.0], complex))
    assert abs(E[0] - 3.0 / (eps + 2.0)) < 1e-9 * abs(3.0 / (eps + 2.0))
    assert abs(E[1]) < 1e-15 and abs(E[2]) < 1e-15
