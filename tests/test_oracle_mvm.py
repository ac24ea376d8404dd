"""Pins for oracle/mvm.py (Eq. 4 discretised; Section I's FFT-accelerated MVM).

Brute force: the FFT MVM equals the literal dense double sum. Structure:
reciprocity of G, translation and rotation/reflection covariance (these catch
swapped or mis-signed tensor components and wrong padding offsets).
"""
import numpy as np
import pytest

from oracle import mvm
from paper_2501_13512_gb300 import inputs

K0 = 2 * np.pi
H = 0.05


@pytest.mark.parametrize("n", [(5, 7, 3), (4, 4, 4), (8, 8, 8), (1, 6, 2), (3, 1, 1)])
def test_fft_equals_dense(n):
    eps_r, _, x = inputs.random_case(n, seed=sum(n))
    A = mvm.dense_operator(eps_r, H, K0)
    yd = mvm.apply_dense(A, x)
    yf = mvm.FFTOperator(eps_r, H, K0)(x)
    assert np.linalg.norm(yf - yd) <= 1e-12 * np.linalg.norm(yd)


@pytest.mark.parametrize("M", [(9, 13, 5), (16, 16, 8), (10, 14, 6)])
def test_padding_invariance(M):
    # every M >= 2n - 1 gives the same Toeplitz product
    eps_r, _, x = inputs.random_case((5, 7, 3), seed=4)
    y0 = mvm.FFTOperator(eps_r, H, K0)(x)
    y1 = mvm.FFTOperator(eps_r, H, K0, M=M)(x)
    assert np.linalg.norm(y1 - y0) <= 1e-13 * np.linalg.norm(y0)


def test_reciprocity():
    G = mvm.dense_G((4, 3, 5), H, K0)
    assert np.abs(G - G.T).max() <= 1e-15 * np.abs(G).max()


def test_translation_covariance():
    rng = np.random.default_rng(7)
    sub = (3, 4, 2)
    chi_s = rng.normal(size=sub[::-1]) + 1j * rng.normal(size=sub[::-1])
    x_s = rng.normal(size=(3,) + sub[::-1]) + 1j * rng.normal(size=(3,) + sub[::-1])
    big = (9, 8, 7)
    outs = []
    for off in [(0, 0, 0), (5, 3, 4), (2, 4, 1)]:
        eps = np.ones(big[::-1], complex)
        x = np.zeros((3,) + big[::-1], complex)
        sl = (slice(off[2], off[2] + sub[2]), slice(off[1], off[1] + sub[1]), slice(off[0], off[0] + sub[0]))
        eps[sl] = 1 + chi_s
        x[(slice(None),) + sl] = x_s
        y = mvm.FFTOperator(eps, H, K0)(x)
        outs.append(y[(slice(None),) + sl])
    for o in outs[1:]:
        assert np.linalg.norm(o - outs[0]) <= 1e-13 * np.linalg.norm(outs[0])


def _rot_z(f):
    # scalar field rotated by +90 deg about z: f'(x, y) = f(y, -x) on a centred cubic grid
    return f[..., ::-1, :].swapaxes(-1, -2)


def test_rotation_covariance():
    n = 6
    eps_r, _, x = inputs.random_case((n, n, n), seed=11)
    y = mvm.FFTOperator(eps_r, H, K0)(x)
    eps_rot = _rot_z(eps_r)
    # vectors rotate too: (vx, vy, vz) -> (-vy, vx, vz)
    x_rot = np.stack([-_rot_z(x[1]), _rot_z(x[0]), _rot_z(x[2])])
    y_rot = np.stack([-_rot_z(y[1]), _rot_z(y[0]), _rot_z(y[2])])
    got = mvm.FFTOperator(eps_rot, H, K0)(x_rot)
    assert np.linalg.norm(got - y_rot) <= 1e-13 * np.linalg.norm(y_rot)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reflection_covariance(axis):
    eps_r, _, x = inputs.random_case((5, 4, 3), seed=12)
    y = mvm.FFTOperator(eps_r, H, K0)(x)
    arr_ax = 2 - axis  # array axis of spatial axis (x->2, y->1, z->0)
    fl = lambda f: np.flip(f, axis=arr_ax)
    sgn = np.ones(3)
    sgn[axis] = -1
    x_m = np.stack([sgn[c] * fl(x[c]) for c in range(3)])
    y_m = np.stack([sgn[c] * fl(y[c]) for c in range(3)])
    got = mvm.FFTOperator(fl(eps_r), H, K0)(x_m)
    assert np.linalg.norm(got - y_m) <= 1e-13 * np.linalg.norm(y_m)


def test_masked_operator_is_principal_submatrix():
    # A_k of Eq. 11: rows and columns of A on a voxel subset
    eps_r, _, x = inputs.random_case((4, 3, 3), seed=5)
    mask = np.random.default_rng(1).uniform(size=eps_r.shape) < 0.6
    A = mvm.dense_operator(eps_r, H, K0)
    idx = np.nonzero(np.tile(mask.ravel(), 3))[0]
    xs = np.where(mask[None], x, 0.0)
    ref = np.zeros(x.size, complex)
    ref[idx] = A[np.ix_(idx, idx)] @ xs.ravel()[idx]
    got = mvm.FFTOperator(eps_r, H, K0, mask=mask)(xs)
    assert np.linalg.norm(got.ravel() - ref) <= 1e-12 * np.linalg.norm(ref)
