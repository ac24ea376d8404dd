"""Oracle: Mie series for a homogeneous sphere (Section III, Figs. 1-2, ref. [30]).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Bohren-Huffman's published method: scattering coefficients a_n, b_n from the
Riccati-Bessel functions of x = k a, with the logarithmic derivative D_n(m x)
taken by downward recurrence, and the amplitude functions S1, S2 from the
angular functions pi_n, tau_n. Bohren-Huffman use exp(-iwt); the refractive
index is therefore m = sqrt(conj(eps_r)) for an eps_r written in this
project's exp(+jwt) convention.

Pinned by tests/test_oracle_mie.py: Qext == Qsca for a lossless sphere (the
optical theorem, which ties S(0) to the coefficient sums), the Rayleigh limit
(8/3) x^4 |(m^2-1)/(m^2+2)|^2, S1(0) == S2(0), and zero scattering at m = 1.
"""
import numpy as np
from scipy.special import spherical_jn, spherical_yn


def coefficients(m, x):
    nstop = int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    mx = m * x
    nmx = int(max(nstop, abs(mx))) + 16
    D = np.zeros(nmx + 1, complex)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    n = np.arange(0, nstop + 1)
    psi = x * spherical_jn(n, x)
    xi = x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))
    nn = n[1:]
    Dn = D[1:nstop + 1]
    ta = Dn / m + nn / x
    tb = m * Dn + nn / x
    a = (ta * psi[1:] - psi[:-1]) / (ta * xi[1:] - xi[:-1])
    b = (tb * psi[1:] - psi[:-1]) / (tb * xi[1:] - xi[:-1])
    return a, b


def efficiencies(m, x):
    a, b = coefficients(m, x)
    n = np.arange(1, a.size + 1)
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    qext = 2.0 / x ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    return qext, qsca


def amplitudes(m, x, theta):
    a, b = coefficients(m, x)
    mu = np.cos(np.atleast_1d(theta))
    S1 = np.zeros(mu.shape, complex)
    S2 = np.zeros(mu.shape, complex)
    pi_prev = np.zeros_like(mu)
    pi_n = np.ones_like(mu)
    for n in range(1, a.size + 1):
        tau_n = n * mu * pi_n - (n + 1) * pi_prev
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_n + b[n - 1] * tau_n)
        S2 += f * (a[n - 1] * tau_n + b[n - 1] * pi_n)
        pi_next = ((2 * n + 1) * mu * pi_n - (n + 1) * pi_prev) / n
        pi_prev, pi_n = pi_n, pi_next
    return S1, S2


def rcs_eplane(eps_r, radius, k, theta):
    """E-plane bistatic RCS 4 pi |S2(theta)|^2 / k^2 for x-polarised incidence along +z."""
    m = np.sqrt(np.conj(complex(eps_r)))
    _, S2 = amplitudes(m, k * radius, theta)
    return 4.0 * np.pi * np.abs(S2) ** 2 / k ** 2
