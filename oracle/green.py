"""Oracle: scalar and dyadic Green's function, self term (Section II.A, Eq. 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Pinned by tests/test_oracle_green.py against: central finite differences of
the scalar Green's function (the dyadic is (I + grad grad / k^2) g), its
static limit, the trace identity tr(k^2 G) = 2 k^2 g, per-axis parities, the
ka -> 0 limit of the self term and the Clausius-Mossotti field of one voxel.
"""
import numpy as np


def scalar_green(R, k):
    """g(R) = exp(-j k R) / (4 pi R), the free-space Green's function after Eq. 1."""
    return np.exp(-1j * k * R) / (4.0 * np.pi * R)


def dyadic_k2(r, k):
    """k^2 G(r) for r != 0, as a 3x3 complex matrix (Eq. 1, G = (I + grad grad/k^2) g).

    Differentiating g twice gives
      k^2 G = g [ (k^2 - jk/R - 1/R^2) I + (-k^2 + 3jk/R + 3/R^2) rhat rhat ].
    """
    r = np.asarray(r, dtype=float)
    R = np.sqrt(np.sum(r * r))
    rh = r / R
    g = scalar_green(R, k)
    a = k * k - 1j * k / R - 1.0 / (R * R)
    b = -k * k + 3j * k / R + 3.0 / (R * R)
    return g * (a * np.eye(3) + b * np.outer(rh, rh))


def equivalent_radius(h):
    """Radius of the sphere with the volume of one h^3 voxel."""
    return h * (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)


def self_term(h, k):
    """Self coefficient s_self of K(0) = s_self I (equivalent-sphere method).

    The paper does not state its singular-integral treatment; this is the
    Livesay-Chen equivalent-sphere result: the principal value of
    k^2 int G over a sphere of radius a is (2/3)[(1 + jka) e^{-jka} - 1] I,
    and the source dyadic of a sphere adds -I/3.
    """
    ka = k * equivalent_radius(h)
    return (2.0 / 3.0) * ((1.0 + 1j * ka) * np.exp(-1j * ka) - 1.0) - 1.0 / 3.0


# component order of the six unique entries of the symmetric tensor
COMPONENTS = ("xx", "xy", "xz", "yy", "yz", "zz")
PAIRS = {"xx": (0, 0), "xy": (0, 1), "xz": (0, 2), "yy": (1, 1), "yz": (1, 2), "zz": (2, 2)}


def kernel_entry(d, h, k):
    """K(D) for an integer lattice offset D = (dx, dy, dz): the 3x3 matrix coupling
    voxel j to voxel i = j + D (Eqs. 1 and 4 with pulse basis, point collocation)."""
    d = np.asarray(d, dtype=float)
    if not np.any(d):
        return self_term(h, k) * np.eye(3, dtype=complex)
    return h ** 3 * dyadic_k2(d * h, k)


def kernel_components(DX, DY, DZ, h, k):
    """Vectorised K(D): dict of the six components on integer offset arrays.

    Written out from the same closed form as dyadic_k2 (checked against it
    entry by entry in the tests)."""
    DX = np.asarray(DX, float)
    DY = np.asarray(DY, float)
    DZ = np.asarray(DZ, float)
    zero = (DX == 0) & (DY == 0) & (DZ == 0)
    rx, ry, rz = DX * h, DY * h, DZ * h
    R = np.sqrt(rx * rx + ry * ry + rz * rz)
    Rs = np.where(zero, 1.0, R)
    g = scalar_green(Rs, k)
    a = k * k - 1j * k / Rs - 1.0 / (Rs * Rs)
    b = -k * k + 3j * k / Rs + 3.0 / (Rs * Rs)
    u = (rx / Rs, ry / Rs, rz / Rs)
    out = {}
    for name, (p, q) in PAIRS.items():
        val = g * b * u[p] * u[q]
        if p == q:
            val = val + g * a
        val = h ** 3 * val
        diag = self_term(h, k) if p == q else 0.0
        out[name] = np.where(zero, diag, val)
    return out


# ---------------------------------------------------------------- near-field variant
# The paper does not say how near-neighbour couplings are integrated; the build's
# primary reading samples K at the source voxel's centre (kernel_entry). The
# variant below integrates k^2 G over the source voxel instead for offsets with
# max |D| <= radius (D != 0): K(D) = int_{cube of side h centred at D h} k^2 G(r) d^3 r,
# by tensor Gauss-Legendre quadrature. The integrand is smooth on those cubes
# (the nearest point of the cube at D != 0 is at least h/2 from the origin).
# Pinned by tests/test_oracle_near.py: convergence in q, an adaptive cubature of
# scipy, the cube mean of a Helmholtz solution (f(c) (1 - (kh)^2 / 24) + O(h^4)),
# parities and reciprocity.

def k2G_at(rx, ry, rz, k):
    """The six components of k^2 G(r) (Eq. 1) at arrays of points r != 0."""
    R = np.sqrt(rx * rx + ry * ry + rz * rz)
    g = scalar_green(R, k)
    a = k * k - 1j * k / R - 1.0 / (R * R)
    b = -k * k + 3j * k / R + 3.0 / (R * R)
    u = (rx / R, ry / R, rz / R)
    return {name: g * b * u[p] * u[q] + (g * a if p == q else 0.0) for name, (p, q) in PAIRS.items()}


def cube_kernel(d, h, k, q):
    """int over the cube of side h centred at d h of k^2 G, six components (d integer, != 0)."""
    t, w = np.polynomial.legendre.leggauss(q)
    x = (d[0] + 0.5 * t) * h
    y = (d[1] + 0.5 * t) * h
    z = (d[2] + 0.5 * t) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :] / 8.0    # mean over the cube
    vals = k2G_at(X, Y, Z, k)
    return {name: h ** 3 * np.sum(W * v) for name, v in vals.items()}


def kernel_components_near(DX, DY, DZ, h, k, radius, q):
    """kernel_components with cube-integrated entries for 0 < max|D| <= radius."""
    out = kernel_components(DX, DY, DZ, h, k)
    DX = np.asarray(DX)
    DY = np.asarray(DY)
    DZ = np.asarray(DZ)
    rng = range(-radius, radius + 1)
    for dz in rng:
        for dy in rng:
            for dx in rng:
                if dx == 0 and dy == 0 and dz == 0:
                    continue
                sel = (DX == dx) & (DY == dy) & (DZ == dz)
                if not np.any(sel):
                    continue
                vals = cube_kernel((dx, dy, dz), h, k, q)
                for name in COMPONENTS:
                    out[name] = np.where(sel, vals[name], out[name])
    return out
