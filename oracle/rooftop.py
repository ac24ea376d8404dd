"""Oracle: the paper's rooftop-basis / pulse-testing discretisation of the VIE (Section II.A, Eqs. 5-9).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The unknown of Eqs. 4-9 is the polarisation current J. Written in w = J / (j w eps0) (units of E;
w = chi E in the continuum), Eq. 4 with Eq. 1 reads

    w / chi - k^2 int g w dv' - grad int g div' w dv' = E_inc,

the three pieces of L^c_ii (contrast term and vector potential, Eq. 8) and L^q_ij (scalar potential,
Eq. 9, read as acting on w_j), with the sign of Eq. 4 (E_tot = E_inc + E_s, Eq. 3). Discretisation
on the uniform grid of cells of edge h (the readings the paper leaves open are listed here and in
the design doc):

* Basis (Eq. 5): component a of w is expanded in rooftops T_(a,c): the hat of half-width h along
  axis a centred on the face between cell c and cell c + e_a, times the pulse of the cell section
  across a. Only faces with both neighbouring cells inside the grid and non-air carry a rooftop
  (the normal current vanishes on the object's surface; the boundary charge is the divergence of the
  last rooftops inside).
* Testing: the a-equation is tested with the pulse on the dual cell centred on the face (Eq. 6).
  The contrast term gives the rooftop/pulse Gram matrix with the face's two cells:
  (3/8)(1/chi_c + 1/chi_(c+e_a)) on the face, (1/8)/chi_c and (1/8)/chi_(c+e_a) on its two
  neighbours along a. Smooth terms (incident field, vector potential) are taken at the face centre.
  The gradient of the scalar potential, tested on the dual cell, is the difference of the cell-centre
  potentials divided by h.
* Charges: div w of the rooftops is constant per cell: rho_c = sum_b (w_(b,c) - w_(b,c-e_b)) / h.
* Integrals: int_cell g = h^3 g(|D| h) at cell-centre offsets D != 0 (the midpoint rule, the same for
  rooftops, whose integral is h^3); for D = 0 the integral over the sphere of volume h^3,
  [(1 + jka) e^{-jka} - 1] / k^2, a = h (3/4pi)^(1/3).

Operator on the face unknowns, components a, b:

    (A w)_(a,c) = [M_chi w]_(a,c) + sum_(b,c') K_ab(c - c') w_(b,c'),
    K_ab(D) = -k^2 delta_ab gh(D) - [gh(D + e_a) - gh(D + e_a - e_b) - gh(D) + gh(D - e_b)] / h^2,

with gh the cell integral of g above. K_ab(D) = K_ba(-D) (reciprocity), so A is complex symmetric.
Vectors: complex128 [3, nz, ny, nx], entry (a, c) on the face between cell c and c + e_a; inactive
faces hold 0.

Pinned by tests/test_oracle_rooftop.py: dense literal operator == FFT operator, A = A^T, the Born
limit (chi -> 0: w -> chi E_inc up to the Gram smoothing), translation covariance, and the bistatic
RCS of the sphere converging to the Mie series with refinement.
"""
import numpy as np

from .green import equivalent_radius, scalar_green
from .solve import voxel_positions


def cell_green(D, h, k):
    """gh(D): the integral of g over the source cell at integer cell offset D (arrays of offsets)."""
    DX, DY, DZ = (np.asarray(d, float) for d in D)
    R = h * np.sqrt(DX * DX + DY * DY + DZ * DZ)
    zero = R == 0
    Rs = np.where(zero, 1.0, R)
    val = h ** 3 * scalar_green(Rs, k)
    ka = k * equivalent_radius(h)
    self_val = ((1.0 + 1j * ka) * np.exp(-1j * ka) - 1.0) / (k * k)
    return np.where(zero, self_val, val)


def active_faces(eps_r):
    """Boolean [3, nz, ny, nx]: face (a, c) carries a rooftop (cells c and c + e_a in the grid, non-air)."""
    solid = (eps_r - 1.0) != 0
    act = np.zeros((3,) + eps_r.shape, bool)
    act[0, :, :, :-1] = solid[:, :, :-1] & solid[:, :, 1:]
    act[1, :, :-1, :] = solid[:, :-1, :] & solid[:, 1:, :]
    act[2, :-1, :, :] = solid[:-1, :, :] & solid[1:, :, :]
    return act


def face_positions(n, h):
    """Coordinates (x, y, z) of the face centres of each component, [3][3][nz, ny, nx]."""
    X, Y, Z = voxel_positions(n, h)
    return [(X + 0.5 * h, Y, Z), (X, Y + 0.5 * h, Z), (X, Y, Z + 0.5 * h)]


def kernel_ab(D, a, b, h, k):
    """K_ab(D) of the module docstring at integer face offsets D = (DX, DY, DZ) (arrays)."""
    e = np.eye(3, dtype=int)
    D = [np.asarray(d) for d in D]
    sh = lambda v: [D[i] + v[i] for i in range(3)]
    T = (cell_green(sh(e[a]), h, k) - cell_green(sh(e[a] - e[b]), h, k)
         - cell_green(D, h, k) + cell_green(sh(-e[b]), h, k)) / (h * h)
    out = -T
    if a == b:
        out = out - k * k * cell_green(D, h, k)
    return out


def gram_apply(w, eps_r, act):
    """[M_chi w]: the contrast term tested on the dual cells (rooftop/pulse Gram with 1/chi per half)."""
    chi = eps_r - 1.0
    inv = np.where(chi != 0, 1.0 / np.where(chi != 0, chi, 1.0), 0.0)
    out = np.zeros_like(w)
    for a in range(3):
        ax = 2 - a                               # array axis of component a's direction
        wa = np.where(act[a], w[a], 0.0)
        lo = inv                                  # cell c (the face's lower cell)
        hi = np.roll(inv, -1, axis=ax)            # cell c + e_a (wrap only reaches inactive faces)
        prev = np.roll(wa, 1, axis=ax)            # w_(a, c - e_a)
        nxt = np.roll(wa, -1, axis=ax)            # w_(a, c + e_a)
        idx = [slice(None)] * 3
        idx[ax] = 0
        prev[tuple(idx)] = 0.0
        idx[ax] = -1
        nxt[tuple(idx)] = 0.0
        out[a] = 0.375 * (lo + hi) * wa + 0.125 * lo * prev + 0.125 * hi * nxt
    return np.where(act, out, 0.0)


def dense_operator(eps_r, h, k):
    """The operator on the active faces as a dense matrix, by the literal sums (small grids)."""
    nz, ny, nx = eps_r.shape
    act = active_faces(eps_r)
    idx = np.argwhere(act)                        # rows (a, z, y, x)
    m = len(idx)
    A = np.zeros((m, m), complex)
    for i, (a, z, y, x) in enumerate(idx):
        for j, (b, z2, y2, x2) in enumerate(idx):
            A[i, j] = kernel_ab(([x - x2], [y - y2], [z - z2]), a, b, h, k)[0]
    # Gram part column by column (unit vectors through gram_apply)
    for j, (b, z2, y2, x2) in enumerate(idx):
        e = np.zeros((3, nz, ny, nx), complex)
        e[b, z2, y2, x2] = 1.0
        col = gram_apply(e, eps_r, act)
        A[:, j] += col[act]
    return A, act


class RooftopOperator:
    """A w through the circulant embedding of each K_ab (padded length 2n per axis)."""

    def __init__(self, eps_r, h, k):
        nz, ny, nx = eps_r.shape
        self.eps_r = eps_r
        self.n = (nx, ny, nz)
        self.act = active_faces(eps_r)
        M = (2 * nx, 2 * ny, 2 * nz)
        self.M = M
        d = [np.where(np.arange(Mi) < ni, np.arange(Mi), np.arange(Mi) - Mi) for Mi, ni in zip(M, self.n)]
        used = [(np.arange(Mi) < ni) | (np.arange(Mi) > Mi - ni) for Mi, ni in zip(M, self.n)]
        DZ, DY, DX = np.meshgrid(d[2], d[1], d[0], indexing="ij")
        U = used[2][:, None, None] & used[1][None, :, None] & used[0][None, None, :]
        s = (M[2], M[1], M[0])
        self.Khat = [[np.fft.fftn(np.where(U, kernel_ab((DX, DY, DZ), a, b, h, k), 0.0), s=s, axes=(0, 1, 2))
                      for b in range(3)]
                     for a in range(3)]

    def apply(self, w):
        nx, ny, nz = self.n
        s = (self.M[2], self.M[1], self.M[0])
        w = np.where(self.act, w, 0.0)
        W = [np.fft.fftn(w[b], s=s, axes=(0, 1, 2)) for b in range(3)]
        u = np.empty_like(w)
        for a in range(3):
            U = sum(self.Khat[a][b] * W[b] for b in range(3))
            u[a] = np.fft.ifftn(U)[:nz, :ny, :nx]
        return np.where(self.act, gram_apply(w, self.eps_r, self.act) + u, 0.0)

    __call__ = apply


def incident(n, h, k, khat, pol, act):
    """E_inc sampled at the face centres of each component (0 on inactive faces)."""
    F = face_positions(n, h)
    out = np.zeros((3,) + tuple(n[::-1]), complex)
    for a in range(3):
        X, Y, Z = F[a]
        out[a] = pol[a] * np.exp(-1j * k * (khat[0] * X + khat[1] * Y + khat[2] * Z))
    return np.where(act, out, 0.0)


def far_field_rcs(w, n, h, k, rhat):
    """Bistatic RCS of the rooftop solution: P(u) = sum_faces w h^3 exp(j k u . r_face) per component."""
    F = face_positions(n, h)
    rhat = np.atleast_2d(rhat)
    out = np.empty(rhat.shape[0])
    for i, u in enumerate(rhat):
        P = np.array([np.sum(w[a] * np.exp(1j * k * (u[0] * F[a][0] + u[1] * F[a][1] + u[2] * F[a][2])))
                      for a in range(3)]) * h ** 3
        Pt = P - u * np.dot(u, P)
        out[i] = k ** 4 / (4 * np.pi) * np.real(np.vdot(Pt, Pt))
    return out
