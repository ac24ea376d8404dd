"""Oracle: the VIE operator y = A x = x - G(chi x), dense and by FFT (Section II, Eqs. 4, 6).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Vectors are complex128 arrays shaped [3, nz, ny, nx] (components x, y, z;
x fastest). The dense form is the literal double sum and is used for grids of
at most 512 voxels; the FFT form is the Toeplitz-to-circulant embedding the
paper uses to accelerate every MVM (Section I: O(N log N) time, O(N) memory),
with numpy's FFT as the library primitive.

Pinned by tests/test_oracle_mvm.py: FFT form == dense form (brute force) on
cubic and ragged grids, reciprocity of the dense G, rotation and translation
covariance, Clausius-Mossotti for one voxel.
"""
import numpy as np

from .green import COMPONENTS, PAIRS, kernel_components, kernel_components_near


def component_name(a, b):
    """Name of the stored entry K_ab = K_ba of the symmetric tensor."""
    p, q = min(a, b), max(a, b)
    return [c for c in COMPONENTS if PAIRS[c] == (p, q)][0]


def voxel_index_coords(n):
    """Integer coordinates (x, y, z) of every voxel, flattened in [z, y, x] order."""
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def _components(DX, DY, DZ, h, k, near):
    if near is None:
        return kernel_components(DX, DY, DZ, h, k)
    return kernel_components_near(DX, DY, DZ, h, k, near[0], near[1])


def dense_G(n, h, k, near=None):
    """The 3N x 3N matrix G with G[(a,i),(b,j)] = K_ab(p_i - p_j) (Eq. 4 discretised).
    near = (radius, q): cube-integrated entries for 0 < max|D| <= radius (green.cube_kernel)."""
    X, Y, Z = voxel_index_coords(n)
    N = X.size
    DX = X[:, None] - X[None, :]
    DY = Y[:, None] - Y[None, :]
    DZ = Z[:, None] - Z[None, :]
    K = _components(DX, DY, DZ, h, k, near)
    G = np.zeros((3 * N, 3 * N), complex)
    for name, (p, q) in PAIRS.items():
        G[p * N:(p + 1) * N, q * N:(q + 1) * N] = K[name]
        if p != q:
            G[q * N:(q + 1) * N, p * N:(p + 1) * N] = K[name]
    return G


def dense_operator(eps_r, h, k, near=None):
    """A = I - G diag(chi) as a dense matrix (literal double sum of Eq. 4)."""
    nz, ny, nx = eps_r.shape
    chi = (eps_r - 1.0).ravel()
    G = dense_G((nx, ny, nz), h, k, near)
    D = np.tile(chi, 3)
    return np.eye(G.shape[0], dtype=complex) - G * D[None, :]


def default_padding(n):
    """Padded FFT length per axis: 2n (any M >= 2n - 1 embeds the Toeplitz sum)."""
    return tuple(2 * v for v in n)


def wrapped_offsets(n_axis, M_axis):
    """Lattice offset stored at each circulant slot, and whether the slot is used."""
    i = np.arange(M_axis)
    d = np.where(i < n_axis, i, i - M_axis)
    used = (i < n_axis) | (i > M_axis - n_axis)
    return d, used


def kernel_array(n, M, h, k, near=None):
    """The six components of K on the padded M grid, offsets wrapped circularly.

    Slot m along an axis holds offset m for m < n and m - M for m > M - n;
    the remaining slots (e.g. m = n when M = 2n) never meet a product of two
    in-grid voxels and are set to zero.
    """
    dx, ux = wrapped_offsets(n[0], M[0])
    dy, uy = wrapped_offsets(n[1], M[1])
    dz, uz = wrapped_offsets(n[2], M[2])
    DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
    used = uz[:, None, None] & uy[None, :, None] & ux[None, None, :]
    K = _components(DX, DY, DZ, h, k, near)
    return {c: np.where(used, K[c], 0.0) for c in COMPONENTS}


class FFTOperator:
    """A x = x - G(chi x) through the circulant embedding (Section I; Eq. 4).

    mask (bool [nz, ny, nx], optional) restricts both the contrast and the
    output to a voxel subset: this is the diagonal block A_k of Eq. 10/11,
    acting on vectors supported on the subset.
    """

    def __init__(self, eps_r, h, k, M=None, mask=None, near=None):
        nz, ny, nx = eps_r.shape
        self.n = (nx, ny, nz)
        self.M = tuple(M) if M is not None else default_padding(self.n)
        chi = eps_r - 1.0
        if mask is not None:
            chi = np.where(mask, chi, 0.0)
        self.chi = chi
        self.mask = mask
        K = kernel_array(self.n, self.M, h, k, near)
        s = (self.M[2], self.M[1], self.M[0])
        self.Khat = {c: np.fft.fftn(K[c], s=s, axes=(0, 1, 2)) for c in COMPONENTS}

    def G(self, w):
        """u = sum_j K(i - j) w_j for all in-grid voxels i (zero-padded circular convolution)."""
        nx, ny, nz = self.n
        s = (self.M[2], self.M[1], self.M[0])
        W = [np.fft.fftn(w[c], s=s, axes=(0, 1, 2)) for c in range(3)]
        u = np.empty((3, nz, ny, nx), complex)
        for a in range(3):
            U = np.zeros(s, complex)
            for b in range(3):
                U += self.Khat[component_name(a, b)] * W[b]
            u[a] = np.fft.ifftn(U)[:nz, :ny, :nx]
        return u

    def apply(self, x):
        y = x - self.G(self.chi[None] * x)
        if self.mask is not None:
            y = np.where(self.mask[None], y, 0.0)
        return y

    __call__ = apply


def apply_dense(A, x):
    return (A @ x.ravel()).reshape(x.shape)
