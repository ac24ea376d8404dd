"""Seeded synthetic workloads (geometry + incidence parameters).

This module is shared by the CUDA path, the tests, the bench and the CPU
oracle. It holds none of the method's arithmetic: it only draws voxel
permittivities, block partitions and incidence parameters. The incident field
itself, the Green's kernel, the FFTs and the solver are computed separately by
each side.

Conventions (Section II.A):
  * grid (nx, ny, nz), voxel edge h, x fastest; arrays are indexed [z, y, x];
  * voxel centre r = (i + 1/2) h - centre of the grid, per axis;
  * time convention exp(+j w t): a lossy medium has Im(eps_r) < 0;
  * block_id[z, y, x] = k >= 0 puts the voxel in subdomain k of the
    block-diagonal preconditioner (Eq. 10); -1 means no block (identity there).

Workloads (synthetic stand-ins for the paper's studies, Section III):
  * sphere:      dielectric sphere, radius 0.25 lambda0, eps_r 4, 16^3 grid,
                 h = lambda0/32 (validation against the Mie series, Figs. 1-2);
  * metasurface: 16 x 16 cylindrical pillars (eps_r 6.25) on a 256x256x16 grid,
                 h = lambda0/20, period 16 voxels, radius ~ U[0.15, 0.4] period,
                 one block per pillar (Section III.A, Eq. 12);
  * solar_cell:  128x128x64 grid, h = 5 nm, lambda0 = 600 nm, absorber slab
                 eps_r 3 - 0.3j (z in [12, 52)), 16 Drude-like spheres
                 eps_r -15 - 1j, radius ~ U[6, 12] voxels; one block per sphere
                 plus the slab split in x into 4 blocks (Section III.B);
  * blob:        cubic grid with a smoothed random level-set blob,
                 eps_r ~ U[2, 8], random incidence (batched instances);
  * serving_draws: a stream of solve requests on n^3 grids (n from a size mix),
                 metasurface tiles and solar-cell slabs rescaled to n, h = 10 nm,
                 wavelengths on a 10 nm grid, tilted plane waves.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    n: tuple            # (nx, ny, nz)
    h: float            # voxel edge, same length unit as lambda0
    lambda0: float
    eps_r: np.ndarray   # complex128 [nz, ny, nx]
    block_id: np.ndarray  # int32 [nz, ny, nx]
    khat: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, 1.0]))
    pol: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.0, 0.0], complex))
    inner_tol: float = 1e-2
    outer_tol: float = 1e-6
    use_precond: bool = True

    @property
    def k0(self) -> float:
        return 2.0 * np.pi / self.lambda0

    @property
    def nvox(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])


def voxel_centres(n, h):
    """Voxel-centre coordinates (x, y, z), each shaped [nz, ny, nx]."""
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) * h - 0.5 * nx * h
    y = (np.arange(ny) + 0.5) * h - 0.5 * ny * h
    z = (np.arange(nz) + 0.5) * h - 0.5 * nz * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def sphere(n=16, eps=4.0, radius_wl=0.25, voxels_per_wl=32, lambda0=1.0):
    """Dielectric sphere centred in an n^3 grid (unpreconditioned solve)."""
    h = lambda0 / voxels_per_wl
    X, Y, Z = voxel_centres((n, n, n), h)
    inside = X**2 + Y**2 + Z**2 <= (radius_wl * lambda0) ** 2
    eps_r = np.where(inside, complex(eps), 1.0 + 0.0j).astype(np.complex128)
    bid = np.full((n, n, n), -1, np.int32)
    return Workload("sphere", (n, n, n), h, lambda0, eps_r, bid, use_precond=False)


def sphere_radius_voxels(n, radius, eps, h, lambda0=1.0):
    """Sphere of a radius given in length units, for resolution sweeps."""
    X, Y, Z = voxel_centres((n, n, n), h)
    inside = X**2 + Y**2 + Z**2 <= radius**2
    eps_r = np.where(inside, complex(eps), 1.0 + 0.0j).astype(np.complex128)
    bid = np.full((n, n, n), -1, np.int32)
    return Workload("sphere", (n, n, n), h, lambda0, eps_r, bid, use_precond=False)


def metasurface(cells=16, period=16, nz=16, eps=6.25, seed=0, voxels_per_wl=20,
                lambda0=1.0, focus=False, focal_wl=10.0, block_cells=0):
    """Array of cylindrical pillars, one preconditioner block per pillar.

    The radius of pillar (a, b) is drawn from U[0.15, 0.4] * period (seeded).
    With focus=True it follows the hyperbolic focusing profile of Eq. 12
    instead: Phi = k (sqrt(x^2 + y^2 + d^2) - d), r = P (0.15 + 0.25 frac(Phi/2pi)).
    block_cells = m > 0 instead makes every m x m group of unit cells one block,
    air voxels included (the unit-cell division of Section III.A and the coarser
    divisions of Table 2's trade-off).
    """
    h = lambda0 / voxels_per_wl
    nx = ny = cells * period
    rng = np.random.default_rng(seed)
    if focus:
        k = 2.0 * np.pi / lambda0
        d = focal_wl * lambda0
        c = (np.arange(cells) + 0.5 - 0.5 * cells) * period * h
        CY, CX = np.meshgrid(c, c, indexing="ij")
        phi = k * (np.sqrt(CX**2 + CY**2 + d**2) - d)
        radii = period * (0.15 + 0.25 * np.mod(phi / (2 * np.pi), 1.0))
    else:
        radii = rng.uniform(0.15, 0.4, size=(cells, cells)) * period
    eps_r = np.ones((nz, ny, nx), np.complex128)
    bid = np.full((nz, ny, nx), -1, np.int32)
    li = np.arange(period) + 0.5 - 0.5 * period
    LY, LX = np.meshgrid(li, li, indexing="ij")
    for a in range(cells):          # a: y cell index
        for b in range(cells):      # b: x cell index
            disk = LX**2 + LY**2 <= radii[a, b] ** 2
            ys = slice(a * period, (a + 1) * period)
            xs = slice(b * period, (b + 1) * period)
            eps_r[:, ys, xs][:, disk] = eps
            bid[:, ys, xs][:, disk] = a * cells + b
    if block_cells > 0:
        m = int(block_cells)
        cy = np.arange(ny) // (period * m)
        cx = np.arange(nx) // (period * m)
        nbx = (cells + m - 1) // m
        bid = np.broadcast_to((cy[:, None] * nbx + cx[None, :]).astype(np.int32), (nz, ny, nx)).copy()
    return Workload("metasurface", (nx, ny, nz), h, lambda0, eps_r, bid,
                    inner_tol=1e-2, outer_tol=1e-6, use_precond=True)


def solar_cell(nx=128, ny=128, nz=64, h=5.0, lambda0=600.0, seed=0,
               eps_slab=3.0 - 0.3j, eps_metal=-15.0 - 1.0j, slab=(12, 52),
               lattice=32, rmin=6, rmax=12, xsplit=4):
    """Absorber slab with an embedded lattice of metal nanospheres."""
    rng = np.random.default_rng(seed)
    eps_r = np.ones((nz, ny, nx), np.complex128)
    bid = np.full((nz, ny, nx), -1, np.int32)
    z0, z1 = slab
    eps_r[z0:z1] = eps_slab
    zc = 0.5 * (z0 + z1)
    Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5,
                          np.arange(nx) + 0.5, indexing="ij")
    cy, cx = ny // lattice, nx // lattice
    k = 0
    for a in range(cy):
        for b in range(cx):
            r = rng.uniform(rmin, rmax)
            jit = max(0.0, 0.5 * lattice - r - 1.0)
            jx, jy = rng.uniform(-jit, jit, size=2)
            px = (b + 0.5) * lattice + jx
            py = (a + 0.5) * lattice + jy
            ball = (X - px) ** 2 + (Y - py) ** 2 + (Z - zc) ** 2 <= r * r
            eps_r[ball] = eps_metal
            bid[ball] = k
            k += 1
    nsph = k
    w = nx // xsplit
    for s in range(xsplit):
        part = np.zeros((nz, ny, nx), bool)
        part[z0:z1, :, s * w:(s + 1) * w] = True
        part &= bid < 0
        bid[part] = nsph + s
    return Workload("solar_cell", (nx, ny, nz), h, lambda0, eps_r, bid,
                    inner_tol=1e-2, outer_tol=1e-6, use_precond=True)


def _smooth(field3, sigma):
    """Separable Gaussian smoothing with periodic wrap (input drawing only)."""
    out = field3
    r = int(np.ceil(3 * sigma))
    t = np.arange(-r, r + 1)
    w = np.exp(-0.5 * (t / sigma) ** 2)
    w /= w.sum()
    for ax in range(3):
        acc = np.zeros_like(out)
        for ti, wi in zip(t, w):
            acc += wi * np.roll(out, ti, axis=ax)
        out = acc
    return out


def random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def blob(n=16, seed=0, voxels_per_wl=20, lambda0=1.0, fill=0.4):
    """Smoothed random level-set blob inside the inscribed sphere of an n^3 grid."""
    rng = np.random.default_rng(seed)
    h = lambda0 / voxels_per_wl
    noise = _smooth(rng.normal(size=(n, n, n)), max(1.0, n / 8))
    X, Y, Z = voxel_centres((n, n, n), h)
    ball = X**2 + Y**2 + Z**2 <= (0.5 * n * h) ** 2
    vals = noise[ball]
    thr = np.quantile(vals, 1.0 - fill)
    inside = ball & (noise >= thr)
    eps = rng.uniform(2.0, 8.0)
    eps_r = np.where(inside, complex(eps), 1.0 + 0.0j).astype(np.complex128)
    bid = np.full((n, n, n), -1, np.int32)
    khat = random_unit(rng)
    a = random_unit(rng)
    p = a - khat * np.dot(a, khat)
    p /= np.linalg.norm(p)
    return Workload("blob", (n, n, n), h, lambda0, eps_r, bid, khat=khat,
                    pol=p.astype(complex), use_precond=False)


def random_case(n, seed, chi_scale=0.5, block_grid=None):
    """Random complex susceptibility and field on an arbitrary (nx, ny, nz) grid.

    Used by parity tests: returns (eps_r, block_id, x) with x shaped
    [3, nz, ny, nx]. block_grid=(bx, by, bz) splits the grid into a regular
    array of blocks (ragged at the edges); voxels whose drawn eps_r is exactly
    1 get block -1.
    """
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    chi = chi_scale * (rng.uniform(-1, 1, (nz, ny, nx))
                       + 1j * rng.uniform(-1, 0, (nz, ny, nx)))
    air = rng.uniform(size=(nz, ny, nx)) < 0.2
    chi[air] = 0.0
    eps_r = (1.0 + chi).astype(np.complex128)
    if block_grid is None:
        bid = np.full((nz, ny, nx), -1, np.int32)
    else:
        bx, by, bz = block_grid
        Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        nbx = -(-nx // bx)
        nby = -(-ny // by)
        bid = ((Z // bz) * nby + (Y // by)) * nbx + (X // bx)
        bid = bid.astype(np.int32)
        bid[air] = -1
    x = rng.normal(size=(3, nz, ny, nx)) + 1j * rng.normal(size=(3, nz, ny, nx))
    return eps_r, bid, x.astype(np.complex128)


WORKLOADS = {
    "sphere": sphere,
    "metasurface": metasurface,
    "solar_cell": solar_cell,
    "blob": blob,
}


SERVING_SIZES = (32, 64, 96, 128)
SERVING_SIZE_WEIGHTS = (0.4, 0.3, 0.2, 0.1)
SERVING_WAVELENGTHS_NM = tuple(range(400, 801, 10))


def serving_geometry(kind, n, sid):
    """The structure `kind` on an n^3 grid (n >= 32), seed sid:
    * 'metasurface': (n/16)^2 unit cells of the metasurface workload (period 16 voxels, pillars
      16 voxels tall, eps_r 6.25, one block per pillar), centred in z in an n^3 box of air;
    * 'solar_cell': the solar-cell workload's recipe on an n x n x n grid: metal spheres (eps_r
      -15 - 1j) on a lattice of min(32, n) voxels, radius U[6, 12] voxels within the slab, in an
      absorber slab (eps_r 3 - 0.3j) 40 voxels thick centred in z (n >= 48; for n = 32 the layers
      [6, 26)), one block per sphere and the slab in 4 blocks along x."""
    if kind == "metasurface":
        cells = n // 16
        tile = metasurface(cells=cells, period=16, nz=16, seed=sid)
        z0 = (n - 16) // 2
        eps_r = np.ones((n, n, n), np.complex128)
        bid = np.full((n, n, n), -1, np.int32)
        eps_r[z0:z0 + 16] = tile.eps_r
        bid[z0:z0 + 16] = tile.block_id
        return Workload("metasurface", (n, n, n), tile.h, tile.lambda0, eps_r, bid, inner_tol=1e-2,
                        outer_tol=1e-6, use_precond=True)
    if kind == "solar_cell":
        z0, z1 = ((n - 40) // 2, (n - 40) // 2 + 40) if n >= 48 else (n // 5, n // 5 + (5 * n) // 8)
        return solar_cell(nx=n, ny=n, nz=n, seed=sid, slab=(z0, z1), lattice=min(32, n), rmin=6,
                          rmax=min(12, (z1 - z0) // 2 - 1))
    raise ValueError(f"unknown structure kind {kind!r}")


def serving_draws(nreq, seed=0, sizes=SERVING_SIZES, weights=SERVING_SIZE_WEIGHTS, structures_per_size=2,
                  kinds=("metasurface", "solar_cell")):
    """Parameters of a seeded stream of solve requests: request i has structure kind kinds[i % len(kinds)],
    a grid size n drawn from `sizes` with probabilities `weights`, one of `structures_per_size` seeded
    geometries of that kind and size, a wavelength from the 10 nm grid 400..800 nm and an incidence angle
    U[0, pi/6] in the xz plane (polarisation in the plane of incidence, perpendicular to khat).
    Returns dicts with keys kind, n, sid, structure (a cache key), lambda_nm, khat, pol."""
    rng = np.random.default_rng(seed)
    out = []
    p = np.asarray(weights, float) / np.sum(weights)
    for i in range(nreq):
        n = int(rng.choice(sizes, p=p))
        kind = kinds[i % len(kinds)]
        sid = int(rng.integers(structures_per_size))
        lam = float(rng.choice(SERVING_WAVELENGTHS_NM))
        th = rng.uniform(0, np.pi / 6)
        out.append({"kind": kind, "n": n, "sid": sid, "structure": f"{kind}-{n}-{sid}", "lambda_nm": lam,
                    "khat": np.array([np.sin(th), 0.0, np.cos(th)]),
                    "pol": np.array([np.cos(th), 0.0, -np.sin(th)], complex)})
    return out
