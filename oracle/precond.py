"""Oracle: block-diagonal preconditioner with inner BiCGSTAB-FFT solves (Section II.B, Eqs. 10-11).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

K2 = diag(A_1, ..., A_N): A_k holds the rows and columns of A that belong to
the voxels S_k of block k, all three field components together (Eq. 11).
Interactions between blocks are dropped (Eq. 10). Each A_k x_k = b_k is solved
by BiCGSTAB with the FFT MVM on the bounding box of S_k, from x_k = 0, to the
loose inner tolerance (Section II.B: "the stopping criteria ... can be
softened"). Voxels outside every block (block id -1) are left unchanged:
their diagonal block is the identity when chi = 0 there.

Pinned by tests/test_oracle_solver.py: against dense per-block LU, and the
single-block case where K2 = A exactly (the outer solve then converges at its
first half-step).

Expanded blocks (the paper's conclusion names enlarged blocks that carry more of
the surrounding field as future work; the reading taken here): with expand = e > 0
block k is solved on S_k+ = S_k plus every voxel with chi != 0 within Chebyshev
distance e of S_k (other blocks' voxels included), and only the values on S_k
are kept (restricted additive Schwarz). Air voxels of the halo are left out:
their columns of A are identity columns, so they cannot change the values on
S_k. Pinned by dense LU on S_k+, e = 0 reducing to the plain blocks, and an
expansion that reaches every voxel giving the exact inverse.
"""
import numpy as np

from .krylov import bicgstab
from .mvm import FFTOperator


class Block:
    def __init__(self, bid, lo, hi, mask):
        self.bid = bid
        self.lo = lo          # (x0, y0, z0) of the bounding box
        self.hi = hi          # exclusive upper corner
        self.mask = mask      # bool [bz, by, bx]: voxels of S_k inside the box

    @property
    def slices(self):
        return (slice(self.lo[2], self.hi[2]), slice(self.lo[1], self.hi[1]),
                slice(self.lo[0], self.hi[0]))


def find_blocks(block_id, expand=0, chi_nonzero=None):
    """The voxel sets S_k and their bounding boxes, in increasing block id.

    expand = e > 0: the box and mask cover S_k+ (S_k plus the voxels with chi != 0
    within Chebyshev distance e, chi_nonzero giving where chi != 0); the block's own
    voxels S_k are in b.core (same shape as b.mask)."""
    blocks = []
    nz, ny, nx = block_id.shape
    for bid in np.unique(block_id):
        if bid < 0:
            continue
        own = block_id == bid
        if expand > 0:
            # dilation of S_k by a (2e+1)^3 cube, then keep S_k and the non-air voxels
            dil = own.copy()
            for ax in range(3):
                acc = dil.copy()
                for d in range(1, expand + 1):
                    acc |= np.roll(dil, d, axis=ax) & _shift_valid(dil.shape, ax, d)
                    acc |= np.roll(dil, -d, axis=ax) & _shift_valid(dil.shape, ax, -d)
                dil = acc
            sel = own | (dil & chi_nonzero)
        else:
            sel = own
        zz, yy, xx = np.nonzero(sel)
        lo = (xx.min(), yy.min(), zz.min())
        hi = (xx.max() + 1, yy.max() + 1, zz.max() + 1)
        b = Block(int(bid), lo, hi, None)
        b.mask = sel[b.slices]
        b.core = own[b.slices]
        blocks.append(b)
    return blocks


def _shift_valid(shape, ax, d):
    """Mask of the positions that np.roll(., d, axis=ax) filled from inside the array (no wrap)."""
    m = np.ones(shape, bool)
    idx = [slice(None)] * 3
    idx[ax] = slice(0, d) if d > 0 else slice(shape[ax] + d, shape[ax])
    m[tuple(idx)] = False
    return m


class BlockPreconditioner:
    """y = K2^{-1} b, each block solved inexactly by inner BiCGSTAB-FFT."""

    def __init__(self, eps_r, block_id, h, k, inner_tol=1e-2, inner_maxit=1000, near=None, expand=0):
        self.blocks = find_blocks(block_id, expand, (eps_r - 1.0) != 0)
        self.ops = []
        for b in self.blocks:
            self.ops.append(FFTOperator(eps_r[b.slices], h, k, mask=b.mask, near=near))
        self.inner_tol = inner_tol
        self.inner_maxit = inner_maxit
        self.last_inner_iters = []

    def apply(self, b):
        y = b.copy()
        self.last_inner_iters = []
        for blk, op in zip(self.blocks, self.ops):
            sl = (slice(None),) + blk.slices
            bk = np.where(blk.mask[None], b[sl], 0.0)
            xk, info = bicgstab(op.apply, bk, self.inner_tol, self.inner_maxit)
            self.last_inner_iters.append(info["iters"])
            sub = y[sl]
            sub[:, blk.core] = xk[:, blk.core]      # only the block's own voxels are kept
            y[sl] = sub
        return y

    __call__ = apply
