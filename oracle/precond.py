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


def find_blocks(block_id):
    """The voxel sets S_k and their bounding boxes, in increasing block id."""
    blocks = []
    for bid in np.unique(block_id):
        if bid < 0:
            continue
        zz, yy, xx = np.nonzero(block_id == bid)
        lo = (xx.min(), yy.min(), zz.min())
        hi = (xx.max() + 1, yy.max() + 1, zz.max() + 1)
        b = Block(int(bid), lo, hi, None)
        b.mask = block_id[b.slices] == bid
        blocks.append(b)
    return blocks


class BlockPreconditioner:
    """y = K2^{-1} b, each block solved inexactly by inner BiCGSTAB-FFT."""

    def __init__(self, eps_r, block_id, h, k, inner_tol=1e-2, inner_maxit=1000, near=None):
        self.blocks = find_blocks(block_id)
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
            sub[:, blk.mask] = xk[:, blk.mask]
            y[sl] = sub
        return y

    __call__ = apply
