"""Writes tests/golden/metasurface_crop_<c>x<c>.npz from the CPU oracle only.

Solves metasurface crops of the benchmark workload's recipe (c x c pillars of
period 16 voxels, eps_r 6.25, 16 z layers, h = lambda0/20, one block per
pillar; Section III.A's setting with the synthetic geometry of
paper_2501_13512_gb300.inputs.metasurface(cells=c, seed=0)) with the oracle's
block-preconditioned BiCGSTAB (inner tolerance 1e-2, Section II.B) to an outer
tolerance of 1e-10, so that the stored field stands for the exact solution of
the discretised system when a solve at 1e-6 is checked against it.

Stored per crop: the oracle's outer iteration count, its true residual, the
field norm and the field at `index` (every entry for c = 4, a seeded sample of
65536 entries for c = 8) as complex128.

Run: python tests/golden/make_crop_references.py [c ...]   (default: 4 8)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, mvm, precond, solve  # noqa: E402
from paper_2501_13512_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-10
FULL_UP_TO = 4          # crops of at most this many cells per side store every entry
NSAMPLE = 65536


def main(cells):
    w = inputs.metasurface(cells=cells, seed=0)
    ein = solve.plane_wave(w.n, w.h, w.k0, w.khat, w.pol)
    A = mvm.FFTOperator(w.eps_r, w.h, w.k0)
    P = precond.BlockPreconditioner(w.eps_r, w.block_id, w.h, w.k0, w.inner_tol, 1000)
    t0 = time.time()
    E, info = krylov.bicgstab(A, ein, TOL, 5000, apply_Kinv=P)
    t_solve = time.time() - t0
    true_res = float(np.linalg.norm(ein - A(E)) / np.linalg.norm(ein))
    flat = E.ravel()
    if cells <= FULL_UP_TO:
        idx = np.arange(flat.size, dtype=np.int64)
    else:
        idx = np.sort(np.random.default_rng(4321).choice(flat.size, size=NSAMPLE, replace=False)).astype(np.int64)
    meta = {
        "_cite": "Section III.A (metasurface, one block per pillar, inner tolerance 1e-2), Eq. 10 block "
                 "preconditioning, Section II.B BiCGSTAB; synthetic geometry inputs.metasurface(cells=%d, seed=0); "
                 "outer tolerance 1e-10; written by tests/golden/make_crop_references.py from oracle/ only." % cells,
        "cells": cells,
        "n": list(w.n),
        "outer_tol": TOL,
        "inner_tol": w.inner_tol,
        "inner_maxit": 1000,
        "outer_iters": info["iters"],
        "status": info["status"],
        "true_rel_res": true_res,
        "field_norm": float(np.linalg.norm(E)),
        "oracle_seconds": t_solve,
    }
    out = os.path.join(HERE, "metasurface_crop_%dx%d.npz" % (cells, cells))
    np.savez_compressed(out, index=idx, value=flat[idx], meta=np.array(json.dumps(meta)))
    print(json.dumps(meta, indent=1))


if __name__ == "__main__":
    for c in (sys.argv[1:] or ["4", "8"]):
        main(int(c))
