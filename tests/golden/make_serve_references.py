"""Writes tests/golden/serve_requests.npz from the CPU oracle only.

The sampled serving requests: requests 0, 2 and 3 of the seeded serving
stream inputs.serving_draws(4, seed=1, sizes=(32, 64), weights=(0.4, 0.3))
(a 32^3 and a 64^3 metasurface tile and a 32^3 solar-cell slab; h = 10 nm,
wavelengths from the 10 nm grid, tilted plane waves), each solved by the
oracle's block-preconditioned BiCGSTAB (Eq. 10 blocks, inner tolerance 1e-2,
Section II.B) to an outer tolerance of 1e-10, so that a served result at 1e-6
can be checked against it.

Stored per sampled request r = 0, 1, 2: meta_r (JSON: the draw, outer iterations, true residual,
field norm, oracle seconds), index_r (a seeded sample of 8192 entries of the
flattened [3, nz, ny, nx] field) and value_r (the field there, complex128).

Run: python tests/golden/make_serve_references.py      (three processes; the solar cell's metal
sphere block takes hundreds of inner iterations per application: about an hour)
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))
SEED, NREQ, SIZES, WEIGHTS = 1, 4, (32, 64), (0.4, 0.3)
PICK = (0, 2, 3)          # indices of the sampled requests in the stream
H_NM = 10.0
TOL = 1e-10
NSAMPLE = 8192


def solve_one(i):
    sys.path.insert(0, ROOT)
    from oracle import krylov, mvm, precond, solve
    from paper_2501_13512_gb300 import inputs
    d = inputs.serving_draws(NREQ, SEED, SIZES, WEIGHTS)[PICK[i]]
    w = inputs.serving_geometry(d["kind"], d["n"], d["sid"])
    k0 = 2 * np.pi / d["lambda_nm"]
    ein = solve.plane_wave(w.n, H_NM, k0, d["khat"], d["pol"])
    t0 = time.time()
    A = mvm.FFTOperator(w.eps_r, H_NM, k0)
    P = precond.BlockPreconditioner(w.eps_r, w.block_id, H_NM, k0, 1e-2, 1000)
    E, info = krylov.bicgstab(A, ein, TOL, 5000, apply_Kinv=P)
    dt = time.time() - t0
    true_res = float(np.linalg.norm(ein - A(E)) / np.linalg.norm(ein))
    flat = E.ravel()
    idx = np.sort(np.random.default_rng(100 + i).choice(flat.size, size=NSAMPLE, replace=False)).astype(np.int64)
    meta = {"request": PICK[i], "kind": d["kind"], "n": d["n"], "sid": d["sid"], "structure": d["structure"],
            "lambda_nm": d["lambda_nm"], "h_nm": H_NM, "outer_tol": TOL, "inner_tol": 1e-2, "inner_maxit": 1000,
            "outer_iters": info["iters"], "status": info["status"], "true_rel_res": true_res,
            "field_norm": float(np.linalg.norm(E)), "oracle_seconds": dt}
    print(json.dumps(meta), flush=True)
    return meta, idx, flat[idx]


def main():
    with mp.get_context("spawn").Pool(len(PICK)) as pool:
        res = pool.map(solve_one, range(len(PICK)))
    arrays = {"_cite": np.array(
        "Sampled serving requests 0, 2, 3 of inputs.serving_draws(4, seed=1, sizes=(32, 64), weights=(0.4, 0.3)), "
        "h = 10 nm; Eq. 10 block preconditioning (inner tolerance 1e-2), Section II.B BiCGSTAB to an outer "
        "tolerance of 1e-10; written by tests/golden/make_serve_references.py from oracle/ only.")}
    for i, (meta, idx, val) in enumerate(res):
        arrays[f"meta_{i}"] = np.array(json.dumps(meta))
        arrays[f"index_{i}"] = idx
        arrays[f"value_{i}"] = val
    np.savez_compressed(os.path.join(HERE, "serve_requests.npz"), **arrays)


if __name__ == "__main__":
    main()
