"""Solves of several requests with merged block-solver launches (vie_solve_many, vie_solve_merged):
each served result is checked against the oracle (the sampled serving requests, solved by the oracle
to 1e-10, tests/golden/serve_requests.npz) and against the same solve run alone, and the blocks of
different requests really share persistent launches.

Tolerances: a solve stopped at a true relative residual of 1e-6 is within 1e-5 of the exact solution
of these systems (the sampled requests' error against the oracle measured on GB300: well below
1e-5 in both modes), and two such solves agree to the same bound."""
import json
import os
import threading

import numpy as np
import pytest
import torch

from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "serve_requests.npz")
H_NM = 10.0


def _sampled():
    gd = np.load(GOLDEN)
    out = []
    draws = inputs.serving_draws(4, 1, (32, 64), (0.4, 0.3))
    for i in range(3):
        meta = json.loads(str(gd[f"meta_{i}"]))
        d = draws[meta["request"]]
        assert d["structure"] == meta["structure"] and d["lambda_nm"] == meta["lambda_nm"]
        w = inputs.serving_geometry(d["kind"], d["n"], d["sid"])
        out.append((w, d, gd[f"index_{i}"], gd[f"value_{i}"]))
    return out


def _problem(w, d, mode, tol):
    g = vie.Grid(w.eps_r, H_NM, w.block_id)
    k0 = 2 * np.pi / d["lambda_nm"]
    sp = g.spectrum(k0)
    return {"grid": g, "spec": sp, "einc": g.plane_wave(k0, d["khat"], d["pol"]), "outer_tol": tol,
            "inner_tol": 1e-2, "mode": mode, "outer_maxit": 1000}


def _close(probs):
    torch.cuda.synchronize()
    for p in probs:
        p["spec"].release()
        p["grid"].close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mode", [vie.MODE_MIXED, vie.MODE_PLAIN_C128])
def test_merged_requests_match_the_oracle_and_their_solves_alone(mode):
    cases = _sampled()
    merged = [_problem(w, d, mode, 1e-6) for (w, d, _, _) in cases]
    res, ms = vie.solve_many(merged)
    alone = [_problem(w, d, mode, 1e-6) for (w, d, _, _) in cases]
    try:
        for (w, d, idx, ref), (e, st), p in zip(cases, res, alone):
            assert st["status"] == vie.VIE_OK and st["true_rel_res"] <= 1e-6
            got = e.cpu().numpy().ravel()[idx]
            err = _rel(got, ref)
            e1, st1 = p["grid"].solve(p["spec"], p["einc"], outer_tol=1e-6, inner_tol=1e-2, mode=mode)
            assert st1["status"] == vie.VIE_OK
            print(f"{d['structure']} lambda {d['lambda_nm']:.0f} nm mode {mode}: merged vs oracle {err:.2e}, "
                  f"merged vs alone {_rel(e.cpu().numpy(), e1.cpu().numpy()):.2e}, outer {st['outer_iters']}")
            assert err <= 1e-5
            assert _rel(e.cpu().numpy(), e1.cpu().numpy()) <= 1e-5
    finally:
        _close(merged + alone)
    if mode == vie.MODE_MIXED:
        # the two metasurface tiles' complex64 blocks (on-chip slab MVM) went through shared launches
        assert ms["launches"] >= 1 and ms["max_solves"] >= 2
    else:
        # complex128 blocks merge only when their grid alone takes the persistent solver (32 blocks or
        # more): these grids keep their own batched launches
        assert ms["launches"] == 0


def test_session_merges_solves_started_from_threads():
    # continuous batching: solves started at different times on their own threads and streams join the
    # session's launches; their results equal their solves alone
    cases = _sampled()
    probs = [_problem(w, d, vie.MODE_MIXED, 1e-6) for (w, d, _, _) in cases]
    sess = vie.MergeSession()
    out = [None] * len(probs)
    errs = []

    def run(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                p = probs[i]
                e, st = p["grid"].solve(p["spec"], p["einc"], outer_tol=1e-6, inner_tol=1e-2, session=sess)
                s.synchronize()
                out[i] = (e, st)
        except Exception as exc:       # reported below
            errs.append(exc)

    th = [threading.Thread(target=run, args=(i,)) for i in range(len(probs))]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    stats = sess.stats()
    sess.close()
    try:
        assert not errs, errs
        for (w, d, idx, ref), (e, st) in zip(cases, out):
            assert st["status"] == vie.VIE_OK
            assert _rel(e.cpu().numpy().ravel()[idx], ref) <= 1e-5
    finally:
        _close(probs)
    assert stats["launches"] >= 1 and stats["max_solves"] >= 2


def test_solve_many_rejects_a_grid_twice_and_runs_one_as_vie_solve():
    w, d, idx, ref = _sampled()[0]
    p = _problem(w, d, vie.MODE_MIXED, 1e-6)
    try:
        with pytest.raises(vie.VieError):
            vie.solve_many([p, dict(p)])
        (e, st), = vie.solve_many([p])[0]
        assert st["status"] == vie.VIE_OK and _rel(e.cpu().numpy().ravel()[idx], ref) <= 1e-5
    finally:
        _close([p])


def _tile(kind, n, sid, lam, mode, tol=1e-6):
    w = inputs.serving_geometry(kind, n, sid)
    d = {"lambda_nm": lam, "khat": np.array([0.3, 0.0, np.sqrt(1 - 0.09)]),
         "pol": np.array([np.sqrt(1 - 0.09), 0.0, -0.3], complex)}
    return _problem(w, d, mode, tol)


def test_solve_many_reports_a_failing_solve_and_finishes_the_others():
    probs = [_tile("metasurface", 32, 0, 500, vie.MODE_MIXED), _tile("metasurface", 32, 1, 620, vie.MODE_MIXED),
             _tile("metasurface", 64, 0, 560, vie.MODE_MIXED)]
    probs[1]["outer_tol"] = 0.0                 # rejected by the solve (VIE_EINVAL) before any block work
    try:
        res, ms = vie.solve_many(probs, check=False)
        assert res[1][1]["status"] == vie.VIE_EINVAL
        for i in (0, 2):
            e, st = res[i]
            assert st["status"] == vie.VIE_OK and st["true_rel_res"] <= 1e-6
            p = probs[i]
            e1, _ = p["grid"].solve(p["spec"], p["einc"], outer_tol=1e-6, mode=vie.MODE_MIXED)
            assert _rel(e.cpu().numpy(), e1.cpu().numpy()) <= 1e-5
        assert ms["launches"] >= 1 and ms["max_solves"] == 2
        with pytest.raises(vie.VieError):
            vie.solve_many(probs)                   # the first failing solve's code, raised
    finally:
        _close(probs)


def test_session_with_mixed_and_fp64_solves_launches_per_precision():
    # complex64 blocks of the mixed solves and complex128 blocks of the FP64 solve (a 96^3 tile: 36
    # blocks, so its grid alone takes the persistent solver) merge in separate launches of one session
    probs = [_tile("metasurface", 96, 0, 600, vie.MODE_MIXED), _tile("metasurface", 96, 1, 610, vie.MODE_MIXED),
             _tile("metasurface", 96, 0, 630, vie.MODE_PLAIN_C128)]
    try:
        res, ms = vie.solve_many(probs)
        for (e, st), p in zip(res, probs):
            assert st["status"] == vie.VIE_OK and st["true_rel_res"] <= 1e-6
            e1, _ = p["grid"].solve(p["spec"], p["einc"], outer_tol=1e-6, mode=p["mode"])
            assert _rel(e.cpu().numpy(), e1.cpu().numpy()) <= 1e-5
        assert ms["launches"] >= 2 and ms["max_solves"] >= 2
    finally:
        _close(probs)
