"""Serving loop logic on the CPU: admission by footprint, slots, bounded skip-ahead, and a
server run against a fake engine (no GPU)."""
import threading
import time

import numpy as np
import pytest

from paper_2501_13512_gb300.serve import Request, Result, Scheduler, Server


def _req(nvox, name="s"):
    n = int(round(nvox ** (1 / 3)))
    return Request(structure=name, eps_r=np.ones((n, n, n), complex), h=1.0, k0=1.0,
                   khat=np.array([0, 0, 1.0]), pol=np.array([1, 0, 0], complex))


def test_admission_respects_budget_slots_and_order():
    s = Scheduler(budget_bytes=100, slots=2, footprint=lambda r: r.nvox)
    a, b, c = _req(64), _req(27), _req(8)      # footprints 64, 27, 8
    for r in (a, b, c):
        s.push(r)
    assert s.next_admissible() is a
    assert s.next_admissible() is b            # 64 + 27 <= 100
    assert s.next_admissible() is None         # slots exhausted
    s.release(a)
    assert s.next_admissible() is c
    assert s.in_use == 27 + 8 and s.running == 2


def test_skip_ahead_is_bounded():
    s = Scheduler(budget_bytes=100, slots=8, max_bypass=2, footprint=lambda r: r.nvox)
    big = _req(64)
    s.push(_req(64))                          # running, holds 64
    assert s.next_admissible() is not None
    s.push(big)                               # does not fit (64 + 64 > 100)
    smalls = [_req(8) for _ in range(5)]
    for r in smalls:
        s.push(r)
    got = [s.next_admissible() for _ in range(4)]
    # two small requests pass the big one, then the line waits for it
    assert got[0] is smalls[0] and got[1] is smalls[1]
    assert got[2] is None and got[3] is None


def test_oversize_request_rejected():
    s = Scheduler(budget_bytes=10, slots=1, footprint=lambda r: r.nvox)
    with pytest.raises(ValueError):
        s.push(_req(27))


class FakeEngine:
    def __init__(self):
        self.lock = threading.Lock()
        self.active = 0
        self.peak = 0

    def run(self, req, stream):
        with self.lock:
            self.active += 1
            self.peak = max(self.peak, self.active)
        time.sleep(0.002 * req.nvox ** (1 / 3))
        with self.lock:
            self.active -= 1
        return Result(None, {"outer_iters": 1.0}, 0.0, 0.0)


def test_server_overlaps_within_slots_and_completes_everything():
    eng = FakeEngine()
    srv = Server(budget_bytes=10 ** 9, slots=3, engine=eng)
    futs = [srv.submit(_req(n ** 3, f"s{n}")) for n in (4, 8, 6, 4, 10, 8, 4, 6)]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    assert len(res) == 8 and all(r.latency_s >= r.queue_s >= 0 for r in res)
    assert 1 < eng.peak <= 3
    st = srv.latency_stats()
    assert st["requests"] == 8 and st["p99_s"] >= st["p50_s"] > 0


def test_server_survives_a_failing_request():
    class Boom(FakeEngine):
        def run(self, req, stream):
            if req.structure == "bad":
                raise RuntimeError("bad geometry")
            return super().run(req, stream)
    srv = Server(budget_bytes=10 ** 9, slots=2, engine=Boom())
    ok = srv.submit(_req(27, "good"))
    bad = srv.submit(_req(27, "bad"))
    with pytest.raises(RuntimeError):
        bad.result(timeout=30)
    assert ok.result(timeout=30).stats["outer_iters"] == 1.0
    srv.close()


def test_engine_keeps_one_merge_session_per_grid_size():
    # the GPU engine's session bookkeeping with a stand-in for the binding's MergeSession (no GPU)
    from paper_2501_13512_gb300.serve import GpuEngine

    class FakeSession:
        made = []

        def __init__(self):
            self.closed = False
            self.st = {"launches": 3 * (len(FakeSession.made) + 1), "max_solves": 2 + len(FakeSession.made),
                       "mean_solves": 1.5}
            FakeSession.made.append(self)

        def stats(self):
            return dict(self.st)

        def close(self):
            self.closed = True

    class FakeVie:
        MergeSession = FakeSession

    eng = GpuEngine(merge=True)
    eng.vie = FakeVie()
    a, b, c = _req(8), _req(27), _req(8)
    sa, sb, sc = eng._session(a), eng._session(b), eng._session(c)
    assert sa is sc and sa is not sb and len(FakeSession.made) == 2
    st = eng.merge_stats()
    assert st["launches"] == 3 + 6 and st["max_solves"] == 3
    assert abs(st["mean_solves"] - 1.5) < 1e-12
    eng.close()
    assert all(s.closed for s in FakeSession.made) and eng.merge_stats()["launches"] == 0
    assert GpuEngine(merge=False)._session(a) is None
