"""Solve server: continuous batching of VIE solve requests on one GPU.

Requests (a structure, a wavelength, an incidence) arrive at any time, as in
the parameter sweeps of metasurface design (Section III.A). The server keeps
grids (per structure) and Green spectra (per structure and wavelength)
resident on the device, admits a queued request as soon as a solve slot and
enough device memory are free (admission by footprint, with bounded
skip-ahead so a large request cannot be starved forever), and runs admitted
requests on separate CUDA streams from separate host threads, so their work
overlaps on the GPU. Each solve is the library's vie_solve; its arithmetic
does not depend on what else runs, so a result is the same alone and in the
mix.

The scheduling logic (Scheduler) is separate from the device engine
(GpuEngine) so it can be tested without a GPU.
"""
from __future__ import annotations

import collections
import concurrent.futures
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Callable, Optional

import numpy as np

# device bytes per voxel of a grid handle with its spectra (workspace, Krylov
# vectors, block scratch, complex128 + complex64 spectra); an upper estimate
# used before the grid exists, replaced by the measured size afterwards
BYTES_PER_VOXEL_ESTIMATE = 3200


@dataclass
class Request:
    structure: str                      # cache key of the geometry
    eps_r: np.ndarray                   # complex [nz, ny, nx]
    h: float
    k0: float
    khat: np.ndarray
    pol: np.ndarray
    block_id: Optional[np.ndarray] = None
    outer_tol: float = 1e-6
    inner_tol: float = 1e-2
    outer_maxit: int = 1000
    mode: int = 1                       # vie.MODE_MIXED
    use_precond: bool = True
    want_field: bool = True             # copy E back to the host
    t_submit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    footprint: int = 0
    future: Any = None

    @property
    def nvox(self) -> int:
        return int(np.prod(self.eps_r.shape))


@dataclass
class Result:
    field: Optional[np.ndarray]
    stats: dict
    latency_s: float
    queue_s: float


class Scheduler:
    """Admission by device-memory footprint with a fixed number of slots.

    next_admissible() returns the first queued request (in arrival order) that
    fits both a free slot and the memory budget; requests may be passed over
    at most `max_bypass` times, after which nothing behind them is admitted.
    """

    def __init__(self, budget_bytes: int, slots: int, max_bypass: int = 8,
                 footprint: Optional[Callable[[Request], int]] = None):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.max_bypass = max_bypass
        self.queue: collections.deque = collections.deque()
        self.in_use = 0
        self.running = 0
        self.bypassed = collections.Counter()
        self.footprint = footprint or (lambda r: r.nvox * BYTES_PER_VOXEL_ESTIMATE)

    def push(self, req: Request):
        req.footprint = int(self.footprint(req))
        if req.footprint > self.budget:
            raise ValueError(f"request needs {req.footprint} bytes, more than the budget {self.budget}")
        self.queue.append(req)

    def next_admissible(self) -> Optional[Request]:
        if self.running >= self.slots:
            return None
        for i, r in enumerate(self.queue):
            if self.in_use + r.footprint <= self.budget:
                del self.queue[i]
                for earlier in list(self.queue)[:i]:
                    self.bypassed[id(earlier)] += 1
                self.in_use += r.footprint
                self.running += 1
                return r
            if self.bypassed[id(r)] >= self.max_bypass:
                return None          # the oldest starved request blocks the line
        return None

    def release(self, req: Request, actual: Optional[int] = None):
        self.in_use -= req.footprint
        self.running -= 1
        self.bypassed.pop(id(req), None)


@dataclass
class GridEntry:
    grid: Any
    busy: bool = True
    last_used: float = 0.0


class GpuEngine:
    """Device side: grid pool per structure, spectrum cache, one stream per worker."""

    def __init__(self, max_spectra: int = 64, cache_bytes: int = 32 << 30, merge: bool = False):
        from . import vie  # noqa: F401  (fails loudly without the CUDA library)
        self.vie = vie
        # merge: concurrent solves of grids of the same size share persistent block-solver launches
        # (continuous batching of the preconditioner's block solves across requests); one session per
        # grid size keeps the solves that wait for one another in lockstep of similar cost
        self.merge = merge
        self.sessions: dict = {}
        self.cache_bytes = cache_bytes
        self.lock = threading.Lock()
        self.grids: dict = collections.defaultdict(list)   # structure -> [GridEntry]
        # (structure, k0) -> [Spectrum, users]; a spectrum serves every grid of its structure
        self.spectra: collections.OrderedDict = collections.OrderedDict()
        self.max_spectra = max_spectra
        self.hits = collections.Counter()

    def _grid(self, req: Request):
        with self.lock:
            for entry in self.grids[req.structure]:
                if not entry.busy:
                    entry.busy = True
                    self.hits["grid_hit"] += 1
                    return entry
        g = self.vie.Grid(req.eps_r, req.h, req.block_id if req.use_precond else None)
        entry = GridEntry(g)
        with self.lock:
            self.grids[req.structure].append(entry)
            self.hits["grid_miss"] += 1
        return entry

    def _spectrum(self, structure, grid, k0):
        key = (structure, float(k0))
        with self.lock:
            ent = self.spectra.get(key)
            if ent is not None:
                ent[1] += 1
                self.spectra.move_to_end(key)
                self.hits["spectrum_hit"] += 1
                return key, ent[0]
        sp = grid.spectrum(k0)
        with self.lock:
            if key in self.spectra:            # made concurrently by another worker: keep the first
                ent = self.spectra[key]
                ent[1] += 1
                extra, sp = sp, ent[0]
            else:
                extra = None
                self.spectra[key] = [sp, 1]
                self.hits["spectrum_miss"] += 1
            self._evict_spectra()
        if extra is not None:
            extra.release()
        return key, sp

    def _evict_spectra(self):
        """Drop least recently used spectra that no running solve holds (lock held)."""
        for key in list(self.spectra):
            if len(self.spectra) <= self.max_spectra:
                break
            if self.spectra[key][1] == 0:
                self.spectra.pop(key)[0].release()

    def _unuse(self, key):
        with self.lock:
            self.spectra[key][1] -= 1
            self._evict_spectra()

    def run(self, req: Request, stream) -> Result:
        import torch
        with torch.cuda.stream(stream):
            entry = self._grid(req)
            skey = None
            try:
                g = entry.grid
                skey, sp = self._spectrum(req.structure, g, req.k0)
                einc = g.plane_wave(req.k0, req.khat, req.pol)
                e, st = g.solve(sp, einc, outer_tol=req.outer_tol, inner_tol=req.inner_tol,
                                use_precond=req.use_precond, mode=req.mode, outer_maxit=req.outer_maxit,
                                session=self._session(req))
                field = e.cpu().numpy() if req.want_field else None
                stream.synchronize()
            finally:
                if skey is not None:
                    self._unuse(skey)
                with self.lock:
                    entry.busy = False
                    entry.last_used = time.perf_counter()
                self._trim()
        return Result(field, st, 0.0, 0.0)

    def _session(self, req):
        if not self.merge:
            return None
        key = tuple(req.eps_r.shape)
        with self.lock:
            if key not in self.sessions:
                self.sessions[key] = self.vie.MergeSession()
            return self.sessions[key]

    def merge_stats(self):
        """Merged launches summed over the sessions (None without merging)."""
        if not self.merge:
            return None
        tot = {"launches": 0, "max_solves": 0, "solve_slots": 0.0}
        for s in self.sessions.values():
            st = s.stats()
            tot["launches"] += st["launches"]
            tot["max_solves"] = max(tot["max_solves"], st["max_solves"])
            tot["solve_slots"] += st["launches"] * st["mean_solves"]
        tot["mean_solves"] = tot.pop("solve_slots") / tot["launches"] if tot["launches"] else 0.0
        return tot

    def close(self):
        for s in self.sessions.values():
            s.close()
        self.sessions = {}

    def _trim(self):
        """Destroy least recently used idle grids (and their spectra) beyond cache_bytes."""
        with self.lock:
            idle = [(e.last_used, key, e) for key, lst in self.grids.items() for e in lst if not e.busy]
            total = sum(e.grid.info()["device_bytes"] for lst in self.grids.values() for e in lst)
            for _, key, e in sorted(idle, key=lambda t: t[0]):
                if total <= self.cache_bytes:
                    break
                g = e.grid
                if len(self.grids[key]) == 1 and any(k[0] == key and v[1] > 0 for k, v in self.spectra.items()):
                    continue                     # its structure's spectra are in use
                total -= g.info()["device_bytes"]
                if len(self.grids[key]) == 1:    # last grid of the structure: its spectra go too
                    for sk in [k for k in self.spectra if k[0] == key]:
                        self.spectra.pop(sk)[0].release()
                self.grids[key].remove(e)
                g.close()


class Server:
    """submit() returns a Future of Result; solves overlap on `slots` streams."""

    def __init__(self, budget_bytes: int, slots: int = 4, engine=None, max_bypass: int = 8, merge: bool = False):
        self.sched = Scheduler(budget_bytes, slots, max_bypass)
        self.engine = engine if engine is not None else GpuEngine(merge=merge)
        self.cv = threading.Condition()
        self.stop = False
        self.done: list = []
        self.workers = []
        self.streams = []
        try:
            import torch
            self.streams = [torch.cuda.Stream() for _ in range(slots)]
        except Exception:
            self.streams = [None] * slots
        for i in range(slots):
            t = threading.Thread(target=self._worker, args=(i,), daemon=True)
            t.start()
            self.workers.append(t)

    def submit(self, req: Request) -> concurrent.futures.Future:
        req.future = concurrent.futures.Future()
        req.t_submit = time.perf_counter()
        with self.cv:
            self.sched.push(req)
            self.cv.notify_all()
        return req.future

    def _worker(self, i):
        while True:
            with self.cv:
                req = None
                while not self.stop:
                    req = self.sched.next_admissible()
                    if req is not None:
                        break
                    self.cv.wait(0.05)
                if req is None:
                    return
            req.t_start = time.perf_counter()
            try:
                res = self.engine.run(req, self.streams[i])
                req.t_done = time.perf_counter()
                res.latency_s = req.t_done - req.t_submit
                res.queue_s = req.t_start - req.t_submit
                req.future.set_result(res)
            except Exception as exc:   # the request fails, the server keeps going
                req.t_done = time.perf_counter()
                req.future.set_exception(exc)
            finally:
                with self.cv:
                    self.sched.release(req)
                    self.done.append(req)
                    self.cv.notify_all()

    def close(self, timeout=None):
        """Stop taking work and wait for the running solves (each is bounded by its outer_maxit)."""
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.workers:
            t.join(timeout=timeout)
        if hasattr(self.engine, "close") and not any(t.is_alive() for t in self.workers):
            self.engine.close()

    def latency_stats(self):
        lat = np.array([r.t_done - r.t_submit for r in self.done if r.t_done > 0])
        if lat.size == 0:
            return {}
        t0 = min(r.t_submit for r in self.done)
        t1 = max(r.t_done for r in self.done)
        by_size = {}
        for r in self.done:
            if r.t_done > 0:
                by_size.setdefault(int(round(r.nvox ** (1 / 3))), []).append(r.t_done - r.t_submit)
        return {"requests": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "solves_per_s": lat.size / max(1e-9, t1 - t0),
                "p50_s_by_size": {n: float(np.percentile(v, 50)) for n, v in sorted(by_size.items())}}


# ---------------------------------------------------------------- synthetic request stream
from .inputs import SERVING_SIZE_WEIGHTS as SIZE_WEIGHTS, SERVING_SIZES as SIZES  # noqa: E402


def make_stream(nreq, seed=0, sizes=SIZES, weights=SIZE_WEIGHTS, h_nm=10.0, structures_per_size=2,
                kinds=("metasurface", "solar_cell"), outer_maxit=1000, mode=1):
    """Serving workload (inputs.serving_draws): grids drawn from `sizes`, structures
    alternating metasurface tiles and particle slabs rescaled to n, wavelength from a
    10 nm sweep grid, random incidence angle (plane waves tilted in the xz plane).
    `mode` is the solve mode of every request (1 mixed, 0 complex128 throughout,
    both with the block preconditioner); the draws do not depend on it, so two
    streams with the same seed hold the same problems."""
    from . import inputs
    geo = {}
    out = []
    for d in inputs.serving_draws(nreq, seed, sizes, weights, structures_per_size, kinds):
        key = d["structure"]
        if key not in geo:
            geo[key] = inputs.serving_geometry(d["kind"], d["n"], d["sid"])
        w = geo[key]
        out.append(Request(structure=key, eps_r=w.eps_r, h=h_nm, k0=2 * np.pi / d["lambda_nm"], khat=d["khat"],
                           pol=d["pol"], block_id=w.block_id, outer_maxit=outer_maxit, mode=mode))
    return out
