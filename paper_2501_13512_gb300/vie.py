"""Python binding of libvie (include/vie.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch provides device memory
and the current stream. Vectors are torch tensors of shape (3, nz, ny, nx),
complex128 (VIE_C128) or complex64 (VIE_C64), contiguous, on the grid's GPU.
If libvie.so is missing this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, byref, c_double, c_int, c_int32, c_int64, c_size_t, c_uint32, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvie.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "vie.h")

VIE_OK, VIE_EINVAL, VIE_ENOMEM, VIE_ECUDA, VIE_ENOTCONV, VIE_EBREAKDOWN, VIE_ETIMEOUT, VIE_EBUSY = range(8)
STATUS_NAMES = {0: "VIE_OK", 1: "VIE_EINVAL", 2: "VIE_ENOMEM", 3: "VIE_ECUDA", 4: "VIE_ENOTCONV",
                5: "VIE_EBREAKDOWN", 6: "VIE_ETIMEOUT", 7: "VIE_EBUSY"}
C128, C64 = 1, 2
INNER_AUTO, INNER_BATCHED, INNER_PERSISTENT = 0, 1, 2
MODE_PLAIN_C128, MODE_MIXED = 0, 1


class VieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("h", c_double),
                ("eps_r", POINTER(c_double)), ("block_id", POINTER(c_int32)), ("flags", c_uint32),
                ("block_expand", c_int32)]


class GridInfo(ctypes.Structure):
    _fields_ = [("nblocks", c_int32), ("ngroups", c_int32), ("Mx", c_int32), ("My", c_int32),
                ("Mz", c_int32), ("device_bytes", c_int64), ("inner_cluster", c_int32 * 2)]


class PrecondStats(ctypes.Structure):
    _fields_ = [("nblocks", c_int32), ("max_iters", c_int32), ("mean_iters", c_double),
                ("not_converged", c_int32), ("breakdowns", c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("outer_tol", c_double), ("inner_tol", c_double), ("outer_maxit", c_int32),
                ("inner_maxit", c_int32), ("use_precond", c_int32), ("mode", c_int32),
                ("max_refinements", c_int32), ("wait_timeout_ms", c_double), ("x0_dev", c_void_p)]


class SolveStats(ctypes.Structure):
    _fields_ = [("outer_iters", c_double), ("inner_iters", c_int64), ("precond_applies", c_int32),
                ("matvecs_c128", c_int32), ("matvecs_c64", c_int32), ("refinements", c_int32),
                ("true_rel_res", c_double), ("status", c_int32), ("rejected", c_int32),
                ("elapsed_ms", c_double)]


class MergeStats(ctypes.Structure):
    _fields_ = [("launches", c_int32), ("max_solves", c_int32), ("mean_solves", c_double)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("h", c_double), ("count", c_int32),
                ("eps_r", POINTER(c_double)), ("flags", c_uint32)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("precision", c_int32), ("launches", c_int64),
                ("total_ms", c_double), ("bytes", c_double)]


def _struct_dict(s):
    return {name: getattr(s, name) for name, _ in s._fields_}


_lib = None


def declared_functions(header=HEADER):
    """Names of the entry points declared in include/vie.h."""
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*int\s+(vie_\w+)\s*\(", text, re.M)))


def load(path=LIB_PATH):
    """Load libvie.so (built by paper_2501_13512_gb300.build) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libvie.so not found at {path}: run paper_2501_13512_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "vie_version": ([], c_int),
        "vie_last_error": ([ctypes.c_char_p, c_size_t], c_int),
        "vie_grid_create": ([POINTER(GridDesc), POINTER(P)], c_int),
        "vie_grid_destroy": ([P], c_int),
        "vie_grid_get_info": ([P, POINTER(GridInfo)], c_int),
        "vie_green_spectrum": ([P, c_double, c_int, P, POINTER(P)], c_int),
        "vie_green_spectrum_near": ([P, c_double, c_int, c_int32, c_int32, P, POINTER(P)], c_int),
        "vie_spectrum_release": ([P], c_int),
        "vie_plane_wave": ([P, c_double, POINTER(c_double), POINTER(c_double), c_int, P, P], c_int),
        "vie_matvec": ([P, P, c_int, P, P, P], c_int),
        "vie_block_precond_apply": ([P, P, c_int, P, P, c_double, c_int, P, POINTER(PrecondStats)], c_int),
        "vie_solve": ([P, P, P, P, POINTER(SolveOpts), P, POINTER(SolveStats)], c_int),
        "vie_solve_host": ([P, P, P, P, POINTER(SolveOpts), P, POINTER(SolveStats)], c_int),
        "vie_merge_session_create": ([POINTER(P)], c_int),
        "vie_merge_session_destroy": ([P], c_int),
        "vie_merge_session_stats": ([P, POINTER(MergeStats)], c_int),
        "vie_solve_merged": ([P, P, P, P, P, POINTER(SolveOpts), P, POINTER(SolveStats)], c_int),
        "vie_solve_many": ([c_int32, POINTER(P), POINTER(P), POINTER(P), POINTER(P), POINTER(SolveOpts), P,
                            POINTER(SolveStats), POINTER(MergeStats)], c_int),
        "vie_matvec_noalloc": ([c_int32, c_int32, c_int32, c_double, c_double, P, P, P, P], c_int),
        "vie_far_field_rcs": ([P, c_double, P, c_int32, POINTER(c_double), POINTER(c_double), P], c_int),
        "vie_batch_create": ([POINTER(BatchDesc), POINTER(P)], c_int),
        "vie_batch_destroy": ([P], c_int),
        "vie_batch_solve": ([P, POINTER(c_double), P, P, POINTER(SolveOpts), P, POINTER(SolveStats)], c_int),
        "vie_batch_get_info": ([P, POINTER(c_int64), POINTER(c_int32)], c_int),
        "vie_batch_solve_many": ([c_int32, POINTER(P), POINTER(P), POINTER(P), POINTER(P), POINTER(SolveOpts), P,
                                  POINTER(P), POINTER(MergeStats)], c_int),
        "vie_profile_enable": ([c_int], c_int),
        "vie_profile_read": ([POINTER(KernelStat), c_int, POINTER(c_int), POINTER(c_int64)], c_int),
        "vie_rooftop_create": ([P, c_double, c_int, P, POINTER(P)], c_int),
        "vie_rooftop_release": ([P], c_int),
        "vie_rooftop_incident": ([P, POINTER(c_double), POINTER(c_double), c_int, P, P], c_int),
        "vie_rooftop_matvec": ([P, c_int, P, P, P], c_int),
        "vie_rooftop_solve": ([P, P, P, c_double, c_int32, c_double, P, POINTER(SolveStats)], c_int),
        "vie_rooftop_far_field_rcs": ([P, P, c_int32, POINTER(c_double), POINTER(c_double), P], c_int),
        "vie_set_device_budget": ([c_int64], c_int),
        "vie_device_usage": ([POINTER(c_int64), POINTER(c_int64)], c_int),
        "vie_fault_inject_alloc": ([c_int32], c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def last_error():
    lib = load()
    buf = ctypes.create_string_buffer(1024)
    lib.vie_last_error(buf, 1024)
    return buf.value.decode()


def _check(rc, allow=()):
    if rc != VIE_OK and rc not in allow:
        raise VieError(rc, last_error())
    return rc


def profile_enable(on=True):
    """Start (clearing) or stop CUDA-event recording of every library launch."""
    _check(load().vie_profile_enable(1 if on else 0))


def profile_read():
    """(per-kernel stats list, total launches since process start)."""
    cap = 64
    arr = (KernelStat * cap)()
    n = c_int()
    tot = c_int64()
    _check(load().vie_profile_read(arr, cap, byref(n), byref(tot)))
    out = []
    for i in range(n.value):
        d = _struct_dict(arr[i])
        d["name"] = arr[i].name.decode()
        d["precision"] = "c128" if arr[i].precision == C128 else "c64"
        out.append(d)
    return out, tot.value


def launch_count():
    tot = c_int64()
    _check(load().vie_profile_read(None, 0, None, byref(tot)))
    return tot.value


def set_device_budget(nbytes):
    """Process-wide cap on the device bytes held by grids, spectra and batches (0: none)."""
    _check(load().vie_set_device_budget(int(nbytes)))


def device_usage():
    """(bytes held by the library's handles, budget) on the device."""
    held, budget = c_int64(), c_int64()
    _check(load().vie_device_usage(byref(held), byref(budget)))
    return held.value, budget.value


def _stream():
    import torch
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype(precision):
    import torch
    return torch.complex128 if precision == C128 else torch.complex64


class Spectrum:
    def __init__(self, grid, handle, k0, mask):
        self.grid = grid
        self.handle = handle
        self.k0 = k0
        self.mask = mask

    def release(self):
        if self.handle:
            _check(load().vie_spectrum_release(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Grid:
    """A voxel grid with its contrast and block partition (vie_grid)."""

    def __init__(self, eps_r, h, block_id=None, inner=INNER_AUTO, expand=0):
        lib = load()
        eps_r = np.ascontiguousarray(eps_r, dtype=np.complex128)
        nz, ny, nx = eps_r.shape
        self.shape = (nz, ny, nx)
        self.n = (nx, ny, nz)
        self.h = float(h)
        self._eps = eps_r.view(np.float64).reshape(-1)
        self._bid = None if block_id is None else np.ascontiguousarray(block_id, dtype=np.int32).reshape(-1)
        d = GridDesc(nx, ny, nz, self.h, self._eps.ctypes.data_as(POINTER(c_double)),
                     None if self._bid is None else self._bid.ctypes.data_as(POINTER(c_int32)), int(inner),
                     int(expand))
        handle = c_void_p()
        _check(lib.vie_grid_create(byref(d), byref(handle)))
        self.handle = handle

    @classmethod
    def from_workload(cls, w, inner=INNER_AUTO, expand=0):
        return cls(w.eps_r, w.h, w.block_id if w.use_precond else None, inner, expand)

    def info(self):
        inf = GridInfo()
        _check(load().vie_grid_get_info(self.handle, byref(inf)))
        d = _struct_dict(inf)
        d["inner_cluster"] = list(inf.inner_cluster)
        return d

    def close(self):
        if self.handle:
            _check(load().vie_grid_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, t, precision, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != _dtype(precision) or tuple(t.shape) != (3,) + self.shape or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {_dtype(precision)} tensor of shape {(3,) + self.shape}")
        return c_void_p(t.data_ptr())

    def empty(self, precision=C128):
        import torch
        return torch.empty((3,) + self.shape, dtype=_dtype(precision), device="cuda")

    def spectrum(self, k0, precision=C128 | C64, near=None):
        """near = (radius, order): cube-integrated near-neighbour entries (vie_green_spectrum_near)."""
        h = c_void_p()
        if near is None:
            _check(load().vie_green_spectrum(self.handle, float(k0), int(precision), _stream(), byref(h)))
        else:
            _check(load().vie_green_spectrum_near(self.handle, float(k0), int(precision), int(near[0]), int(near[1]),
                                                  _stream(), byref(h)))
        return Spectrum(self, h, float(k0), precision)

    def plane_wave(self, k0, khat, pol, precision=C128, out=None):
        out = self.empty(precision) if out is None else out
        kh = (c_double * 3)(*[float(v) for v in khat])
        p = np.asarray(pol, dtype=np.complex128)
        pv = (c_double * 6)(p[0].real, p[0].imag, p[1].real, p[1].imag, p[2].real, p[2].imag)
        _check(load().vie_plane_wave(self.handle, float(k0), kh, pv, precision,
                                     self._vec(out, precision, "out"), _stream()))
        return out

    def matvec(self, spec, x, y=None, precision=None):
        precision = precision or (C128 if x.dtype == _dtype(C128) else C64)
        y = self.empty(precision) if y is None else y
        _check(load().vie_matvec(self.handle, spec.handle, precision, self._vec(x, precision, "x"),
                                 self._vec(y, precision, "y"), _stream()))
        return y

    def precond(self, spec, b, y=None, inner_tol=1e-2, inner_maxit=1000, precision=None):
        precision = precision or (C128 if b.dtype == _dtype(C128) else C64)
        y = self.empty(precision) if y is None else y
        st = PrecondStats()
        _check(load().vie_block_precond_apply(self.handle, spec.handle, precision, self._vec(b, precision, "b"),
                                              self._vec(y, precision, "y"), float(inner_tol), int(inner_maxit),
                                              _stream(), byref(st)))
        return y, _struct_dict(st)

    def _opts(self, outer_tol=1e-6, inner_tol=1e-2, outer_maxit=1000, inner_maxit=1000, use_precond=True,
              mode=MODE_MIXED, max_refinements=0, wait_timeout_ms=0.0, x0=None):
        return SolveOpts(float(outer_tol), float(inner_tol), int(outer_maxit), int(inner_maxit), int(bool(use_precond)),
                         int(mode), int(max_refinements), float(wait_timeout_ms),
                         None if x0 is None else self._vec(x0, C128, "x0"))

    def solve(self, spec, einc, e=None, outer_tol=1e-6, inner_tol=1e-2, outer_maxit=1000, inner_maxit=1000,
              use_precond=True, mode=MODE_MIXED, max_refinements=0, wait_timeout_ms=0.0, x0=None, check=True,
              session=None):
        """x0: initial guess (complex128 CUDA tensor, may be `e` itself), None for zero.
        session: a MergeSession whose concurrent solves share block-solver launches (vie_solve_merged)."""
        e = self.empty(C128) if e is None else e
        o = self._opts(outer_tol, inner_tol, outer_maxit, inner_maxit, use_precond, mode, max_refinements,
                       wait_timeout_ms, x0)
        st = SolveStats()
        args = (self.handle, spec.handle, self._vec(einc, C128, "einc"), self._vec(e, C128, "e"), byref(o),
                _stream(), byref(st))
        if session is None:
            rc = load().vie_solve(*args)
        else:
            rc = load().vie_solve_merged(session.handle, *args)
        if check:
            _check(rc, allow=(VIE_ENOTCONV,))
        return e, _struct_dict(st)

    def far_field_rcs(self, k0, e, dirs):
        """Bistatic RCS of the field e (complex128 CUDA tensor) in the unit directions dirs (n x 3)."""
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
        out = np.empty(d.shape[0], dtype=np.float64)
        _check(load().vie_far_field_rcs(self.handle, float(k0), self._vec(e, C128, "e"), d.shape[0],
                                        d.ctypes.data_as(POINTER(c_double)), out.ctypes.data_as(POINTER(c_double)),
                                        _stream()))
        return out

    def solve_host(self, spec, einc_host, out_host, outer_tol=1e-6, inner_tol=1e-2, outer_maxit=1000,
                   inner_maxit=1000, use_precond=True, mode=MODE_MIXED, max_refinements=0, wait_timeout_ms=0.0,
                   check=True):
        """End-to-end solve from host memory (vie_solve_host): einc_host and out_host are contiguous complex128
        CPU tensors of shape (3, nz, ny, nx) (pinned for full-speed copies); E_inc in, E out, both copies
        inside the call."""
        import torch
        for t, name in ((einc_host, "einc_host"), (out_host, "out_host")):
            if (not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.complex128
                    or tuple(t.shape) != (3,) + self.shape or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous complex128 CPU tensor of shape {(3,) + self.shape}")
        o = self._opts(outer_tol, inner_tol, outer_maxit, inner_maxit, use_precond, mode, max_refinements,
                       wait_timeout_ms)
        st = SolveStats()
        rc = load().vie_solve_host(self.handle, spec.handle, c_void_p(einc_host.data_ptr()),
                                   c_void_p(out_host.data_ptr()), byref(o), _stream(), byref(st))
        if check:
            _check(rc, allow=(VIE_ENOTCONV,))
        return out_host, _struct_dict(st)


class MergeSession:
    """Solves run concurrently (own threads and streams) inside a session share persistent block-solver
    launches (vie_merge_session_*)."""

    def __init__(self):
        h = c_void_p()
        _check(load().vie_merge_session_create(byref(h)))
        self.handle = h

    def stats(self):
        ms = MergeStats()
        _check(load().vie_merge_session_stats(self.handle, byref(ms)))
        return _struct_dict(ms)

    def close(self):
        if self.handle:
            _check(load().vie_merge_session_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _addr(p):
    return p.value if isinstance(p, c_void_p) else p


def solve_many(problems, check=True):
    """Solves several systems at once (vie_solve_many): each problem is a dict with keys grid, spec, einc,
    optionally e, and any option of Grid.solve (outer_tol, inner_tol, mode, ...); the grids must be distinct.
    Block-preconditioner applications of all solves share persistent launches. Returns
    ([(e, stats) per problem], merge stats)."""
    n = len(problems)
    grids = (c_void_p * n)()
    specs = (c_void_p * n)()
    ein = (c_void_p * n)()
    eout = (c_void_p * n)()
    opts = (SolveOpts * n)()
    stats = (SolveStats * n)()
    fields = []
    for i, p in enumerate(problems):
        g = p["grid"]
        e = p.get("e")
        e = g.empty(C128) if e is None else e
        fields.append(e)
        kw = {k: v for k, v in p.items() if k not in ("grid", "spec", "einc", "e")}
        grids[i] = _addr(g.handle)
        specs[i] = _addr(p["spec"].handle)
        ein[i] = _addr(g._vec(p["einc"], C128, "einc"))
        eout[i] = _addr(g._vec(e, C128, "e"))
        opts[i] = g._opts(**kw)
    ms = MergeStats()
    rc = load().vie_solve_many(n, grids, specs, ein, eout, opts, _stream(), stats, byref(ms))
    if check:
        _check(rc, allow=(VIE_ENOTCONV,))
    return [(fields[i], _struct_dict(stats[i])) for i in range(n)], _struct_dict(ms)


class Rooftop:
    """The paper's rooftop / pulse discretisation of a grid's permittivity (vie_rooftop): unknown
    w = J / (j w eps0) on faces, vectors (3, nz, ny, nx) with component a at the face above cell c."""

    def __init__(self, grid, k0, precision=C128 | C64):
        self.grid = grid
        self.k0 = float(k0)
        h = c_void_p()
        _check(load().vie_rooftop_create(grid.handle, self.k0, int(precision), _stream(), byref(h)))
        self.handle = h

    def incident(self, khat, pol, precision=C128):
        out = self.grid.empty(precision)
        kh = (c_double * 3)(*[float(v) for v in khat])
        p = np.asarray(pol, dtype=np.complex128)
        pv = (c_double * 6)(p[0].real, p[0].imag, p[1].real, p[1].imag, p[2].real, p[2].imag)
        _check(load().vie_rooftop_incident(self.handle, kh, pv, precision, self.grid._vec(out, precision, "out"),
                                           _stream()))
        return out

    def matvec(self, w, y=None):
        precision = C128 if w.dtype == _dtype(C128) else C64
        y = self.grid.empty(precision) if y is None else y
        _check(load().vie_rooftop_matvec(self.handle, precision, self.grid._vec(w, precision, "w"),
                                         self.grid._vec(y, precision, "y"), _stream()))
        return y

    def solve(self, b, w=None, tol=1e-6, maxit=1000, wait_timeout_ms=0.0, check=True):
        w = self.grid.empty(C128) if w is None else w
        st = SolveStats()
        rc = load().vie_rooftop_solve(self.handle, self.grid._vec(b, C128, "b"), self.grid._vec(w, C128, "w"),
                                      float(tol), int(maxit), float(wait_timeout_ms), _stream(), byref(st))
        if check:
            _check(rc, allow=(VIE_ENOTCONV,))
        return w, _struct_dict(st)

    def far_field_rcs(self, w, dirs):
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
        out = np.empty(d.shape[0], dtype=np.float64)
        _check(load().vie_rooftop_far_field_rcs(self.handle, self.grid._vec(w, C128, "w"), d.shape[0],
                                                d.ctypes.data_as(POINTER(c_double)),
                                                out.ctypes.data_as(POINTER(c_double)), _stream()))
        return out

    def close(self):
        if self.handle:
            _check(load().vie_rooftop_release(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent instances of one grid shape solved together (vie_batch)."""

    def __init__(self, eps_list, h):
        lib = load()
        eps = np.ascontiguousarray(np.stack([np.asarray(e, dtype=np.complex128) for e in eps_list]))
        self.count, nz, ny, nx = eps.shape
        self.shape = (nz, ny, nx)
        self._eps = eps.view(np.float64).reshape(-1)
        d = BatchDesc(nx, ny, nz, float(h), self.count, self._eps.ctypes.data_as(POINTER(c_double)), 0)
        handle = c_void_p()
        _check(lib.vie_batch_create(byref(d), byref(handle)))
        self.handle = handle

    def info(self):
        nbytes, pers = c_int64(), c_int32()
        _check(load().vie_batch_get_info(self.handle, byref(nbytes), byref(pers)))
        return {"device_bytes": nbytes.value, "persistent": bool(pers.value)}

    def empty(self):
        import torch
        return torch.empty((self.count, 3) + self.shape, dtype=torch.complex128, device="cuda")

    def solve(self, k0s, einc, e=None, outer_tol=1e-6, outer_maxit=1000, max_refinements=0, wait_timeout_ms=0.0,
              check=True):
        import torch
        if tuple(einc.shape) != (self.count, 3) + self.shape or einc.dtype != torch.complex128 or not einc.is_cuda:
            raise ValueError("einc must be a complex128 CUDA tensor of shape (count, 3, nz, ny, nx)")
        e = self.empty() if e is None else e
        k = (c_double * self.count)(*[float(v) for v in np.broadcast_to(np.asarray(k0s, float), (self.count,))])
        o = self._opts(outer_tol, outer_maxit, max_refinements, wait_timeout_ms)
        st = (SolveStats * self.count)()
        rc = load().vie_batch_solve(self.handle, k, c_void_p(einc.data_ptr()), c_void_p(e.data_ptr()), byref(o),
                                    _stream(), st)
        if check:
            _check(rc, allow=(VIE_ENOTCONV,))
        return e, [_struct_dict(x) for x in st]

    def _opts(self, outer_tol=1e-6, outer_maxit=1000, max_refinements=0, wait_timeout_ms=0.0):
        return SolveOpts(float(outer_tol), 0.0, int(outer_maxit), 1, 0, MODE_MIXED, int(max_refinements),
                         float(wait_timeout_ms))

    def close(self):
        if self.handle:
            _check(load().vie_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve_many(jobs, check=True):
    """Solves several batches (vie_batch_solve_many) of different grid shapes together: each job is a dict
    with keys batch, k0s, einc, optionally e, and options of Batch.solve. The persistent correction launches
    of all batches run merged. Returns ([(e, [stats per instance]) per job], merge stats)."""
    import torch
    n = len(jobs)
    bh = (c_void_p * n)()
    kp = (c_void_p * n)()
    ein = (c_void_p * n)()
    eout = (c_void_p * n)()
    opts = (SolveOpts * n)()
    stp = (c_void_p * n)()
    keep = []
    out = []
    for i, j in enumerate(jobs):
        b = j["batch"]
        einc = j["einc"]
        if tuple(einc.shape) != (b.count, 3) + b.shape or einc.dtype != torch.complex128 or not einc.is_cuda:
            raise ValueError("einc must be a complex128 CUDA tensor of shape (count, 3, nz, ny, nx)")
        e = j.get("e")
        e = b.empty() if e is None else e
        k = (c_double * b.count)(*[float(v) for v in np.broadcast_to(np.asarray(j["k0s"], float), (b.count,))])
        st = (SolveStats * b.count)()
        keep += [k, st]
        bh[i] = _addr(b.handle)
        kp[i] = ctypes.cast(k, c_void_p).value
        ein[i] = einc.data_ptr()
        eout[i] = e.data_ptr()
        opts[i] = b._opts(**{k_: v for k_, v in j.items() if k_ not in ("batch", "k0s", "einc", "e")})
        stp[i] = ctypes.cast(st, c_void_p).value
        out.append((e, st))
    ms = MergeStats()
    rc = load().vie_batch_solve_many(n, bh, kp, ein, eout, opts, _stream(), stp, byref(ms))
    if check:
        _check(rc, allow=(VIE_ENOTCONV,))
    return [(e, [_struct_dict(x) for x in st]) for e, st in out], _struct_dict(ms)
