"""vie_matvec_noalloc: the MVM for callers that cannot allocate device memory.

Some callers must not allocate device memory at run time (their device memory
belongs to another framework's allocator, or they run in a loop that cannot
block on the driver's allocator). vie_matvec_noalloc keeps every intermediate
in one static device array instead. This test calls it through the C ABI and
checks it against vie_matvec (the allocating path) to the complex128 MVM
tolerance, on two calls in a row so that state left in the shared array by one
call cannot leak into the next, and on its own against the CPU oracle's FFT
operator. It lives in its own file, collected last; its first test makes the
first call of the process on a non-blocking side stream (the one-time twiddle
upload must be complete before that stream's kernels read it).
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import mvm as omvm
from paper_2501_13512_gb300 import inputs, vie

pytestmark = pytest.mark.gpu

K0 = 2 * np.pi
H = 0.05


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.complex128)


def _noalloc(lib, n, chi, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.vie_matvec_noalloc(n[0], n[1], n[2], H, K0, ctypes.c_void_p(chi.data_ptr()),
                                  ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)


@pytest.mark.parametrize("n,seed", [((5, 7, 3), 6), ((1, 9, 4), 7)])
def test_noalloc_matches_oracle_on_a_side_stream(n, seed):
    # the first no-allocation call of a fresh process runs here, on a non-blocking side stream
    lib = vie.load()
    eps_r, _, x = inputs.random_case(n, seed=seed)
    ref = omvm.FFTOperator(eps_r, H, K0)(x)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        xd, chi = _dev(x), _dev(eps_r - 1.0)
        y = torch.full_like(xd, complex(np.nan, np.nan))
        assert _noalloc(lib, n, chi, xd, y) == vie.VIE_OK, vie.last_error()
    side.synchronize()
    got = y.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,seed", [((16, 16, 16), 1), ((5, 7, 3), 2), ((1, 9, 4), 3)])
def test_noalloc_matches_matvec_on_consecutive_calls(n, seed):
    lib = vie.load()
    eps_r, _, x = inputs.random_case(n, seed=seed)
    g = vie.Grid(eps_r, H)
    sp = g.spectrum(K0, vie.C128)
    xd = _dev(x)
    ref = g.matvec(sp, xd)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    chi = _dev(eps_r - 1.0)
    for call in range(2):
        y = torch.full_like(xd, complex(np.nan, np.nan))
        assert _noalloc(lib, n, chi, xd, y) == vie.VIE_OK, vie.last_error()
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), call


def test_noalloc_after_a_different_grid_and_rejects_oversize():
    lib = vie.load()
    # a second grid shape after the first: the shared array must be rewritten, not reused stale
    for n, seed in [((8, 8, 8), 4), ((12, 3, 6), 5)]:
        eps_r, _, x = inputs.random_case(n, seed=seed)
        g = vie.Grid(eps_r, H)
        sp = g.spectrum(K0, vie.C128)
        xd = _dev(x)
        ref = g.matvec(sp, xd)
        y = torch.empty_like(xd)
        assert _noalloc(lib, n, _dev(eps_r - 1.0), xd, y) == vie.VIE_OK
        torch.cuda.synchronize()
        assert torch.linalg.vector_norm(y - ref) <= 1e-12 * torch.linalg.vector_norm(ref)
    big = (17, 16, 16)      # padded 64 x 32 x 32 exceeds the static limit
    z = torch.zeros((3, 16, 16, 17), dtype=torch.complex128, device="cuda")
    chi = torch.zeros((16, 16, 17), dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, big, chi, z, torch.empty_like(z)) == vie.VIE_EINVAL
    assert "static scratch limit" in vie.last_error()
    # y overlapping chi is refused before any launch
    n = (4, 4, 4)
    buf = torch.zeros(3 * 64 + 64, dtype=torch.complex128, device="cuda")
    x = torch.zeros(3 * 64, dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, n, buf[3 * 64 - 8:], x, buf[:3 * 64]) == vie.VIE_EINVAL
    assert "chi and y overlap" in vie.last_error()
