"""tl_dtg_batched_noalloc: the batched forward for callers that cannot let the library allocate device
memory (their device memory belongs to a caching allocator or a fixed budget, they cannot afford
cudaMalloc's device-wide synchronisation, or they are handed only their buffers).  Its scratch lives
in a fixed device array inside the library.  Called through the C ABI and compared with the
single-grid entry point tl_dtg_forward on two calls in a row, the second with different grids, so stale
scratch contents from the first call would show."""
import ctypes

import numpy as np
import pytest

import gridgen
from tests.parity import TOL_F64, assert_components

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_1804_10120_gb300 import build, lib
    build.build()
    L = lib()
    vp = ctypes.c_void_p
    L.tl_dtg_batched_noalloc.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int, vp]
    L.tl_dtg_batched_noalloc.restype = ctypes.c_int
    return L


def _grids(sides, seed):
    dev = torch.device("cuda", 0)
    xs, ys = [], []
    for d, side in enumerate(sides):
        n = side ** 3
        xs.append(torch.from_numpy(gridgen.random_grid(n, seed, stream_base=64 * d)).to(dev))
        ys.append(torch.full((39, n), float("nan"), dtype=torch.float64, device=dev))
    G = len(sides)
    tin = (ctypes.c_void_p * (43 * G))()
    tout = (ctypes.c_void_p * (39 * G))()
    ns = (ctypes.c_int64 * G)()
    for d, (x, y) in enumerate(zip(xs, ys)):
        n = x.shape[1]
        ns[d] = n
        for s in range(43):
            tin[43 * d + s] = x[s].data_ptr() if n else 16
        for s in range(39):
            tout[39 * d + s] = y[s].data_ptr() if n else 16
    return xs, ys, tin, tout, ns


def test_noalloc_matches_forward_on_two_calls():
    import paper_1804_10120_gb300 as tl
    L = _lib()
    for seed, sides in [(61, [9, 14, 3, 0, 21, 7, 16, 11, 5, 18, 2, 12]), (62, [6, 19, 1, 10, 15])]:
        xs, ys, tin, tout, ns = _grids(sides, seed)
        rc = L.tl_dtg_batched_noalloc(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(ns), len(sides), 0, None)
        assert rc == 0, L.tl_last_error()
        torch.cuda.synchronize()
        for x, y in zip(xs, ys):
            ref = tl.tl_dtg_forward(x)
            torch.cuda.synchronize()
            assert_components(y.cpu().numpy(), ref.cpu().numpy(), TOL_F64, what="noalloc vs forward")


def test_noalloc_rejects_more_than_its_maximum():
    L = _lib()
    G = 1025
    tin = (ctypes.c_void_p * (43 * G))(*([16] * (43 * G)))
    tout = (ctypes.c_void_p * (39 * G))(*([16] * (39 * G)))
    ns = (ctypes.c_int64 * G)()
    assert L.tl_dtg_batched_noalloc(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(ns), G, 0, None) == 1
    assert b"1024" in L.tl_last_error()
