"""tl_dtg_batched_noalloc: the batched forward for callers that cannot let the library allocate device
memory (their device memory belongs to a caching allocator or a fixed budget, they cannot afford
cudaMalloc's device-wide synchronisation, or they are handed only their buffers).  Its scratch lives
in a fixed device array inside the library that every call reuses.

Called through the C ABI for every storage type, three times in a row with the number of grids
shrinking and then growing, so that tables left in the scratch by an earlier call would show.  Each
call is compared bit for bit with the single-grid entry point (tl_dtg_forward) and with a batch plan
launch of the same grids (the same per-point code), and with the CPU oracle within the tolerance the
other parity tests use.  Collected last, so a run that stops at its first failure has run every other
test by then."""
import ctypes

import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import TOL_F64, assert_components, component_errors, OUT_NAMES

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F32_COMPUTE = 2e-6
DTYPE_CODE = {"f64": 0, "f32": 1, "f64_ff": 2}
CALLS = [(61, [9, 14, 3, 0, 21, 7, 16, 11, 5, 18, 2, 12]),          # 12 grids (one empty)
         (62, [6, 19, 1, 10, 15]),                                   # fewer grids: stale tables past G=5
         (63, [4, 13, 8, 17, 1, 20, 3, 11, 6, 9, 2, 14, 7, 5, 16, 10, 12, 15, 19, 22])]   # more grids


def _lib():
    from paper_1804_10120_gb300 import build, lib
    build.build()
    L = lib()
    vp = ctypes.c_void_p
    L.tl_dtg_batched_noalloc.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int, vp]
    L.tl_dtg_batched_noalloc.restype = ctypes.c_int
    return L


def _grids(sides, seed, dtype):
    dev = torch.device("cuda", 0)
    td = torch.float32 if dtype == "f32" else torch.float64
    xs_host, xs, ys = [], [], []
    for d, side in enumerate(sides):
        n = side ** 3
        x = gridgen.random_grid(n, seed, stream_base=64 * d)
        if dtype == "f32":
            x = x.astype(np.float32)
        xs_host.append(x)
        xs.append(torch.from_numpy(x).to(dev))
        ys.append(torch.full((39, n), float("nan"), dtype=td, device=dev))
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
    return xs_host, xs, ys, tin, tout, ns


def _bits(t):
    return t.view(torch.int32 if t.dtype == torch.float32 else torch.int64)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64_ff"])
def test_noalloc_matches_forward_plan_and_oracle_on_three_calls(dtype):
    import paper_1804_10120_gb300 as tl
    L = _lib()
    stream = torch.cuda.current_stream(torch.device("cuda", 0))
    for seed, sides in CALLS:
        xs_host, xs, ys, tin, tout, ns = _grids(sides, seed, dtype)
        rc = L.tl_dtg_batched_noalloc(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(ns), len(sides),
                                      DTYPE_CODE[dtype], ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.tl_last_error()
        torch.cuda.synchronize()
        # a batch plan over the same grids, written to separate outputs
        yp = [torch.full_like(y, float("nan")) for y in ys]
        plan = tl.BatchPlan(xs, yp, dtype=dtype)
        plan.launch(stream)
        torch.cuda.synchronize()
        plan.close()
        for d, (xh, x, y) in enumerate(zip(xs_host, xs, ys)):
            if x.shape[1] == 0:
                continue
            ref = tl.tl_dtg_forward(x, dtype=dtype)
            torch.cuda.synchronize()
            assert torch.equal(_bits(y), _bits(ref)), (dtype, seed, d)
            assert torch.equal(_bits(y), _bits(yp[d])), (dtype, seed, d)
            yo = oracle.forward(xh.astype(np.float64))
            if dtype == "f32":
                err = component_errors(y.cpu().numpy().astype(np.float64), yo)
                assert err.max() <= TOL_F32_COMPUTE, dict(zip(OUT_NAMES, err))
            else:
                assert_components(y.cpu().numpy(), yo, TOL_F64, what="noalloc %s grid %d" % (dtype, d))


def test_noalloc_refused_during_stream_capture():
    """The call reuses a static host image of the tables, so it refuses to run while its stream is being
    captured; nothing is enqueued and the capture stays valid."""
    L = _lib()
    dev = torch.device("cuda", 0)
    _, xs, ys, tin, tout, ns = _grids([5, 7], 64, "f64")
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    marker = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = L.tl_dtg_batched_noalloc(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(ns), 2, 0,
                                      ctypes.c_void_p(side.cuda_stream))
        marker.add_(1.0)                                     # the capture goes on after the refusal
    assert rc == 3, rc
    assert b"captured" in L.tl_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert marker.item() == 1.0
    assert all(bool(torch.isnan(y).all()) for y in ys)      # the refused call enqueued nothing


def test_noalloc_rejects_more_than_its_maximum():
    L = _lib()
    G = 1025
    tin = (ctypes.c_void_p * (43 * G))(*([16] * (43 * G)))
    tout = (ctypes.c_void_p * (39 * G))(*([16] * (39 * G)))
    ns = (ctypes.c_int64 * G)()
    assert L.tl_dtg_batched_noalloc(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(ns), G, 0, None) == 1
    assert b"1024" in L.tl_last_error()
