"""The C-ABI library: it loads, exports every symbol include/tl.h declares, and its host-side argument
checks reject bad calls before touching a device (no GPU needed; nothing is computed here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1804_10120_gb300 import build, lib
    build.build()
    return lib()


def declared_symbols():
    syms = []
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            syms += re.findall(r"TL_API\s+[\w\s\*]+?\b(tl_\w+)\s*\(", text)
    return syms


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert "tl_dtg_forward" in syms and "tl_dtg_backward" in syms
    for s in syms:
        assert hasattr(L, s), s


def test_status_strings(L):
    for code, name in [(0, b"TL_OK"), (1, b"TL_ERR_INVALID_ARG"), (2, b"TL_ERR_ALIGNMENT"),
                       (3, b"TL_ERR_UNSUPPORTED"), (4, b"TL_ERR_CUDA"), (5, b"TL_ERR_TIMEOUT"),
                       (6, b"TL_ERR_PLAN_MISMATCH")]:
        assert L.tl_status_string(code) == name


def _tabs(base=1 << 20, n=16, esz=8, stride=None):
    stride = stride or n * esz
    tin = (ctypes.c_void_p * 43)(*[base + s * stride for s in range(43)])
    tout = (ctypes.c_void_p * 39)(*[base + (43 + s) * stride for s in range(39)])
    return tin, tout


def test_forward_argument_checks(L):
    tin, tout = _tabs()
    f = L.tl_dtg_forward
    assert f(None, ctypes.byref(tout), 16, 0, None) == 1
    assert f(ctypes.byref(tin), ctypes.byref(tout), -1, 0, None) == 1
    assert f(ctypes.byref(tin), ctypes.byref(tout), 16, 7, None) == 1
    bad = (ctypes.c_void_p * 43)(*tin); bad[5] = None
    assert f(ctypes.byref(bad), ctypes.byref(tout), 16, 0, None) == 1
    assert b"in[5]" in L.tl_last_error()
    mis = (ctypes.c_void_p * 43)(*tin); mis[3] = tin[3] + 4
    assert f(ctypes.byref(mis), ctypes.byref(tout), 16, 0, None) == 2
    # binary32 needs only 4-byte alignment, but then the 4-byte shift overlaps nothing in this layout
    # output aliasing an input
    alias = (ctypes.c_void_p * 39)(*tout); alias[2] = tin[7]
    assert f(ctypes.byref(tin), ctypes.byref(alias), 16, 0, None) == 1
    # two outputs overlapping partially
    ov = (ctypes.c_void_p * 39)(*tout); ov[4] = tout[3] + 8
    assert f(ctypes.byref(tin), ctypes.byref(ov), 16, 0, None) == 1
    # inputs may overlap each other (read-only)
    rd = (ctypes.c_void_p * 43)(*tin); rd[1] = tin[0]
    assert f(ctypes.byref(rd), ctypes.byref(tout), 0, 0, None) == 0
    # n == 0: nothing to do, no device touched
    assert f(ctypes.byref(tin), ctypes.byref(tout), 0, 0, None) == 0


def test_backward_argument_checks(L):
    tin, tout = _tabs()
    gout = (ctypes.c_void_p * 39)(*([None] * 39))
    gin = (ctypes.c_void_p * 43)(*[(1 << 30) + s * 128 for s in range(43)])
    b = L.tl_dtg_backward
    assert b(ctypes.byref(tin), ctypes.byref(gout), ctypes.byref(gin), 0, 0, None) == 0   # NULL gouts allowed
    assert b(ctypes.byref(tin), ctypes.byref(gout), ctypes.byref(gin), 0, 1, None) == 3   # no f32 adjoint
    g2 = (ctypes.c_void_p * 43)(*gin); g2[0] = tin[0]
    assert b(ctypes.byref(tin), ctypes.byref(gout), ctypes.byref(g2), 16, 0, None) == 1


def test_forward_backward_argument_checks(L):
    tin, tout = _tabs()
    gout = (ctypes.c_void_p * 39)(*([None] * 39))
    gin = (ctypes.c_void_p * 43)(*[(1 << 30) + s * 128 for s in range(43)])
    f = L.tl_dtg_forward_backward
    f.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    assert f(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(gout), ctypes.byref(gin), 0, 0, None) == 0
    assert f(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(gout), ctypes.byref(gin), 16, 1, None) == 3  # no f32
    assert f(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(gout), ctypes.byref(gin), -1, 0, None) == 1
    assert f(None, ctypes.byref(tout), ctypes.byref(gout), ctypes.byref(gin), 16, 0, None) == 1
    g2 = (ctypes.c_void_p * 43)(*gin); g2[3] = tout[5]           # an input gradient over an output
    assert f(ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(gout), ctypes.byref(g2), 16, 0, None) == 1
    assert b"overlap" in L.tl_last_error()
    nul = (ctypes.c_void_p * 39)(*tout); nul[38] = None           # outputs are all required
    assert f(ctypes.byref(tin), ctypes.byref(nul), ctypes.byref(gout), ctypes.byref(gin), 16, 0, None) == 1


def test_host_workspace_size(L):
    L.tl_dtg_host_workspace_bytes.restype = ctypes.c_size_t
    L.tl_dtg_host_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int]
    assert L.tl_dtg_host_workspace_bytes(0, 0) == 0
    assert L.tl_dtg_host_workspace_bytes(100, 0) == 100 * 82 * 8
    assert L.tl_dtg_host_workspace_bytes(100, 1) == 100 * 82 * 4
    big = 1 << 24
    assert L.tl_dtg_host_workspace_bytes(big, 0) == 3 * (1 << 19) * 82 * 8
    assert L.tl_dtg_host_workspace_bytes((1 << 19) + 1, 1) == 2 * (1 << 19) * 82 * 4


def test_batched_prepare_argument_checks(L):
    """Batch validation runs on the host before any device work: overlaps across grids, NULL entries
    and negative sizes are rejected."""
    vp = ctypes.c_void_p
    L.tl_dtg_batched_prepare.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int, ctypes.POINTER(vp)]
    L.tl_dtg_batched_prepare.restype = ctypes.c_int
    G, n = 3, 16
    ins = (vp * (43 * G))(*[(1 << 24) + (d * 82 + s) * n * 8 for d in range(G) for s in range(43)])
    outs = (vp * (39 * G))(*[(1 << 24) + (d * 82 + 43 + s) * n * 8 for d in range(G) for s in range(39)])
    ns = (ctypes.c_int64 * G)(n, n, n)
    h = vp()
    bad = (vp * (39 * G))(*outs); bad[39 + 5] = ins[0]            # grid 1 writes over grid 0's g_00
    assert L.tl_dtg_batched_prepare(ctypes.byref(ins), ctypes.byref(bad), ctypes.byref(ns), G, 0, ctypes.byref(h)) == 1
    assert b"overlap" in L.tl_last_error()
    nul = (vp * (43 * G))(*ins); nul[43 * 2 + 7] = None
    assert L.tl_dtg_batched_prepare(ctypes.byref(nul), ctypes.byref(outs), ctypes.byref(ns), G, 0, ctypes.byref(h)) == 1
    neg = (ctypes.c_int64 * G)(n, -1, n)
    assert L.tl_dtg_batched_prepare(ctypes.byref(ins), ctypes.byref(outs), ctypes.byref(neg), G, 0, ctypes.byref(h)) == 1
    assert L.tl_dtg_batched_prepare(ctypes.byref(ins), ctypes.byref(outs), ctypes.byref(ns), -1, 0, ctypes.byref(h)) == 1
    assert L.tl_dtg_batched_prepare(ctypes.byref(ins), ctypes.byref(outs), ctypes.byref(ns), G, 9, ctypes.byref(h)) == 1


def test_bench_traffic_is_tied_to_kernel_sources(monkeypatch, tmp_path):
    """bench.py reports an ncu DRAM figure only for the kernel sources it was captured on: scaled to
    the benchmark's point count when the recorded source digest matches, None otherwise."""
    import json
    import bench
    kernel = "dtg_fwd_f64_kernel"
    entry = {"dram_bytes": 4.0e9, "n": 1 << 22, "src_digest": bench.src_digest(kernel), "ncu_duration_s": 1e-3}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({kernel: entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "src_digest", lambda k=None: entry["src_digest"])
    assert bench.traffic_per_launch(kernel, 1 << 24) == 4 * 4.0e9
    monkeypatch.setattr(bench, "src_digest", lambda k=None: "changed")
    assert bench.traffic_per_launch(kernel, 1 << 24) is None
    assert bench.traffic_per_launch("no_such_kernel", 1 << 24) is None


def test_pipe_rate_probe_argument_checks(L):
    """The FP64 pipe-rate probe hook rejects bad arguments on the host, before any launch."""
    f = L.tl_testing_pipe_rate
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    sink = ctypes.c_void_p(1 << 20)
    assert f(9, 16, 1, 256, sink, None) == 1          # no such operation
    assert f(-1, 16, 1, 256, sink, None) == 1
    assert f(0, -1, 1, 256, sink, None) == 1          # negative rounds
    assert f(0, 16, 0, 256, sink, None) == 1          # no blocks
    assert f(0, 16, 1, 33, sink, None) == 1           # not whole warps
    assert f(0, 16, 1, 2048, sink, None) == 1         # beyond 1024 threads
    assert f(0, 16, 1, 256, None, None) == 1          # no sink


def test_bench_floor_and_nominal_bandwidth(monkeypatch):
    """The FP64 floor is the operation mix over the measured rates; the nominal HBM figure is memory
    clock x 2 x bus width from the device properties, and absent when they are not exposed."""
    import types
    import torch
    import bench
    n = 1 << 24
    rates = (2.0e9 * 152 * 2.07, 1.68e9 * 152 * 2.07)
    split = bench.fp64_floor_ms((71, 18), n, rates)
    all_dfma = bench.fp64_floor_ms((89, 0), n, rates)
    assert abs(split - (71 / rates[0] + 18 / rates[1]) * n * 1e3) < 1e-12
    assert all_dfma < split
    assert abs(all_dfma - 2.37) < 0.02            # 89 x 2^24 / (2 x 152 x 2.07e9) s
    props = types.SimpleNamespace(memory_clock_rate=3996000, memory_bus_width=8192)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: props)
    gbs, src = bench.nominal_hbm_gbs(None)
    assert abs(gbs - 3996e6 * 2 * 1024 / 1e9) < 1e-6 and "8192-bit" in src
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: types.SimpleNamespace())
    if not torch.cuda.is_available():
        assert bench.nominal_hbm_gbs(torch.device("cuda", 0)) is None   # no device to query either


def test_memory_info_argument_checks(L):
    """The device memory query rejects NULL outputs before any CUDA call."""
    f = L.tl_testing_memory_info
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    v = ctypes.c_int32()
    assert f(0, None, ctypes.byref(v)) == 1 and f(0, ctypes.byref(v), None) == 1
