"""The bounded waits of the staged binary32 kernel, exercised without a fault: a test hook makes
every stage announce 16 bytes more than its bulk copies deliver, so no stage completes and each
block's wait runs out.  The launch must end by itself, count one timeout per block, write nothing,
and leave the context usable for the next (normal) call."""
import ctypes
import time

import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import component_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_staged_wait_runs_out_and_is_reported():
    import paper_1804_10120_gb300 as tl
    dev = torch.device("cuda", 0)
    n = 4 * 512                                   # four tiles: four blocks, one wait each
    x_np = gridgen.random_grid(n, 45).astype(np.float32)
    x = torch.from_numpy(x_np).to(dev)
    y = torch.full((39, n), float("nan"), dtype=torch.float32, device=dev)
    itab = tl._table(tl._rows(x, 43, "inputs"), 43, n, torch.float32, "cuda", "inputs")
    otab = tl._table(tl._rows(y, 39, "outputs"), 39, n, torch.float32, "cuda", "outputs")
    L = tl.lib()
    L.tl_testing_f32_staged_stall.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    L.tl_testing_f32_staged_stall.restype = ctypes.c_int
    before = tl.tl_wait_timeouts()
    t0 = time.time()
    tl._check(L.tl_testing_f32_staged_stall(ctypes.byref(itab), ctypes.byref(otab), n,
                                            tl._stream_handle(None, dev)))
    torch.cuda.synchronize()
    elapsed = time.time() - t0
    assert tl.tl_wait_timeouts() - before == 4
    assert elapsed < 10.0
    assert bool(torch.isnan(y).all())             # the blocks left before computing anything
    # the context is intact: the normal staged call on the same buffers is correct
    tl.tl_dtg_forward(x, y, dtype="f32")
    torch.cuda.synchronize()
    err = component_errors(y.cpu().numpy().astype(np.float64), oracle.forward(x_np.astype(np.float64)))
    assert err.max() <= 2e-6
    assert tl.tl_wait_timeouts() - before == 4


def test_stall_hook_rejects_unaligned_inputs():
    import paper_1804_10120_gb300 as tl
    dev = torch.device("cuda", 0)
    n = 1024
    buf = torch.zeros((43, n + 1), dtype=torch.float32, device=dev)
    y = torch.zeros((39, n), dtype=torch.float32, device=dev)
    itab = tl._table([buf[k, 1:] for k in range(43)], 43, n, torch.float32, "cuda", "inputs")
    otab = tl._table(tl._rows(y, 39, "outputs"), 39, n, torch.float32, "cuda", "outputs")
    L = tl.lib()
    L.tl_testing_f32_staged_stall.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    L.tl_testing_f32_staged_stall.restype = ctypes.c_int
    assert L.tl_testing_f32_staged_stall(ctypes.byref(itab), ctypes.byref(otab), n, tl._stream_handle(None, dev)) == 2


def test_staged_batched_waits_give_up_and_leave_outputs_untouched():
    """The staged batched kernel's waits on its bulk copies are bounded as well: with every stage
    announcing 16 bytes that never arrive, each block gives up, counts it, lets its copies land and
    leaves; nothing is written, and the next normal launch of the same plan is correct."""
    import paper_1804_10120_gb300 as tl
    from tests.test_gpu_batched import make_batch
    hosts, xs, ys = make_batch([8, 12, 6], 27)
    plan = tl.BatchPlan(xs, ys)
    plan.set_config(128, 1, 1)
    plan.set_staging(2)
    L = tl.lib()
    L.tl_testing_batched_staged_stall.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.tl_testing_batched_staged_stall.restype = ctypes.c_int
    dev = torch.device("cuda", 0)
    tiles = sum((x.shape[1] + 127) // 128 for x in xs)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = min(tiles, sms)
    before = tl.tl_wait_timeouts()
    t0 = time.time()
    tl._check(L.tl_testing_batched_staged_stall(plan._h, tl._stream_handle(None, dev)))
    torch.cuda.synchronize()
    assert time.time() - t0 < 10.0
    assert tl.tl_wait_timeouts() - before == blocks
    assert all(bool(torch.isnan(y).all()) for y in ys)
    plan.launch()
    torch.cuda.synchronize()
    for x, y in zip(xs, ys):
        assert torch.equal(tl.tl_dtg_forward(x), y)
    plan.check()
    plan.set_staging(0)
    with pytest.raises(tl.TLError):
        tl._check(L.tl_testing_batched_staged_stall(plan._h, tl._stream_handle(None, dev)))
    plan.close()
