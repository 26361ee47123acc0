"""Binary64 operations done on the integer pipes (mul_int in the kernels) against the IEEE operation
computed by the host CPU, bit for bit: random bit patterns over the whole format (zeros, subnormals,
inf, nan included), products near overflow and underflow, and constructed rounding ties."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(op, a, b, c=None):
    import paper_1804_10120_gb300 as tl
    dev = torch.device("cuda", 0)
    ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    tc = torch.from_numpy(c).to(dev) if c is not None else None
    y = torch.empty_like(ta)
    L = tl.lib()
    L.tl_testing_f64_int.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    L.tl_testing_f64_int.restype = ctypes.c_int
    st = torch.cuda.current_stream(dev).cuda_stream
    assert L.tl_testing_f64_int(op, ta.data_ptr(), tb.data_ptr(), tc.data_ptr() if tc is not None else None,
                                y.data_ptr(), len(a), st) == 0
    torch.cuda.synchronize()
    return y.cpu().numpy()


def same_bits(y, ref):
    yb, rb = y.view(np.uint64), ref.view(np.uint64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(y), nan)
    bad = np.nonzero((yb != rb) & ~nan)[0]
    assert bad.size == 0, [(float.hex(float(y[i])), float.hex(float(ref[i]))) for i in bad[:5]]


def operands(rng, n):
    cases = []
    # uniformly random bit patterns: every exponent, sign, zeros, subnormals, inf, nan
    cases.append((rng.integers(0, 2**64, n, dtype=np.uint64).view(np.float64),
                  rng.integers(0, 2**64, n, dtype=np.uint64).view(np.float64)))
    # the kernels' working range
    cases.append((rng.normal(size=n) * 2.0 ** rng.integers(-30, 30, n), rng.normal(size=n) * 2.0 ** rng.integers(-30, 30, n)))
    # products near the overflow and underflow thresholds, and into the subnormal range
    for lo, hi in ((1000, 1030), (-1080, -1000)):
        ea = rng.integers(lo // 2 - 20, hi // 2 + 20, n)
        cases.append((rng.uniform(1, 2, n) * 2.0 ** ea, rng.uniform(1, 2, n) * 2.0 ** (rng.integers(lo, hi, n) - ea)))
    # exact ties: significand ma times 1.5 leaves exactly half an ulp when ma is odd
    ma = rng.integers(2**52, 2**53, n, dtype=np.int64)
    a = np.ldexp(ma.astype(np.float64), -52) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    cases.append((a, np.full(n, 1.5) * 2.0 ** rng.integers(-5, 5, n)))
    # zeros and infinities against finite and special values
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
                        1.7976931348623157e308, 1.0, -1.0, 3.0])
    sa, sb = np.meshgrid(special, special)
    cases.append((sa.ravel(), sb.ravel()))
    return cases


def test_mul_int_equals_ieee_product():
    rng = np.random.default_rng(7)
    with np.errstate(all="ignore"):
        for a, b in operands(rng, 1 << 20):
            a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
            same_bits(run(0, a, b), a * b)


def rcp_operands(rng, n):
    """Divisors for the reciprocal: the binary32-seeded window [2^-124, 2^125) in magnitude (random
    significands over its whole exponent range, powers of two, all-ones significands, both edges), and
    operands just outside it and special values, which take the IEEE quotient."""
    sign = np.where(rng.random(n) < 0.5, np.uint64(1) << np.uint64(63), np.uint64(0))
    frac = rng.integers(0, 2**52, n, dtype=np.uint64)
    inside = []
    for e in (rng.integers(899, 1148, n), np.full(n, 899), np.full(n, 1147)):
        inside.append(sign | (e.astype(np.uint64) << np.uint64(52)) | frac)
    e = rng.integers(899, 1148, 64).astype(np.uint64) << np.uint64(52)
    inside.append(np.concatenate([e, e | np.uint64(2**52 - 1)]))
    inside = np.concatenate(inside).view(np.float64)
    outside = np.concatenate([
        (sign | (np.full(n, 898, np.uint64) << np.uint64(52)) | frac).view(np.float64),
        (sign | (np.full(n, 1148, np.uint64) << np.uint64(52)) | frac).view(np.float64),
        rng.integers(0, 2**64, n, dtype=np.uint64).view(np.float64),
        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -2.5e-310, 2.2250738585072014e-308,
                  1.7976931348623157e308, 2.0 ** -125, 2.0 ** 125])])
    return inside, outside


def in_window(d):
    """Operands whose reciprocal takes the binary32-seeded path: biased exponent in [899, 1147]."""
    e = (d.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7ff)
    return (e >= 899) & (e <= 1147)


def ulp_distance(y, ref):
    """|y - ref| in units of ref's last place, from the ordered integer images of the two values."""
    def ordered(v):
        b = v.view(np.int64)
        return np.where(b < 0, np.int64(-2**63) - b, b)
    return np.abs(ordered(y) - ordered(ref))


def test_rcp_f64_within_one_ulp_of_ieee_quotient():
    """The kernels' reciprocal (binary32 seed, one third-order step) is within one ulp of the host's IEEE
    1/d everywhere in its window, and equals it bit for bit outside (where it divides)."""
    rng = np.random.default_rng(17)
    inside, outside = rcp_operands(rng, 1 << 20)
    with np.errstate(all="ignore"):
        y = run(1, inside, inside)
        ref = 1.0 / inside
        d = ulp_distance(y, ref)
        assert d.max() <= 1, [(float.hex(float(inside[i])), float.hex(float(y[i]))) for i in np.argsort(d)[-3:]]
        assert (d == 0).mean() > 0.99      # almost always the correctly rounded quotient
        yo = run(1, outside, outside)
        win = in_window(outside)           # random bit patterns land inside the window too
        assert ulp_distance(yo[win], 1.0 / outside[win]).max(initial=0) <= 1
        same_bits(yo[~win], 1.0 / outside[~win])


def test_generated_reciprocal_within_one_ulp():
    """The runtime generator's reciprocal (emitted as CUDA source for a scalar divisor) on the same
    operands, through a one-statement program y = a / s with a = 1."""
    import paper_1804_10120_gb300 as tl
    rng = np.random.default_rng(19)
    inside, outside = rcp_operands(rng, 1 << 18)
    k = tl.JitKernel("in a; in s; out y; y = a / s;")
    dev = torch.device("cuda", 0)
    with np.errstate(all="ignore"):
        for ops, exact in ((inside, False), (outside, True)):
            x = np.stack([np.ones_like(ops), ops])
            y = k.launch(torch.from_numpy(x).to(dev))
            torch.cuda.synchronize()
            y = y.cpu().numpy()[0]
            win = in_window(ops)
            assert ulp_distance(y[win], 1.0 / ops[win]).max(initial=0) <= 1
            same_bits(y[~win], 1.0 / ops[~win])
            assert exact or win.all()
    k.close()


def test_pipe_rate_probe_runs_and_writes_nothing():
    """Every operation of the FP64 pipe-rate probe launches, finishes, and leaves its sink unwritten (the
    chains only decide a store that the probe's operands never trigger); the DFMA rate comes out in
    the range two operations per clock per SM allows."""
    import paper_1804_10120_gb300 as tl
    dev = torch.device("cuda", 0)
    L = tl.lib()
    L.tl_testing_pipe_rate.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p]
    L.tl_testing_pipe_rate.restype = ctypes.c_int
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * sms, 256
    sink = torch.full((blocks * threads,), float("nan"), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    for op in range(9):
        assert L.tl_testing_pipe_rate(op, 64, blocks, threads, sink.data_ptr(), st.cuda_stream) == 0
    torch.cuda.synchronize()
    assert bool(torch.isnan(sink).all())
    iters = 4096
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    assert L.tl_testing_pipe_rate(0, iters, blocks, threads, sink.data_ptr(), st.cuda_stream) == 0
    e1.record(st)
    torch.cuda.synchronize()
    per_s = blocks * threads * 8 * iters / (e0.elapsed_time(e1) * 1e-3)
    per_clk_sm = per_s / (sms * 2.07e9)                # at the highest SM clock of the part
    assert 0.5 < per_clk_sm < 2.2, per_clk_sm


def test_memory_info_gives_the_nominal_hbm_bandwidth():
    """The device memory query: clock x 2 x bus width / 8 is the part's nominal HBM bandwidth, above
    the measured copy bandwidth (which reads a little below nominal)."""
    import json
    import os
    import bench
    import paper_1804_10120_gb300 as tl
    L = tl.lib()
    L.tl_testing_memory_info.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.tl_testing_memory_info.restype = ctypes.c_int
    c, b = ctypes.c_int32(), ctypes.c_int32()
    assert L.tl_testing_memory_info(0, ctypes.byref(c), ctypes.byref(b)) == 0
    gbs = c.value * 1e3 * 2 * b.value / 8 / 1e9
    nominal = bench.nominal_hbm_gbs(torch.device("cuda", 0))
    assert nominal is not None and abs(nominal[0] - gbs) < 1e-6 * gbs
    peaks = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    measured = json.load(open(peaks))["hbm_gbs"] if os.path.exists(peaks) else 6000.0
    assert measured < gbs < 2 * measured, (gbs, measured)
