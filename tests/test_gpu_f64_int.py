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
