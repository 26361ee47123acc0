"""The float-float primitives of the TL_F64_FF kernels against exact rational arithmetic, through the
tl_testing_ff hook (include/tl_testing.h)."""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def hook():
    import paper_1804_10120_gb300 as tl
    L = tl.lib()
    f = L.tl_testing_ff
    f.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 7 + [ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def run(op, *arrays):
    dev = torch.device("cuda", 0)
    ts = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays]
    n = ts[0].numel()
    y = torch.empty(n, dtype=torch.float64, device=dev)
    ptrs = [t.data_ptr() for t in ts] + [None] * (6 - len(ts))
    rc = hook()(op, *ptrs, y.data_ptr(), n, None)
    assert rc == 0
    torch.cuda.synchronize()
    return y.cpu().numpy()


def sample(n, seed, lo_exp=-70, hi_exp=62):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n)
    ex = rng.integers(lo_exp, hi_exp, n)
    sign = rng.choice([-1.0, 1.0], n)
    v = sign * np.ldexp(mant, ex)
    special = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** 40, 2.0 ** -60, np.nextafter(2.0, 0), np.nextafter(1.0, 2),
                        1.0 + 2.0 ** -52, -(2.0 - 2.0 ** -52), 3.0, 1 / 3, np.pi, -np.e])
    return np.concatenate([special, v])


def test_roundtrip():
    x = sample(20000, 1)
    y = run(0, x)
    for a, b in zip(x, y):
        if a == 0:
            assert b == 0
            continue
        assert abs(Fraction(b) - Fraction(a)) <= Fraction(2) ** -47 * abs(Fraction(a)), (a, b)


def test_subtraction_with_cancellation():
    a = sample(5000, 2, -30, 30)
    rng = np.random.default_rng(3)
    # b close to a: heavy cancellation; b random: none
    b = np.where(rng.random(a.size) < 0.5, a * (1 + rng.normal(0, 1e-9, a.size)), sample(5000, 4, -30, 30)[:a.size])
    y = run(1, a, b)
    for u, v, r in zip(a, b, y):
        exact = Fraction(u) - Fraction(v)
        scale = max(abs(Fraction(u)), abs(Fraction(v)))
        assert abs(Fraction(r) - exact) <= Fraction(2) ** -46 * scale, (u, v, r)


def test_dot3():
    rng = np.random.default_rng(5)
    arrs = [rng.normal(0, 1, 5000) * np.ldexp(1.0, rng.integers(-20, 20, 5000)) for _ in range(6)]
    arrs[0][:10] = 0.0
    y = run(2, *arrs)
    for k in range(5000):
        t = [Fraction(arrs[2 * q][k]) * Fraction(arrs[2 * q + 1][k]) for q in range(3)]
        exact = sum(t)
        scale = sum(abs(v) for v in t)
        # input splits 2 x 2^-48, dropped lo*lo 2^-48, two cross-term roundings and four low-order
        # additions of ~2^-47 each, merge 2^-52:  below 2^-44 of the sum of |terms|
        assert abs(Fraction(y[k]) - exact) <= Fraction(2) ** -44 * scale, k
