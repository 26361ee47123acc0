"""GPU parity of the fused forward chain against the CPU oracle, through the C ABI.

Binary64 forms are gated per output component at max|y - y_ref| <= 1e-12 * max|y_ref| (parity.py);
the binary32-storage form at the bound derived for it (TOL_F32_* below)."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import TOL_F64, POINTWISE_F64, POINTWISE_FF, assert_components, assert_pointwise, component_errors, OUT_NAMES

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Binary32 form.  Computation error alone (oracle evaluated on the binary32-rounded inputs): the chain
# is at most ~6 dependent roundings deep (bracket 2, raise 3, covariant derivative 3, Eq. 5 2) and each
# output is a short sum whose terms are bounded by its component's maximum, so a normwise error of a
# few tens of ulp(2^-24 = 6e-8) bounds it: 2e-6.  End to end against the binary64 inputs the storage
# rounding of the 43 inputs (relative 2^-24 each) enters with the same conditioning: 5e-6.
TOL_F32_COMPUTE = 2e-6
TOL_F32_E2E = 5e-6


def dev():
    return torch.device("cuda", 0)


def run_f64(x_np, dtype="f64"):
    import paper_1804_10120_gb300 as tl
    x = torch.from_numpy(x_np).to(dev())
    y = tl.tl_dtg_forward(x, dtype=dtype)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_config0_f64_all_components():
    x = gridgen.random_grid(4096, 0)
    y = run_f64(x)
    y_ref = oracle.forward(x)
    assert_components(y, y_ref, TOL_F64, what="N=4096 seed 0 f64")
    assert_pointwise(y, y_ref, POINTWISE_F64, what="N=4096 seed 0 f64")


@pytest.mark.parametrize("n", [1, 2, 31, 255, 257, 4097, 100003])
def test_ragged_sizes_f64(n):
    x = gridgen.random_grid(n, 100 + n)
    y = run_f64(x)
    assert_components(y, oracle.forward(x), TOL_F64, what="n=%d" % n)


def test_empty_grid():
    import paper_1804_10120_gb300 as tl
    x = torch.empty((43, 0), dtype=torch.float64, device=dev())
    y = tl.tl_dtg_forward(x)
    torch.cuda.synchronize()
    assert y.shape == (39, 0)


def test_unaligned_and_scattered_tables():
    """Arrays that are only 8-byte aligned, each from its own allocation, with a stream that is not the
    default one."""
    import paper_1804_10120_gb300 as tl
    n = 5001
    x = gridgen.random_grid(n, 77)
    ins = []
    for s in range(43):
        buf = torch.empty(n + 1, dtype=torch.float64, device=dev())
        v = buf[1:]                        # shifted by 8 bytes
        v.copy_(torch.from_numpy(x[s]))
        ins.append(v)
    outs = []
    for s in range(39):
        buf = torch.empty(n + 3, dtype=torch.float64, device=dev())
        outs.append(buf[3:])
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    tl.tl_dtg_forward(ins, outs, stream=st)
    st.synchronize()
    y = np.stack([o.cpu().numpy() for o in outs])
    assert_components(y, oracle.forward(x), TOL_F64, what="unaligned")


def test_conformal_grid_exact_zeros_f64():
    """Conformally flat metric, beta = K = 0: nabla beta and d_t g vanish exactly; Gamma matches."""
    side = 32
    x = gridgen.conformal_grid(side)
    y = run_f64(x)
    assert np.all(y[24:39] == 0.0)
    assert_components(y, oracle.forward(x), TOL_F64, what="conformal f64")


def test_full_size_sampled_f64():
    """N = 2^24 (256^3), seed 1, in the launch configuration the benchmark times; the oracle checks a
    sample of 65536 points (random, plus the first and last 1024)."""
    import paper_1804_10120_gb300 as tl
    n = 1 << 24
    x = gridgen.random_grid(n, 1)
    xd = torch.from_numpy(x).to(dev())
    y = tl.tl_dtg_forward(xd)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([np.arange(1024), np.arange(n - 1024, n), rng.integers(0, n, 63488)]))
    ys = y[:, torch.from_numpy(idx).to(dev())].cpu().numpy()
    y_ref = oracle.forward(np.ascontiguousarray(x[:, idx]))
    assert_components(ys, y_ref, TOL_F64, what="N=2^24 sampled")
    assert_pointwise(ys, y_ref, POINTWISE_F64, what="N=2^24 sampled")
    # every output written: no NaN / untouched memory anywhere
    assert bool(torch.isfinite(y).all())


def test_f32_storage_form():
    x = gridgen.random_grid(1 << 16, 4)
    x32 = x.astype(np.float32)
    import paper_1804_10120_gb300 as tl
    y = tl.tl_dtg_forward(torch.from_numpy(x32).to(dev()), dtype="f32")
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    compute = component_errors(y, oracle.forward(x32.astype(np.float64)))
    e2e = component_errors(y, oracle.forward(x))
    assert compute.max() <= TOL_F32_COMPUTE, dict(zip(OUT_NAMES, compute))
    assert e2e.max() <= TOL_F32_E2E, dict(zip(OUT_NAMES, e2e))


def test_f32_conformal_exact_zeros():
    side = 32
    x = gridgen.conformal_grid(side).astype(np.float32)
    import paper_1804_10120_gb300 as tl
    y = tl.tl_dtg_forward(torch.from_numpy(x).to(dev()), dtype="f32")
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    assert np.all(y[24:39] == 0.0)
    err = component_errors(y.astype(np.float64), oracle.forward(x.astype(np.float64)))
    assert err.max() <= TOL_F32_COMPUTE


def test_host_buffer_entry_point():
    """tl_dtg_forward_host: page-locked host arrays in and out, ragged chunking (n not a multiple of the
    pipeline chunk)."""
    import paper_1804_10120_gb300 as tl
    n = (1 << 20) * 2 + 12345
    x = gridgen.random_grid(n, 8)
    xin = torch.from_numpy(x).pin_memory()
    yout = torch.empty((39, n), dtype=torch.float64).pin_memory()
    tl.tl_dtg_forward_host(xin, yout)
    torch.cuda.synchronize()
    y = yout.numpy()
    rng = np.random.default_rng(8)
    idx = np.unique(np.concatenate([np.arange(2048), np.arange((1 << 20) - 1024, (1 << 20) + 1024),
                                    np.arange(n - 2048, n), rng.integers(0, n, 20000)]))
    assert_components(y[:, idx], oracle.forward(np.ascontiguousarray(x[:, idx])), TOL_F64, what="host path")


def test_host_entry_point_separate_arrays_and_f32():
    """Host tables whose arrays are separate allocations (per-array copies), binary32, n spanning four
    chunks with a ragged tail, called twice in a row on a non-default stream."""
    import paper_1804_10120_gb300 as tl
    n = 3 * (1 << 19) + 777
    x = gridgen.random_grid(n, 9).astype(np.float32)
    ins = [torch.from_numpy(x[s].copy()).pin_memory() for s in range(43)]
    outs = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(39)]
    st = torch.cuda.Stream()
    for _ in range(2):
        for o in outs:
            o.fill_(float("nan"))
        tl.tl_dtg_forward_host(ins, outs, dtype="f32", stream=st)
        st.synchronize()
        y = np.stack([o.numpy() for o in outs]).astype(np.float64)
        rng = np.random.default_rng(9)
        idx = np.unique(np.concatenate([np.arange(1000), np.arange(n - 1000, n), rng.integers(0, n, 20000)]))
        err = component_errors(y[:, idx], oracle.forward(np.ascontiguousarray(x[:, idx].astype(np.float64))))
        assert err.max() <= TOL_F32_COMPUTE
        assert not np.isnan(y).any()


def test_device_check_rejects_nothing_on_sm103():
    import paper_1804_10120_gb300 as tl
    assert torch.cuda.get_device_capability(0) == (10, 3)
    assert tl.lib().tl_version() >= 10000


# --------------------------------------------------------------------------- float-float contractions

def test_ff_config0_all_components():
    x = gridgen.random_grid(4096, 0)
    y = run_f64(x, dtype="f64_ff")
    assert_components(y, oracle.forward(x), TOL_F64, what="N=4096 seed 0 f64_ff")
    assert_pointwise(y, oracle.forward(x), POINTWISE_FF, what="N=4096 seed 0 f64_ff")


@pytest.mark.parametrize("n", [1, 33, 4099, 100003])
def test_ff_ragged_sizes(n):
    x = gridgen.random_grid(n, 200 + n)
    assert_components(run_f64(x, dtype="f64_ff"), oracle.forward(x), TOL_F64, what="ff n=%d" % n)


def test_ff_full_size_sampled():
    import paper_1804_10120_gb300 as tl
    n = 1 << 24
    x = gridgen.random_grid(n, 1)
    y = tl.tl_dtg_forward(torch.from_numpy(x).to(dev()), dtype="f64_ff")
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([np.arange(1024), np.arange(n - 1024, n), rng.integers(0, n, 63488)]))
    ys = y[:, torch.from_numpy(idx).to(dev())].cpu().numpy()
    y_ref = oracle.forward(np.ascontiguousarray(x[:, idx]))
    assert_components(ys, y_ref, TOL_F64, what="ff N=2^24 sampled")
    assert_pointwise(ys, y_ref, POINTWISE_FF, what="ff N=2^24 sampled")
    assert bool(torch.isfinite(y).all())


def test_ff_exact_zero_cases():
    """Flat metric (Gamma = 0), conformal grid with beta = K = 0 (nabla beta = d_t g = 0): exact zeros
    survive the pair arithmetic."""
    x = gridgen.conformal_grid(24)
    y = run_f64(x, dtype="f64_ff")
    assert np.all(y[24:39] == 0.0)
    assert_components(y, oracle.forward(x), TOL_F64, what="ff conformal")
    x = gridgen.random_grid(777, 31)
    x[0:6] = np.array([1, 0, 0, 1, 0, 1.0])[:, None]
    x[6:24] = 0.0
    y = run_f64(x, dtype="f64_ff")
    assert np.all(y[6:24] == 0.0)
    # d_j beta_i passes through a pair (48 significant bits): equal within the gate, not bitwise
    assert_components(y, oracle.forward(x), TOL_F64, what="ff flat")


def test_ff_extreme_values_and_fallback():
    """Values the pair format cannot carry (|x| >= 2^63, inf) send their point through the all-binary64
    evaluation; tiny, subnormal, power-of-two and negative-zero values go through the pairs."""
    n = 4096
    x = gridgen.random_grid(n, 41)
    x[31, 0:8] = 2.0 ** 70                 # huge shift: fallback path
    x[34, 8:16] = -3.0e30                  # huge d_j beta_i (below 2^127 but above 2^63): fallback
    x[6 + 5, 16:24] = 1e300                # huge metric derivative: fallback
    x[31:34, 24:32] = 1e-40                # tiny shift (no lo part)
    x[34:43, 32:40] = 5e-324               # subnormal d beta
    x[6:24, 40:48] = 2.0 ** -30            # powers of two in the bracket
    x[0:6, 48:56] = np.array([2.0, 0, 0, 4.0, 0, 8.0])[:, None]   # diagonal powers of two: exact inverse
    x[31:34, 56:64] = -0.0
    y = run_f64(x, dtype="f64_ff")
    y_ref = oracle.forward(x)
    # huge values make the per-component maxima huge; check the extreme rows pointwise in their own
    # scale and the rest of the grid with the standard gate
    for lo, hi in [(0, 8), (8, 16), (16, 24)]:
        assert_components(y[:, lo:hi], y_ref[:, lo:hi], TOL_F64, what="fallback rows %d-%d" % (lo, hi))
    assert_components(y[:, 24:], y_ref[:, 24:], TOL_F64, what="tiny/pow2 rows")
    x[31, 64:72] = np.inf
    y = run_f64(x[:, 64:72].copy(), dtype="f64_ff")
    y_ref = oracle.forward(x[:, 64:72].copy())
    assert np.array_equal(np.isnan(y), np.isnan(y_ref)) and np.array_equal(np.isinf(y), np.isinf(y_ref))


def test_f32_rare_operands_take_general_conversions():
    """Subnormal binary32 metric entries (outside the integer fast conversion's range) are evaluated by
    the out-of-line general path and still match."""
    x = gridgen.random_grid(2048, 43).astype(np.float32)
    x[1, 0:64] = np.float32(1e-40)        # subnormal g_01
    x[2, 64:128] = np.float32(0.0)
    x[2, 128:192] = np.float32(-0.0)
    import paper_1804_10120_gb300 as tl
    y = tl.tl_dtg_forward(torch.from_numpy(x).to(dev()), dtype="f32")
    torch.cuda.synchronize()
    err = component_errors(y.cpu().numpy().astype(np.float64), oracle.forward(x.astype(np.float64)))
    assert err.max() <= TOL_F32_COMPUTE


@pytest.mark.parametrize("n", [1, 255, 256, 257, 4099, 3 * 256 * 152 + 77])
def test_f32_staged_equals_plain_kernel_bitwise(n):
    """16-byte aligned input tables take the shared-memory-staged kernel (tiles of 256 points, the
    last n % 256 points by the plain kernel); the same inputs one element off alignment take the plain
    kernel alone.  Both evaluate the same binary32 chain, so the outputs agree bit for bit, and they
    meet the oracle bound; no bounded wait gives up."""
    import paper_1804_10120_gb300 as tl
    timeouts = tl.tl_wait_timeouts()
    x = gridgen.random_grid(n, 44).astype(np.float32)
    npad = (n + 3) // 4 * 4                       # rows start on 16-byte boundaries
    abuf = torch.zeros((43, npad), dtype=torch.float32, device=dev())
    abuf[:, :n] = torch.from_numpy(x).to(dev())
    xa = [abuf[k, :n] for k in range(43)]
    assert all(r.data_ptr() % 16 == 0 for r in xa)
    buf = torch.empty((43, n + 1), dtype=torch.float32, device=dev())
    buf[:, 1:] = abuf[:, :n]
    xu = buf[:, 1:]
    assert xu[0].data_ptr() % 16 != 0
    ya = tl.tl_dtg_forward(xa, dtype="f32")
    yu = tl.tl_dtg_forward([xu[k] for k in range(43)], dtype="f32")
    torch.cuda.synchronize()
    assert torch.equal(ya, yu)
    idx = np.unique(np.linspace(0, n - 1, min(n, 3000)).astype(np.int64))
    err = component_errors(ya.cpu().numpy()[:, idx].astype(np.float64), oracle.forward(x[:, idx].astype(np.float64)))
    assert err.max() <= TOL_F32_COMPUTE
    assert tl.tl_wait_timeouts() == timeouts


@pytest.mark.parametrize("dtype", ["f64", "f64_ff", "f32"])
def test_single_grid_forward_in_cuda_graph(dtype):
    """Each forward form captured in a CUDA graph (the staged binary32 kernel included: its launch
    sets a function attribute, which is not a stream operation) replays to the eager result, bit for
    bit, with a ragged tail."""
    import paper_1804_10120_gb300 as tl
    n = 5 * 512 * 152 + 300
    td = torch.float32 if dtype == "f32" else torch.float64
    x = torch.from_numpy(gridgen.random_grid(n, 46)).to(dev(), td)
    y_eager = tl.tl_dtg_forward(x, dtype=dtype)
    y = torch.empty_like(y_eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tl.tl_dtg_forward(x, y, dtype=dtype, stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, y_eager)


def test_integer_pipe_products_equal_fp64_products_on_extreme_values():
    """The binary64 kernel forms its stand-alone products on the integer pipes; the float-float
    kernel's fallback path evaluates the same chain with FP64 multiplies.  With beta_0 = 1e30 every
    point takes that fallback, so on inputs full of zeros, subnormals, huge values, infinities and
    NaNs (products overflowing, underflowing, special) the two must agree bit for bit."""
    import paper_1804_10120_gb300 as tl
    n = 1 << 16
    rng = np.random.default_rng(11)
    x = gridgen.random_grid(n, 47)
    specials = np.array([0.0, -0.0, 5e-324, -2.5e-310, 1e-160, 3e-155, 1e155, -7e160, 1e300, np.inf,
                         -np.inf, np.nan, 2.0 ** 1023, 2.0 ** -1022])
    pts = rng.integers(0, n, n // 2)
    comps = rng.integers(0, 43, n // 2)
    x[comps, pts] = specials[rng.integers(0, len(specials), n // 2)]
    scale = 2.0 ** rng.integers(-500, 500, n)      # whole points scaled towards both thresholds
    with np.errstate(over="ignore"):
        x[:, : n // 4] *= scale[: n // 4]
    x[31] = 1e30                                   # beta_0 outside the pair range: every point falls back
    y64 = run_f64(x, "f64")
    yff = run_f64(x, "f64_ff")
    assert np.array_equal(np.isnan(y64), np.isnan(yff))
    ok = np.isnan(y64) | (y64.view(np.uint64) == yff.view(np.uint64))
    assert ok.all(), np.argwhere(~ok)[:5]


def test_f32_full_size_sampled_and_conformal_256():
    """The binary32 workloads at full size in the benchmark's launch configuration (the staged kernel:
    16-byte aligned rows of a [43, 2^24] buffer): N = 2^24 random grid (seed 4) and the conformal 256^3
    grid, each checked on 65536 sampled points against the oracle on the binary32-rounded inputs;
    every output written; the conformal grid's exact zeros stay exact everywhere."""
    import paper_1804_10120_gb300 as tl
    n = 1 << 24
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([np.arange(1024), np.arange(n - 1024, n), rng.integers(0, n, 63488)]))
    for x in (gridgen.random_grid(n, 4).astype(np.float32), gridgen.conformal_grid(256).astype(np.float32)):
        xd = torch.from_numpy(x).to(dev())
        assert xd[1].data_ptr() % 16 == 0
        y = tl.tl_dtg_forward(xd, dtype="f32")
        torch.cuda.synchronize()
        ys = y[:, torch.from_numpy(idx).to(dev())].cpu().numpy().astype(np.float64)
        err = component_errors(ys, oracle.forward(np.ascontiguousarray(x[:, idx]).astype(np.float64)))
        assert err.max() <= TOL_F32_COMPUTE, dict(zip(OUT_NAMES, err))
        assert bool(torch.isfinite(y).all())
        del xd, y
    y = tl.tl_dtg_forward(torch.from_numpy(x).to(dev()), dtype="f32")
    assert bool((y[24:39] == 0).all())              # conformal: dbcov and dtg vanish exactly


@pytest.mark.parametrize("dtype", ["f64", "f64_ff"])
def test_singular_metric_matches_oracle_special_values(dtype):
    """The degenerate case of the method: a singular metric (det g = 0; rank 2 and rank 1, and the same
    metrics negated).  g^ij = cofactor / det becomes +-inf or NaN and propagates through every output;
    the kernel's reciprocal-times-cofactor form must give the oracle's pattern of NaN and signed
    infinities."""
    n = 64
    x = gridgen.random_grid(n, 51)
    rank2 = np.array([1.0, 1.0, 0.0, 1.0, 0.0, 2.0])      # rows 0 and 1 equal
    rank1 = np.array([1.0, 2.0, 3.0, 4.0, 6.0, 9.0])      # outer product of (1, 2, 3)
    x[0:6, 0:32] = rank2[:, None]
    x[0:6, 32:64] = rank1[:, None]
    x[0:6, 16:32] *= -1.0                                 # the rank-2 metric negated
    with np.errstate(all="ignore"):
        y_ref = oracle.forward(x)
    y = run_f64(x, dtype=dtype)
    assert np.array_equal(np.isnan(y), np.isnan(y_ref))
    assert np.array_equal(np.isposinf(y), np.isposinf(y_ref)) and np.array_equal(np.isneginf(y), np.isneginf(y_ref))


def test_small_grid_kernel_equals_full_kernel_bitwise():
    """Grids of less than one block per SM run a kernel with FP64 multiplies instead of the integer-pipe
    products; the results are the same bits.  A 4096-point grid (the small kernel) against the same
    points repeated 16 times (65536 points: the full kernel), on random and extreme inputs."""
    n = 4096
    rng = np.random.default_rng(23)
    x = gridgen.random_grid(n, 23)
    specials = np.array([0.0, -0.0, 5e-324, 1e-160, 1e155, -7e160, np.inf, np.nan, 2.0 ** -1022])
    pts = rng.integers(0, n, n // 4)
    x[rng.integers(0, 43, n // 4), pts] = specials[rng.integers(0, len(specials), n // 4)]
    with np.errstate(over="ignore"):
        x[:, : n // 8] *= 2.0 ** rng.integers(-500, 500, n // 8)
    y_small = run_f64(x)
    y_full = run_f64(np.ascontiguousarray(np.tile(x, (1, 16))))
    for k in range(16):
        yk = y_full[:, k * n:(k + 1) * n]
        assert np.array_equal(np.isnan(y_small), np.isnan(yk))
        ok = np.isnan(y_small) | (y_small.view(np.uint64) == yk.view(np.uint64))
        assert ok.all(), np.argwhere(~ok)[:5]
