"""The fused forward + adjoint (tl_dtg_forward_backward): outputs bit for bit those of tl_dtg_forward,
input gradients against the CPU oracle's adjoint, for every combination of upstream-gradient groups,
ragged sizes and the full N = 2^22 grid in the benchmark's launch configuration."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import TOL_F64, POINTWISE_F64, POINTWISE_FF, assert_components, assert_pointwise, IN_NAMES
from tests.test_gpu_backward import upstream

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda", 0)


def run_fused(x, gout):
    import paper_1804_10120_gb300 as tl
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    y, gin = tl.tl_dtg_forward_backward(xd, gd)
    y_sep = tl.tl_dtg_forward(xd)
    torch.cuda.synchronize()
    return y.cpu().numpy(), gin.cpu().numpy(), y_sep.cpu().numpy()


@pytest.mark.parametrize("which", [("gamma", "dtg"), ("ginv", "gamma", "dbcov", "dtg"), ("dtg",), ("gamma",),
                                   ("dbcov",), ("ginv",), ("ginv", "dtg"), ()])
def test_fused_matches_forward_and_oracle_adjoint(which):
    n = 4096
    x = gridgen.random_grid(n, 3)
    gout = upstream(n, 3, which)
    y, gin, y_sep = run_fused(x, gout)
    assert np.array_equal(y.view(np.uint64), y_sep.view(np.uint64))
    if not which:
        assert np.all(gin == 0.0)
        return
    assert_components(gin, oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="fused adjoint %s" % (which,))


@pytest.mark.parametrize("n", [1, 2, 127, 129, 255, 65537])
def test_fused_ragged(n):
    x = gridgen.random_grid(n, 70 + n)
    gout = upstream(n, 70 + n, ("ginv", "gamma", "dbcov", "dtg"))
    y, gin, y_sep = run_fused(x, gout)
    assert np.array_equal(y.view(np.uint64), y_sep.view(np.uint64))
    assert_components(gin, oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="fused n=%d" % n)


def test_fused_partial_groups_and_conformal_grid():
    n = 1000
    x = gridgen.random_grid(n, 5)
    gout = upstream(n, 5, ("gamma", "dtg", "dbcov"))
    gout[24 + 4] = None
    gout[6 + 7] = None
    _, gin, _ = run_fused(x, gout)
    assert_components(gin, oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="fused partial")
    x = gridgen.conformal_grid(16)
    gout = upstream(x.shape[1], 6, ("ginv", "gamma", "dbcov", "dtg"))
    y, gin, y_sep = run_fused(x, gout)
    assert np.array_equal(y.view(np.uint64), y_sep.view(np.uint64))
    assert_components(gin, oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="fused conformal")


def test_fused_full_size():
    """N = 2^22, seed 3, loss sum W dtg + V Gamma, in the benchmark's launch: outputs bitwise equal to
    the forward kernel on every point, gradients within the gate of the (finite-difference-checked)
    adjoint kernel on every point and of the oracle on a sample."""
    import paper_1804_10120_gb300 as tl
    n = 1 << 22
    x = gridgen.random_grid(n, 3)
    gout = upstream(n, 3)
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    y, gin = tl.tl_dtg_forward_backward(xd, gd)
    assert torch.equal(y.view(torch.int64), tl.tl_dtg_forward(xd).view(torch.int64))
    gsep = tl.tl_dtg_backward(xd, gd)
    err = ((gin - gsep).abs().amax(dim=1) / gsep.abs().amax(dim=1)).max().item()
    assert err <= TOL_F64, err
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([np.arange(300), np.arange(n - 300, n), rng.integers(0, n, 15000)]))
    ref = oracle.backward(np.ascontiguousarray(x[:, idx]),
                          [None if g is None else np.ascontiguousarray(g[idx]) for g in gout])
    gi = gin[:, torch.from_numpy(idx).to(dev())].cpu().numpy()
    assert_components(gi, ref, TOL_F64, names=IN_NAMES, what="N=2^22 sampled fused adjoint")
    assert_pointwise(gi, ref, POINTWISE_F64, names=IN_NAMES, what="N=2^22 sampled fused adjoint")


def test_fused_empty_and_unsupported():
    import paper_1804_10120_gb300 as tl
    x = torch.empty((43, 0), dtype=torch.float64, device=dev())
    y, gin = tl.tl_dtg_forward_backward(x, [None] * 39)
    assert y.shape == (39, 0) and gin.shape == (43, 0)
    x = torch.from_numpy(gridgen.random_grid(16, 1)).to(dev(), torch.float32)
    with pytest.raises(tl.TLError) as e:
        tl.tl_dtg_forward_backward(x, [None] * 39, dtype="f32")
    assert e.value.status == 3


def run_fused_ff(x, gout):
    import paper_1804_10120_gb300 as tl
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    y, gin = tl.tl_dtg_forward_backward(xd, gd, dtype="f64_ff")
    y_sep = tl.tl_dtg_forward(xd, dtype="f64_ff")
    torch.cuda.synchronize()
    return y.cpu().numpy(), gin.cpu().numpy(), y_sep.cpu().numpy()


@pytest.mark.parametrize("which", [("gamma", "dtg"), ("ginv", "gamma", "dbcov", "dtg"), ("dtg",), ("gamma",),
                                   ("dbcov",), ("ginv",), ("ginv", "dtg")])
def test_fused_ff_matches_ff_forward_and_oracle_adjoint(which):
    n = 4096
    x = gridgen.random_grid(n, 3)
    gout = upstream(n, 3, which)
    y, gin, y_sep = run_fused_ff(x, gout)
    assert np.array_equal(y.view(np.uint64), y_sep.view(np.uint64))
    ref = oracle.backward(x, gout)
    assert_components(gin, ref, TOL_F64, names=IN_NAMES, what="fused ff %s" % (which,))
    assert_pointwise(gin, ref, POINTWISE_FF, names=IN_NAMES, what="fused ff %s" % (which,))


@pytest.mark.parametrize("n", [1, 129, 255, 65537])
def test_fused_ff_ragged_and_conformal(n):
    x = gridgen.random_grid(n, 90 + n)
    gout = upstream(n, 90 + n, ("ginv", "gamma", "dbcov", "dtg"))
    y, gin, y_sep = run_fused_ff(x, gout)
    assert np.array_equal(y.view(np.uint64), y_sep.view(np.uint64))
    assert_components(gin, oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="fused ff n=%d" % n)
    x = gridgen.conformal_grid(12)
    gout = upstream(x.shape[1], 91, ("ginv", "gamma", "dbcov", "dtg"))
    y, gin, y_sep = run_fused_ff(x, gout)
    assert np.array_equal(y.view(np.uint64), y_sep.view(np.uint64))
    assert_components(gin, oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="fused ff conformal")


def test_fused_ff_binary64_fallback():
    """Points whose inputs fall outside the pair range (beta_0 = 2^70) are evaluated in binary64, outputs
    and gradients: bit for bit the binary64 fused pass (the float-float forward also takes binary64
    there).  Points whose upstream gradients do (a Gamma^0_12 upstream gradient of 1e200) keep their
    float-float outputs and take their gradients from the binary64 adjoint, bit for bit those of
    tl_dtg_backward.  So the outputs equal the float-float forward's at every point.  The oracle gates
    the untouched points and the points 0-8; at the points 8-16 its own sum adds and removes terms of
    ~1e199 (the two halves of the bracket's d_2 g_12 - d_2 g_21) and drops the O(1) terms between
    them, so the exact gradient there is the one without cancellation."""
    import paper_1804_10120_gb300 as tl
    n = 2048
    x = gridgen.random_grid(n, 44)
    x[31, 0:8] = 2.0 ** 70
    gout = upstream(n, 45, ("ginv", "gamma", "dbcov", "dtg"))
    gout[6 + 4][8:16] = 1e200
    y, gin, y_sep = run_fused_ff(x, gout)
    assert np.array_equal(y.view(np.uint64), y_sep.view(np.uint64))
    ref = oracle.backward(x, gout)
    for lo, hi in [(0, 8), (16, n)]:
        assert_components(gin[:, lo:hi], ref[:, lo:hi], TOL_F64, names=IN_NAMES, what="fused ff rows %d-%d" % (lo, hi))
    y64, gin64, _ = run_fused(x, gout)
    assert np.array_equal(y[:, 0:8].view(np.uint64), y64[:, 0:8].view(np.uint64))
    assert np.array_equal(gin[:, 0:8].view(np.uint64), gin64[:, 0:8].view(np.uint64))
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    gb = tl.tl_dtg_backward(xd, gd).cpu().numpy()
    assert np.array_equal(gin[:, 8:16].view(np.uint64), gb[:, 8:16].view(np.uint64))


def test_fused_ff_full_size():
    import paper_1804_10120_gb300 as tl
    n = 1 << 22
    x = gridgen.random_grid(n, 3)
    gout = upstream(n, 3)
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    y, gin = tl.tl_dtg_forward_backward(xd, gd, dtype="f64_ff")
    assert torch.equal(y.view(torch.int64), tl.tl_dtg_forward(xd, dtype="f64_ff").view(torch.int64))
    rng = np.random.default_rng(41)
    idx = np.unique(np.concatenate([np.arange(300), np.arange(n - 300, n), rng.integers(0, n, 15000)]))
    ref = oracle.backward(np.ascontiguousarray(x[:, idx]),
                          [None if g is None else np.ascontiguousarray(g[idx]) for g in gout])
    gi = gin[:, torch.from_numpy(idx).to(dev())].cpu().numpy()
    assert_components(gi, ref, TOL_F64, names=IN_NAMES, what="N=2^22 sampled fused ff adjoint")


def test_fused_in_cuda_graph_and_with_scattered_tables():
    """The fused entry point only enqueues a launch, so it can be captured in a CUDA graph; and it takes
    any element-aligned tables: rows of buffers at irregular offsets (not 16-byte aligned) give the
    same bits as the contiguous [43, n] layout."""
    import paper_1804_10120_gb300 as tl
    n = 5000
    x = gridgen.random_grid(n, 8)
    gout = upstream(n, 8, ("ginv", "gamma", "dbcov", "dtg"))
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    y_ref, g_ref = tl.tl_dtg_forward_backward(xd, gd)
    torch.cuda.synchronize()

    def scattered(count, like=None):
        offs = [k * (n + 40) + (k % 3) for k in range(count)]      # element offsets 0, 1, 2 mod 3
        buf = torch.full((offs[-1] + n + 4,), float("nan"), dtype=torch.float64, device=dev())
        rows = [buf[o:o + n] for o in offs]
        if like is not None:
            for r, src in zip(rows, like):
                r.copy_(src)
        return rows
    xr = scattered(43, xd)
    yr, gr = scattered(39), scattered(43)
    tl.tl_dtg_forward_backward(xr, gd, yr, gr)
    torch.cuda.synchronize()
    assert torch.equal(torch.stack(yr), y_ref) and torch.equal(torch.stack(gr), g_ref)

    y = torch.full_like(y_ref, float("nan"))
    g = torch.full_like(g_ref, float("nan"))
    side = torch.cuda.Stream(dev())
    side.wait_stream(torch.cuda.current_stream(dev()))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        tl.tl_dtg_forward_backward(xd, gd, y, g, stream=side)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref) and torch.equal(g, g_ref)


def test_fused_on_extreme_values():
    """Inputs and upstream gradients full of zeros, subnormals, huge values, infinities and NaNs on some
    points: the fused kernel's outputs stay bit for bit those of the forward kernel (the same body, its
    integer-pipe products falling back to the FP64 multiply where they must), and on the points left
    untouched the gradients still meet the oracle's gate."""
    import paper_1804_10120_gb300 as tl
    n = 1 << 14
    rng = np.random.default_rng(33)
    x = gridgen.random_grid(n, 33)
    gout = upstream(n, 34, ("ginv", "gamma", "dbcov", "dtg"))
    specials = np.array([0.0, -0.0, 5e-324, -2.5e-310, 1e-160, 1e155, -7e160, 1e300, np.inf, -np.inf, np.nan])
    hit = np.zeros(n, dtype=bool)
    pts = rng.integers(0, n // 2, n // 4)
    x[rng.integers(0, 43, n // 4), pts] = specials[rng.integers(0, len(specials), n // 4)]
    hit[pts] = True
    for g in gout:
        k = rng.integers(0, n // 2, n // 32)
        g[k] = specials[rng.integers(0, len(specials), n // 32)]
        hit[k] = True
    with np.errstate(all="ignore"):
        y, gin, y_sep = run_fused(x, gout)
    assert np.array_equal(np.isnan(y), np.isnan(y_sep))
    ok = np.isnan(y) | (y.view(np.uint64) == y_sep.view(np.uint64))
    assert ok.all(), np.argwhere(~ok)[:5]
    clean = np.nonzero(~hit)[0]
    assert clean.size > n // 3
    ref = oracle.backward(np.ascontiguousarray(x[:, clean]), [np.ascontiguousarray(g[clean]) for g in gout])
    assert_components(gin[:, clean], ref, TOL_F64, names=IN_NAMES, what="fused, untouched points")
