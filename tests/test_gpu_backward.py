"""GPU adjoint (tl_dtg_backward and the autograd Function) against the CPU oracle's adjoint, central
finite differences of the GPU forward, and torch autograd through the oracle-checked chain."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import TOL_F64, POINTWISE_F64, POINTWISE_FF, assert_components, assert_pointwise, IN_NAMES

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda", 0)


def upstream(n, seed, which=("gamma", "dtg")):
    """Upstream gradients N(0,1); entries of absent groups are None."""
    g = [None] * 39
    if "ginv" in which:
        g[0:6] = list(gridgen.normal_fields(6, n, seed, 900))
    if "gamma" in which:
        g[6:24] = list(gridgen.normal_fields(18, n, seed, 1100))
    if "dbcov" in which:
        g[24:33] = list(gridgen.normal_fields(9, n, seed, 1200))
    if "dtg" in which:
        g[33:39] = list(gridgen.normal_fields(6, n, seed, 1000))
    return g


def run_bwd(x, gout, dtype="f64"):
    import paper_1804_10120_gb300 as tl
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    gin = tl.tl_dtg_backward(xd, gd, dtype=dtype)
    torch.cuda.synchronize()
    return gin.cpu().numpy()


@pytest.mark.parametrize("dtype", ["f64", "f64_ff"])
@pytest.mark.parametrize("which", [("gamma", "dtg"), ("ginv", "gamma", "dbcov", "dtg"), ("dtg",), ("gamma",),
                                   ("dbcov",), ("ginv",), ("ginv", "dtg")])
def test_adjoint_matches_oracle(which, dtype):
    n = 4096
    x = gridgen.random_grid(n, 3)
    gout = upstream(n, 3, which)
    g = run_bwd(x, gout, dtype)
    ref = oracle.backward(x, gout)
    assert_components(g, ref, TOL_F64, names=IN_NAMES, what="adjoint %s %s" % (dtype, which))
    assert_pointwise(g, ref, POINTWISE_F64 if dtype == "f64" else POINTWISE_FF, names=IN_NAMES,
                     what="adjoint %s %s" % (dtype, which))


def test_ff_adjoint_special_cases():
    """Exact zeros (conformal grid with beta = K = 0), values outside the pair range (binary64 fallback
    per point) and a partially absent upstream group, for the float-float adjoint."""
    x = gridgen.conformal_grid(16)
    n = x.shape[1]
    gout = upstream(n, 4, ("ginv", "gamma", "dbcov", "dtg"))
    assert_components(run_bwd(x, gout, "f64_ff"), oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="ff conformal")
    n = 2048
    x = gridgen.random_grid(n, 44)
    x[31, 0:8] = 2.0 ** 70
    x[6 + 4, 8:16] = -1e200
    gout = upstream(n, 44, ("gamma", "dtg", "dbcov"))
    gout[24 + 2] = None
    y = run_bwd(x, gout, "f64_ff")
    ref = oracle.backward(x, gout)
    for lo, hi in [(0, 8), (8, 16), (16, n)]:
        assert_components(y[:, lo:hi], ref[:, lo:hi], TOL_F64, names=IN_NAMES, what="ff rows %d-%d" % (lo, hi))


def test_adjoint_partial_group_and_all_null():
    n = 1000
    x = gridgen.random_grid(n, 5)
    gout = upstream(n, 5, ("gamma", "dtg", "dbcov"))
    gout[24 + 4] = None          # one nabla beta entry absent inside a present group
    gout[6 + 7] = None
    assert_components(run_bwd(x, gout), oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="partial")
    zero = run_bwd(x, [None] * 39)
    assert np.all(zero == 0.0)


@pytest.mark.parametrize("dtype", ["f64", "f64_ff"])
@pytest.mark.parametrize("n", [1, 127, 129, 65537])
def test_adjoint_ragged(n, dtype):
    x = gridgen.random_grid(n, 50 + n)
    gout = upstream(n, 50 + n, ("ginv", "gamma", "dbcov", "dtg"))
    assert_components(run_bwd(x, gout, dtype), oracle.backward(x, gout), TOL_F64, names=IN_NAMES,
                      what="%s n=%d" % (dtype, n))


def _loss_points(y, gout_d):
    s = torch.zeros(y.shape[1], dtype=torch.float64, device=y.device)
    for c, g in enumerate(gout_d):
        if g is not None:
            s += g * y[c]
    return s


def test_full_size_adjoint_finite_differences():
    """N = 2^22, seed 3, loss sum W dtg + V Gamma.  Central differences (h = 1e-6) of the GPU forward
    on every point at once (points are independent, so perturbing input s everywhere changes each point's
    loss only through its own value), compared with the adjoint at every point for every input array;
    and the oracle's adjoint on a sample of points."""
    import paper_1804_10120_gb300 as tl
    n = 1 << 22
    x = gridgen.random_grid(n, 3)
    gout = upstream(n, 3)
    xd = torch.from_numpy(x).to(dev())
    gd = [None if g is None else torch.from_numpy(g).to(dev()) for g in gout]
    gin = tl.tl_dtg_backward(xd, gd)
    h = 1e-6
    worst = 0.0
    for s in range(43):
        xp = xd.clone(); xp[s] += h
        xm = xd.clone(); xm[s] -= h
        fd = (_loss_points(tl.tl_dtg_forward(xp), gd) - _loss_points(tl.tl_dtg_forward(xm), gd)) / (2 * h)
        err = ((fd - gin[s]).abs() / gin[s].abs().clamp(min=1.0)).max().item()
        worst = max(worst, err)
        assert err <= 1e-7, (IN_NAMES[s], err)
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([np.arange(512), np.arange(n - 512, n), rng.integers(0, n, 15000)]))
    ref = oracle.backward(np.ascontiguousarray(x[:, idx]), [None if g is None else np.ascontiguousarray(g[idx])
                                                            for g in gout])
    gi = gin[:, torch.from_numpy(idx).to(dev())].cpu().numpy()
    assert_components(gi, ref, TOL_F64, names=IN_NAMES, what="N=2^22 sampled adjoint")
    assert_pointwise(gi, ref, POINTWISE_F64, names=IN_NAMES, what="N=2^22 sampled adjoint")
    gin_ff = tl.tl_dtg_backward(xd, gd, dtype="f64_ff")
    gi = gin_ff[:, torch.from_numpy(idx).to(dev())].cpu().numpy()
    assert_components(gi, ref, TOL_F64, names=IN_NAMES, what="N=2^22 sampled float-float adjoint")


def test_autograd_function_matches_oracle_and_torch_autograd():
    """DtgFunction's backward equals the oracle adjoint; at N=64, equals torch autograd through a plain
    float64 torch transcription of the chain."""
    import paper_1804_10120_gb300 as tl
    n = 64
    x = gridgen.random_grid(n, 3)
    gout = upstream(n, 3)
    X = torch.from_numpy(x).to(dev()).requires_grad_(True)
    ginv, gamma, dbcov, dtg = tl.dtg(X)
    V = torch.from_numpy(np.stack(gout[6:24])).to(dev())
    W = torch.from_numpy(np.stack(gout[33:39])).to(dev())
    L = (V * gamma).sum() + (W * dtg).sum()
    L.backward()
    g_ours = X.grad.cpu().numpy()
    assert_components(g_ours, oracle.backward(x, gout), TOL_F64, names=IN_NAMES, what="autograd fn")

    # plain torch transcription (CPU, float64), differentiated by torch autograd
    P = {}
    for p, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        P[(a, b)] = P[(b, a)] = p
    Xc = torch.tensor(x, requires_grad=True)
    idx = torch.tensor([[P[(a, b)] for b in range(3)] for a in range(3)])
    Gm = Xc[0:6][idx]
    Dm = Xc[6:24].reshape(6, 3, n)[idx]
    H = torch.linalg.inv(Gm.permute(2, 0, 1)).permute(1, 2, 0)
    Tm = Dm.permute(1, 0, 2, 3) + Dm.permute(0, 2, 1, 3) - Dm.permute(2, 0, 1, 3)
    Gam = 0.5 * torch.einsum("iln,ljkn->ijkn", H, Tm)
    Nb = Xc[34:43].reshape(3, 3, n) - torch.einsum("kijn,kn->ijn", Gam, Xc[31:34])
    dtgm = -2 * Xc[30] * Xc[24:30][idx] + Nb.permute(1, 0, 2) + Nb
    Lc = 0.0
    for p, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        Lc = Lc + (torch.tensor(gout[33 + p]) * dtgm[a, b]).sum()
        for i in range(3):
            Lc = Lc + (torch.tensor(gout[6 + 6 * i + p]) * Gam[i, a, b]).sum()
    Lc.backward()
    assert_components(g_ours, Xc.grad.numpy(), TOL_F64, names=IN_NAMES, what="vs torch autograd")


def test_autograd_gradcheck_small():
    import paper_1804_10120_gb300 as tl
    x = torch.from_numpy(gridgen.random_grid(8, 9)).to(dev()).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: tl.dtg(t), (x,), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("which", [("gamma", "dtg"), ("ginv", "gamma", "dbcov", "dtg")])
def test_integer_pipe_products_equal_fp64_products_on_extreme_values(which):
    """The binary64 adjoint forms its 59 stand-alone products on the integer pipes; the float-float
    adjoint's fallback evaluates the same reverse pass with FP64 multiplies and is taken at every
    point when beta_0 = 1e30.  On inputs and upstream gradients full of zeros, subnormals, huge values,
    infinities and NaNs the two agree bit for bit."""
    n = 1 << 15
    rng = np.random.default_rng(12)
    x = gridgen.random_grid(n, 48)
    gout = upstream(n, 49, which)
    specials = np.array([0.0, -0.0, 5e-324, -2.5e-310, 1e-160, 1e155, -7e160, 1e300, np.inf, -np.inf,
                         np.nan, 2.0 ** 1023, 2.0 ** -1022])
    pts = rng.integers(0, n, n // 2)
    x[rng.integers(0, 43, n // 2), pts] = specials[rng.integers(0, len(specials), n // 2)]
    for g in gout:
        if g is not None:
            k = rng.integers(0, n, n // 16)
            g[k] = specials[rng.integers(0, len(specials), n // 16)]
    with np.errstate(over="ignore"):
        x[:, : n // 4] *= 2.0 ** rng.integers(-500, 500, n // 4)
    x[31] = 1e30
    g64 = run_bwd(x, gout, "f64")
    gff = run_bwd(x, gout, "f64_ff")
    assert np.array_equal(np.isnan(g64), np.isnan(gff))
    ok = np.isnan(g64) | (g64.view(np.uint64) == gff.view(np.uint64))
    assert ok.all(), np.argwhere(~ok)[:5]
