"""The on-grid forward (derivatives by finite differences inside the kernel) against the FD oracle
followed by the chain oracle."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import TOL_F64, assert_components

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(shape, order, dtype, seed=5, h=None):
    import paper_1804_10120_gb300 as tl
    f = gridgen.periodic_fields(shape, seed)
    h = h or tuple(1.0 / m for m in shape)
    y = tl.tl_dtg_forward_fd(torch.from_numpy(f).to(torch.device("cuda", 0)), shape, h, order, dtype=dtype)
    torch.cuda.synchronize()
    return f, h, y


@pytest.mark.parametrize("dtype", ["f64", "f64_ff"])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("shape", [(16, 12, 10), (1, 1, 9), (3, 2, 1), (37, 5, 7)])
@pytest.mark.parametrize("spacing", ["per_axis", "equal"])
def test_fd_forward_matches_oracle(shape, order, dtype, spacing):
    """Spacings 1/n_axis (unequal: each derivative scaled in the stencil) and 0.07 on every axis
    (equal: the kernel forms plain differences and the chain applies the common factor once)."""
    f, h, y = run(shape, order, dtype, h=(0.07, 0.07, 0.07) if spacing == "equal" else None)
    ref = oracle.forward(oracle.fd_inputs(f, shape, h, order))
    assert_components(y.cpu().numpy(), ref, TOL_F64, what="fd %s order %d %s %s" % (shape, order, dtype, spacing))


def test_fd_forward_full_grid_sampled():
    """256^3 = 2^24 points (the benchmark grid); the oracle evaluates 4 z-planes' worth of points."""
    import paper_1804_10120_gb300 as tl
    shape = (256, 256, 256)
    f, h, y = run(shape, 4, "f64", seed=1)
    # the derivative table of 4 sampled z-planes needs their +-2 neighbours: the oracle runs on the
    # 8-plane sub-box z0-2 .. z0+5 (periodic in x and y like the grid; its own z wrap only affects the
    # two planes at each end, which are not compared)
    z0 = 100
    sub = f.reshape(16, 256, 256, 256)[:, z0 - 2:z0 + 6]            # z planes z0-2 .. z0+5
    sub_flat = np.ascontiguousarray(sub.reshape(16, -1))
    full = oracle.fd_inputs(sub_flat, (256, 256, 8), h, 4)           # periodic in z is wrong only at the ends
    x43 = np.ascontiguousarray(full.reshape(43, 8, 256 * 256)[:, 2:6].reshape(43, -1))
    ref = oracle.forward(x43)
    got = y.reshape(39, 256, 256 * 256)[:, z0:z0 + 4].reshape(39, -1).cpu().numpy()
    assert_components(got, ref, TOL_F64, what="256^3 planes %d-%d" % (z0, z0 + 3))
    assert bool(torch.isfinite(y).all())


def test_fd_argument_checks():
    import paper_1804_10120_gb300 as tl
    f = torch.zeros((16, 27), dtype=torch.float64, device=torch.device("cuda", 0))
    with pytest.raises(tl.TLError):
        tl.tl_dtg_forward_fd(f, (3, 3, 3), (0.1, 0.1, 0.1), order=3)
    with pytest.raises(tl.TLError):
        tl.tl_dtg_forward_fd(f, (3, 3, 3), (0.1, 0.0, 0.1))
    with pytest.raises(tl.TLError):
        tl.tl_dtg_forward_fd(f, (3, 3, 3), (0.1, 0.1, 0.1), dtype="f32")


@pytest.mark.parametrize("dtype", ["f64", "f64_ff"])
@pytest.mark.parametrize("order", [2, 4])
def test_fd_constant_fields_give_exact_zeros(order, dtype):
    """Fields constant over the grid (a constant non-diagonal metric, K, alpha, beta): every difference
    is exactly zero, so Gamma and nabla beta are exactly 0 and d_t g_ij = -2 alpha K_ij to the last bit
    of the oracle's value; g^ij within the binary64 gate of the oracle."""
    import paper_1804_10120_gb300 as tl
    shape = (9, 7, 5)
    n = 9 * 7 * 5
    const = np.array([1.2, 0.1, -0.05, 0.9, 0.07, 1.1,            # g (SPD)
                      0.3, -0.2, 0.1, 0.25, -0.15, 0.05,          # K
                      0.8,                                        # alpha
                      0.4, -0.3, 0.2])                            # beta
    f = np.repeat(const[:, None], n, axis=1)
    y = tl.tl_dtg_forward_fd(torch.from_numpy(f).to(torch.device("cuda", 0)), shape, (0.1, 0.2, 0.3), order,
                             dtype=dtype).cpu().numpy()
    assert np.all(y[6:33] == 0.0)                                 # Gamma and nabla beta
    ref = oracle.forward(oracle.fd_inputs(f, shape, (0.1, 0.2, 0.3), order))
    assert np.array_equal(y[33:39], ref[33:39])                   # -2 alpha K, one exact scaling and a product
    assert_components(y, ref, TOL_F64, what="constant fields")
