"""Pins of the on-grid derivative oracle: the exact discrete derivative of a Fourier mode, the
convergence order of both stencils, the axis / index placement, and the untouched copies."""
import numpy as np
import pytest

import gridgen
import oracle


def _mode_fields(shape, kvec, phase, which):
    """16 fields: zero except field `which` = sin(2 pi k.x + phase) (g and alpha keep a base so the table
    is a valid chain input)."""
    nx, ny, nz = shape
    ix, iy, iz = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny, np.arange(nz) / nz, indexing="ij")
    arg = 2 * np.pi * (kvec[0] * ix + kvec[1] * iy + kvec[2] * iz) + phase
    f = np.zeros((16, nx * ny * nz))
    f[which] = np.sin(arg).transpose(2, 1, 0).reshape(-1)          # x fastest
    return f, np.cos(arg).transpose(2, 1, 0).reshape(-1)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("field,first", [(13, 34), (4, 6 + 3 * 4)], ids=["beta_0", "g_12"])
def test_discrete_derivative_of_a_mode_is_exact(order, field, first):
    """For sin(k x + phi) the centred differences are exactly cos(k x + phi) times
    sin(kh)/h (order 2) or (8 sin(kh) - sin(2kh)) / (6h) (order 4), along each axis with its own
    spacing; checked for a shift component (d_j beta_0 at 34 + j) and a metric component
    (d_k g_12 at 6 + 3 p(1,2) + k)."""
    shape = (20, 12, 10)
    kv = (3, -2, 1)
    f, c = _mode_fields(shape, kv, 0.7, field)
    h = (1 / 20, 1 / 12, 1 / 10)
    x = oracle.fd_inputs(f, shape, h, order)
    for axis in range(3):
        k = 2 * np.pi * kv[axis]
        if order == 2:
            factor = np.sin(k * h[axis]) / h[axis]
        else:
            factor = (8 * np.sin(k * h[axis]) - np.sin(2 * k * h[axis])) / (6 * h[axis])
        assert np.abs(x[first + axis] - factor * c).max() <= 1e-12 * abs(factor)
    others = [r for r in list(range(6, 24)) + list(range(34, 43)) if not first <= r < first + 3]
    assert np.all(x[others] == 0.0)              # every other derivative entry is zero


@pytest.mark.parametrize("order", [2, 4])
def test_convergence_order(order):
    errs = []
    for n in (16, 32, 64):
        shape = (n, 4, 4)
        f, c = _mode_fields(shape, (1, 0, 0), 0.3, 0)    # g_00 varies along x
        x = oracle.fd_inputs(f, shape, (1 / n, 1 / 4, 1 / 4), order)
        errs.append(np.abs(x[6] - 2 * np.pi * c).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.1 for r in rates), rates


def test_axis_placement_and_copies():
    shape = (6, 7, 5)
    f = gridgen.periodic_fields(shape, 2)
    x = oracle.fd_inputs(f, shape, (1 / 6, 1 / 7, 1 / 5), 4)
    assert np.array_equal(x[0:6], f[0:6]) and np.array_equal(x[24:30], f[6:12])
    assert np.array_equal(x[30], f[12]) and np.array_equal(x[31:34], f[13:16])
    # a field varying only along y has only d_1 non-zero: dg[3p+1]
    g, _ = _mode_fields(shape, (0, 2, 0), 0.1, 4)        # g_12
    g[0] = g[3] = g[5] = 1.0
    x = oracle.fd_inputs(g, shape, (1 / 6, 1 / 7, 1 / 5), 2)
    assert np.all(x[6 + 3 * 4 + 0] == 0) and np.all(x[6 + 3 * 4 + 2] == 0) and np.abs(x[6 + 3 * 4 + 1]).max() > 1


def test_constant_fields_have_zero_derivatives():
    shape = (5, 3, 4)
    f = np.ones((16, 60)) * 0.25
    x = oracle.fd_inputs(f, shape, (0.1, 0.2, 0.3), 4)
    assert np.all(x[6:24] == 0) and np.all(x[34:43] == 0)
