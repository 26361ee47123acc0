"""Pins of the benchmark-expression oracle (Sec. 5.1, Eqs. 9-21) against numpy (a library routine:
einsum / elementwise arithmetic in the same order) and exact special cases; and the effective-bandwidth
element counts N_e of each expression (Eq. 8)."""
import numpy as np
import pytest

import gridgen
import oracle
from paper_1804_10120_gb300.bweff import Idx, Ref, count_elements

N = 257


def inputs(eq, seed=0):
    n_in, _ = oracle.EXPR_ARITY[eq]
    return gridgen.normal_fields(n_in, N, seed + eq, 5000)


def test_assign_add_outer_bitwise():
    for eq in (9, 10, 11):
        x = inputs(eq)
        assert np.array_equal(oracle.expr(eq, x), x)
    for eq in (12, 13, 14):
        x = inputs(eq)
        ops = x.reshape(eq - 10, 3, N)
        ref = ops[0].copy()
        for t in range(1, eq - 10):
            ref = ref + ops[t]
        assert np.array_equal(oracle.expr(eq, x), ref)
    for eq in (15, 16, 17):
        R = eq - 13
        x = inputs(eq)
        v = x.reshape(R, 3, N)
        ref = v[0]
        for t in range(1, R):
            ref = (ref[..., None, :] * v[t][None, :, :].reshape((1,) * (ref.ndim - 1) + (3, N)))
        assert np.array_equal(oracle.expr(eq, x), ref.reshape(-1, N))


def test_contractions_against_einsum():
    x = inputs(18)
    B, E = x[:9].reshape(3, 3, N), x[9:].reshape(3, 3, 3, 3, N)
    ref = np.einsum("imx,mjklx->ijklx", B, E).reshape(81, N)
    assert np.abs(oracle.expr(18, x) - ref).max() <= 1e-14 * np.abs(ref).max()
    x = inputs(19)
    B, C, E = x[:9].reshape(3, 3, N), x[9:18].reshape(3, 3, N), x[18:].reshape(3, 3, 3, 3, N)
    ref = np.einsum("jnx,imx,mnklx->ijklx", C, B, E).reshape(81, N)
    assert np.abs(oracle.expr(19, x) - ref).max() <= 1e-14 * np.abs(ref).max()
    x = inputs(20)
    B, C, D, E = (x[:9].reshape(3, 3, N), x[9:18].reshape(3, 3, N), x[18:27].reshape(3, 3, N),
                  x[27:].reshape(3, 3, 3, 3, N))
    ref = np.einsum("kox,jnx,imx,mnolx->ijklx", D, C, B, E).reshape(81, N)
    assert np.abs(oracle.expr(20, x) - ref).max() <= 1e-14 * np.abs(ref).max()


def test_contractions_with_identity_factors_are_exact():
    for eq, nm in ((18, 1), (19, 2), (20, 3)):
        x = inputs(eq)
        eye = np.eye(3).reshape(9, 1) * np.ones((1, N))
        for q in range(nm):
            x[9 * q:9 * q + 9] = eye
        assert np.array_equal(oracle.expr(eq, x), x[9 * nm:])


def test_kij():
    x = inputs(21)
    x[0] = gridgen.uniform(N, 1, 77, 0.5, 1.5)
    P = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    ref = np.stack([(2.0 * x[0]) * x[1 + p] + x[7 + i] * x[7 + j] for p, (i, j) in enumerate(P)])
    assert np.array_equal(oracle.expr(21, x), ref)
    x[7:10] = 0.0
    assert np.array_equal(oracle.expr(21, x), (2.0 * x[0]) * x[1:7])


def test_element_counts():
    """N_e of Eq. 8 for each expression (all indices dimension 3, K and g symmetric)."""
    i, j, k, l, m, n, o = (Idx(c) for c in "ijklmno")
    d = {c: 3 for c in "ijklmno"}
    cases = {
        9: [Ref("A", (i,)), Ref("B", (i,))],
        12: [Ref("A", (i,)), Ref("B", (i,)), Ref("C", (i,))],
        17: [Ref("A", (i, j, k, l)), Ref("B", (i,)), Ref("C", (j,)), Ref("D", (k,)), Ref("E", (l,))],
        18: [Ref("A", (i, j, k, l)), Ref("B", (i, m)), Ref("E", (m, j, k, l))],
        20: [Ref("A", (i, j, k, l)), Ref("D", (k, o)), Ref("C", (j, n)), Ref("B", (i, m)), Ref("E", (m, n, o, l))],
        21: [Ref("K", (i, j), ((0, 1),)), Ref("alpha", ()), Ref("g", (i, j), ((0, 1),)), Ref("beta", (i,))],
    }
    for eq, refs in cases.items():
        n_in, n_out = oracle.EXPR_ARITY[eq]
        assert count_elements(refs, d) == n_in + n_out, eq


def test_bad_expression_id():
    with pytest.raises(KeyError):
        oracle.expr(8, np.zeros((3, 2)))
