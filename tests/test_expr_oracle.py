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


def test_sums_and_outer_products_exact_on_integers():
    """Eqs. 12-17 on integer-valued operands in [-20, 20]: every sum and product is exact in binary64,
    so the oracle must reproduce the exact integer result, formed here by brute force over the index
    tuples in int64 (component order row-major over the indices as written)."""
    import itertools
    rng = np.random.default_rng(11)
    for eq in (12, 13, 14):
        t = eq - 10
        xi = rng.integers(-20, 21, size=(3 * t, N))
        ref = np.stack([sum(xi[3 * q + i] for q in range(t)) for i in range(3)])
        assert np.array_equal(oracle.expr(eq, xi.astype(np.float64)), ref.astype(np.float64)), eq
    for eq in (15, 16, 17):
        R = eq - 13
        xi = rng.integers(-20, 21, size=(3 * R, N))
        rows = []
        for idx in itertools.product(range(3), repeat=R):
            prod = np.ones(N, dtype=np.int64)
            for q, i in enumerate(idx):
                prod = prod * xi[3 * q + i]
            rows.append(prod)
        assert np.array_equal(oracle.expr(eq, xi.astype(np.float64)), np.stack(rows).astype(np.float64)), eq


def test_contractions_exact_on_integers():
    """Eqs. 18-20 on integer-valued operands in [-5, 5]: at most 27 terms of four-factor products, all
    exact in binary64; the exact sums are formed by brute force over every index value in int64."""
    import itertools
    rng = np.random.default_rng(12)
    for eq, nf in ((18, 1), (19, 2), (20, 3)):
        n_in, _ = oracle.EXPR_ARITY[eq]
        xi = rng.integers(-5, 6, size=(n_in, N))
        fac = [xi[9 * q:9 * q + 9].reshape(3, 3, N) for q in range(nf)]     # B, C, D: F[a][b] = F_ab
        E = xi[9 * nf:].reshape(3, 3, 3, 3, N)
        ref = np.zeros((3, 3, 3, 3, N), dtype=np.int64)
        for i, j, k, l in itertools.product(range(3), repeat=4):
            free = (i, j, k)
            for summed in itertools.product(range(3), repeat=nf):
                # factor q carries free index q and summed index q; E takes the summed indices first
                term = E[summed + free[nf:] + (l,)].copy()
                for q in range(nf):
                    term = term * fac[q][free[q], summed[q]]
                ref[i, j, k, l] += term
        assert np.array_equal(oracle.expr(eq, xi.astype(np.float64)), ref.reshape(81, N).astype(np.float64)), eq


def test_kij_minus_lapse_term_is_rank_one():
    """Eq. 21: K_ij - 2 alpha g_ij = beta_i beta_j is a rank-one matrix with a non-negative diagonal:
    (K - 2 alpha g)_ij^2 = (K - 2 alpha g)_ii (K - 2 alpha g)_jj for every pair, and its diagonal is
    beta_i^2 (recovered up to sign by the square root)."""
    x = inputs(21, seed=3)
    x[0] = gridgen.uniform(N, 3, 78, 0.5, 1.5)
    K = oracle.expr(21, x)
    P = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    M = {ij: K[p] - 2.0 * x[0] * x[1 + p] for ij, p in P.items()}
    scale = np.abs(x[7:10]).max() ** 2
    for i in range(3):
        assert np.abs(np.sqrt(np.abs(M[(i, i)])) - np.abs(x[7 + i])).max() <= 1e-7 * np.sqrt(scale)
        for j in range(i + 1, 3):
            assert np.abs(M[(i, j)] ** 2 - M[(i, i)] * M[(j, j)]).max() <= 1e-12 * scale ** 2


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
