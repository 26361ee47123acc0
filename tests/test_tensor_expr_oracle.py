"""Pins of the tensor-index program interpreter (the runtime generator's oracle): the whole metric
evolution chain written as a program equals the chain oracle; the benchmark expressions equal their
literal oracle bit for bit; the paper's two contraction listings equal numpy.einsum."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle.tensor_expr import Program

CHAIN = """
in g(3,3) sym(0,1); in dg(3,3,3) sym(0,1); in K(3,3) sym(0,1); in alpha; in beta(3); in db(3,3);
temp c(3,3) sym(0,1); temp det; temp T(3,3,3) sym(1,2);
out ginv(3,3) sym(0,1); out Gamma(3,3,3) sym(1,2); out dbcov(3,3); out dtg(3,3) sym(0,1);
c(0,0) = g(1,1)*g(2,2) - g(1,2)*g(1,2);
c(0,1) = g(0,2)*g(1,2) - g(0,1)*g(2,2);
c(0,2) = g(0,1)*g(1,2) - g(0,2)*g(1,1);
c(1,1) = g(0,0)*g(2,2) - g(0,2)*g(0,2);
c(1,2) = g(0,1)*g(0,2) - g(0,0)*g(1,2);
c(2,2) = g(0,0)*g(1,1) - g(0,1)*g(0,1);
det = g(0,0)*c(0,0) + g(0,1)*c(0,1) + g(0,2)*c(0,2);
ginv(i,j) = c(i,j) / det;
T(l,j,k) = dg(j,l,k) + dg(l,k,j) - dg(j,k,l);        # the bracket of Eq. 6
Gamma(i,j,k) = 0.5*Sum(l, ginv(i,l)*T(l,j,k));       # Eq. 6
dbcov(i,j) = db(i,j) - Sum(k, Gamma(k,i,j)*beta(k)); # footnote to Listing 1
dtg(i,j) = -2*alpha*K(i,j) + dbcov(j,i) + dbcov(i,j);  # Eq. 5
"""

EXPR_PROGRAMS = {
    9: "in B(3); out A(3); A(i) = B(i);",
    11: "in B(3,3,3); out A(3,3,3); A(i,j,k) = B(i,j,k);",
    14: "in B(3); in C(3); in D(3); in E(3); out A(3); A(i) = B(i) + C(i) + D(i) + E(i);",
    17: "in B(3); in C(3); in D(3); in E(3); out A(3,3,3,3); A(i,j,k,l) = B(i)*C(j)*D(k)*E(l);",
    18: "in B(3,3); in E(3,3,3,3); out A(3,3,3,3); A(i,j,k,l) = Sum(m, B(i,m)*E(m,j,k,l));",
    19: "in B(3,3); in C(3,3); in E(3,3,3,3); out A(3,3,3,3); A(i,j,k,l) = Sum(m, Sum(n, C(j,n)*B(i,m)*E(m,n,k,l)));",
    21: "in alpha; in g(3,3) sym(0,1); in beta(3); out K(3,3) sym(0,1); K(i,j) = 2*alpha*g(i,j) + beta(i)*beta(j);",
}


@pytest.mark.parametrize("which", ["transcribed here", "shipped with the package", "symmetric footnote sum"])
def test_chain_program_equals_chain_oracle(which):
    from paper_1804_10120_gb300.programs import CHAIN as PACKAGE_CHAIN, CHAIN_SYM
    p = Program({"transcribed here": CHAIN, "shipped with the package": PACKAGE_CHAIN,
                 "symmetric footnote sum": CHAIN_SYM}[which])
    assert len(p.inputs()) == 43 and len(p.outputs()) == 39
    x = gridgen.random_grid(2000, 13)
    y = p.run(x)
    ref = oracle.forward(x)
    scale = np.abs(ref).max(axis=1)
    assert (np.abs(y - ref).max(axis=1) <= 1e-14 * scale).all()


def test_benchmark_expressions_bitwise():
    for eq, text in EXPR_PROGRAMS.items():
        p = Program(text)
        n_in, n_out = oracle.EXPR_ARITY[eq]
        assert (len(p.inputs()), len(p.outputs())) == (n_in, n_out)
        x = gridgen.normal_fields(n_in, 300, eq, 5000)
        y = p.run(x)
        ref = oracle.expr(eq, x)
        if eq == 19:     # same terms, summed m-outer / n-inner in both
            assert np.abs(y - ref).max() <= 1e-15 * np.abs(ref).max()
        else:
            assert np.array_equal(y, ref), eq


def test_paper_listings_against_einsum():
    """The rank-2 symmetric contraction of Listing 15 (spacetime indices) and the fixed / offset
    index example of Listing 17."""
    n = 50
    rng = np.random.default_rng(4)
    p = Program("in A(4,4); in B(4,4); out C(4,4) sym(0,1); C(a,b) = Sum(c, A(a,c)*B(c,b));")
    A, B = rng.normal(size=(4, 4, n)), rng.normal(size=(4, 4, n))
    y = p.run(np.concatenate([A.reshape(16, n), B.reshape(16, n)]))
    full = np.einsum("acx,cbx->abx", A, B)
    ref = np.stack([full[a, b] for a in range(4) for b in range(a, 4)])
    assert np.abs(y - ref).max() <= 1e-14
    assert y.shape[0] == 10                      # N_e counts 10 stored elements of C
    p = Program("index i(3); in E(4,4); in F(4,4); out D(4,4) sym(0,1); D(i,0) = Sum(c, E(i+1,c)*F(c,0));"
                "D(3,0) = E(0,0); D(1,1) = E(0,0); D(1,2) = E(0,0); D(1,3) = E(0,0); D(2,2) = E(0,0);"
                "D(2,3) = E(0,0); D(3,3) = E(0,0);")
    E, F = rng.normal(size=(4, 4, n)), rng.normal(size=(4, 4, n))
    y = p.run(np.concatenate([E.reshape(16, n), F.reshape(16, n)]))
    ref = np.einsum("icx,cx->ix", E[1:4], F[:, 0])
    # D(i,0), i = 0..2 (spatial), land on the stored elements (0,0), (0,1), (0,2) of the symmetric D
    assert np.abs(y[0:3] - ref).max() <= 1e-14
    assert np.array_equal(y[3], E[0, 0])         # D(3,0) = D(0,3)


def test_sum_over_a_declared_range_against_einsum():
    """A contraction letter with its own range and an offset: the spatial part (slots 1..3) of a
    4-dimensional index, v_a = sum_{m<3} E_a,m+1 F_m+1."""
    n = 40
    rng = np.random.default_rng(5)
    p = Program("index m(3); in E(4,4); in F(4); out v(4); v(a) = Sum(m, E(a,m+1)*F(m+1));")
    E, F = rng.normal(size=(4, 4, n)), rng.normal(size=(4, n))
    y = p.run(np.concatenate([E.reshape(16, n), F]))
    ref = np.einsum("amx,mx->ax", E[:, 1:4], F[1:4])
    assert np.abs(y - ref).max() <= 1e-14
