"""Tensor-index programs shared by the generator tests (plain text; no arithmetic here).  "chain" is
the package's own program, the one the benchmark compiles; the interpreter pins check it against the
chain oracle."""
from paper_1804_10120_gb300.programs import CHAIN, CHAIN_SYM
from tests.test_tensor_expr_oracle import EXPR_PROGRAMS

PROGRAMS = {
    "chain": CHAIN,
    "chain_sym": CHAIN_SYM,
    "eq9": EXPR_PROGRAMS[9],
    "eq14": EXPR_PROGRAMS[14],
    "eq17": EXPR_PROGRAMS[17],
    "eq18": EXPR_PROGRAMS[18],
    "eq19": EXPR_PROGRAMS[19],
    "eq20": "in B(3,3); in C(3,3); in D(3,3); in E(3,3,3,3); out A(3,3,3,3);"
            "A(i,j,k,l) = Sum(m, Sum(n, Sum(o, D(k,o)*C(j,n)*B(i,m)*E(m,n,o,l))));",
    "eq21": EXPR_PROGRAMS[21],
    "listing15": "in A(4,4); in B(4,4); out C(4,4) sym(0,1); C(a,b) = Sum(c, A(a,c)*B(c,b));",
    "listing17": "index i(3); in E(4,4); in F(4,4); out D(4,4) sym(0,1); D(i,0) = Sum(c, E(i+1,c)*F(c,0));"
                 "D(3,0) = E(0,0); D(1,1) = E(0,0); D(1,2) = E(0,0); D(1,3) = E(0,0); D(2,2) = E(0,0);"
                 "D(2,3) = E(0,0); D(3,3) = E(0,0);",
    "trace_div": "in B(3,3); in s; out t; out u(3); t = Sum(i, B(i,i)); u(i) = B(i,0) / (s*s + 1);",
    "spatial_slice": "in psi(4,4) sym(0,1); out g(3,3) sym(0,1); out beta(3); g(i,j) = psi(i+1,j+1); beta(i) = psi(i+1,0);",
    "spatial_contraction": "index m(3); in E(4,4); in F(4); out v(4); v(a) = Sum(m, E(a,m+1)*F(m+1));",
}

BAD = {
    "in B(3); out A(3); A(i) = B(j);": "free indices",
    "in B(3); in C(3); out A(3); A(i) = B(i)*C(i);": "both factors",
    "in B(3); out A(3); A(i) = B(i+1);": "out of range",
    "in B(3); out A(3); A(0) = B(0);": "never assigned",
    "in B(3); in C(3,3); out A(3); A(i) = B(i) + C(i,i);": "repeated",
    "in B(3); out A(3); A(i) = B(i) / B(i);": "scalar",
    "out A(3); A(i) = Q(i);": "unknown tensor",
    "in B(3); out A(3); B(i) = A(i);": "input",
    "in B(3); out A(4); A(i) = B(i);": "out of range",
    "in B(3); in C(4); out A; A = Sum(i, B(i)*C(i));": "declare its range",
    "in B(3) sym(0,1); out A(3); A(i) = B(i);": "sym",
    "in B(3); temp T(3); out A(3); A(i) = T(i) + B(i);": "before it is assigned",
}
