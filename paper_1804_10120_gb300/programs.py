"""Tensor-index programs shipped with the package (plain text for the runtime generator,
``JitKernel(text)``; no arithmetic happens here).

CHAIN is the metric-evolution chain of the hand-written kernels as a program: the cofactor inverse of
g_ij, the bracket and the Christoffel symbols of Eq. 6, the covariant derivative of the shift (the
footnote to Listing 1) and d_t g_ij of Eq. 5.  Its component tables coincide with the 43 + 39 layout
of tl_dtg_forward (symmetric pairs stored once, ascending).

CHAIN_SYM is the same chain with the footnote's sum Gamma^k_ij beta_k written as a temporary tensor
symmetric in ij, so that the generator (which evaluates each stored element of a symmetric left-hand
side once) forms its 6 distinct values instead of 9 chains, as the hand-written kernel does."""

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

CHAIN_SYM = CHAIN.replace(
    "temp T(3,3,3) sym(1,2);", "temp T(3,3,3) sym(1,2); temp S(3,3) sym(0,1);").replace(
    "dbcov(i,j) = db(i,j) - Sum(k, Gamma(k,i,j)*beta(k)); # footnote to Listing 1",
    "S(i,j) = Sum(k, Gamma(k,i,j)*beta(k));              # symmetric in ij: 6 sums\n"
    "dbcov(i,j) = db(i,j) - S(i,j);                       # footnote to Listing 1")
