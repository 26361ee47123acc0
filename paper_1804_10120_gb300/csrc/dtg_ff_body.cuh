// dtg_ff_body.cuh -- the float-float chain body (binary64 inverse, bracket, shift subtraction and
// Eq. 5; the Eq. 6 contraction and Gamma^k_ij beta_k in pairs), shared by the kernels that use it.
#pragma once
#include "dtg_fwd_body.cuh"
#include "ff.cuh"

namespace tl {

// Intermediates of the float-float chain at one point that the fused forward + adjoint reuses: g^ij in
// binary64, and 1/2 g^ij, the Eq. 6 bracket, Gamma and beta as pairs.
struct ChainFFKeep {
    double ginv[6];
    ff h[6], T[3][6], gam[3][6], b[3];
};

// The chain on one point's 43 input values (in registers, input-table order), outputs to o.out[s][x],
// intermediates to k.  Returns false, having stored nothing but g^ij, when a value falls outside the
// pair format's range; the caller then evaluates the point in binary64.  kScaled and sd as for
// chain_f64: the 27 derivative entries are differences still to be multiplied by sd.
template <class OutTable, bool kScaled = false>
__device__ __forceinline__ bool chain_ff_keep(const double (&v)[N_IN], const OutTable &o, int64_t x, double sd,
                                              ChainFFKeep &k)
{
    const double g00 = v[IN_G + 0], g01 = v[IN_G + 1],
                 g02 = v[IN_G + 2], g11 = v[IN_G + 3],
                 g12 = v[IN_G + 4], g22 = v[IN_G + 5];
    double dg[18];
#pragma unroll
    for (int s = 0; s < 18; ++s)
        dg[s] = v[IN_DG + s];

    // step 1 in binary64
    double c[6];
    c[0] = fma(g11, g22, -(g12 * g12));
    c[1] = fma(g02, g12, -(g01 * g22));
    c[2] = fma(g01, g12, -(g02 * g11));
    c[3] = fma(g00, g22, -(g02 * g02));
    c[4] = fma(g01, g02, -(g00 * g12));
    c[5] = fma(g00, g11, -(g01 * g01));
    const double det = fma(g00, c[0], fma(g01, c[1], g02 * c[2]));
    const double rdet = rcp_f64(det);
    uint32_t big = 0;
    ff h[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        const double gi = c[p] * rdet;
        st_stream(o.out[OUT_GINV + p] + x, gi);
        k.ginv[p] = gi;
        if constexpr (kScaled)
            h[p] = split_ff(gi * half_exact(sd), big);
        else
            h[p] = split_ff(half_exact(gi), big);
    }

    // bracket of Eq. 6 in binary64, then pairs
    double Td[3][6];
    christoffel_bracket<double>(dg, Td);
    ff T[3][6];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int p = 0; p < 6; ++p)
            T[l][p] = split_ff(Td[l][p], big);

    const double b0 = v[IN_BETA + 0], b1 = v[IN_BETA + 1],
                 b2 = v[IN_BETA + 2];
    const ff bf0 = split_ff(b0, big), bf1 = split_ff(b1, big), bf2 = split_ff(b2, big);

    if (big)
        return false;
#pragma unroll
    for (int p = 0; p < 6; ++p)
        k.h[p] = h[p];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int p = 0; p < 6; ++p)
            k.T[l][p] = T[l][p];
    k.b[0] = bf0;
    k.b[1] = bf1;
    k.b[2] = bf2;

    // step 2: Eq. 6 contraction in pairs
    ff gam[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            gam[i][p] = dot3_ff(h[sym(i, 0)], T[0][p], h[sym(i, 1)], T[1][p], h[sym(i, 2)], T[2][p]);
            st_stream(o.out[OUT_GAMMA + 6 * i + p] + x, merge_ff(gam[i][p]));
            k.gam[i][p] = gam[i][p];
        }

    // step 3: S_ij = Gamma^k_ij beta_k (symmetric in ij: 6 sums) in pairs, then
    // nabla_j beta_i = d_j beta_i - S_ij in binary64 (exactly d_j beta_i where S vanishes)
    double S6[6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
        S6[p] = merge_ff(dot3_ff(gam[0][p], bf0, gam[1][p], bf1, gam[2][p], bf2));
    double nb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if constexpr (kScaled)
                nb[i][j] = fma(sd, v[IN_DBETA + 3 * i + j], -S6[sym(i, j)]);
            else
                nb[i][j] = v[IN_DBETA + 3 * i + j] - S6[sym(i, j)];
            st_stream(o.out[OUT_DBCOV + 3 * i + j] + x, nb[i][j]);
        }

    // step 4: Eq. 5 in binary64
    const double m2a = neg_exact(twice_exact(v[IN_ALPHA]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const int p = sym(i, j);
            const double K = v[IN_K + p];
            const double s = (i == j) ? twice_exact(nb[i][i]) : nb[i][j] + nb[j][i];
            st_stream(o.out[OUT_DTG + p] + x, fma(m2a, K, s));
        }
    return true;
}

// The chain alone (the intermediates are dropped; the compiler removes the copies).
template <class OutTable, bool kScaled = false>
__device__ __forceinline__ bool chain_ff(const double (&v)[N_IN], const OutTable &o, int64_t x, double sd = 1.0)
{
    ChainFFKeep unused;
    return chain_ff_keep<OutTable, kScaled>(v, o, x, sd, unused);
}

}  // namespace tl
