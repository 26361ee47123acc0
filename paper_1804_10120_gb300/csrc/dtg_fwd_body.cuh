// dtg_fwd_body.cuh -- per-point device bodies of the forward chain shared by the forward kernels.
#pragma once
#include "tl_common.cuh"
#include "tl_kernels.h"

namespace tl {

// The bracket of Eq. 6 for the stored pairs, T[l][p(j,k)] = d_k g_jl + d_j g_lk - d_l g_jk, from
// D(a,b,c) = d_c g_ab.  When l is one of j, k two terms cancel identically:
//   l == j: T = d_k g_jj;   l == k: T = d_j g_kk;   j == k != l: T = 2 d_j g_jl - d_l g_jj.
// Only the three (j<k, l outside {j,k}) entries need the full three-term sum.
template <typename R>
__device__ __forceinline__ R dgc(const R (&dg)[18], int i, int j, int k) { return dg[3 * sym(i, j) + k]; }

__device__ __forceinline__ double negate(double x) { return neg_exact(x); }
__device__ __forceinline__ float negate(float x) { return -x; }

template <typename R>
__device__ __forceinline__ void christoffel_bracket(const R (&dg)[18], R (&T)[3][6])
{
#define D(i_, j_, k_) dgc<R>(dg, i_, j_, k_)
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = j; k < 3; ++k) {
                const int p = sym(j, k);
                if (l == j)
                    T[l][p] = D(j, j, k);
                else if (l == k)
                    T[l][p] = D(k, k, j);
                else if (j == k)
                    T[l][p] = fma((R)2, D(j, l, j), negate(D(j, j, l)));
                else
                    T[l][p] = (D(j, l, k) + D(l, k, j)) - D(j, k, l);
            }
#undef D
}

// ------------------------------------------------------------------------------------ binary64 forward
// Product for the binary64 chain: on the integer pipes (mul_int, bit-identical to the FP64 multiply)
// where the FP64 pipe is the binding unit; the FP64 multiply in rarely taken fallback paths, whose
// register needs would otherwise raise those of the kernels that call them.
template <bool kIntMul> __device__ __forceinline__ double mul64(double a, double b)
{
    return kIntMul ? mul_int(a, b) : a * b;
}

// Intermediates of the binary64 chain at one point that the fused forward + adjoint kernel reuses:
// g^ij, 1/2 g^ij, the Eq. 6 bracket and Gamma (packed as in the output table).
struct ChainF64Keep {
    double ginv[6], h[6], T[3][6], gam[3][6];
};

// The chain on one point's 43 input values (in registers, in the input-table order); the 39 outputs go
// to o.out[s][x] (o: any argument block with an `out` table) and the intermediates to k.  kLate: the
// entries of v from K_ij on (K, alpha, beta, d_j beta_i: 19 values that only steps 3 and 4 use) are
// not yet loaded; `late` fills them just before step 3 (by default from o.in[s][x], which the caller
// has prefetched into L1), so their registers are free while the inverse and Eq. 6 are formed.
// kScaled: the d_k g_ij and d_j beta_i entries of v are differences that still need one common factor
// sd (a finite-difference stencil on a grid with equal spacings); sd is then applied once to
// 1/2 g^il and fused into nabla_j beta_i instead of to each of the 27 derivatives.  kIntMul: the 37
// products that are not fused into an FMA go to the integer pipes (mul_int); the results are the same
// bits either way.
// The late entries of v (K, alpha, beta, d_j beta_i) read from the input table o.in.
struct LoadLate {
    template <class OutTable> __device__ __forceinline__ void operator()(const OutTable &o, int64_t x, double (&vl)[N_IN]) const
    {
#pragma unroll
        for (int s = IN_K; s < N_IN; ++s)
            vl[s] = ld_stream(o.in[s] + x);
    }
};

template <class OutTable, bool kScaled = false, bool kIntMul = true, bool kLate = false, class Late = LoadLate>
__device__ __forceinline__ void chain_f64_keep(const double (&v0)[N_IN], const OutTable &o, int64_t x, double sd,
                                               ChainF64Keep &k, const Late &late = Late())
{
    double vl[N_IN];
#pragma unroll
    for (int s = 0; s < N_IN; ++s)
        vl[s] = v0[s];
    const double (&v)[N_IN] = vl;
    // step 1: inverse metric by cofactors; det by first-row expansion
    const double g00 = v[IN_G + 0], g01 = v[IN_G + 1],
                 g02 = v[IN_G + 2], g11 = v[IN_G + 3],
                 g12 = v[IN_G + 4], g22 = v[IN_G + 5];
    double dg[18];
#pragma unroll
    for (int s = 0; s < 18; ++s)
        dg[s] = v[IN_DG + s];

    double c[6];
    c[0] = fma(g11, g22, -mul64<kIntMul>(g12, g12));
    c[1] = fma(g02, g12, -mul64<kIntMul>(g01, g22));
    c[2] = fma(g01, g12, -mul64<kIntMul>(g02, g11));
    c[3] = fma(g00, g22, -mul64<kIntMul>(g02, g02));
    c[4] = fma(g01, g02, -mul64<kIntMul>(g00, g12));
    c[5] = fma(g00, g11, -mul64<kIntMul>(g01, g01));
    const double det = fma(g00, c[0], fma(g01, c[1], mul64<kIntMul>(g02, c[2])));
    const double rdet = rcp_f64(det);
    double ginv[6], h[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        ginv[p] = mul64<kIntMul>(c[p], rdet);
        if constexpr (kScaled)
            h[p] = mul64<kIntMul>(ginv[p], half_exact(sd));
        else
            h[p] = half_exact(ginv[p]);      // 1/2 g^il of Eq. 6
        st_stream(o.out[OUT_GINV + p] + x, ginv[p]);
        k.ginv[p] = ginv[p];
        k.h[p] = h[p];
    }

    // step 2: Christoffel symbols, Eq. 6
    double T[3][6];
    christoffel_bracket<double>(dg, T);
    double gam[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            gam[i][p] = fma(h[sym(i, 2)], T[2][p], fma(h[sym(i, 1)], T[1][p], mul64<kIntMul>(h[sym(i, 0)], T[0][p])));
            st_stream(o.out[OUT_GAMMA + 6 * i + p] + x, gam[i][p]);
            k.T[i][p] = T[i][p];
            k.gam[i][p] = gam[i][p];
        }

    if constexpr (kLate) {
        asm volatile("" ::: "memory");   // the late inputs are loaded here, not hoisted above Eq. 6
        late(o, x, vl);
    }
    // step 3: nabla_j beta_i = d_j beta_i - Gamma^k_ij beta_k.  Gamma^k_ij beta_k is symmetric in ij, so
    // its 6 distinct sums are formed once (a product and 2 FMAs each) and subtracted from the 9
    // derivatives: 21 FP64-pipe operations instead of the 27 FMAs of 9 separate chains.
    const double b0 = v[IN_BETA + 0], b1 = v[IN_BETA + 1],
                 b2 = v[IN_BETA + 2];
    double nb[3][3], S6[6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
        S6[p] = fma(gam[2][p], b2, fma(gam[1][p], b1, mul64<kIntMul>(gam[0][p], b0)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int p = sym(i, j);
            const double B = v[IN_DBETA + 3 * i + j];
            if constexpr (kScaled)
                nb[i][j] = fma(sd, B, -S6[p]);
            else
                nb[i][j] = B - S6[p];
            st_stream(o.out[OUT_DBCOV + 3 * i + j] + x, nb[i][j]);
        }

    // step 4: Eq. 5, d_t g_ij = -2 alpha K_ij + nabla_i beta_j + nabla_j beta_i
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
}

// The chain alone (the intermediates are dropped; the compiler removes the copies).
template <class OutTable, bool kScaled = false, bool kIntMul = true>
__device__ __forceinline__ void chain_f64(const double (&v)[N_IN], const OutTable &o, int64_t x, double sd = 1.0)
{
    ChainF64Keep unused;
    chain_f64_keep<OutTable, kScaled, kIntMul>(v, o, x, sd, unused);
}

// One point of the forward.  The 24 inputs of the inverse and Eq. 6 (g_ij, d_k g_ij) are loaded before
// any arithmetic; the other 19 are prefetched into L1 and loaded before step 3, which leaves room for
// three 256-thread blocks per SM (80 registers, 24 warps): 2.77 -> 2.75 ms at N = 2^24 against every
// input loaded up front at two blocks (128 registers).
template <bool kIntMul = true> __device__ __forceinline__ void fwd_point_f64(const FwdArgs<double> &a, int64_t x)
{
    double v[N_IN];
#pragma unroll
    for (int s = 0; s < IN_K; ++s)
        v[s] = ld_stream(a.in[s] + x);
#pragma unroll
    for (int s = IN_K; s < N_IN; ++s) {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.in[s] + x));
        v[s] = 0.0;
    }
    asm volatile("" ::: "memory");   // the first 24 loads are issued before any arithmetic
    ChainF64Keep unused;
    chain_f64_keep<FwdArgs<double>, false, kIntMul, true>(v, a, x, 1.0, unused);
}

}  // namespace tl
