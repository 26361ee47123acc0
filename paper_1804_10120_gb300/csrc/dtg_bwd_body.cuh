// dtg_bwd_body.cuh -- per-point pieces of the binary64 adjoint, shared by the adjoint kernel and the
// fused forward + adjoint kernel.  The paper has no adjoint: these are the reverse-mode derivatives of
// Eq. 5, the footnote to Listing 1, Eq. 6 and the inverse metric, taken in reverse order.
//
// Notation (per point): H = g^ij, h = H / 2, T the Eq. 6 bracket (Gamma^i_p = sum_l h_il T_lp),
// W, V, U, Y the upstream gradients of d_t g, Gamma, nabla beta and g^ij, Nbar the gradient of
// nabla_j beta_i, S_p its symmetric fold, Gbar the gradient of Gamma, Tbar that of the bracket.
//
// The gradient of the stored metric follows from dH = -H dG H: with Hbar the gradient of the nine
// entries of H and A = Hbar + Hbar^T, gbar_ij = -(H A H)_ij (i < j) and -(H A H)_ii / 2.  Through
// Eq. 6, Hbar = 1/2 Gbar T^T and Tbar = h Gbar, so H Hbar = Tbar T^T =: P, and H Hbar H = P H = X;
// then H A H = X + X^T.  So
//   gbar_ii = -X_ii,   gbar_ij = -(X_ij + X_ji)   (i < j),
// which needs P (9 dot products of length 6) and the six folded entries of P H (27 terms) instead of
// Hbar, the product H A and the six entries of (H A) H.  When Gamma is at hand (the fused kernel),
// T^T H = 2 Gamma^T gives X = 2 Tbar Gamma^T directly and P is not formed at all.
#pragma once
#include "dtg_fwd_body.cuh"

namespace tl {

template <typename T> __device__ __forceinline__ T ld_opt(const T *p, int64_t x)
{
    return p ? ld_stream(p + x) : T(0);
}

// Reverse of Eq. 5 and of the footnote: stores Kbar_p = -2 alpha W_p, alphabar = -2 sum_p K_p W_p and
// dbetabar_ij = Nbar_ij (Nbar_ij = W_p(ij), doubled on the diagonal since d_t g_ii holds nabla_i beta_i
// twice, plus U_ij when kU), and returns S_p = Nbar_ij + Nbar_ji (i < j) or Nbar_ii.
template <bool kU, bool kIntMul, class Args>
__device__ __forceinline__ void adj_eq5_footnote(const Args &a, int64_t x, const double (&W)[6], const double (&K)[6],
                                                 double alpha, double (&S)[6])
{
    const double m2a = neg_exact(twice_exact(alpha));
    double asum = 0.0;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        st_stream(a.gin[IN_K + p] + x, mul64<kIntMul>(m2a, W[p]));
        asum = (p == 0) ? mul64<kIntMul>(K[p], W[p]) : fma(K[p], W[p], asum);
    }
    st_stream(a.gin[IN_ALPHA] + x, neg_exact(twice_exact(asum)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int p = sym(i, j);
            double nbar = (i == j) ? twice_exact(W[p]) : W[p];
            if (kU)
                nbar += ld_opt(a.gout[OUT_DBCOV + 3 * i + j], x);
            st_stream(a.gin[IN_DBETA + 3 * i + j] + x, nbar);
            if (kU) {
                if (i <= j)
                    S[p] = nbar;
                else
                    S[p] += nbar;
            }
        }
    if (!kU) {
#pragma unroll
        for (int p = 0; p < 6; ++p)
            S[p] = twice_exact(W[p]);
    }
}

// Tbar_lp = sum_i h_il Gbar_ip.
template <bool kIntMul>
__device__ __forceinline__ void adj_tbar(const double (&h)[6], const double (&gb)[3][6], double (&Tb)[3][6])
{
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int p = 0; p < 6; ++p)
            Tb[l][p] = fma(h[sym(2, l)], gb[2][p], fma(h[sym(1, l)], gb[1][p], mul64<kIntMul>(h[sym(0, l)], gb[0][p])));
}

// Reverse of the bracket: every term of T_lp scattered onto the stored derivative d_k g_ij it reads, then
// stored.  The first contribution to an entry is assigned rather than added to zero (one FP64 addition
// saved per entry; `seen` is resolved at compile time once the loops are unrolled).
template <class Args>
__device__ __forceinline__ void adj_bracket_store(const Args &a, int64_t x, const double (&Tb)[3][6])
{
    double dgb[18];
    bool seen[18] = {};
    auto put = [&](int s, double t) {
        dgb[s] = seen[s] ? dgb[s] + t : t;
        seen[s] = true;
    };
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = j; k < 3; ++k) {
                const double t = Tb[l][sym(j, k)];
                if (l == j) {                       // T = d_k g_jj
                    put(3 * sym(j, j) + k, t);
                } else if (l == k) {                // T = d_j g_kk
                    put(3 * sym(k, k) + j, t);
                } else if (j == k) {                // T = 2 d_j g_jl - d_l g_jj
                    put(3 * sym(j, l) + j, twice_exact(t));
                    put(3 * sym(j, j) + l, -t);
                } else {                            // T = d_k g_jl + d_j g_lk - d_l g_jk
                    put(3 * sym(j, l) + k, t);
                    put(3 * sym(l, k) + j, t);
                    put(3 * sym(j, k) + l, -t);
                }
            }
#pragma unroll
    for (int s = 0; s < 18; ++s)
        st_stream(a.gin[IN_DG + s] + x, dgb[s]);
}

// P += h A_Y with A_Y the symmetric matrix of the g^ij upstream gradient as it enters A = Hbar + Hbar^T
// (Y_p off the diagonal, 2 Y_p on it: the stored entry g^ij is one element of H).
template <bool kIntMul>
__device__ __forceinline__ void adj_add_hAY(const double (&h)[6], const double (&Y)[6], double (&P)[3][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            double s = P[i][l];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const double y = (m == l) ? twice_exact(Y[sym(m, l)]) : Y[sym(m, l)];
                s = fma(h[sym(i, m)], y, s);
            }
            P[i][l] = s;
        }
}

// The six folded entries of X = P H: F_ii = X_ii, F_ij = X_ij + X_ji (i < j), packed.
template <bool kIntMul>
__device__ __forceinline__ void adj_fold_PH(const double (&P)[3][3], const double (&H)[6], double (&F)[6])
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double s = mul64<kIntMul>(P[i][0], H[sym(0, j)]);
            s = fma(P[i][1], H[sym(1, j)], s);
            s = fma(P[i][2], H[sym(2, j)], s);
            if (i != j) {
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    s = fma(P[j][m], H[sym(m, i)], s);
            }
            F[sym(i, j)] = s;
        }
}

// The binary64 adjoint at one point (a: any argument block with `in`, `gout` and `gin` tables).  kU:
// upstream gradient of nabla beta present; kG: upstream gradient of g^ij present.  kIntMul: the 59
// products not fused into an FMA run on the integer pipes (mul_int, the same bits as the FP64 multiply).
template <bool kU, bool kG, bool kIntMul = true, class Args = BwdArgs<double>>
__device__ __forceinline__ void bwd_point_f64(const Args &a, int64_t x)
{
    // ---- recompute: inverse metric and bracket
    const double g00 = ld_stream(a.in[IN_G + 0] + x), g01 = ld_stream(a.in[IN_G + 1] + x),
                 g02 = ld_stream(a.in[IN_G + 2] + x), g11 = ld_stream(a.in[IN_G + 3] + x),
                 g12 = ld_stream(a.in[IN_G + 4] + x), g22 = ld_stream(a.in[IN_G + 5] + x);
    double dg[18];
#pragma unroll
    for (int s = 0; s < 18; ++s)
        dg[s] = ld_stream(a.in[IN_DG + s] + x);
    double H[6], h[6];
    {
        double c[6];
        c[0] = fma(g11, g22, -mul64<kIntMul>(g12, g12));
        c[1] = fma(g02, g12, -mul64<kIntMul>(g01, g22));
        c[2] = fma(g01, g12, -mul64<kIntMul>(g02, g11));
        c[3] = fma(g00, g22, -mul64<kIntMul>(g02, g02));
        c[4] = fma(g01, g02, -mul64<kIntMul>(g00, g12));
        c[5] = fma(g00, g11, -mul64<kIntMul>(g01, g01));
        const double det = fma(g00, c[0], fma(g01, c[1], mul64<kIntMul>(g02, c[2])));
        const double rdet = rcp_f64(det);
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            H[p] = mul64<kIntMul>(c[p], rdet);
            h[p] = half_exact(H[p]);
        }
    }
    double T[3][6];
    christoffel_bracket<double>(dg, T);

    // ---- Eq. 5 and the footnote, reversed
    double W[6], K[6], S[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        W[p] = ld_opt(a.gout[OUT_DTG + p], x);
        K[p] = ld_stream(a.in[IN_K + p] + x);
    }
    adj_eq5_footnote<kU, kIntMul>(a, x, W, K, ld_stream(a.in[IN_ALPHA] + x), S);

    // betabar_k = -sum_p S_p Gamma^k_p = -sum_l h_kl u_l with u_l = sum_p S_p T_lp: Gamma itself is
    // never needed by the adjoint
    double u[3], beta[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        double s = mul64<kIntMul>(S[0], T[l][0]);
#pragma unroll
        for (int p = 1; p < 6; ++p)
            s = fma(S[p], T[l][p], s);
        u[l] = s;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        beta[k] = ld_stream(a.in[IN_BETA + k] + x);
        // the sign on the integer pipe: the compiler negates a binary64 result with an FP64 addition
        st_stream(a.gin[IN_BETA + k] + x,
                  neg_exact(fma(h[sym(k, 2)], u[2], fma(h[sym(k, 1)], u[1], mul64<kIntMul>(h[sym(k, 0)], u[0])))));
    }

    // ---- Gamma: Gammabar = V - beta_k S_p
    double gbar[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int p = 0; p < 6; ++p)
            gbar[k][p] = fma(-beta[k], S[p], ld_opt(a.gout[OUT_GAMMA + 6 * k + p], x));

    // ---- Eq. 6: Tbar, scattered onto d_k g_ij
    double Tb[3][6];
    adj_tbar<kIntMul>(h, gbar, Tb);
    adj_bracket_store(a, x, Tb);

    // ---- inverse: P = Tbar T^T (= H Hbar), plus h A_Y; gbar = -fold(P H)
    double P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            double s = mul64<kIntMul>(Tb[i][0], T[l][0]);
#pragma unroll
            for (int p = 1; p < 6; ++p)
                s = fma(Tb[i][p], T[l][p], s);
            P[i][l] = s;
        }
    if (kG) {
        double Y[6];
#pragma unroll
        for (int p = 0; p < 6; ++p)
            Y[p] = ld_opt(a.gout[OUT_GINV + p], x);
        adj_add_hAY<kIntMul>(h, Y, P);
    }
    double F[6];
    adj_fold_PH<kIntMul>(P, H, F);
#pragma unroll
    for (int p = 0; p < 6; ++p)
        st_stream(a.gin[IN_G + p] + x, neg_exact(F[p]));
}

}  // namespace tl
