// dtg_bwd.cu -- adjoint of the fused chain: given upstream gradients of the 39 outputs, the gradient of
// L = sum gout * out with respect to the 43 stored inputs.  The paper has no adjoint; this is the
// reverse-mode derivative of Eq. 5, the footnote to Listing 1, Eq. 6 and the inverse metric, taken in
// reverse order.  g^ij and the bracket T of Eq. 6 are recomputed in registers from the inputs (never
// stored or re-read; Gamma itself is not needed, see betabar below), so one launch reads the inputs
// the gradient depends on plus the upstream gradients present and writes 43 input gradients.
//
// Per point, with h = g^ij / 2, Gamma^i_p = sum_l h_il T_lp, Nbar the gradient of nabla_j beta_i:
//   Kbar_p = -2 alpha W_p,  abar = -2 sum_p K_p W_p,  Nbar_ij = U_ij + (W_p(ij), doubled on the diagonal)
//   dbetabar_ij = Nbar_ij,  S_p = Nbar_ij + Nbar_ji (i<j) or Nbar_ii,
//   betabar_k = -sum_p S_p Gamma^k_p = -sum_l h_kl u_l,  u_l = sum_p S_p T_lp
//   Gammabar_kp = V_kp - beta_k S_p
//   Tbar_lp = sum_i h_il Gammabar_ip, scattered through the bracket's three terms onto d_k g_ij
//   P = Tbar T^T (+ h A_Y),  gbar_ii = -(P H)_ii,  gbar_ij = -((P H)_ij + (P H)_ji)   (i < j)
// where W, V, U, Y are the upstream gradients of d_t g, Gamma, nabla beta and g^ij (the last line is
// -H A H folded onto the stored pairs, A = Hbar + Hbar^T; dtg_bwd_body.cuh derives it).
#include "dtg_bwd_body.cuh"
#include "ff.cuh"
#include "tl_kernels.h"

namespace tl {

// ------------------------------------------------------------------------------ float-float adjoint
// The binary64 adjoint needs 240 binary64 operations per point (181 of them on the 1/64-rate FP64
// pipe once its 59 stand-alone products run on the integer pipes).  Here the
// inverse, the bracket, Kbar, abar and the folds of the upstream gradients stay in binary64, and every
// contraction -- betabar, Gammabar, Hbar, Tbar, the bracket's scatter onto d_k g_ij and -H A H --
// runs in float-float pairs (ff.cuh); points with values the pairs cannot carry take the
// binary64 body.
template <bool kU, bool kG>
__device__ __noinline__ void bwd_point_f64_general(const BwdArgs<double> &a, int64_t x)
{
    bwd_point_f64<kU, kG, false>(a, x);
}

template <bool kU, bool kG> __device__ __forceinline__ void bwd_point_ff(const BwdArgs<double> &a, int64_t x)
{
    // every load first: the 34 inputs the gradient depends on (not d_j beta_i) and the upstream gradients
    double g[6], dg[18], K[6], W[6], V[18], beta[3];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        g[p] = ld_stream(a.in[IN_G + p] + x);
        K[p] = ld_stream(a.in[IN_K + p] + x);
        W[p] = ld_opt(a.gout[OUT_DTG + p], x);
    }
#pragma unroll
    for (int s = 0; s < 18; ++s) {
        dg[s] = ld_stream(a.in[IN_DG + s] + x);
        V[s] = ld_opt(a.gout[OUT_GAMMA + s], x);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        beta[k] = ld_stream(a.in[IN_BETA + k] + x);
    const double alpha = ld_stream(a.in[IN_ALPHA] + x);
    asm volatile("" ::: "memory");

    // binary64: inverse metric and bracket
    double H[6];
    {
        double c[6];
        c[0] = fma(g[3], g[5], -(g[4] * g[4]));
        c[1] = fma(g[2], g[4], -(g[1] * g[5]));
        c[2] = fma(g[1], g[4], -(g[2] * g[3]));
        c[3] = fma(g[0], g[5], -(g[2] * g[2]));
        c[4] = fma(g[1], g[2], -(g[0] * g[4]));
        c[5] = fma(g[0], g[3], -(g[1] * g[1]));
        const double det = fma(g[0], c[0], fma(g[1], c[1], g[2] * c[2]));
        const double rdet = rcp_f64(det);
#pragma unroll
        for (int p = 0; p < 6; ++p)
            H[p] = c[p] * rdet;
    }
    double Td[3][6];
    christoffel_bracket<double>(dg, Td);

    // binary64: Eq. 5 and the folds of the upstream gradients
    const double m2a = neg_exact(twice_exact(alpha));
    double asum = 0.0;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        st_stream(a.gin[IN_K + p] + x, m2a * W[p]);
        asum = (p == 0) ? K[p] * W[p] : fma(K[p], W[p], asum);
    }
    st_stream(a.gin[IN_ALPHA] + x, neg_exact(twice_exact(asum)));
    double S[6];
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

    // pairs
    uint32_t big = 0;
    ff hf[6], Sf[6], Tf[3][6], Vf[3][6], bf[3], Wgf[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        hf[p] = split_ff(half_exact(H[p]), big);
        Sf[p] = split_ff(S[p], big);
        Wgf[p] = kG ? split_ff(ld_opt(a.gout[OUT_GINV + p], x), big) : ff{0.0f, 0.0f};
    }
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            Tf[l][p] = split_ff(Td[l][p], big);
            Vf[l][p] = split_ff(V[6 * l + p], big);
        }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        bf[k] = split_ff(beta[k], big);
    if (big) {
        bwd_point_f64_general<kU, kG>(a, x);
        return;
    }

    // betabar_k = -sum_p S_p Gamma^k_p = -sum_l h_kl u_l with u_l = sum_p S_p T_lp
    ff uf[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        ffacc U = acc_prod(Sf[0], Tf[l][0]);
#pragma unroll
        for (int p = 1; p < 6; ++p)
            acc_add_prod(U, Sf[p], Tf[l][p]);
        uf[l] = acc_result(U);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ffacc B = acc_prod(hf[sym(k, 0)], uf[0]);
        acc_add_prod(B, hf[sym(k, 1)], uf[1]);
        acc_add_prod(B, hf[sym(k, 2)], uf[2]);
        st_stream(a.gin[IN_BETA + k] + x, neg_exact(merge_ff(acc_result(B))));
    }

    // Gammabar_kp = V_kp - beta_k S_p
    ff gb[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            ffacc A = acc_from(Vf[k][p]);
            acc_add_prod(A, ff_neg(bf[k]), Sf[p]);
            gb[k][p] = acc_result(A);
        }

    // Hbar_il = 1/2 sum_p Gammabar_ip T_lp ; A = Hbar + Hbar^T (+ the g^ij upstream gradient)
    ff Hb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            ffacc A = acc_prod(gb[i][0], Tf[l][0]);
#pragma unroll
            for (int p = 1; p < 6; ++p)
                acc_add_prod(A, gb[i][p], Tf[l][p]);
            Hb[i][l] = ff_scale(acc_result(A), 0.5f);
        }

    // Tbar_lp = sum_i h_il Gammabar_ip, scattered through the bracket onto d_k g_ij
    ffacc D[18];
    bool seen[18] = {};
    auto put = [&](int s, ff t) {   // first contribution assigned (resolved at compile time)
        if (seen[s])
            acc_add(D[s], t);
        else
            D[s] = acc_from(t);
        seen[s] = true;
    };
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = j; k < 3; ++k) {
                const int p = sym(j, k);
                ffacc A = acc_prod(hf[sym(0, l)], gb[0][p]);
                acc_add_prod(A, hf[sym(1, l)], gb[1][p]);
                acc_add_prod(A, hf[sym(2, l)], gb[2][p]);
                const ff t = acc_result(A);
                if (l == j) {
                    put(3 * sym(j, j) + k, t);
                } else if (l == k) {
                    put(3 * sym(k, k) + j, t);
                } else if (j == k) {
                    put(3 * sym(j, l) + j, ff_scale(t, 2.0f));
                    put(3 * sym(j, j) + l, ff_neg(t));
                } else {
                    put(3 * sym(j, l) + k, t);
                    put(3 * sym(l, k) + j, t);
                    put(3 * sym(j, k) + l, ff_neg(t));
                }
            }
#pragma unroll
    for (int s = 0; s < 18; ++s)
        st_stream(a.gin[IN_DG + s] + x, merge_ff(acc_result(D[s])));

    // inverse: gbar = fold of -H Hbar H with A = Hbar + Hbar^T
    ff Af[6], Hf[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const int p = sym(i, j);
            ffacc A = acc_from(i == j ? ff_scale(Hb[i][i], 2.0f) : Hb[i][j]);
            if (i != j)
                acc_add(A, Hb[j][i]);
            if (kG)
                acc_add(A, i == j ? ff_scale(Wgf[p], 2.0f) : Wgf[p]);
            Af[p] = acc_result(A);
            Hf[p] = ff_scale(hf[p], 2.0f);
        }
    ff M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            ffacc A = acc_prod(Hf[sym(i, 0)], Af[sym(0, j)]);
            acc_add_prod(A, Hf[sym(i, 1)], Af[sym(1, j)]);
            acc_add_prod(A, Hf[sym(i, 2)], Af[sym(2, j)]);
            M[i][j] = acc_result(A);
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            ffacc A = acc_prod(M[i][0], Hf[sym(0, j)]);
            acc_add_prod(A, M[i][1], Hf[sym(1, j)]);
            acc_add_prod(A, M[i][2], Hf[sym(2, j)]);
            ff v = acc_result(A);
            if (i == j)
                v = ff_scale(v, 0.5f);
            st_stream(a.gin[IN_G + sym(i, j)] + x, neg_exact(merge_ff(v)));
        }
}

// The float-float body is ~6000 instructions per point, and the kernel runs at 8 warps per SM (197
// registers): instruction fetch is what it waits on most.  One 256-thread block per SM walks the points
// in block-sized strides with a barrier after each, so the block's warps run the same stretch of code
// together and share its fetches (1.46 -> 1.29 ms at N = 2^22 against 128-thread blocks walking a
// grid stride).  The trip count depends only on the block, so every thread meets every barrier.
template <bool kU, bool kG>
__global__ void __launch_bounds__(kBwdFfThreads) dtg_bwd_ff_kernel(const BwdArgs<double> a, int64_t n)
{
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        if (base + threadIdx.x < n)
            bwd_point_ff<kU, kG>(a, base + threadIdx.x);
        __syncthreads();
    }
}

// Block-strided with a barrier per point, like the float-float adjoint (about 1 % over a grid stride).
// Four 128-thread blocks per SM (128 registers, 48 bytes spilled): 1.47 -> 1.40 ms at N = 2^22 against
// three blocks at 162 registers.
template <bool kU, bool kG>
__global__ void __launch_bounds__(kBwdThreads, 4) dtg_bwd_f64_kernel(const BwdArgs<double> a, int64_t n)
{
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        if (base + threadIdx.x < n)
            bwd_point_f64<kU, kG>(a, base + threadIdx.x);
        __syncthreads();
    }
}

static bool any_present(const double *const *p, int count)
{
    for (int i = 0; i < count; ++i)
        if (p[i])
            return true;
    return false;
}

// The upstream gradients of nabla beta and g^ij are often absent altogether; kernels specialised on
// their presence skip that work.  Within a group, NULL entries read as zero.
cudaError_t launch_bwd_f64(const BwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s)
{
    const bool hasU = any_present(a.gout + OUT_DBCOV, 9), hasG = any_present(a.gout + OUT_GINV, 6);
    if (hasU && hasG)
        dtg_bwd_f64_kernel<true, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasU)
        dtg_bwd_f64_kernel<true, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasG)
        dtg_bwd_f64_kernel<false, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else
        dtg_bwd_f64_kernel<false, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_bwd_ff(const BwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s)
{
    const bool hasU = any_present(a.gout + OUT_DBCOV, 9), hasG = any_present(a.gout + OUT_GINV, 6);
    if (hasU && hasG)
        dtg_bwd_ff_kernel<true, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasU)
        dtg_bwd_ff_kernel<true, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasG)
        dtg_bwd_ff_kernel<false, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else
        dtg_bwd_ff_kernel<false, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t occupancy_bwd(int *f64, int *ff)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(f64, dtg_bwd_f64_kernel<true, true>, kBwdThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ff, dtg_bwd_ff_kernel<false, false>, kBwdFfThreads, 0);
    return e;
}

}  // namespace tl
