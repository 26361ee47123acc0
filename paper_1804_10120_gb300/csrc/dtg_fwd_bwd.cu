// dtg_fwd_bwd.cu -- the forward chain and its adjoint in one pass, for a functional whose upstream
// gradients are known before the forward runs (L = sum gout * out with gout given, as for a loss that
// is linear in the outputs).  One launch reads the 43 inputs and the upstream gradients present, and
// writes the 39 outputs and the 43 input gradients: 1192 bytes per point for the loss
// sum W d_t g + V Gamma, against 656 + 808 for the forward and the adjoint launched one after the other.
//
// The forward is the binary64 body of tl_dtg_forward (outputs bit for bit the same).  The adjoint reuses
// what the forward formed in registers -- g^ij, the Eq. 6 bracket T and Gamma -- so it does not invert
// the metric or form the bracket again, and with Gamma at hand two of its contractions get shorter:
//   betabar_k = -sum_p S_p Gamma^k_p                          (18 terms)
//   gbar_ii = -2 sum_p Tbar_ip Gamma^i_p,
//   gbar_ij = -2 sum_p (Tbar_ip Gamma^j_p + Tbar_jp Gamma^i_p)   (i < j)
// the second because T^T g^ij = 2 Gamma^T turns -g^ij A g^ij (A = Hbar + Hbar^T, from dH = -H dG H)
// into -(X + X^T) with X = 2 Tbar Gamma^T (dtg_bwd_body.cuh gives the derivation).
#include "dtg_bwd_body.cuh"
#include "dtg_ff_body.cuh"
#include "tl_kernels.h"

namespace tl {

template <bool kU, bool kG>
__device__ __forceinline__ void fwdbwd_point_f64(const FwdBwdArgs<double> &a, int64_t x)
{
    double v[N_IN];
#pragma unroll
    for (int s = 0; s < N_IN; ++s)
        v[s] = ld_stream(a.in[s] + x);
    double W[6], V[3][6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
        W[p] = ld_opt(a.gout[OUT_DTG + p], x);
    asm volatile("" ::: "memory");   // the inputs and W are loaded before any arithmetic

    ChainF64Keep c;
    chain_f64_keep<FwdBwdArgs<double>, false, true>(v, a, x, 1.0, c);
    // the upstream gradients of Gamma are loaded only now, when the forward has released most of the
    // inputs' registers (164 registers without spills, against 168 with spills when loaded up front:
    // 1.78 against 1.85 ms at N = 2^22)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int p = 0; p < 6; ++p)
            V[k][p] = ld_opt(a.gout[OUT_GAMMA + 6 * k + p], x);

    // ---- Eq. 5 and the footnote, reversed
    double K[6], S[6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
        K[p] = v[IN_K + p];
    adj_eq5_footnote<kU, true>(a, x, W, K, v[IN_ALPHA], S);

    // betabar_k = -sum_p S_p Gamma^k_p
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double s = mul_int(S[0], c.gam[k][0]);
#pragma unroll
        for (int p = 1; p < 6; ++p)
            s = fma(S[p], c.gam[k][p], s);
        st_stream(a.gin[IN_BETA + k] + x, neg_exact(s));
    }

    // Gammabar_kp = V_kp - beta_k S_p
    double gbar[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int p = 0; p < 6; ++p)
            gbar[k][p] = fma(-v[IN_BETA + k], S[p], V[k][p]);

    // Eq. 6: Tbar, scattered onto d_k g_ij
    double Tb[3][6];
    adj_tbar<true>(c.h, gbar, Tb);
    adj_bracket_store(a, x, Tb);

    // inverse: gbar = -(X + X^T) folded, X = 2 Tbar Gamma^T (+ the g^ij upstream gradient's -H A_Y H)
    double F[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double s = mul_int(Tb[i][0], c.gam[j][0]);
#pragma unroll
            for (int p = 1; p < 6; ++p)
                s = fma(Tb[i][p], c.gam[j][p], s);
            if (i != j) {
#pragma unroll
                for (int p = 0; p < 6; ++p)
                    s = fma(Tb[j][p], c.gam[i][p], s);
            }
            F[sym(i, j)] = twice_exact(s);
        }
    if (kG) {
        double Y[6], P[3][3] = {}, FY[6];
#pragma unroll
        for (int p = 0; p < 6; ++p)
            Y[p] = ld_opt(a.gout[OUT_GINV + p], x);
        adj_add_hAY<true>(c.h, Y, P);
        adj_fold_PH<true>(P, c.ginv, FY);
#pragma unroll
        for (int p = 0; p < 6; ++p)
            F[p] += FY[p];
    }
#pragma unroll
    for (int p = 0; p < 6; ++p)
        st_stream(a.gin[IN_G + p] + x, neg_exact(F[p]));
}

// Block-strided with a barrier per point, like the adjoint kernels: the block's warps run the same
// stretch of the long straight-line body together and share its instruction fetches.  The trip count
// depends only on the block, so every thread meets every barrier.  Three 128-thread blocks per SM
// (<= 168 registers): 1.85 ms at N = 2^22 against 2.12 ms at two blocks (182 registers), and 2.08 ms
// at four (128 registers, 224 bytes spilled).
template <bool kU, bool kG>
__global__ void __launch_bounds__(kFwdBwdThreads, 3) dtg_fwdbwd_f64_kernel(const FwdBwdArgs<double> a, int64_t n)
{
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        if (base + threadIdx.x < n)
            fwdbwd_point_f64<kU, kG>(a, base + threadIdx.x);
        __syncthreads();
    }
}

// ------------------------------------------------------------------- float-float forward + adjoint
// The same pass with the float-float arithmetic of TL_F64_FF: the inverse, the Eq. 6 bracket, the
// folds of the upstream gradients and Eq. 5 in binary64, every contraction -- Eq. 6 and the footnote in
// the forward, betabar, Gammabar, Tbar, the bracket's scatter and the folded -H A H in the adjoint --
// in float-float pairs reusing the forward's h, T and Gamma.  A point whose inputs fall outside the
// pair format's range is evaluated again, outputs and gradients, by the binary64 pass (the float-float
// forward takes binary64 for such a point too); one whose upstream gradients or S do keeps its outputs
// and takes its gradients from the binary64 adjoint.
template <bool kU, bool kG> __device__ __noinline__ void fwdbwd_point_f64_general(const FwdBwdArgs<double> &a, int64_t x)
{
    fwdbwd_point_f64<kU, kG>(a, x);
}

// The gradients alone, by the binary64 adjoint's body (the same bits as tl_dtg_backward with TL_F64),
// for a point whose float-float outputs are already stored.
template <bool kU, bool kG> __device__ __noinline__ void fwdbwd_point_grad_f64(const FwdBwdArgs<double> &a, int64_t x)
{
    bwd_point_f64<kU, kG, false>(a, x);
}

template <bool kU, bool kG>
__device__ __forceinline__ void fwdbwd_point_ff(const FwdBwdArgs<double> &a, int64_t x)
{
    double v[N_IN];
#pragma unroll
    for (int s = 0; s < N_IN; ++s)
        v[s] = ld_stream(a.in[s] + x);
    double W[6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
        W[p] = ld_opt(a.gout[OUT_DTG + p], x);
    asm volatile("" ::: "memory");

    ChainFFKeep c;
    if (!chain_ff_keep<FwdBwdArgs<double>, false>(v, a, x, 1.0, c)) {
        fwdbwd_point_f64_general<kU, kG>(a, x);
        return;
    }
    uint32_t big = 0;
    ff V[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int p = 0; p < 6; ++p)
            V[k][p] = split_ff(ld_opt(a.gout[OUT_GAMMA + 6 * k + p], x), big);

    // Eq. 5 and the footnote reversed, in binary64
    double K[6], S[6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
        K[p] = v[IN_K + p];
    adj_eq5_footnote<kU, false>(a, x, W, K, v[IN_ALPHA], S);
    ff Sf[6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
        Sf[p] = split_ff(S[p], big);
    if (big) {   // the outputs stand; the gradients come from the binary64 adjoint
        fwdbwd_point_grad_f64<kU, kG>(a, x);
        return;
    }

    // betabar_k = -sum_p S_p Gamma^k_p
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ffacc B = acc_prod(Sf[0], c.gam[k][0]);
#pragma unroll
        for (int p = 1; p < 6; ++p)
            acc_add_prod(B, Sf[p], c.gam[k][p]);
        st_stream(a.gin[IN_BETA + k] + x, neg_exact(merge_ff(acc_result(B))));
    }

    // Gammabar_kp = V_kp - beta_k S_p
    ff gb[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            ffacc A = acc_from(V[k][p]);
            acc_add_prod(A, ff_neg(c.b[k]), Sf[p]);
            gb[k][p] = acc_result(A);
        }

    // Tbar_lp = sum_i h_il Gammabar_ip, scattered through the bracket onto d_k g_ij
    ff Tb[3][6];
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
                ffacc A = acc_prod(c.h[sym(0, l)], gb[0][p]);
                acc_add_prod(A, c.h[sym(1, l)], gb[1][p]);
                acc_add_prod(A, c.h[sym(2, l)], gb[2][p]);
                const ff t = acc_result(A);
                Tb[l][p] = t;
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

    // inverse: gbar = -(X + X^T) folded, X = 2 Tbar Gamma^T (+ the g^ij upstream gradient's -H A_Y H)
    double F[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            ffacc A = acc_prod(Tb[i][0], c.gam[j][0]);
#pragma unroll
            for (int p = 1; p < 6; ++p)
                acc_add_prod(A, Tb[i][p], c.gam[j][p]);
            if (i != j) {
#pragma unroll
                for (int p = 0; p < 6; ++p)
                    acc_add_prod(A, Tb[j][p], c.gam[i][p]);
            }
            F[sym(i, j)] = twice_exact(merge_ff(acc_result(A)));
        }
    if (kG) {
        double Y[6], h[6], P[3][3] = {}, FY[6];
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            Y[p] = ld_opt(a.gout[OUT_GINV + p], x);
            h[p] = half_exact(c.ginv[p]);
        }
        adj_add_hAY<false>(h, Y, P);
        adj_fold_PH<false>(P, c.ginv, FY);
#pragma unroll
        for (int p = 0; p < 6; ++p)
            F[p] += FY[p];
    }
#pragma unroll
    for (int p = 0; p < 6; ++p)
        st_stream(a.gin[IN_G + p] + x, neg_exact(F[p]));
}

// One 256-thread block per SM walking block-sized strides with a barrier per point, as the float-float
// adjoint does (its body is of the same length).
template <bool kU, bool kG>
__global__ void __launch_bounds__(kFwdBwdFfThreads) dtg_fwdbwd_ff_kernel(const FwdBwdArgs<double> a, int64_t n)
{
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        if (base + threadIdx.x < n)
            fwdbwd_point_ff<kU, kG>(a, base + threadIdx.x);
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

cudaError_t launch_fwdbwd_f64(const FwdBwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s)
{
    const bool hasU = any_present(a.gout + OUT_DBCOV, 9), hasG = any_present(a.gout + OUT_GINV, 6);
    if (hasU && hasG)
        dtg_fwdbwd_f64_kernel<true, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasU)
        dtg_fwdbwd_f64_kernel<true, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasG)
        dtg_fwdbwd_f64_kernel<false, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else
        dtg_fwdbwd_f64_kernel<false, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_fwdbwd_ff(const FwdBwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s)
{
    const bool hasU = any_present(a.gout + OUT_DBCOV, 9), hasG = any_present(a.gout + OUT_GINV, 6);
    if (hasU && hasG)
        dtg_fwdbwd_ff_kernel<true, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasU)
        dtg_fwdbwd_ff_kernel<true, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else if (hasG)
        dtg_fwdbwd_ff_kernel<false, true><<<sh.grid, sh.threads, 0, s>>>(a, n);
    else
        dtg_fwdbwd_ff_kernel<false, false><<<sh.grid, sh.threads, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t occupancy_fwdbwd(int *f64, int *ff)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(f64, dtg_fwdbwd_f64_kernel<true, true>, kFwdBwdThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ff, dtg_fwdbwd_ff_kernel<false, false>, kFwdBwdFfThreads, 0);
    return e;
}

}  // namespace tl
