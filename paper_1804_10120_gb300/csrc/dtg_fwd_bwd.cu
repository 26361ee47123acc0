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

cudaError_t occupancy_fwdbwd(int *f64)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(f64, dtg_fwdbwd_f64_kernel<true, true>, kFwdBwdThreads, 0);
}

}  // namespace tl
