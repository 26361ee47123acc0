// dtg_fwd_ff.cu -- forward chain with float-float contractions (TL_F64_FF).
//
// GB300 issues FP64 arithmetic at 1/64 of its FP32 rate (two FP64 operations per clock per SM), and
// the all-binary64 chain needs ~126 of them per point: that alone caps it near 45 % of the HBM
// roofline.  This kernel keeps binary64 hardware for the cancellation-prone parts -- the cofactors,
// determinant and inverse of g_ij, the bracket of Eq. 6 and Eq. 5 itself -- and evaluates the two
// contractions, Gamma^i_jk = sum_l (g^il / 2) T_ljk (Eq. 6) and sum_k Gamma^k_ij beta_k (footnote to
// Listing 1), in float-float pairs on the FP32 pipes, converting between binary64 and pairs with
// integer operations (ff.cuh).  FP64 work drops to ~54 operations per point.  Points whose values
// fall outside the pair format's safe range (|x| >= 2^63, inf, nan) are evaluated by the
// all-binary64 path instead.
#include "dtg_batched.cuh"
#include "dtg_fwd_body.cuh"
#include <algorithm>

#include "../../include/tl_testing.h"
#include "ff.cuh"
#include "tl_kernels.h"

namespace tl {

// The all-binary64 evaluation, out of line (only points outside the pair format's range take it).
__device__ __noinline__ void fwd_point_f64_general(const FwdArgs<double> &a, int64_t x) { fwd_point_f64(a, x); }

__device__ __forceinline__ void fwd_point_ff(const FwdArgs<double> &a, int64_t x)
{
    double v[N_IN];
#pragma unroll
    for (int s = 0; s < N_IN; ++s)
        v[s] = ld_stream(a.in[s] + x);
    asm volatile("" ::: "memory");   // every load is issued before any arithmetic
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
        st_stream(a.out[OUT_GINV + p] + x, gi);
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

    if (big) {   // outside the pair format's range: the all-binary64 evaluation of this point
        fwd_point_f64_general(a, x);
        return;
    }

    // step 2: Eq. 6 contraction in pairs
    ff gam[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            gam[i][p] = dot3_ff(h[sym(i, 0)], T[0][p], h[sym(i, 1)], T[1][p], h[sym(i, 2)], T[2][p]);
            st_stream(a.out[OUT_GAMMA + 6 * i + p] + x, merge_ff(gam[i][p]));
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
            nb[i][j] = v[IN_DBETA + 3 * i + j] - S6[sym(i, j)];
            st_stream(a.out[OUT_DBCOV + 3 * i + j] + x, nb[i][j]);
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
            st_stream(a.out[OUT_DTG + p] + x, fma(m2a, K, s));
        }
}

__global__ void __launch_bounds__(kFwdThreads) dtg_fwd_ff_kernel(const FwdArgs<double> a, int64_t n)
{
    const GridStride gs;
    for (int64_t x = gs.first; x < n; x += gs.step)
        fwd_point_ff(a, x);
}

cudaError_t launch_fwd_ff(const FwdArgs<double> &a, int64_t n, int grid, cudaStream_t s)
{
    dtg_fwd_ff_kernel<<<grid, kFwdThreads, 0, s>>>(a, n);
    return cudaGetLastError();
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads) dtg_batched_ff_kernel(const BatchView v)
{
    __shared__ FwdArgs<double> s_args;
    batched_loop<double>(v, s_args, [](const FwdArgs<double> &a, int64_t x) { fwd_point_ff(a, x); });
}

cudaError_t launch_batched_ff(const BatchView &v, int threads, int grid, cudaStream_t s)
{
    switch (threads) {
    case 128: dtg_batched_ff_kernel<128><<<grid, 128, 0, s>>>(v); break;
    case 256: dtg_batched_ff_kernel<256><<<grid, 256, 0, s>>>(v); break;
    case 512: dtg_batched_ff_kernel<512><<<grid, 512, 0, s>>>(v); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t occupancy_batched_ff(int threads, int *blocks)
{
    switch (threads) {
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_ff_kernel<128>, 128, 0);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_ff_kernel<256>, 256, 0);
    case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_ff_kernel<512>, 512, 0);
    }
    return cudaErrorInvalidValue;
}

cudaError_t occupancy_fwd_ff(int *ff_blocks)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ff_blocks, dtg_fwd_ff_kernel, kFwdThreads, 0);
}

}  // namespace tl

// ------------------------------------------------------------------------------- test hook (tl_testing.h)
namespace tl {

__global__ void ff_testing_kernel(int op, const double *a, const double *b, const double *c, const double *d,
                                  const double *e, const double *f, double *y, int64_t n)
{
    const GridStride gs;
    for (int64_t i = gs.first; i < n; i += gs.step) {
        uint32_t big = 0;
        if (op == 0) {
            y[i] = merge_ff(normalize_ff(split_ff(a[i], big)));
        } else if (op == 1) {
            const ff pa = split_ff(a[i], big), pb = split_ff(b[i], big);
            y[i] = merge_ff(sub_ff(pa, pb));
        } else {
            const ff pa = split_ff(a[i], big), pb = split_ff(b[i], big), pc = split_ff(c[i], big),
                     pd = split_ff(d[i], big), pe = split_ff(e[i], big), pf = split_ff(f[i], big);
            y[i] = merge_ff(dot3_ff(pa, pb, pc, pd, pe, pf));
        }
    }
}

}  // namespace tl

extern "C" TL_API tl_status tl_testing_ff(int op, const double *a, const double *b, const double *c,
                                          const double *d, const double *e, const double *f, double *y,
                                          int64_t n, tl_stream stream)
{
    if (op < 0 || op > 2 || n < 0 || !a || !y || (op >= 1 && !b) || (op == 2 && (!c || !d || !e || !f)))
        return TL_ERR_INVALID_ARG;
    if (n == 0)
        return TL_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    tl::ff_testing_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(op, a, b, c, d, e, f, y, n);
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}
