// dtg_fwd_ff.cu -- forward chain with float-float contractions (TL_F64_FF).
//
// GB300 issues FP64 arithmetic at 1/64 of its FP32 rate (two FP64 operations per clock per SM), and
// the all-binary64 chain needs 126 binary64 operations per point (89 on the FP64 pipe when its
// stand-alone products run on the integer pipes): that alone caps it near 48-68 % of the HBM
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
#include "dtg_ff_body.cuh"
#include "ff.cuh"
#include "tl_kernels.h"

namespace tl {

// The all-binary64 evaluation, out of line (only points outside the pair format's range take it).
__device__ __noinline__ void fwd_point_f64_general(const FwdArgs<double> &a, int64_t x) { fwd_point_f64<false>(a, x); }

__device__ __forceinline__ void fwd_point_ff(const FwdArgs<double> &a, int64_t x)
{
    double v[N_IN];
#pragma unroll
    for (int s = 0; s < N_IN; ++s)
        v[s] = ld_stream(a.in[s] + x);
    asm volatile("" ::: "memory");   // every load is issued before any arithmetic
    if (!chain_ff(v, a, x))          // outside the pair format's range: all-binary64 evaluation
        fwd_point_f64_general(a, x);
}

// Blocks walk block-sized strides with a barrier per point, which keeps a block's warps on the same
// stretch of the ~3000-instruction body (2.47 -> 2.43 ms at N = 2^24; the same walk lifted the
// float-float adjoint, whose body is twice as long, by 11 %).  The trip count depends only on the block.
__global__ void __launch_bounds__(kFwdThreads, 2) dtg_fwd_ff_kernel(const FwdArgs<double> a, int64_t n)
{
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        if (base + threadIdx.x < n)
            fwd_point_ff(a, base + threadIdx.x);
        __syncthreads();
    }
}

cudaError_t launch_fwd_ff(const FwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s)
{
    dtg_fwd_ff_kernel<<<sh.grid, sh.threads, 0, s>>>(a, n);
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

// The integer-pipe binary64 operations against the hardware ones (tl_testing.h).
namespace tl {

__global__ void f64_int_testing_kernel(int op, const double *a, const double *b, const double *c, double *y,
                                       int64_t n)
{
    const GridStride gs;
    for (int64_t i = gs.first; i < n; i += gs.step) {
        if (op == 0)
            y[i] = mul_int(a[i], b[i]);
        else if (op == 1)
            y[i] = rcp_f64(a[i]);
        else
            y[i] = fma(a[i], b[i], c[i]);
    }
}

}  // namespace tl

extern "C" TL_API tl_status tl_testing_f64_int(int op, const double *a, const double *b, const double *c, double *y,
                                               int64_t n, tl_stream stream)
{
    if (op < 0 || op > 3 || op == 2 || n < 0 || !a || !y || (op != 1 && !b) || (op == 3 && !c))
        return TL_ERR_INVALID_ARG;
    if (n == 0)
        return TL_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    tl::f64_int_testing_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(op, a, b, c, y, n);
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}
