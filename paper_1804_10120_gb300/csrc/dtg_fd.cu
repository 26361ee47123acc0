// dtg_fd.cu -- the fused chain with the spatial derivatives formed on the grid.
//
// The paper's kernels take d_k g_ij and d_j beta_i as inputs (27 arrays; Listing 3's dg).  Here they
// are computed inside the kernel by centred finite differences on a periodic nx x ny x nz grid (x
// fastest), of order 2,  (f(x+h) - f(x-h)) / (2h),  or 4,  (8 (f(x+h) - f(x-h)) - (f(x+2h) - f(x-2h)))
// / (12h), so one launch reads 16 arrays (g, K, alpha, beta) instead of 43 and writes the same 39:
// 440 instead of 656 bytes per point.  One thread per point; the neighbours of a point are shared with
// the threads around it, and the z-planes a wave of blocks touches (a few MB) stay in L2, so each array
// still crosses HBM about once.  The chain itself is the single-grid kernel's body (binary64 or
// float-float contractions).
#include <cmath>

#include "dtg_ff_body.cuh"
#include "tl_host.h"
#include "tl_kernels.h"

namespace tl {

enum : int { FD_G = 0, FD_K = 6, FD_ALPHA = 12, FD_BETA = 13, FD_N_IN = 16 };

struct FdArgs {
    const double *in[FD_N_IN];
    double *out[N_OUT];
    int64_t nx, ny, nz;
    double c1[3], c2[3];   // per axis: 1/(2h) (order 2) or 8/(12h), 1/(12h) (order 4)
};

// With equal spacings along the three axes every derivative is c1 times a plain difference,
//   order 2:  f(x+h) - f(x-h),      order 4:  (f(x+h) - f(x-h)) - (f(x+2h) - f(x-2h)) / 8,
// (8/12 = c1 h and 1/12 = c1 h / 8), so the kernel forms the differences and the chain applies c1 once
// (to 1/2 g^il and inside nabla_j beta_i): 21 fewer binary64 operations per point.

// Coordinate of the neighbour at offset o (|o| <= 2) along a periodic axis of length m: (i + o) mod m.
// One conditional correction suffices when m >= 3; shorter axes take the modulo.
__device__ __forceinline__ int wrapc(int i, int o, int m)
{
    int j = i + o;
    if (m >= 3)
        return (j >= m) ? j - m : (j < 0 ? j + m : j);
    return ((j % m) + m) % m;
}

// Per grid row (iy, iz): element offsets of the +-1, +-2 neighbour rows along y and z, relative to the
// row's own start (index 0..3 = offset -2, -1, +1, +2).
struct RowNeighbours {
    int64_t y[4], z[4];
};

template <int ORDER, bool UNIFORM>
__device__ __forceinline__ double fd_axis(const double *__restrict__ f, int64_t x, const int64_t (&off)[4], double c1,
                                          double c2)
{
    const double d1 = __ldg(f + x + off[2]) - __ldg(f + x + off[1]);
    if (ORDER == 2)
        return UNIFORM ? d1 : d1 * c1;
    const double d2 = __ldg(f + x + off[3]) - __ldg(f + x + off[0]);
    return UNIFORM ? fma(d2, -0.125, d1) : fma(d1, c1, -(d2 * c2));
}

template <int ORDER, bool UNIFORM>
__device__ __forceinline__ void fd_inputs(const FdArgs &a, int64_t x, const int64_t (&xo)[4], const RowNeighbours &rn,
                                          double (&v)[N_IN])
{
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        const double *f = a.in[FD_G + p];
        v[IN_G + p] = __ldg(f + x);
        v[IN_DG + 3 * p + 0] = fd_axis<ORDER, UNIFORM>(f, x, xo, a.c1[0], a.c2[0]);
        v[IN_DG + 3 * p + 1] = fd_axis<ORDER, UNIFORM>(f, x, rn.y, a.c1[1], a.c2[1]);
        v[IN_DG + 3 * p + 2] = fd_axis<ORDER, UNIFORM>(f, x, rn.z, a.c1[2], a.c2[2]);
        v[IN_K + p] = ld_stream(a.in[FD_K + p] + x);
    }
    v[IN_ALPHA] = ld_stream(a.in[FD_ALPHA] + x);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double *f = a.in[FD_BETA + i];
        v[IN_BETA + i] = __ldg(f + x);
        v[IN_DBETA + 3 * i + 0] = fd_axis<ORDER, UNIFORM>(f, x, xo, a.c1[0], a.c2[0]);
        v[IN_DBETA + 3 * i + 1] = fd_axis<ORDER, UNIFORM>(f, x, rn.y, a.c1[1], a.c2[1]);
        v[IN_DBETA + 3 * i + 2] = fd_axis<ORDER, UNIFORM>(f, x, rn.z, a.c1[2], a.c2[2]);
    }
}

// The binary64 form loads g and forms d_k g_ij first (the inverse and Eq. 6 need nothing else), and
// K, alpha, beta and the d_j beta_i stencils only after Eq. 6, through the chain's late-input hook, so
// that their registers are free meanwhile: 80 -> 52 bytes spilled at 128 registers, order 4 at 256^3
// 5.65 -> 5.46 ms.
template <int ORDER, bool UNIFORM>
__device__ __forceinline__ void fd_inputs_early(const FdArgs &a, int64_t x, const int64_t (&xo)[4], const RowNeighbours &rn,
                                                double (&v)[N_IN])
{
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        const double *f = a.in[FD_G + p];
        v[IN_G + p] = __ldg(f + x);
        v[IN_DG + 3 * p + 0] = fd_axis<ORDER, UNIFORM>(f, x, xo, a.c1[0], a.c2[0]);
        v[IN_DG + 3 * p + 1] = fd_axis<ORDER, UNIFORM>(f, x, rn.y, a.c1[1], a.c2[1]);
        v[IN_DG + 3 * p + 2] = fd_axis<ORDER, UNIFORM>(f, x, rn.z, a.c1[2], a.c2[2]);
    }
#pragma unroll
    for (int s = IN_K; s < N_IN; ++s)
        v[s] = 0.0;
}

template <int ORDER, bool UNIFORM> struct FdLate {
    const int64_t (&xo)[4];
    const RowNeighbours &rn;
    __device__ __forceinline__ void operator()(const FdArgs &a, int64_t x, double (&v)[N_IN]) const
    {
#pragma unroll
        for (int p = 0; p < 6; ++p)
            v[IN_K + p] = ld_stream(a.in[FD_K + p] + x);
        v[IN_ALPHA] = ld_stream(a.in[FD_ALPHA] + x);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double *f = a.in[FD_BETA + i];
            v[IN_BETA + i] = __ldg(f + x);
            v[IN_DBETA + 3 * i + 0] = fd_axis<ORDER, UNIFORM>(f, x, xo, a.c1[0], a.c2[0]);
            v[IN_DBETA + 3 * i + 1] = fd_axis<ORDER, UNIFORM>(f, x, rn.y, a.c1[1], a.c2[1]);
            v[IN_DBETA + 3 * i + 2] = fd_axis<ORDER, UNIFORM>(f, x, rn.z, a.c1[2], a.c2[2]);
        }
    }
};

// Blocks walk grid rows (iy, iz); the threads of a block walk the row's points.  All coordinate
// arithmetic is per row except the x wrap.
template <int ORDER, bool FF, bool UNIFORM>
__global__ void __launch_bounds__(256, 2) dtg_fd_kernel(const FdArgs a, int64_t n)
{
    (void)n;
    const int nx = (int)a.nx, ny = (int)a.ny, nz = (int)a.nz;
    const int64_t plane = (int64_t)nx * ny;
    for (int r = blockIdx.x; r < ny * nz; r += gridDim.x) {
        const int iy = r % ny, iz = r / ny;
        RowNeighbours rn;
        const int offs[4] = {-2, -1, 1, 2};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            rn.y[q] = (int64_t)(wrapc(iy, offs[q], ny) - iy) * nx;
            rn.z[q] = (int64_t)(wrapc(iz, offs[q], nz) - iz) * plane;
        }
        const int64_t row = (int64_t)r * nx;
        for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
            int64_t xo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                xo[q] = wrapc(ix, offs[q], nx) - ix;
            const int64_t x = row + ix;
            double v[N_IN];
            if (FF) {
                fd_inputs<ORDER, UNIFORM>(a, x, xo, rn, v);
                if (!chain_ff<FdArgs, UNIFORM>(v, a, x, a.c1[0]))
                    chain_f64<FdArgs, UNIFORM, false>(v, a, x, a.c1[0]);
            } else {
                fd_inputs_early<ORDER, UNIFORM>(a, x, xo, rn, v);
                asm volatile("" ::: "memory");   // d_k g_ij formed before the chain starts
                ChainF64Keep unused;
                chain_f64_keep<FdArgs, UNIFORM, true, true, FdLate<ORDER, UNIFORM>>(v, a, x, a.c1[0], unused,
                                                                                    FdLate<ORDER, UNIFORM>{xo, rn});
            }
        }
    }
}

// A block walks whole grid rows, so a block wider than a row leaves threads idle on every row: the
// block is the row length rounded up to whole warps, at most 256 threads (128^3: 128-thread blocks,
// four per SM, instead of 256-thread blocks with half their threads idle).
template <int ORDER, bool FF, bool UNIFORM>
static cudaError_t fd_launch(const FdArgs &a, int64_t n, int sms, cudaStream_t s)
{
    const int threads = (int)std::min<int64_t>(256, std::max<int64_t>(32, (a.nx + 31) / 32 * 32));
    int blocks = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, dtg_fd_kernel<ORDER, FF, UNIFORM>, threads, 0);
    if (e != cudaSuccess)
        return e;
    const int64_t rows = a.ny * a.nz;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(rows, (int64_t)sms * std::max(blocks, 1)));
    dtg_fd_kernel<ORDER, FF, UNIFORM><<<grid, threads, 0, s>>>(a, n);
    return cudaGetLastError();
}

template <int ORDER, bool FF> static cudaError_t fd_launch(const FdArgs &a, int64_t n, int sms, cudaStream_t s, bool uniform)
{
    return uniform ? fd_launch<ORDER, FF, true>(a, n, sms, s) : fd_launch<ORDER, FF, false>(a, n, sms, s);
}

}  // namespace tl

using namespace tl;

extern "C" tl_status tl_dtg_forward_fd(const tl_dtg_grid_in *in, const tl_dtg_out *out, const tl_grid3d *grid,
                                       tl_dtype dtype, tl_stream stream)
{
    if (!in || !out || !grid)
        return fail(TL_ERR_INVALID_ARG, "NULL argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
        return fail(TL_ERR_INVALID_ARG, "grid extents must be >= 1");
    if (!(grid->hx > 0 && grid->hy > 0 && grid->hz > 0) || !std::isfinite(grid->hx) || !std::isfinite(grid->hy) ||
        !std::isfinite(grid->hz))
        return fail(TL_ERR_INVALID_ARG, "grid spacings must be positive and finite");
    if (grid->order != 2 && grid->order != 4)
        return fail(TL_ERR_INVALID_ARG, "finite-difference order must be 2 or 4");
    if (dtype != TL_F64 && dtype != TL_F64_FF)
        return fail(TL_ERR_UNSUPPORTED, "the on-grid form is provided for TL_F64 and TL_F64_FF");
    if (grid->nx > INT32_MAX || grid->ny > INT32_MAX || grid->nz > INT32_MAX || grid->ny * grid->nz > INT32_MAX ||
        grid->nx > (int64_t(1) << 40) / grid->ny / grid->nz)
        return fail(TL_ERR_INVALID_ARG, "grid too large (ny*nz and each extent must fit in 32 bits)");
    const int64_t n = grid->nx * grid->ny * grid->nz;
    const void *const *tabs[2] = {(const void *const *)in, (const void *const *)out};
    const int counts[2] = {FD_N_IN, N_OUT};
    const bool writes[2] = {false, true}, nullable[2] = {false, false};
    const char *const names[2] = {"in", "out"};
    std::vector<Range> rs;
    tl_status s = collect_ranges(rs, tabs, counts, writes, nullable, names, 2, n, sizeof(double), -1);
    if (s == TL_OK)
        s = check_overlaps(rs);
    if (s != TL_OK)
        return s;
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    FdArgs a;
    for (int q = 0; q < FD_N_IN; ++q)
        a.in[q] = (const double *)((const void *const *)in)[q];
    for (int q = 0; q < N_OUT; ++q)
        a.out[q] = (double *)((void *const *)out)[q];
    a.nx = grid->nx;
    a.ny = grid->ny;
    a.nz = grid->nz;
    const double h[3] = {grid->hx, grid->hy, grid->hz};
    for (int k = 0; k < 3; ++k) {
        a.c1[k] = grid->order == 2 ? 1.0 / (2.0 * h[k]) : 8.0 / (12.0 * h[k]);
        a.c2[k] = grid->order == 2 ? 0.0 : 1.0 / (12.0 * h[k]);
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const bool ff = dtype == TL_F64_FF;
    const bool u = grid->hx == grid->hy && grid->hy == grid->hz;
    cudaError_t e = grid->order == 2
                        ? (ff ? fd_launch<2, true>(a, n, d->sms, st, u) : fd_launch<2, false>(a, n, d->sms, st, u))
                        : (ff ? fd_launch<4, true>(a, n, d->sms, st, u) : fd_launch<4, false>(a, n, d->sms, st, u));
    if (e != cudaSuccess)
        return cuda_fail(e, "on-grid forward launch");
    return TL_OK;
}
