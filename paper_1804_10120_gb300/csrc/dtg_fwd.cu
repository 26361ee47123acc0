// dtg_fwd.cu -- fused forward kernels: inverse metric -> Christoffel symbols (Eq. 6) -> covariant
// derivative of the shift (footnote to Listing 1) -> d_t g_ij (Eq. 5), one grid point per thread.
//
// Each thread reads the 43 input components of its point once, keeps every intermediate in
// registers and writes the 39 outputs once: 656 bytes of HBM traffic per point in binary64, the
// paper's effective-bandwidth count N_e = 82 (Sec. 5.1, Eq. 8).  Unlike the paper's generated
// kernels (one thread per point and output component, one kernel per expression, pointer tables
// read from global memory; Sec. 4), the whole chain is one kernel and the pointer tables are kernel
// parameters.
#include <algorithm>

#include "bulk.cuh"
#include "dtg_batched.cuh"
#include "dtg_fwd_body.cuh"

namespace tl {

__global__ void __launch_bounds__(kFwdF64Threads, kFwdF64Blocks) dtg_fwd_f64_kernel(const FwdArgs<double> a, int64_t n)
{
    const GridStride gs;
    for (int64_t x = gs.first; x < n; x += gs.step)
        fwd_point_f64(a, x);
}

// Grids too small to give every SM a full block (fewer than SMs x 256 points) run at most a warp or a
// few per SM, so the time is one warp's path through the body rather than the FP64 pipe's throughput.
// There the products stay FP64 multiplies (the same bits as the integer-pipe form): about 1400 fewer
// instructions per point, 12.3 -> 10.2 us at N = 4096.
__global__ void __launch_bounds__(kFwdF64Threads, kFwdF64Blocks) dtg_fwd_f64_small_kernel(const FwdArgs<double> a,
                                                                                           int64_t n)
{
    const GridStride gs;
    for (int64_t x = gs.first; x < n; x += gs.step)
        fwd_point_f64<false>(a, x);
}

// ------------------------------------------------------------------------------------ binary32 forward
// Storage and arithmetic in binary32, except det(g) and the 3x3 inverse, which are formed in binary64
// from the (exactly widened) binary32 metric and rounded once to binary32.
template <bool kIntConv>
__device__ __forceinline__ double widen(float f, uint32_t &rare)
{
    return kIntConv ? f32_to_f64(f, rare) : (double)f;
}
template <bool kIntConv>
__device__ __forceinline__ float narrow(double d, uint32_t &rare)
{
    return kIntConv ? f64_to_f32(d, rare) : (float)d;
}

// The chain on one point's 43 binary32 inputs (in registers, input-table order), outputs to
// a.out[s][x].  kIntConv: binary32 <-> binary64 conversions on the integer pipe (returns false, having
// written nothing, when an operand needs the general conversions); otherwise the compiler's F2F
// conversions.
template <bool kIntConv>
__device__ __forceinline__ bool chain_f32(const float (&v)[N_IN], const FwdArgs<float> &a, int64_t x)
{
    // step 1 in binary64 from the exactly widened metric; g^ij rounded once to binary32
    uint32_t rare = 0;
    const double g00 = widen<kIntConv>(v[IN_G + 0], rare), g01 = widen<kIntConv>(v[IN_G + 1], rare),
                 g02 = widen<kIntConv>(v[IN_G + 2], rare), g11 = widen<kIntConv>(v[IN_G + 3], rare),
                 g12 = widen<kIntConv>(v[IN_G + 4], rare), g22 = widen<kIntConv>(v[IN_G + 5], rare);
    double c[6];
    c[0] = fma(g11, g22, -(g12 * g12));
    c[1] = fma(g02, g12, -(g01 * g22));
    c[2] = fma(g01, g12, -(g02 * g11));
    c[3] = fma(g00, g22, -(g02 * g02));
    c[4] = fma(g01, g02, -(g00 * g12));
    c[5] = fma(g00, g11, -(g01 * g01));
    const double det = fma(g00, c[0], fma(g01, c[1], g02 * c[2]));
    const double rdet = rcp_f64(det);
    float h[6], gi[6];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        gi[p] = narrow<kIntConv>(c[p] * rdet, rare);
        h[p] = 0.5f * gi[p];
    }
    if (kIntConv && rare)
        return false;
#pragma unroll
    for (int p = 0; p < 6; ++p)
        st_stream(a.out[OUT_GINV + p] + x, gi[p]);

    // step 2: Eq. 6
    float dg[18];
#pragma unroll
    for (int s = 0; s < 18; ++s)
        dg[s] = v[IN_DG + s];
    float T[3][6];
    christoffel_bracket<float>(dg, T);
    float gam[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            gam[i][p] = fmaf(h[sym(i, 2)], T[2][p], fmaf(h[sym(i, 1)], T[1][p], h[sym(i, 0)] * T[0][p]));
            st_stream(a.out[OUT_GAMMA + 6 * i + p] + x, gam[i][p]);
        }

    // step 3: nabla_j beta_i = d_j beta_i - Gamma^k_ij beta_k
    const float b0 = v[IN_BETA + 0], b1 = v[IN_BETA + 1], b2 = v[IN_BETA + 2];
    float nb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int p = sym(i, j);
            nb[i][j] = fmaf(-gam[2][p], b2, fmaf(-gam[1][p], b1, fmaf(-gam[0][p], b0, v[IN_DBETA + 3 * i + j])));
            st_stream(a.out[OUT_DBCOV + 3 * i + j] + x, nb[i][j]);
        }

    // step 4: Eq. 5
    const float m2a = -2.0f * v[IN_ALPHA];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const int p = sym(i, j);
            const float s = (i == j) ? 2.0f * nb[i][i] : nb[i][j] + nb[j][i];
            st_stream(a.out[OUT_DTG + p] + x, fmaf(m2a, v[IN_K + p], s));
        }
    return true;
}

template <bool kIntConv>
__device__ __forceinline__ bool fwd_point_f32(const FwdArgs<float> &a, int64_t x)
{
    float v[N_IN];
#pragma unroll
    for (int s = 0; s < N_IN; ++s)
        v[s] = ld_stream(a.in[s] + x);
    asm volatile("" ::: "memory");   // every load is issued before any arithmetic
    return chain_f32<kIntConv>(v, a, x);
}

// The general-conversion evaluation of one point, out of line (rare operands only).
__device__ __noinline__ void fwd_point_f32_general(const FwdArgs<float> &a, int64_t x) { fwd_point_f32<false>(a, x); }

__global__ void __launch_bounds__(kFwdThreads) dtg_fwd_f32_kernel(const FwdArgs<float> a, int64_t n)
{
    const GridStride gs;
    for (int64_t x = gs.first; x < n; x += gs.step)
        if (!fwd_point_f32<true>(a, x))
            fwd_point_f32_general(a, x);
}

// ------------------------------------------------------------------- binary32 forward, staged inputs
// The binary32 form moves 328 bytes per point against 24 FP64 operations, so it is bound by how many
// loads are in flight rather than by arithmetic.  Here the 43 input streams of a tile of TILE points
// are brought into shared memory by the bulk-copy engine, STAGES tiles ahead of the threads that
// compute on them: one thread issues 43 copies of TILE * 4 contiguous bytes per tile, completion is
// counted in bytes on one mbarrier per stage, and the loads overlap the arithmetic of earlier tiles.
// 512 points x 2 stages (176 KB: one block, 16 warps per SM) measured best, 0.94 ms at N = 2^24
// against 1.00 ms for the plain kernel; 256 x 4 and 384 x 3 (8 and 12 warps) leave the binary64
// inverse latency-bound, and 640 x 2 or 768 x 2 (K and alpha then read directly) were slower, as were
// 256 x 2 at two blocks per SM (1.05 ms) and 128 x 3 at three (1.18 ms).
// Each block walks tiles blockIdx.x, + gridDim.x, ...
// One __syncthreads per tile (after the wait) certifies that every thread has finished the previous
// tile, whose stage is then refilled.  Requires 16-byte aligned input streams; the last n % TILE
// points are left to the plain kernel.
__device__ unsigned int g_wait_timeouts;   // waits that gave up (a bulk copy never completed)

constexpr uint32_t kWaitPolls = 1u << 20;
constexpr uint64_t kWaitNs = 500000000ull;   // 0.5 s: a stage normally lands within microseconds

// extra_tx: bytes announced beyond what is copied; 0 in use.  The test hook passes a nonzero value so
// that no stage ever completes and the bounded waits run out (the failure path, without any fault).
template <int TILE, int STAGES>
__global__ void __launch_bounds__(TILE) dtg_fwd_f32_staged_kernel(const FwdArgs<float> a, int64_t ntiles, uint32_t extra_tx)
{
    extern __shared__ __align__(128) float stage_buf[];   // [STAGES][N_IN][TILE]
    __shared__ __align__(8) uint64_t full[STAGES];
    const int tid = threadIdx.x;
    const int64_t count = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s)
            mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int64_t i) {   // thread 0: the block's tile i into stage i % STAGES
        const int s = (int)(i % STAGES);
        const int64_t t = (int64_t)blockIdx.x + i * gridDim.x;
        float *dst = stage_buf + (size_t)s * N_IN * TILE;
        mbar_arrive_expect_tx(&full[s], N_IN * TILE * (uint32_t)sizeof(float) + extra_tx);
#pragma unroll 1
        for (int k = 0; k < N_IN; ++k)
            bulk_copy_g2s(dst + k * TILE, a.in[k] + t * TILE, TILE * (uint32_t)sizeof(float), &full[s]);
    };
    if (tid == 0)
        for (int64_t i = 0; i < STAGES - 1 && i < count; ++i)
            issue(i);
    for (int64_t i = 0; i < count; ++i) {
        const int s = (int)(i % STAGES);
        const bool ok = mbar_wait(&full[s], (uint32_t)((i / STAGES) & 1), kWaitPolls, kWaitNs);
        if (__syncthreads_or(!ok)) {   // block-uniform: record, let issued copies land, leave
            if (tid == 0) {
                atomicAdd(&g_wait_timeouts, 1u);
                for (int64_t j = i; j < count && j < i + STAGES - 1; ++j)
                    mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1), kWaitPolls, kWaitNs);
            }
            return;
        }
        if (tid == 0 && i + STAGES - 1 < count)
            issue(i + STAGES - 1);
        const float *src = stage_buf + (size_t)s * N_IN * TILE + tid;
        float v[N_IN];
#pragma unroll
        for (int k = 0; k < N_IN; ++k)
            v[k] = src[k * TILE];
        const int64_t x = ((int64_t)blockIdx.x + i * gridDim.x) * TILE + tid;
        if (!chain_f32<true>(v, a, x))
            fwd_point_f32_general(a, x);
    }
}

template <int TILE, int STAGES>
static cudaError_t launch_f32_staged(const FwdArgs<float> &a, int64_t ntiles, int sms, cudaStream_t s,
                                     uint32_t extra_tx = 0)
{
    const size_t smem = (size_t)STAGES * N_IN * TILE * sizeof(float);
    auto kern = dtg_fwd_f32_staged_kernel<TILE, STAGES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int blocks = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, TILE, smem);
    if (e != cudaSuccess)
        return e;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sms * std::max(blocks, 1)));
    kern<<<grid, TILE, smem, s>>>(a, ntiles, extra_tx);
    return cudaGetLastError();
}

cudaError_t launch_fwd_f32_staged_stalled(const FwdArgs<float> &a, int64_t n, int sms, cudaStream_t s)
{
    return n / kF32StagedTile > 0 ? launch_f32_staged<kF32StagedTile, kF32StagedStages>(a, n / kF32StagedTile, sms, s, 16)
                                  : cudaSuccess;
}

cudaError_t read_wait_timeouts(unsigned int *count)
{
    return cudaMemcpyFromSymbol(count, g_wait_timeouts, sizeof(unsigned int));
}

// ------------------------------------------------------------------------------------ batched forward
template <int kThreads>
__global__ void __launch_bounds__(kThreads) dtg_batched_f64_kernel(const BatchView v)
{
    __shared__ FwdArgs<double> s_args;
    batched_loop<double>(v, s_args, [](const FwdArgs<double> &a, int64_t x) { fwd_point_f64(a, x); });
}

template <int kThreads>
__global__ void __launch_bounds__(kThreads) dtg_batched_f32_kernel(const BatchView v)
{
    __shared__ FwdArgs<float> s_args;
    batched_loop<float>(v, s_args, [](const FwdArgs<float> &a, int64_t x) {
        if (!fwd_point_f32<true>(a, x))
            fwd_point_f32_general(a, x);
    });
}

// ---------------------------------------------------------------- batched forward, staged inputs
// The batched loop with the 43 input rows of each tile brought into shared memory by bulk copies,
// STAGES tiles ahead of the threads that compute on them: the staging depth, which the tuner searches
// next to the block size and the blocks per SM (depth 0 is the register-loading kernel above).  A tile
// is THREADS points of one grid, one per thread.  Thread 0 also produces: it walks the CTA's run of
// tiles STAGES - 1 ahead of the others, keeping the input table of the grid it is in (and whether all
// 43 rows start on a 16-byte boundary) in shared memory, and for each tile copies the 16-byte-aligned
// prefix of each row, which is the whole tile unless the tile ends its grid at a byte length that is
// not a multiple of 16.  The points beyond that prefix, and every point of a grid whose rows are not
// 16-byte aligned, are loaded directly.  Completion is counted in bytes on one mbarrier per stage; a
// stage with nothing to copy completes on the producer's arrival alone.  The waits are bounded as in
// the single-grid staged kernel: a block whose wait gives up counts it (tl_wait_timeouts), lets the
// copies it issued land (bounded again) and returns.
template <typename T, int THREADS, int STAGES>
__global__ void __launch_bounds__(THREADS) dtg_batched_staged_kernel(const BatchView v)
{
    extern __shared__ __align__(128) unsigned char staged_smem[];
    T *const stage_buf = (T *)staged_smem;   // [STAGES][N_IN][THREADS]
    __shared__ __align__(8) uint64_t full[STAGES];
    __shared__ FwdArgs<T> s_args;            // consumers: table of the grid being computed
    __shared__ const T *p_in[N_IN];          // producer: input table of the grid being copied
    __shared__ int p_aligned;
    const int tid = threadIdx.x;
    const int64_t per = (v.total_tiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t_end = (t0 + per < v.total_tiles) ? t0 + per : v.total_tiles;
    if (t0 >= t_end)
        return;
    const int64_t count = t_end - t0;
    int lo = 0, hi = v.G;                    // grid of tile t0: last d with tile_prefix[d] <= t0
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (v.tile_prefix[mid] <= t0)
            lo = mid;
        else
            hi = mid;
    }
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s)
            mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    int pd = lo, p_loaded = -1;              // producer state (thread 0 only)
    auto issue = [&](int64_t i) {            // tile t0 + i into stage i % STAGES
        const int64_t t = t0 + i;
        while (pd < v.G && t >= v.tile_prefix[pd + 1])
            ++pd;
        const int s = (int)(i % STAGES);
        uint32_t row = 0;
        int64_t x0 = 0;
        if (pd < v.G) {
            if (pd != p_loaded) {
                int al = 1;
                for (int k = 0; k < N_IN; ++k) {
                    p_in[k] = (const T *)v.tables[(int64_t)pd * (N_IN + N_OUT) + k];
                    al &= ((uintptr_t)p_in[k] % 16 == 0) ? 1 : 0;
                }
                p_aligned = al;
                p_loaded = pd;
            }
            x0 = (t - v.tile_prefix[pd]) * THREADS;
            const int64_t m = (v.n[pd] - x0 < THREADS) ? v.n[pd] - x0 : THREADS;
            row = p_aligned ? (uint32_t)(m * (int64_t)sizeof(T)) & ~15u : 0u;
        }
        mbar_arrive_expect_tx(&full[s], N_IN * row + v.extra_tx);
        if (row) {
            T *dst = stage_buf + (size_t)s * N_IN * THREADS;
            for (int k = 0; k < N_IN; ++k)
                bulk_copy_g2s(dst + k * THREADS, p_in[k] + x0, row, &full[s]);
        }
    };
    if (tid == 0)
        for (int64_t i = 0; i < STAGES - 1 && i < count; ++i)
            issue(i);

    int d = lo, loaded = -1, aligned = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t t = t0 + i;
        while (d < v.G && t >= v.tile_prefix[d + 1])
            ++d;
        const int s = (int)(i % STAGES);
        const bool ok = mbar_wait(&full[s], (uint32_t)((i / STAGES) & 1), kWaitPolls, kWaitNs);
        // block-uniform; also certifies that every thread is done with tile i - 1 (its stage and table).
        // d >= G cannot happen for a consistent plan.  Either way the block leaves once the copies it
        // issued have landed.
        const bool bad_plan = d >= v.G;
        if (__syncthreads_or(!ok || bad_plan)) {
            if (tid == 0) {
                if (!ok)
                    atomicAdd(&g_wait_timeouts, 1u);
                else
                    atomicCAS(v.status, 0u, 6u);   // TL_ERR_PLAN_MISMATCH
                for (int64_t j = ok ? i + 1 : i; j < count && j < i + STAGES - 1; ++j)
                    mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1), kWaitPolls, kWaitNs);
            }
            return;
        }
        if (d != loaded) {
            bool al = true;
            if (tid < N_IN + N_OUT) {
                const void *q = v.tables[(int64_t)d * (N_IN + N_OUT) + tid];
                ((const void **)&s_args)[tid] = q;
                al = tid >= N_IN || (uintptr_t)q % 16 == 0;
            }
            aligned = __syncthreads_and(al);
            loaded = d;
        }
        if (tid == 0 && i + STAGES - 1 < count)
            issue(i + STAGES - 1);
        const int64_t x0 = (t - v.tile_prefix[d]) * THREADS;
        const int64_t m = (v.n[d] - x0 < THREADS) ? v.n[d] - x0 : THREADS;
        const int64_t staged = aligned ? (int64_t)(((uint32_t)(m * (int64_t)sizeof(T)) & ~15u) / sizeof(T)) : 0;
        if (tid < m) {
            const int64_t x = x0 + tid;
            T val[N_IN];
            if (tid < staged) {
                const T *src = stage_buf + (size_t)s * N_IN * THREADS + tid;
#pragma unroll
                for (int k = 0; k < N_IN; ++k)
                    val[k] = src[k * THREADS];
            } else {
#pragma unroll
                for (int k = 0; k < N_IN; ++k)
                    val[k] = ld_stream(s_args.in[k] + x);
            }
            if constexpr (sizeof(T) == 8) {
                chain_f64(val, s_args, x);
            } else {
                if (!chain_f32<true>(val, s_args, x))
                    fwd_point_f32_general(s_args, x);
            }
        }
    }
}

// Staging depths provided per element type and block size (shared memory per block <= 227 KB):
// binary64 128 x {2, 3}, 256 x 2; binary32 128 x {2, 3}, 256 x {2, 3}, 512 x 2.
template <typename T, int THREADS, int STAGES>
static cudaError_t staged_kernel_op(bool launch, const BatchView *v, int grid, cudaStream_t s, int *blocks)
{
    const size_t smem = (size_t)STAGES * N_IN * THREADS * sizeof(T);
    auto kern = dtg_batched_staged_kernel<T, THREADS, STAGES>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    if (!launch)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, THREADS, smem);
    kern<<<grid, THREADS, smem, s>>>(*v);
    return cudaGetLastError();
}

static cudaError_t staged_dispatch(int dtype, int threads, int stages, bool launch, const BatchView *v, int grid,
                                   cudaStream_t s, int *blocks)
{
    const int key = (dtype == 0 ? 0 : 1000) + threads * 10 + stages;
    switch (key) {
    case 1282: return staged_kernel_op<double, 128, 2>(launch, v, grid, s, blocks);
    case 1283: return staged_kernel_op<double, 128, 3>(launch, v, grid, s, blocks);
    case 2562: return staged_kernel_op<double, 256, 2>(launch, v, grid, s, blocks);
    case 2282: return staged_kernel_op<float, 128, 2>(launch, v, grid, s, blocks);
    case 2283: return staged_kernel_op<float, 128, 3>(launch, v, grid, s, blocks);
    case 3562: return staged_kernel_op<float, 256, 2>(launch, v, grid, s, blocks);
    case 3563: return staged_kernel_op<float, 256, 3>(launch, v, grid, s, blocks);
    case 6122: return staged_kernel_op<float, 512, 2>(launch, v, grid, s, blocks);
    }
    return cudaErrorNotSupported;
}

bool batched_staging_provided(int dtype, int threads, int stages)
{
    if (dtype != 0 && dtype != 1)
        return false;
    const int key = (dtype == 0 ? 0 : 1000) + threads * 10 + stages;
    return key == 1282 || key == 1283 || key == 2562 || key == 2282 || key == 2283 || key == 3562 || key == 3563 ||
           key == 6122;
}

cudaError_t launch_batched_staged(int dtype, const BatchView &v, int threads, int stages, int grid, cudaStream_t s)
{
    return staged_dispatch(dtype, threads, stages, true, &v, grid, s, nullptr);
}

cudaError_t occupancy_batched_staged(int dtype, int threads, int stages, int *blocks)
{
    *blocks = 0;
    return staged_dispatch(dtype, threads, stages, false, nullptr, 0, nullptr, blocks);
}

template <typename K> static cudaError_t launch_k(K k, const BatchView &v, int threads, int grid, cudaStream_t s)
{
    k<<<grid, threads, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_batched(int dtype, const BatchView &v, int threads, int grid, cudaStream_t s)
{
    if (dtype == 2)
        return launch_batched_ff(v, threads, grid, s);
    switch (threads) {
    case 128: return dtype == 0 ? launch_k(dtg_batched_f64_kernel<128>, v, 128, grid, s)
                                : launch_k(dtg_batched_f32_kernel<128>, v, 128, grid, s);
    case 256: return dtype == 0 ? launch_k(dtg_batched_f64_kernel<256>, v, 256, grid, s)
                                : launch_k(dtg_batched_f32_kernel<256>, v, 256, grid, s);
    case 512: return dtype == 0 ? launch_k(dtg_batched_f64_kernel<512>, v, 512, grid, s)
                                : launch_k(dtg_batched_f32_kernel<512>, v, 512, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t occupancy_batched(int dtype, int threads, int *blocks)
{
    if (dtype == 2)
        return occupancy_batched_ff(threads, blocks);
    switch (threads) {
    case 128: return dtype == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_f64_kernel<128>, 128, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_f32_kernel<128>, 128, 0);
    case 256: return dtype == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_f64_kernel<256>, 256, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_f32_kernel<256>, 256, 0);
    case 512: return dtype == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_f64_kernel<512>, 512, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dtg_batched_f32_kernel<512>, 512, 0);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------- launchers
cudaError_t launch_fwd_f64(const FwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s)
{
    if (sh.threads < kFwdF64Threads)   // the block was shrunk: a grid of less than one block per SM
        dtg_fwd_f64_small_kernel<<<sh.grid, sh.threads, 0, s>>>(a, n);
    else
        dtg_fwd_f64_kernel<<<sh.grid, sh.threads, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_fwd_f32(const FwdArgs<float> &a, int64_t n, LaunchShape sh, cudaStream_t s)
{
    dtg_fwd_f32_kernel<<<sh.grid, sh.threads, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_fwd_f32_staged(const FwdArgs<float> &a, int64_t n, int sms, LaunchShape tail, cudaStream_t s)
{
    constexpr int kTile = kF32StagedTile;
    bool aligned = true;
    for (int k = 0; k < N_IN; ++k)
        aligned = aligned && ((uintptr_t)a.in[k] % 16 == 0);
    const int64_t ntiles = aligned ? n / kTile : 0;
    cudaError_t e = cudaSuccess;
    if (ntiles > 0)
        e = launch_f32_staged<kTile, kF32StagedStages>(a, ntiles, sms, s);
    const int64_t done = ntiles * kTile;
    if (e != cudaSuccess || done == n)
        return e;
    FwdArgs<float> t = a;   // the remaining points: plain kernel on the shifted tables
    for (int k = 0; k < N_IN; ++k)
        t.in[k] += done;
    for (int k = 0; k < N_OUT; ++k)
        t.out[k] += done;
    // the tail is at most kF32StagedTile - 1 points, or the whole grid when the inputs are not aligned
    const int64_t m = n - done;
    if (ntiles > 0)
        tail = LaunchShape{(int)((m + kFwdThreads - 1) / kFwdThreads), kFwdThreads};
    return launch_fwd_f32(t, m, tail, s);
}

cudaError_t occupancy_fwd(int *f64, int *f32, int *ff)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(f64, dtg_fwd_f64_kernel, kFwdF64Threads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(f32, dtg_fwd_f32_kernel, kFwdThreads, 0);
    if (e == cudaSuccess)
        e = occupancy_fwd_ff(ff);
    return e;
}

}  // namespace tl
