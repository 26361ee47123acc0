// dtg_batched.cuh -- persistent multi-grid loop shared by the batched forward kernels.
//
// Many subgrids of uneven size (the paper's multi-domain grids, Sec. 1) run in ONE launch.  The plan
// cuts every grid into tiles of blockDim.x x ppt points (ppt points per thread, strided by blockDim.x)
// and lays the tiles of all grids end to end; CTA c takes a contiguous run of about
// total_tiles / gridDim.x tiles, so it crosses few grid boundaries.
// The component pointer tables of all grids live in device memory (uploaded once by the plan, like the
// paper's cached GPUPointers, Sec. 4); a CTA copies the table of its current grid into shared memory
// only when it crosses into a new grid, and the per-point bodies read their pointers from there.
#pragma once
#include "tl_common.cuh"

namespace tl {

// Device-side view of a batch plan, passed by value.
struct BatchView {
    const void *const *tables;     // G x 82 device pointers: 43 inputs then 39 outputs per grid
    const int64_t *n;              // G grid sizes
    const int64_t *tile_prefix;    // G + 1 running tile counts for this block size
    int64_t total_tiles;
    int32_t G;
    int32_t ppt;                   // points per thread in a tile (the tile holds blockDim.x x ppt points)
    uint32_t *status;              // 0 = fine; a TL_ERR_* code if the plan looked inconsistent
    uint32_t extra_tx;             // staged kernels: bytes announced per stage beyond the copies; 0 in use
                                   // (a test hook sets it so that no stage completes)
};

template <typename T, typename Body>
__device__ __forceinline__ void batched_loop(const BatchView &v, FwdArgs<T> &s_args, Body body)
{
    const int64_t per = (v.total_tiles + gridDim.x - 1) / gridDim.x;
    int64_t t = (int64_t)blockIdx.x * per;
    const int64_t t_end = (t + per < v.total_tiles) ? t + per : v.total_tiles;
    if (t >= t_end)
        return;
    // grid holding tile t: last d with tile_prefix[d] <= t (binary search, identical in every thread)
    int lo = 0, hi = v.G;                       // invariant: prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (v.tile_prefix[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    int d = lo, loaded = -1;
    for (; t < t_end; ++t) {
        while (d < v.G && t >= v.tile_prefix[d + 1])
            ++d;
        if (d >= v.G) {                         // cannot happen for a consistent plan
            if (threadIdx.x == 0)
                atomicCAS(v.status, 0u, 6u);    // TL_ERR_PLAN_MISMATCH
            return;
        }
        if (d != loaded) {
            __syncthreads();                    // everyone is done with the previous grid's table
            if (threadIdx.x < N_IN + N_OUT)
                ((const void **)&s_args)[threadIdx.x] = v.tables[(int64_t)d * (N_IN + N_OUT) + threadIdx.x];
            __syncthreads();
            loaded = d;
        }
        const int64_t x0 = (t - v.tile_prefix[d]) * ((int64_t)blockDim.x * v.ppt) + threadIdx.x;
#pragma unroll 1
        for (int k = 0; k < v.ppt; ++k) {
            const int64_t x = x0 + (int64_t)k * blockDim.x;
            if (x < v.n[d])
                body(s_args, x);
        }
    }
}

}  // namespace tl
