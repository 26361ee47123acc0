// tl_kernels.h -- internal launchers (C++; not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "tl_common.cuh"

namespace tl {

constexpr int kFwdThreads = 256;
// The binary64 forward kernel (dtg_fwd_f64_kernel): threads per block and blocks per SM it is built for.
constexpr int kFwdF64Threads = 256, kFwdF64Blocks = 3;

// Grid and block size of a one-dimensional launch.
struct LaunchShape {
    int grid, threads;
};

constexpr int kBwdThreads = 128;
constexpr int kBwdFfThreads = 256;   // the float-float adjoint (one block per SM, see dtg_bwd.cu)

cudaError_t launch_fwd_f64(const FwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s);
cudaError_t launch_fwd_f32(const FwdArgs<float> &a, int64_t n, LaunchShape sh, cudaStream_t s);
// Binary32 forward with the inputs staged through shared memory by bulk copies (tiles of
// kF32StagedTile points, kF32StagedStages deep); falls back to launch_fwd_f32 (shape `tail`) for
// unaligned inputs and for the last n % kF32StagedTile points.
constexpr int kF32StagedTile = 512;
constexpr int kF32StagedStages = 2;
cudaError_t launch_fwd_f32_staged(const FwdArgs<float> &a, int64_t n, int sms, LaunchShape tail, cudaStream_t s);
// Test hook: the staged kernel over the full tiles of n points with 16 bytes announced per stage that
// never arrive, so every block's first wait runs out (about 1 s) and the block leaves without output.
cudaError_t launch_fwd_f32_staged_stalled(const FwdArgs<float> &a, int64_t n, int sms, cudaStream_t s);
// Number of bounded waits in the staged kernels that gave up since the library was loaded.
cudaError_t read_wait_timeouts(unsigned int *count);
cudaError_t launch_fwd_ff(const FwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s);
cudaError_t launch_bwd_f64(const BwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s);
cudaError_t launch_bwd_ff(const BwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s);
// Forward and adjoint of one functional in one pass (binary64).
constexpr int kFwdBwdThreads = 128;
constexpr int kFwdBwdFfThreads = 256;   // the float-float form (one block per SM)
cudaError_t launch_fwdbwd_f64(const FwdBwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s);
cudaError_t launch_fwdbwd_ff(const FwdBwdArgs<double> &a, int64_t n, LaunchShape sh, cudaStream_t s);
cudaError_t occupancy_fwdbwd(int *f64, int *ff);

struct BatchView;
// Batched forward: one persistent launch over all grids of a plan; `threads` in {128, 256, 512}.
cudaError_t launch_batched(int dtype, const BatchView &v, int threads, int grid, cudaStream_t s);
// Resident blocks per SM of the batched kernel for dtype and block size.
cudaError_t occupancy_batched(int dtype, int threads, int *blocks);
cudaError_t launch_batched_ff(const BatchView &v, int threads, int grid, cudaStream_t s);
// Batched forward with the inputs staged through shared memory `stages` tiles deep (tiles of `threads`
// points, one per thread: the plan's points-per-thread-1 tiling).  dtype 0 or 1; see
// batched_staging_provided for the (threads, stages) pairs built.
bool batched_staging_provided(int dtype, int threads, int stages);
cudaError_t launch_batched_staged(int dtype, const BatchView &v, int threads, int stages, int grid, cudaStream_t s);
cudaError_t occupancy_batched_staged(int dtype, int threads, int stages, int *blocks);
cudaError_t occupancy_batched_ff(int threads, int *blocks);

// Resident blocks per SM of each kernel (0 where a kernel is not provided).
cudaError_t occupancy_fwd(int *f64, int *f32, int *ff);
cudaError_t occupancy_bwd(int *f64, int *ff);
cudaError_t occupancy_fwd_ff(int *ff);

}  // namespace tl
