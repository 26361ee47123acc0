// dtg_bwd.cu -- adjoint of the fused chain.
#include "tl_common.cuh"
#include "tl_kernels.h"

namespace tl {

cudaError_t launch_bwd_f64(const BwdArgs<double> &, int64_t, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_bwd_ff(const BwdArgs<double> &, int64_t, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t occupancy_bwd(int *f64, int *ff)
{
    *f64 = 0;
    *ff = 0;
    return cudaSuccess;
}

}  // namespace tl
