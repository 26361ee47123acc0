// dtg_fwd_ff.cu -- forward chain with float-float contractions (TL_F64_FF).
#include "tl_common.cuh"
#include "tl_kernels.h"

namespace tl {

cudaError_t launch_fwd_ff(const FwdArgs<double> &, int64_t, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t occupancy_fwd_ff(int *ff)
{
    *ff = 0;
    return cudaSuccess;
}

}  // namespace tl
