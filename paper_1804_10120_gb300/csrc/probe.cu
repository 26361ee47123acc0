// probe.cu -- issue-rate probe of the arithmetic pipes that bound the binary64 kernels (a test hook,
// tl_testing.h).  Each thread runs eight independent dependency chains of one operation for `iters`
// rounds, so the launch is throughput-bound on that operation's pipe once a few warps share an SM;
// the host times it and divides the operation count by the time.  The chains' results decide a
// store that never happens for the operands the host passes, so nothing can be removed.
// Ops 0-4 take their second and third operands straight from the parameter bank; ops 5-8 take them
// from registers, as the kernels' operations do (values the compiler cannot see: broadcast by a warp
// shuffle), and op 8 is an addition written as an FMA whose factor 1.0 is read from constant memory.
#include "tl_common.cuh"
#include "../../include/tl_testing.h"

namespace tl {

constexpr int kProbeChains = 8;

static __constant__ double c_probe_unit = 1.0;

template <int OP>
__global__ void __launch_bounds__(1024) pipe_rate_kernel(double *sink, int64_t iters, double a, double b)
{
    double v[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k)
        v[k] = 1.0 + 1e-3 * threadIdx.x + k;
    const float fa = (float)a;
    const double ra = __shfl_sync(0xffffffffu, a, 0), rb = __shfl_sync(0xffffffffu, b, 0);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) {
            if (OP == 0)
                v[k] = fma(v[k], a, b);                   // DFMA
            else if (OP == 1)
                v[k] = v[k] + b;                          // DADD
            else if (OP == 2)
                v[k] = v[k] * a;                          // DMUL
            else if (OP == 3) {                           // F2F.F32.F64, FMUL, F2F.F64.F32
                float f;
                asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(v[k]));
                f *= fa;
                asm volatile("cvt.f64.f32 %0, %1;" : "=d"(v[k]) : "f"(f));
            } else if (OP == 4) {
                asm volatile("fma.rn.f64 %0, %1, 0d3FF0000000000000, %2;" : "=d"(v[k]) : "d"(v[k]), "d"(b));   // v*1 + b
            } else if (OP == 5) {
                v[k] = fma(v[k], ra, rb);                 // DFMA, register operands
            } else if (OP == 6) {
                v[k] = v[k] + rb;                         // DADD, register operands
            } else if (OP == 7) {
                v[k] = v[k] * ra;                         // DMUL, register operands
            } else {
                v[k] = fma(v[k], c_probe_unit, rb);       // v*1 + b, the 1.0 from constant memory
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k)
        s += v[k];
    if (s == b * 1e300)   // false for the probe's operands (b = 0)
        sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace tl

extern "C" TL_API tl_status tl_testing_pipe_rate(int op, int64_t iters, int32_t blocks, int32_t threads, double *sink,
                                                 tl_stream stream)
{
    if (op < 0 || op > 8 || iters < 0 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || !sink)
        return TL_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    // a = 1 keeps every chain finite and exact (b = 0 for the additions); the pipe cost is the same
    switch (op) {
    case 0: tl::pipe_rate_kernel<0><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    case 1: tl::pipe_rate_kernel<1><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    case 2: tl::pipe_rate_kernel<2><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    case 3: tl::pipe_rate_kernel<3><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    case 4: tl::pipe_rate_kernel<4><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    case 5: tl::pipe_rate_kernel<5><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    case 6: tl::pipe_rate_kernel<6><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    case 7: tl::pipe_rate_kernel<7><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    default: tl::pipe_rate_kernel<8><<<blocks, threads, 0, s>>>(sink, iters, 1.0, 0.0); break;
    }
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}

extern "C" TL_API tl_status tl_testing_memory_info(int32_t device, int32_t *clock_khz, int32_t *bus_bits)
{
    if (!clock_khz || !bus_bits)
        return TL_ERR_INVALID_ARG;
    int c = 0, b = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMemoryClockRate, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b, cudaDevAttrGlobalMemoryBusWidth, device) != cudaSuccess) {
        (void)cudaGetLastError();
        return TL_ERR_CUDA;
    }
    *clock_khz = c;
    *bus_bits = b;
    return TL_OK;
}
