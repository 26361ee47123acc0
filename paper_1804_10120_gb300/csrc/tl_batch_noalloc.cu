// tl_batch_noalloc.cu -- the batched forward without any allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: code that runs inside a caching allocator or a
// fixed memory budget that owns all device memory, loops that cannot afford cudaMalloc's implicit
// device synchronisation, or plug-ins that are handed only their input and output buffers.  For them,
// tl_dtg_batched_noalloc runs the same persistent batched kernel as tl_dtg_batched, but keeps the
// kernel's scratch -- the per-grid pointer tables, grid sizes, tile prefix sums and the status word,
// which a batch plan would allocate -- in one file-scope device array of fixed size, kNoAllocBytes,
// which every GPU that loads this library holds until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "dtg_batched.cuh"
#include "tl_host.h"
#include "tl_kernels.h"

namespace tl {
namespace {

constexpr int kNoAllocMaxGrids = 1024;
constexpr int kNoAllocThreads = 256;
constexpr size_t kTablesBytes = (size_t)kNoAllocMaxGrids * (N_IN + N_OUT) * sizeof(void *);
constexpr size_t kNBytes = (size_t)kNoAllocMaxGrids * sizeof(int64_t);
constexpr size_t kPrefixBytes = (size_t)(kNoAllocMaxGrids + 1) * sizeof(int64_t);
constexpr size_t kStatusOffset = kTablesBytes + kNBytes + kPrefixBytes;
constexpr size_t kNoAllocBytes = kStatusOffset + 256;   // 688,392 bytes

// The scratch.  In host code this name is only a stand-in for the device array; the device address is
// obtained with cudaGetSymbolAddress (once per device, below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int sms = 0;
    int blocks[3] = {0, 0, 0};          // resident blocks per SM at 256 threads, by dtype
};
NoAllocDevice g_na[kMaxDevices];
std::mutex g_na_mu;   // guards the per-device set-up and the host staging image below

// Host image of the scratch, staged here (static storage: nothing is allocated per call).
unsigned char g_host_image[kStatusOffset];
Range g_ranges[(size_t)kNoAllocMaxGrids * (N_IN + N_OUT)];

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" TL_API tl_status tl_dtg_batched_noalloc(const tl_dtg_in *in, const tl_dtg_out *out, const int64_t *n,
                                                   int32_t G, tl_dtype dtype, tl_stream stream)
{
    if (G < 0 || (G > 0 && (!in || !out || !n)))
        return fail(TL_ERR_INVALID_ARG, "G = %d with NULL in/out/n", (int)G);
    if (G > kNoAllocMaxGrids)
        return fail(TL_ERR_INVALID_ARG, "G = %d exceeds the allocation-free maximum of %d grids", (int)G,
                    kNoAllocMaxGrids);
    if (!dtype_ok(dtype))
        return fail(TL_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    // The tables travel through a static host image that the next call overwrites, so a copy recorded
    // into a graph would replay the wrong grids' tables: refuse during stream capture, before anything
    // (including the one-time set-up) touches the stream or the device.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(TL_ERR_UNSUPPORTED, "tl_dtg_batched_noalloc cannot be called while its stream is being captured");
    const DeviceInfo *di = nullptr;
    tl_status s = device_info(&di);
    if (s != TL_OK)
        return s;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");

    std::lock_guard<std::mutex> lk(g_na_mu);
    NoAllocDevice &D = g_na[dev];
    if (!D.ready) {   // once per device, with that device current
        void *ptr = nullptr;
        if ((e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch)) != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress (allocation-free scratch)");
        for (int t = 0; t < 3; ++t)
            if ((e = occupancy_batched(t, kNoAllocThreads, &D.blocks[t])) != cudaSuccess)
                return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        D.scratch = (unsigned char *)ptr;
        D.sms = di->sms;
        D.ready = true;
    }

    // validation, in static storage
    const size_t esz = elem_size(dtype);
    size_t nr = 0;
    int64_t tiles = 0;
    void **tables = (void **)g_host_image;
    int64_t *hn = (int64_t *)(g_host_image + kTablesBytes);
    int64_t *hp = (int64_t *)(g_host_image + kTablesBytes + kNBytes);
    for (int32_t d = 0; d < G; ++d) {
        if (n[d] < 0)
            return fail(TL_ERR_INVALID_ARG, "n[%d] = %lld < 0", (int)d, (long long)n[d]);
        const void *const *ip = (const void *const *)&in[d];
        void *const *op = (void *const *)&out[d];
        for (int q = 0; q < N_IN + N_OUT; ++q) {
            const void *p = q < N_IN ? ip[q] : op[q - N_IN];
            if (!p)
                return fail(TL_ERR_INVALID_ARG, "grid %d: %s[%d] is NULL", (int)d, q < N_IN ? "in" : "out",
                            q < N_IN ? q : q - N_IN);
            if ((uintptr_t)p % esz)
                return fail(TL_ERR_ALIGNMENT, "grid %d: array %d is not %zu-byte aligned", (int)d, q, esz);
            if (n[d] > 0)
                g_ranges[nr++] = {(uintptr_t)p, (uintptr_t)p + (uintptr_t)n[d] * esz, q >= N_IN,
                                  q < N_IN ? "in" : "out", q < N_IN ? q : q - N_IN, (int)d};
            tables[(size_t)d * (N_IN + N_OUT) + q] = (void *)p;
        }
        hn[d] = n[d];
        hp[d] = tiles;
        tiles += (n[d] + kNoAllocThreads - 1) / kNoAllocThreads;
    }
    hp[G] = tiles;
    std::sort(g_ranges, g_ranges + nr, [](const Range &a, const Range &b) { return a.lo < b.lo; });
    size_t open_any = SIZE_MAX, open_w = SIZE_MAX;
    for (size_t i = 0; i < nr; ++i) {
        const Range &r = g_ranges[i];
        if ((r.write && open_any != SIZE_MAX && g_ranges[open_any].hi > r.lo) ||
            (open_w != SIZE_MAX && g_ranges[open_w].hi > r.lo))
            return fail(TL_ERR_INVALID_ARG, "grid %d: %s[%d] overlaps another array: outputs must not alias", r.grid,
                        r.name, r.index);
        if (open_any == SIZE_MAX || r.hi > g_ranges[open_any].hi)
            open_any = i;
        if (r.write && (open_w == SIZE_MAX || r.hi > g_ranges[open_w].hi))
            open_w = i;
    }
    if (tiles == 0)
        return TL_OK;

    // upload the tables, sizes and prefix sums into the scratch (from pageable static memory: the copy
    // has consumed the host image when cudaMemcpyAsync returns), and clear the status word
    const cudaStream_t st = (cudaStream_t)stream;
    unsigned char *dsc = D.scratch;
    if ((e = cudaMemcpyAsync(dsc, tables, (size_t)G * (N_IN + N_OUT) * sizeof(void *), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dsc + kTablesBytes, hn, (size_t)G * sizeof(int64_t), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(dsc + kTablesBytes + kNBytes, hp, (size_t)(G + 1) * sizeof(int64_t),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(dsc + kStatusOffset, 0, sizeof(uint32_t), st)) != cudaSuccess)
        return cuda_fail(e, "staging the allocation-free scratch");
    BatchView v;
    v.tables = (const void *const *)dsc;
    v.n = (const int64_t *)(dsc + kTablesBytes);
    v.tile_prefix = (const int64_t *)(dsc + kTablesBytes + kNBytes);
    v.total_tiles = tiles;
    v.ppt = 1;
    v.G = G;
    v.status = (uint32_t *)(dsc + kStatusOffset);
    v.extra_tx = 0;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)D.sms * D.blocks[dtype], tiles));
    if ((e = launch_batched((int)dtype, v, kNoAllocThreads, grid, st)) != cudaSuccess)
        return cuda_fail(e, "allocation-free batched launch");
    return TL_OK;
}
