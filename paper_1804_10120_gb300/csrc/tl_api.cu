// tl_api.cu -- the C ABI: argument validation, launch configuration, host-buffer pipeline, errors.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tl.h"
#include "tl_host.h"
#include "../../include/tl_testing.h"
#include "tl_kernels.h"

namespace tl {

thread_local std::string g_last_error;

tl_status fail(tl_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

tl_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(TL_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---- per-device facts, queried once ------------------------------------------------------------------
DeviceInfo g_dev[kMaxDevices];
std::mutex g_dev_mu;

tl_status device_info(const DeviceInfo **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(TL_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceInfo &d = g_dev[dev];
    if (!d.ready) {
        int major = 0, minor = 0;
        if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        d.supported = (major == 10 && minor == 3);
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
            strncpy(d.name, prop.name, sizeof d.name - 1);
            for (char *c = d.name; *c; ++c)
                if (*c == ' ' || *c == '|')
                    *c = '_';
        }
        if (d.supported) {
            e = occupancy_fwd(&d.fwd_f64_blocks, &d.fwd_f32_blocks, &d.fwd_ff_blocks);
            if (e == cudaSuccess)
                e = occupancy_bwd(&d.bwd_f64_blocks, &d.bwd_ff_blocks);
            if (e == cudaSuccess)
                e = occupancy_fwdbwd(&d.fwdbwd_f64_blocks, &d.fwdbwd_ff_blocks);
            if (e != cudaSuccess)
                return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        }
        d.ready = true;
    }
    if (!d.supported)
        return fail(TL_ERR_UNSUPPORTED, "device %d is not sm_103 (the library is built for sm_103a only)", dev);
    *out = &d;
    return TL_OK;
}

// Launch shape of the one-point-per-thread kernels (grid-stride or block-strided loops over n points).
// A grid of at least one full wave (every SM holding blocks_per_sm blocks of max_threads) gets that
// wave and loops.  A smaller grid would leave SMs idle with full-size blocks (N = 4096 in 256-thread
// blocks occupies 16 of 152 SMs), so the block shrinks, in whole warps, to about n / sms threads: the
// points spread over all SMs and each SM's share of the FP64-bound work drops by the same factor.
LaunchShape shape_for(int64_t n, int max_threads, int sms, int blocks_per_sm)
{
    const int64_t wave = (int64_t)sms * std::max(1, blocks_per_sm) * max_threads;
    if (n >= wave)
        return LaunchShape{(int)(wave / max_threads), max_threads};
    int64_t t = (n + sms - 1) / std::max(1, sms);
    t = std::min<int64_t>(max_threads, std::max<int64_t>(32, (t + 31) / 32 * 32));
    return LaunchShape{(int)std::max<int64_t>(1, (n + t - 1) / t), (int)t};
}

// ---- argument checks ---------------------------------------------------------------------------------
size_t elem_size(tl_dtype t) { return t == TL_F32 ? 4 : 8; }
bool dtype_ok(int t) { return t == TL_F64 || t == TL_F32 || t == TL_F64_FF; }

// Collect the ranges of a set of tables: all pointers non-null (unless nullable) and element-aligned.
tl_status collect_ranges(std::vector<Range> &rs, const void *const *tabs[], const int counts[], const bool writes[],
                         const bool nullable[], const char *const names[], int ntabs, int64_t n, size_t esz, int grid)
{
    for (int t = 0; t < ntabs; ++t)
        for (int s = 0; s < counts[t]; ++s) {
            const void *p = tabs[t][s];
            if (!p) {
                if (nullable[t])
                    continue;
                return grid < 0 ? fail(TL_ERR_INVALID_ARG, "%s[%d] is NULL", names[t], s)
                                : fail(TL_ERR_INVALID_ARG, "grid %d: %s[%d] is NULL", grid, names[t], s);
            }
            if ((uintptr_t)p % esz)
                return fail(TL_ERR_ALIGNMENT, "%s[%d]=%p is not %zu-byte aligned", names[t], s, p, esz);
            if (n > 0)
                rs.push_back({(uintptr_t)p, (uintptr_t)p + (uintptr_t)n * esz, writes[t], names[t], s, grid});
        }
    return TL_OK;
}

// No written range may intersect any other range (read/read overlap is allowed).
tl_status check_overlaps(std::vector<Range> &rs)
{
    std::sort(rs.begin(), rs.end(), [](const Range &a, const Range &b) { return a.lo < b.lo; });
    // sweep with the furthest-reaching written and any range seen so far
    size_t open_any = SIZE_MAX, open_w = SIZE_MAX;
    for (size_t i = 0; i < rs.size(); ++i) {
        const Range &r = rs[i];
        const Range *hit = nullptr;
        if (r.write && open_any != SIZE_MAX && rs[open_any].hi > r.lo)
            hit = &rs[open_any];
        else if (open_w != SIZE_MAX && rs[open_w].hi > r.lo)
            hit = &rs[open_w];
        if (hit)
            return fail(TL_ERR_INVALID_ARG, "%s[%d] (grid %d) overlaps %s[%d] (grid %d): outputs must not alias",
                        hit->name, hit->index, hit->grid, r.name, r.index, r.grid);
        if (open_any == SIZE_MAX || r.hi > rs[open_any].hi)
            open_any = i;
        if (r.write && (open_w == SIZE_MAX || r.hi > rs[open_w].hi))
            open_w = i;
    }
    return TL_OK;
}

tl_status check_tables(const void *const *tabs[], const int counts[], const bool writes[], const bool nullable[],
                       const char *const names[], int ntabs, int64_t n, size_t esz)
{
    std::vector<Range> rs;
    rs.reserve(128);
    tl_status s = collect_ranges(rs, tabs, counts, writes, nullable, names, ntabs, n, esz, -1);
    return s != TL_OK ? s : check_overlaps(rs);
}

template <typename T> FwdArgs<T> fwd_args(const tl_dtg_in *in, const tl_dtg_out *out)
{
    FwdArgs<T> a;
    const void *const *ip = (const void *const *)in;
    void *const *op = (void *const *)out;
    for (int s = 0; s < N_IN; ++s)
        a.in[s] = (const T *)ip[s];
    for (int s = 0; s < N_OUT; ++s)
        a.out[s] = (T *)op[s];
    return a;
}

static_assert(sizeof(tl_dtg_in) == N_IN * sizeof(void *), "tl_dtg_in must be 43 packed pointers");
static_assert(sizeof(tl_dtg_out) == N_OUT * sizeof(void *), "tl_dtg_out must be 39 packed pointers");
static_assert(sizeof(tl_dtg_gout) == N_OUT * sizeof(void *), "tl_dtg_gout must be 39 packed pointers");
static_assert(sizeof(tl_dtg_gin) == N_IN * sizeof(void *), "tl_dtg_gin must be 43 packed pointers");

tl_status launch_forward(const DeviceInfo &d, const tl_dtg_in *in, const tl_dtg_out *out, int64_t n,
                         tl_dtype dtype, cudaStream_t st)
{
    cudaError_t e;
    switch (dtype) {
    case TL_F64:
        e = launch_fwd_f64(fwd_args<double>(in, out), n, shape_for(n, kFwdF64Threads, d.sms, d.fwd_f64_blocks), st);
        break;
    case TL_F32:
        e = launch_fwd_f32_staged(fwd_args<float>(in, out), n, d.sms, shape_for(n, kFwdThreads, d.sms, d.fwd_f32_blocks),
                                  st);
        break;
    case TL_F64_FF:
        e = launch_fwd_ff(fwd_args<double>(in, out), n, shape_for(n, kFwdThreads, d.sms, d.fwd_ff_blocks), st);
        break;
    default:
        return fail(TL_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    }
    if (e == cudaErrorNotSupported)
        return fail(TL_ERR_UNSUPPORTED, "dtype %d has no forward kernel in this build", (int)dtype);
    if (e != cudaSuccess)
        return cuda_fail(e, "forward launch");
    return TL_OK;
}

tl_status check_forward(const tl_dtg_in *in, const tl_dtg_out *out, int64_t n, tl_dtype dtype)
{
    if (!in || !out)
        return fail(TL_ERR_INVALID_ARG, "NULL table");
    if (n < 0)
        return fail(TL_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (!dtype_ok(dtype))
        return fail(TL_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    const void *const *tabs[2] = {(const void *const *)in, (const void *const *)out};
    const int counts[2] = {N_IN, N_OUT};
    const bool writes[2] = {false, true}, nullable[2] = {false, false};
    const char *const names[2] = {"in", "out"};
    return check_tables(tabs, counts, writes, nullable, names, 2, n, elem_size(dtype));
}

// ---- host-buffer pipeline ----------------------------------------------------------------------------
// Chunks of kHostChunk points flow through three streams -- host->device copies, kernel, device->host
// copies -- over kHostSlots workspace slots, so that both copy directions and the kernel overlap.
constexpr int64_t kHostChunk = int64_t(1) << 19;   // points per pipeline chunk
constexpr int kHostSlots = 3;

struct HostPipe {
    std::mutex mu;
    bool ready = false;
    cudaStream_t h2d = nullptr, cmp = nullptr, d2h = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t in_ready[kHostSlots] = {}, done[kHostSlots] = {}, slot_free[kHostSlots] = {};
};
HostPipe g_pipes[kMaxDevices];
std::mutex g_pipes_mu;

tl_status host_pipe(HostPipe **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_pipes_mu);
    HostPipe &P = g_pipes[dev];
    if (!P.ready) {
        cudaStream_t *ss[3] = {&P.h2d, &P.cmp, &P.d2h};
        for (cudaStream_t *sp : ss)
            if ((e = cudaStreamCreateWithFlags(sp, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreateWithFlags");
        cudaEvent_t *es[2 + 3 * kHostSlots];
        int k = 0;
        es[k++] = &P.fork;
        es[k++] = &P.join;
        for (int i = 0; i < kHostSlots; ++i) {
            es[k++] = &P.in_ready[i];
            es[k++] = &P.done[i];
            es[k++] = &P.slot_free[i];
        }
        for (int i = 0; i < k; ++i)
            if ((e = cudaEventCreateWithFlags(es[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreateWithFlags");
        P.ready = true;
    }
    *out = &P;
    return TL_OK;
}

// The byte stride between consecutive arrays of a table if it is uniform (a [count, n] array), else 0.
size_t uniform_stride(const char *const *p, int count, size_t row_bytes)
{
    const intptr_t st = (intptr_t)(p[1] - p[0]);
    if (st < (intptr_t)row_bytes)
        return 0;
    for (int q = 2; q < count; ++q)
        if ((intptr_t)(p[q] - p[q - 1]) != st)
            return 0;
    return (size_t)st;
}

// Copies of m points of a table between host arrays (offset x0) and a slot's contiguous rows.  With a
// uniform host stride the rows move as one 2-D copy; equally spaced arrays may still be separate
// allocations, which the runtime rejects for a 2-D copy (invalid value): then *hstride is cleared and
// the rows are copied one by one from here on.
cudaError_t copy_table(char *const *host, int count, int64_t x0, int64_t m, char *slot, int64_t chunk, size_t esz,
                       size_t *hstride, bool to_device, cudaStream_t st)
{
    const cudaMemcpyKind kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    if (*hstride) {
        char *h = host[0] + x0 * esz;
        const cudaError_t e = to_device ? cudaMemcpy2DAsync(slot, chunk * esz, h, *hstride, m * esz, count, kind, st)
                                        : cudaMemcpy2DAsync(h, *hstride, slot, chunk * esz, m * esz, count, kind, st);
        if (e != cudaErrorInvalidValue)
            return e;
        (void)cudaGetLastError();   // not sticky; fall back to one copy per array
        *hstride = 0;
    }
    for (int q = 0; q < count; ++q) {
        char *h = host[q] + x0 * esz, *d = slot + (size_t)q * chunk * esz;
        const cudaError_t e = to_device ? cudaMemcpyAsync(d, h, m * esz, kind, st) : cudaMemcpyAsync(h, d, m * esz, kind, st);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace tl

using namespace tl;

extern "C" {

const char *tl_status_string(tl_status s)
{
    switch (s) {
    case TL_OK: return "TL_OK";
    case TL_ERR_INVALID_ARG: return "TL_ERR_INVALID_ARG";
    case TL_ERR_ALIGNMENT: return "TL_ERR_ALIGNMENT";
    case TL_ERR_UNSUPPORTED: return "TL_ERR_UNSUPPORTED";
    case TL_ERR_CUDA: return "TL_ERR_CUDA";
    case TL_ERR_TIMEOUT: return "TL_ERR_TIMEOUT";
    case TL_ERR_PLAN_MISMATCH: return "TL_ERR_PLAN_MISMATCH";
    }
    return "TL_ERR_UNKNOWN";
}

const char *tl_last_error(void) { return g_last_error.c_str(); }

int tl_version(void) { return 10000; }

tl_status tl_wait_timeouts(uint32_t *count)
{
    if (!count)
        return fail(TL_ERR_INVALID_ARG, "NULL count");
    const DeviceInfo *d = nullptr;
    tl_status s = device_info(&d);
    if (s != TL_OK)
        return s;
    unsigned int c = 0;
    cudaError_t e = read_wait_timeouts(&c);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the wait-timeout counter");
    *count = c;
    return TL_OK;
}

tl_status tl_dtg_forward(const tl_dtg_in *in, const tl_dtg_out *out, int64_t n, tl_dtype dtype, tl_stream stream)
{
    tl_status s = check_forward(in, out, n, dtype);
    if (s != TL_OK || n == 0)
        return s;
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    return launch_forward(*d, in, out, n, dtype, (cudaStream_t)stream);
}

tl_status tl_testing_f32_staged_stall(const tl_dtg_in *in, const tl_dtg_out *out, int64_t n, tl_stream stream)
{
    tl_status s = check_forward(in, out, n, TL_F32);
    if (s != TL_OK || n == 0)
        return s;
    for (int k = 0; k < N_IN; ++k)
        if ((uintptr_t)((const void *const *)in)[k] % 16 != 0)
            return fail(TL_ERR_ALIGNMENT, "the staged kernel needs 16-byte aligned inputs");
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    const cudaError_t e = launch_fwd_f32_staged_stalled(fwd_args<float>(in, out), n, d->sms, (cudaStream_t)stream);
    return e == cudaSuccess ? TL_OK : cuda_fail(e, "staged kernel launch");
}

tl_status tl_dtg_backward(const tl_dtg_in *in, const tl_dtg_gout *gout, const tl_dtg_gin *gin, int64_t n,
                          tl_dtype dtype, tl_stream stream)
{
    if (!in || !gout || !gin)
        return fail(TL_ERR_INVALID_ARG, "NULL table");
    if (n < 0)
        return fail(TL_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (!dtype_ok(dtype))
        return fail(TL_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (dtype == TL_F32)
        return fail(TL_ERR_UNSUPPORTED, "the adjoint is provided for TL_F64 and TL_F64_FF");
    const void *const *tabs[3] = {(const void *const *)in, (const void *const *)gout, (const void *const *)gin};
    const int counts[3] = {N_IN, N_OUT, N_IN};
    const bool writes[3] = {false, false, true}, nullable[3] = {false, true, false};
    const char *const names[3] = {"in", "gout", "gin"};
    tl_status s = check_tables(tabs, counts, writes, nullable, names, 3, n, elem_size(dtype));
    if (s != TL_OK || n == 0)
        return s;
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    BwdArgs<double> a;
    for (int q = 0; q < N_IN; ++q) {
        a.in[q] = (const double *)((const void *const *)in)[q];
        a.gin[q] = (double *)((void *const *)gin)[q];
    }
    for (int q = 0; q < N_OUT; ++q)
        a.gout[q] = (const double *)((const void *const *)gout)[q];
    cudaError_t e = (dtype == TL_F64)
                        ? launch_bwd_f64(a, n, shape_for(n, kBwdThreads, d->sms, d->bwd_f64_blocks), (cudaStream_t)stream)
                        : launch_bwd_ff(a, n, shape_for(n, kBwdFfThreads, d->sms, d->bwd_ff_blocks), (cudaStream_t)stream);
    if (e == cudaErrorNotSupported)
        return fail(TL_ERR_UNSUPPORTED, "dtype %d has no adjoint kernel in this build", (int)dtype);
    if (e != cudaSuccess)
        return cuda_fail(e, "backward launch");
    return TL_OK;
}

tl_status tl_dtg_forward_backward(const tl_dtg_in *in, const tl_dtg_out *out, const tl_dtg_gout *gout,
                                  const tl_dtg_gin *gin, int64_t n, tl_dtype dtype, tl_stream stream)
{
    if (!in || !out || !gout || !gin)
        return fail(TL_ERR_INVALID_ARG, "NULL table");
    if (n < 0)
        return fail(TL_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (!dtype_ok(dtype))
        return fail(TL_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (dtype == TL_F32)
        return fail(TL_ERR_UNSUPPORTED, "the fused forward + adjoint is provided for TL_F64 and TL_F64_FF");
    const void *const *tabs[4] = {(const void *const *)in, (const void *const *)out, (const void *const *)gout,
                                  (const void *const *)gin};
    const int counts[4] = {N_IN, N_OUT, N_OUT, N_IN};
    const bool writes[4] = {false, true, false, true}, nullable[4] = {false, false, true, false};
    const char *const names[4] = {"in", "out", "gout", "gin"};
    tl_status s = check_tables(tabs, counts, writes, nullable, names, 4, n, elem_size(dtype));
    if (s != TL_OK || n == 0)
        return s;
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    FwdBwdArgs<double> a;
    for (int q = 0; q < N_IN; ++q) {
        a.in[q] = (const double *)((const void *const *)in)[q];
        a.gin[q] = (double *)((void *const *)gin)[q];
    }
    for (int q = 0; q < N_OUT; ++q) {
        a.out[q] = (double *)((void *const *)out)[q];
        a.gout[q] = (const double *)((const void *const *)gout)[q];
    }
    const cudaError_t e =
        dtype == TL_F64 ? launch_fwdbwd_f64(a, n, shape_for(n, kFwdBwdThreads, d->sms, d->fwdbwd_f64_blocks), (cudaStream_t)stream)
                        : launch_fwdbwd_ff(a, n, shape_for(n, kFwdBwdFfThreads, d->sms, d->fwdbwd_ff_blocks), (cudaStream_t)stream);
    return e == cudaSuccess ? TL_OK : cuda_fail(e, "forward + adjoint launch");
}

size_t tl_dtg_host_workspace_bytes(int64_t n, tl_dtype dtype)
{
    if (n <= 0 || !dtype_ok(dtype))
        return 0;
    const int64_t chunk = std::min<int64_t>(n, kHostChunk);
    const int64_t slots = std::min<int64_t>(kHostSlots, (n + chunk - 1) / chunk);
    return (size_t)(slots * (N_IN + N_OUT) * chunk) * elem_size(dtype);
}

tl_status tl_dtg_forward_host(const tl_dtg_in *in, const tl_dtg_out *out, int64_t n, tl_dtype dtype,
                              void *workspace, size_t workspace_bytes, tl_stream stream)
{
    tl_status s = check_forward(in, out, n, dtype);
    if (s != TL_OK || n == 0)
        return s;
    const size_t need = tl_dtg_host_workspace_bytes(n, dtype);
    if (!workspace || workspace_bytes < need)
        return fail(TL_ERR_INVALID_ARG, "workspace %p of %zu bytes; %zu needed", workspace, workspace_bytes, need);
    if ((uintptr_t)workspace % 16)
        return fail(TL_ERR_ALIGNMENT, "workspace must be 16-byte aligned");
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    HostPipe *P = nullptr;
    if ((s = host_pipe(&P)) != TL_OK)
        return s;
    // the pipeline's streams and events are shared per device: one caller enqueues at a time
    std::lock_guard<std::mutex> enqueue_lock(P->mu);
    const size_t esz = elem_size(dtype);
    const int64_t chunk = std::min<int64_t>(n, kHostChunk);
    const cudaStream_t user = (cudaStream_t)stream;
    char *const *hin = (char *const *)in;
    char *const *hout = (char *const *)out;
    size_t sin = uniform_stride(hin, N_IN, n * esz), sout = uniform_stride(hout, N_OUT, n * esz);
    cudaError_t e;
    if ((e = cudaEventRecord(P->fork, user)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
    for (cudaStream_t st : {P->h2d, P->cmp, P->d2h})
        if ((e = cudaStreamWaitEvent(st, P->fork, 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    int64_t c = 0;
    for (int64_t x0 = 0; x0 < n; x0 += chunk, ++c) {
        const int b = (int)(c % kHostSlots);
        const int64_t m = std::min(chunk, n - x0);
        char *base = (char *)workspace + (size_t)b * (N_IN + N_OUT) * chunk * esz;
        char *slot_in = base, *slot_out = base + (size_t)N_IN * chunk * esz;
        if (c >= kHostSlots && (e = cudaStreamWaitEvent(P->h2d, P->slot_free[b], 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
        if ((e = copy_table((char *const *)hin, N_IN, x0, m, slot_in, chunk, esz, &sin, true, P->h2d)) != cudaSuccess)
            return cuda_fail(e, "host->device copy");
        if ((e = cudaEventRecord(P->in_ready[b], P->h2d)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(P->cmp, P->in_ready[b], 0)) != cudaSuccess)
            return cuda_fail(e, "pipeline event");
        tl_dtg_in din;
        tl_dtg_out dout;
        const void **dinp = (const void **)&din;
        void **doutp = (void **)&dout;
        for (int q = 0; q < N_IN; ++q)
            dinp[q] = slot_in + (size_t)q * chunk * esz;
        for (int q = 0; q < N_OUT; ++q)
            doutp[q] = slot_out + (size_t)q * chunk * esz;
        if ((s = launch_forward(*d, &din, &dout, m, dtype, P->cmp)) != TL_OK)
            return s;
        if ((e = cudaEventRecord(P->done[b], P->cmp)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(P->d2h, P->done[b], 0)) != cudaSuccess)
            return cuda_fail(e, "pipeline event");
        if ((e = copy_table(hout, N_OUT, x0, m, slot_out, chunk, esz, &sout, false, P->d2h)) != cudaSuccess)
            return cuda_fail(e, "device->host copy");
        if ((e = cudaEventRecord(P->slot_free[b], P->d2h)) != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord");
    }
    // the last device->host copy follows every earlier operation of the pipeline
    if ((e = cudaEventRecord(P->join, P->d2h)) != cudaSuccess || (e = cudaStreamWaitEvent(user, P->join, 0)) != cudaSuccess)
        return cuda_fail(e, "pipeline join");
    return TL_OK;
}

}  // extern "C"
