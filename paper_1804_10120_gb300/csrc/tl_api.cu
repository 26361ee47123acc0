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

int grid_for(int64_t n, int threads, int sms, int blocks_per_sm)
{
    const int64_t need = (n + threads - 1) / threads;
    const int64_t resident = (int64_t)sms * std::max(1, blocks_per_sm);
    return (int)std::max<int64_t>(1, std::min(need, resident));
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
        e = launch_fwd_f64(fwd_args<double>(in, out), n, grid_for(n, kFwdThreads, d.sms, d.fwd_f64_blocks), st);
        break;
    case TL_F32:
        e = launch_fwd_f32(fwd_args<float>(in, out), n, grid_for(n, kFwdThreads, d.sms, d.fwd_f32_blocks), st);
        break;
    case TL_F64_FF:
        e = launch_fwd_ff(fwd_args<double>(in, out), n, grid_for(n, kFwdThreads, d.sms, d.fwd_ff_blocks), st);
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
constexpr int64_t kHostChunk = int64_t(1) << 20;   // points per pipeline chunk
constexpr int kHostLanes = 2;                      // chunks in flight (double buffering)

struct HostLanes {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s[kHostLanes] = {};
    cudaEvent_t fork = nullptr, join[kHostLanes] = {};
};
HostLanes g_lanes[kMaxDevices];
std::mutex g_lanes_mu;

tl_status host_lanes(HostLanes **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_lanes_mu);
    HostLanes &L = g_lanes[dev];
    if (!L.ready) {
        for (int i = 0; i < kHostLanes; ++i) {
            if ((e = cudaStreamCreateWithFlags(&L.s[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreateWithFlags");
            if ((e = cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreateWithFlags");
        }
        if ((e = cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreateWithFlags");
        L.ready = true;
    }
    *out = &L;
    return TL_OK;
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
                        ? launch_bwd_f64(a, n, grid_for(n, kBwdThreads, d->sms, d->bwd_f64_blocks), (cudaStream_t)stream)
                        : launch_bwd_ff(a, n, grid_for(n, kBwdThreads, d->sms, d->bwd_ff_blocks), (cudaStream_t)stream);
    if (e == cudaErrorNotSupported)
        return fail(TL_ERR_UNSUPPORTED, "dtype %d has no adjoint kernel in this build", (int)dtype);
    if (e != cudaSuccess)
        return cuda_fail(e, "backward launch");
    return TL_OK;
}

size_t tl_dtg_host_workspace_bytes(int64_t n, tl_dtype dtype)
{
    if (n <= 0 || !dtype_ok(dtype))
        return 0;
    const int64_t chunk = std::min<int64_t>(n, kHostChunk);
    const int64_t lanes = std::min<int64_t>(kHostLanes, (n + chunk - 1) / chunk);
    return (size_t)(lanes * (N_IN + N_OUT) * chunk) * elem_size(dtype);
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
    HostLanes *L = nullptr;
    if ((s = host_lanes(&L)) != TL_OK)
        return s;
    // the lanes and their events are shared per device: one caller enqueues at a time
    std::lock_guard<std::mutex> enqueue_lock(L->mu);
    const size_t esz = elem_size(dtype);
    const int64_t chunk = std::min<int64_t>(n, kHostChunk);
    const cudaStream_t user = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaEventRecord(L->fork, user)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
    for (int i = 0; i < kHostLanes; ++i)
        if ((e = cudaStreamWaitEvent(L->s[i], L->fork, 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    const char *const *hin = (const char *const *)in;
    char *const *hout = (char *const *)out;
    int64_t c = 0;
    for (int64_t x0 = 0; x0 < n; x0 += chunk, ++c) {
        const int lane = (int)(c % kHostLanes);
        const cudaStream_t st = L->s[lane];
        const int64_t m = std::min(chunk, n - x0);
        char *base = (char *)workspace + (size_t)lane * (N_IN + N_OUT) * chunk * esz;
        tl_dtg_in din;
        tl_dtg_out dout;
        const void **dinp = (const void **)&din;
        void **doutp = (void **)&dout;
        for (int q = 0; q < N_IN; ++q) {
            dinp[q] = base + (size_t)q * chunk * esz;
            if ((e = cudaMemcpyAsync((void *)dinp[q], hin[q] + x0 * esz, m * esz, cudaMemcpyHostToDevice, st)) !=
                cudaSuccess)
                return cuda_fail(e, "cudaMemcpyAsync host->device");
        }
        for (int q = 0; q < N_OUT; ++q)
            doutp[q] = base + (size_t)(N_IN + q) * chunk * esz;
        if ((s = launch_forward(*d, &din, &dout, m, dtype, st)) != TL_OK)
            return s;
        for (int q = 0; q < N_OUT; ++q)
            if ((e = cudaMemcpyAsync(hout[q] + x0 * esz, doutp[q], m * esz, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
                return cuda_fail(e, "cudaMemcpyAsync device->host");
    }
    for (int i = 0; i < kHostLanes; ++i) {
        if ((e = cudaEventRecord(L->join[i], L->s[i])) != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(user, L->join[i], 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    }
    return TL_OK;
}

}  // extern "C"
