// tl_batch.cu -- batch plans (many grids, one persistent launch) and their autotuner.
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "dtg_batched.cuh"
#include "tl_host.h"
#include "../../include/tl_testing.h"
#include "tl_kernels.h"

namespace tl {
namespace {

constexpr uint64_t kPlanMagic = 0x746c5f706c616e31ull;   // "tl_plan1"
constexpr int kThreadOptions[3] = {128, 256, 512};
constexpr int kPptOptions[3] = {1, 2, 4};   // points per thread in a tile

int thread_slot(int threads)
{
    for (int i = 0; i < 3; ++i)
        if (kThreadOptions[i] == threads)
            return i;
    return -1;
}

int ppt_slot(int ppt)
{
    for (int i = 0; i < 3; ++i)
        if (kPptOptions[i] == ppt)
            return i;
    return -1;
}

constexpr int kStageOptions[3] = {0, 2, 3};   // staging depth (0: inputs loaded straight into registers)

// ---- tuning cache: one line per key, "key threads blocks_per_sm points_per_thread stages ms" ----------
std::mutex g_cache_mu;

std::string cache_path()
{
    const char *p = getenv("TL_TUNE_CACHE");
    if (p && *p)
        return strcmp(p, "off") == 0 ? std::string() : std::string(p);
    const char *home = getenv("HOME");
    if (!home || !*home)
        return std::string();
    return std::string(home) + "/.cache/tl_dtg_tune.txt";
}

bool cache_lookup(const std::string &key, int *threads, int *bps, int *ppt, int *stages)
{
    std::lock_guard<std::mutex> lk(g_cache_mu);
    const std::string path = cache_path();
    if (path.empty())
        return false;
    FILE *f = fopen(path.c_str(), "r");
    if (!f)
        return false;
    char line[768], k[512];
    int t = 0, b = 0, q = 0, st = 0;
    double ms = 0;
    bool found = false;
    while (fgets(line, sizeof line, f))
        if (sscanf(line, "%511s %d %d %d %d %lf", k, &t, &b, &q, &st, &ms) == 6 && key == k && thread_slot(t) >= 0 &&
            b >= 1 && ppt_slot(q) >= 0 && st >= 0) {
            *threads = t;
            *bps = b;
            *ppt = q;
            *stages = st;
            found = true;          // the last entry for a key wins
        }
    fclose(f);
    return found;
}

void cache_store(const std::string &key, int threads, int bps, int ppt, int stages, double ms)
{
    std::lock_guard<std::mutex> lk(g_cache_mu);
    const std::string path = cache_path();
    if (path.empty())
        return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos && slash > 0)
        mkdir(path.substr(0, slash).c_str(), 0755);   // one level; EEXIST is fine
    if (FILE *f = fopen(path.c_str(), "a")) {
        fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), threads, bps, ppt, stages, ms);
        fclose(f);
    }
}

}  // namespace
}  // namespace tl

struct tl_batch_plan {
    uint64_t magic = 0;
    int device = -1;
    tl_dtype dtype = TL_F64;
    int32_t G = 0;
    int64_t total_points = 0;
    int sms = 0;
    int max_blocks[3] = {0, 0, 0};          // occupancy per thread option
    int threads = 256, blocks_per_sm = 0;   // launch configuration
    int ppt = 1;                            // points per thread in a tile
    int stages = 0;                         // staging depth (0: registers; else ppt == 1)
    std::string key;                        // tuning-cache key
    // device data
    void **d_tables = nullptr;              // G x 82
    int64_t *d_n = nullptr;                 // G
    int64_t *d_prefix = nullptr;            // 9 x (G + 1): thread option x points-per-thread option
    uint32_t *d_status = nullptr;
    int64_t total_tiles[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

using namespace tl;

static tl_status plan_ok(const tl_batch_plan *p)
{
    if (!p || p->magic != kPlanMagic)
        return fail(TL_ERR_PLAN_MISMATCH, "not a live batch plan");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device)
        return fail(TL_ERR_PLAN_MISMATCH, "plan belongs to device %d, device %d is current", p->device, dev);
    return TL_OK;
}

static BatchView view_of(const tl_batch_plan *p, int slot)
{
    BatchView v;
    v.tables = (const void *const *)p->d_tables;
    v.n = p->d_n;
    v.tile_prefix = p->d_prefix + (size_t)slot * (p->G + 1);
    v.total_tiles = p->total_tiles[slot];
    v.ppt = kPptOptions[slot % 3];
    v.G = p->G;
    v.status = p->d_status;
    v.extra_tx = 0;
    return v;
}

static void plan_free(tl_batch_plan *p)
{
    cudaFree(p->d_tables);
    cudaFree(p->d_n);
    cudaFree(p->d_prefix);
    cudaFree(p->d_status);
    p->magic = 0;
    delete p;
}

extern "C" {

tl_status tl_dtg_batched_prepare(const tl_dtg_in *in, const tl_dtg_out *out, const int64_t *n, int32_t G,
                                 tl_dtype dtype, tl_batch_plan **plan)
{
    if (!plan)
        return fail(TL_ERR_INVALID_ARG, "plan is NULL");
    *plan = nullptr;
    if (G < 0 || (G > 0 && (!in || !out || !n)))
        return fail(TL_ERR_INVALID_ARG, "G = %d with NULL in/out/n", (int)G);
    if (!dtype_ok(dtype))
        return fail(TL_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    const size_t esz = elem_size(dtype);
    std::vector<Range> rs;
    rs.reserve((size_t)G * (N_IN + N_OUT));
    int64_t total = 0;
    for (int32_t d = 0; d < G; ++d) {
        if (n[d] < 0)
            return fail(TL_ERR_INVALID_ARG, "n[%d] = %lld < 0", (int)d, (long long)n[d]);
        const void *const *tabs[2] = {(const void *const *)&in[d], (const void *const *)&out[d]};
        const int counts[2] = {N_IN, N_OUT};
        const bool writes[2] = {false, true}, nullable[2] = {false, false};
        const char *const names[2] = {"in", "out"};
        tl_status s = collect_ranges(rs, tabs, counts, writes, nullable, names, 2, n[d], esz, d);
        if (s != TL_OK)
            return s;
        total += n[d];
    }
    tl_status s = check_overlaps(rs);
    if (s != TL_OK)
        return s;
    const DeviceInfo *di = nullptr;
    if ((s = device_info(&di)) != TL_OK)
        return s;

    tl_batch_plan *p = new tl_batch_plan();
    cudaGetDevice(&p->device);
    p->dtype = dtype;
    p->G = G;
    p->total_points = total;
    p->sms = di->sms;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = occupancy_batched((int)dtype, kThreadOptions[i], &p->max_blocks[i]);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    }
    // host images of the device data
    std::vector<void *> tables((size_t)std::max(G, 1) * (N_IN + N_OUT));
    for (int32_t d = 0; d < G; ++d) {
        memcpy(&tables[(size_t)d * (N_IN + N_OUT)], &in[d], N_IN * sizeof(void *));
        memcpy(&tables[(size_t)d * (N_IN + N_OUT) + N_IN], &out[d], N_OUT * sizeof(void *));
    }
    std::vector<int64_t> prefix((size_t)9 * (G + 1));
    for (int i = 0; i < 9; ++i) {
        const int64_t tile = (int64_t)kThreadOptions[i / 3] * kPptOptions[i % 3];
        int64_t acc = 0;
        for (int32_t d = 0; d < G; ++d) {
            prefix[(size_t)i * (G + 1) + d] = acc;
            acc += (n[d] + tile - 1) / tile;
        }
        prefix[(size_t)i * (G + 1) + G] = acc;
        p->total_tiles[i] = acc;
    }
    const size_t gG = (size_t)std::max(G, 1);
    if ((e = cudaMalloc((void **)&p->d_tables, tables.size() * sizeof(void *))) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_n, gG * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_prefix, prefix.size() * sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_status, sizeof(uint32_t))) != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "cudaMalloc (batch plan)");
    }
    std::vector<int64_t> nn(gG, 0);
    for (int32_t d = 0; d < G; ++d)
        nn[d] = n[d];
    if ((e = cudaMemcpy(p->d_tables, tables.data(), tables.size() * sizeof(void *), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(p->d_n, nn.data(), gG * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_prefix, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemset(p->d_status, 0, sizeof(uint32_t))) != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "upload of the batch plan");
    }
    // tuning-cache key: GPU, SMs, dtype, batch shape (G and the size of the batch in powers of two)
    char key[512];
    snprintf(key, sizeof key, "%s|sm%d|dtype%d|batched3|G%d|log2pts%d", di->name, di->sms, (int)dtype, (int)G,
             total > 0 ? (int)std::floor(std::log2((double)total)) : 0);
    p->key = key;
    p->threads = 256;
    p->blocks_per_sm = p->max_blocks[1];
    p->ppt = 1;
    int t = 0, b = 0, q = 0, st = 0, sb = 0;
    if (cache_lookup(p->key, &t, &b, &q, &st)) {
        if (st == 0 && b <= p->max_blocks[thread_slot(t)]) {
            p->threads = t;
            p->blocks_per_sm = b;
            p->ppt = q;
        } else if (st > 0 && q == 1 && batched_staging_provided((int)dtype, t, st) &&
                   occupancy_batched_staged((int)dtype, t, st, &sb) == cudaSuccess && b <= sb) {
            p->threads = t;
            p->blocks_per_sm = b;
            p->ppt = 1;
            p->stages = st;
        }
    }
    p->magic = kPlanMagic;
    *plan = p;
    return TL_OK;
}

tl_status tl_dtg_batched(const tl_batch_plan *p, tl_stream stream)
{
    tl_status s = plan_ok(p);
    if (s != TL_OK)
        return s;
    const int slot = thread_slot(p->threads) * 3 + ppt_slot(p->ppt);
    if (p->total_tiles[slot] == 0)
        return TL_OK;
    const int64_t want = (int64_t)p->sms * p->blocks_per_sm;
    const int grid = (int)std::max<int64_t>(1, std::min(want, p->total_tiles[slot]));
    cudaError_t e = p->stages > 0 ? launch_batched_staged((int)p->dtype, view_of(p, slot), p->threads, p->stages, grid,
                                                          (cudaStream_t)stream)
                                  : launch_batched((int)p->dtype, view_of(p, slot), p->threads, grid, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "batched launch");
    return TL_OK;
}

tl_status tl_batch_plan_config(const tl_batch_plan *p, int32_t *threads, int32_t *blocks_per_sm)
{
    if (!p || p->magic != kPlanMagic)
        return fail(TL_ERR_PLAN_MISMATCH, "not a live batch plan");
    if (threads)
        *threads = p->threads;
    if (blocks_per_sm)
        *blocks_per_sm = p->blocks_per_sm;
    return TL_OK;
}

tl_status tl_batch_plan_set_config(tl_batch_plan *p, int32_t threads, int32_t blocks_per_sm)
{
    if (!p || p->magic != kPlanMagic)
        return fail(TL_ERR_PLAN_MISMATCH, "not a live batch plan");
    const int slot = thread_slot(threads);
    if (slot < 0)
        return fail(TL_ERR_INVALID_ARG, "threads must be 128, 256 or 512 (got %d)", (int)threads);
    int maxb = p->max_blocks[slot];
    if (p->stages > 0) {
        if (!batched_staging_provided((int)p->dtype, threads, p->stages))
            return fail(TL_ERR_INVALID_ARG, "staging depth %d is not provided for %d threads", p->stages, (int)threads);
        const cudaError_t e = occupancy_batched_staged((int)p->dtype, threads, p->stages, &maxb);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    }
    if (blocks_per_sm < 1 || blocks_per_sm > maxb)
        return fail(TL_ERR_INVALID_ARG, "blocks_per_sm must be in [1, %d] for %d threads", maxb, (int)threads);
    p->threads = threads;
    p->blocks_per_sm = blocks_per_sm;
    return TL_OK;
}

tl_status tl_batch_plan_points_per_thread(const tl_batch_plan *p, int32_t *ppt)
{
    if (!p || p->magic != kPlanMagic)
        return fail(TL_ERR_PLAN_MISMATCH, "not a live batch plan");
    if (ppt)
        *ppt = p->ppt;
    return TL_OK;
}

tl_status tl_batch_plan_set_points_per_thread(tl_batch_plan *p, int32_t ppt)
{
    if (!p || p->magic != kPlanMagic)
        return fail(TL_ERR_PLAN_MISMATCH, "not a live batch plan");
    if (ppt_slot(ppt) < 0)
        return fail(TL_ERR_INVALID_ARG, "points per thread must be 1, 2 or 4 (got %d)", (int)ppt);
    if (p->stages > 0 && ppt != 1)
        return fail(TL_ERR_INVALID_ARG, "a staged plan computes one point per thread");
    p->ppt = ppt;
    return TL_OK;
}

tl_status tl_batch_plan_staging(const tl_batch_plan *p, int32_t *stages)
{
    if (!p || p->magic != kPlanMagic)
        return fail(TL_ERR_PLAN_MISMATCH, "not a live batch plan");
    if (stages)
        *stages = p->stages;
    return TL_OK;
}

tl_status tl_batch_plan_set_staging(tl_batch_plan *p, int32_t stages)
{
    tl_status s = plan_ok(p);
    if (s != TL_OK)
        return s;
    if (stages == 0) {
        p->stages = 0;
        p->blocks_per_sm = std::min(p->blocks_per_sm, p->max_blocks[thread_slot(p->threads)]);
        return TL_OK;
    }
    if (p->dtype == TL_F64_FF)
        return fail(TL_ERR_UNSUPPORTED, "staged inputs are provided for TL_F64 and TL_F32");
    if (!batched_staging_provided((int)p->dtype, p->threads, stages))
        return fail(TL_ERR_INVALID_ARG, "staging depth %d is not provided for %d threads", (int)stages, p->threads);
    int maxb = 0;
    const cudaError_t e = occupancy_batched_staged((int)p->dtype, p->threads, stages, &maxb);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (maxb < 1)
        return fail(TL_ERR_UNSUPPORTED, "the staged kernel does not fit on an SM");
    p->stages = stages;
    p->ppt = 1;
    p->blocks_per_sm = std::max(1, std::min(p->blocks_per_sm, maxb));
    return TL_OK;
}

tl_status tl_dtg_batched_tune(tl_batch_plan *p, tl_stream stream)
{
    tl_status s = plan_ok(p);
    if (s != TL_OK)
        return s;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    const int keep_t = p->threads, keep_b = p->blocks_per_sm, keep_q = p->ppt, keep_s = p->stages;
    int best_t = keep_t, best_b = keep_b, best_q = keep_q, best_s = keep_s;
    float best = 1e30f;
    // threads x points per thread x staging depth; a staged kernel computes one point per thread
    for (int j = 0; j < 27 && s == TL_OK; ++j) {
        const int i = j / 9, T = kThreadOptions[i], Q = kPptOptions[(j / 3) % 3], S = kStageOptions[j % 3];
        int maxb = p->max_blocks[i];
        if (S > 0) {
            if (Q != 1 || !batched_staging_provided((int)p->dtype, T, S))
                continue;
            if ((e = occupancy_batched_staged((int)p->dtype, T, S, &maxb)) != cudaSuccess) {
                s = cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
                break;
            }
        }
        int cands[4] = {1, 2, 4, maxb};
        for (int c = 0; c < 4 && s == TL_OK; ++c) {
            const int B = cands[c];
            if (B < 1 || B > maxb || (c < 3 && B == maxb))
                continue;
            p->threads = T;
            p->blocks_per_sm = B;
            p->ppt = Q;
            p->stages = S;
            if ((s = tl_dtg_batched(p, stream)) != TL_OK)   // warm-up
                break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && s == TL_OK; ++r)
                s = tl_dtg_batched(p, stream);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                s = cuda_fail(e, "cudaEventSynchronize");
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (s == TL_OK && ms < best) {
                best = ms;
                best_t = T;
                best_b = B;
                best_q = Q;
                best_s = S;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->threads = best_t;
    p->blocks_per_sm = best_b;
    p->ppt = best_q;
    p->stages = best_s;
    if (s == TL_OK && best < 1e30f)
        cache_store(p->key, best_t, best_b, best_q, best_s, best / 3.0);
    return s;
}

tl_status tl_testing_batched_staged_stall(const tl_batch_plan *p, tl_stream stream)
{
    tl_status s = plan_ok(p);
    if (s != TL_OK)
        return s;
    if (p->stages == 0)
        return fail(TL_ERR_INVALID_ARG, "the plan does not stage its inputs");
    const int slot = thread_slot(p->threads) * 3 + ppt_slot(p->ppt);
    if (p->total_tiles[slot] == 0)
        return TL_OK;
    const int64_t want = (int64_t)p->sms * p->blocks_per_sm;
    const int grid = (int)std::max<int64_t>(1, std::min(want, p->total_tiles[slot]));
    BatchView v = view_of(p, slot);
    v.extra_tx = 16;
    const cudaError_t e = launch_batched_staged((int)p->dtype, v, p->threads, p->stages, grid, (cudaStream_t)stream);
    return e == cudaSuccess ? TL_OK : cuda_fail(e, "staged batched launch");
}

tl_status tl_batch_plan_check(const tl_batch_plan *p)
{
    tl_status s = plan_ok(p);
    if (s != TL_OK)
        return s;
    uint32_t w = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(&w, p->d_status, sizeof w, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && w != 0)
        e = cudaMemset(p->d_status, 0, sizeof w);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the batch status word");
    if (w != 0)
        return fail((tl_status)w, "a batched launch recorded status %u", w);
    return TL_OK;
}

void tl_batch_plan_destroy(tl_batch_plan *p)
{
    if (!p || p->magic != kPlanMagic)
        return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device)
        cudaSetDevice(p->device);
    plan_free(p);
    if (cur >= 0 && cur != p->device)
        cudaSetDevice(cur);
}

}  // extern "C"
