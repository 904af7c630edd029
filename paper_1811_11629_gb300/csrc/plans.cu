// Launch plans, CUDA-graph capture, host-buffer generation and the autotuner.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "api_internal.hpp"

using namespace rsaprng;

struct rsaprng_plan {
    rsaprng_ctx *ctx = nullptr;
    DevPlan dp;
    rsaprng_config cfg{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;
};

namespace {

// Tuned configurations, kept per (device, workload signature, exponent
// class) for the life of the process (and across processes through
// rsaprng_autotune_cache_save / _load).
std::mutex g_tune_mu;
std::map<std::string, rsaprng_config> g_tune_cache;

// The cache key. Device: compute capability and SM count. Workload: the
// request count, mean and longest request (log2 buckets) and the output
// kind. Exponent class: the mean cost per output in Montgomery products
// (the planner's weight), in steps of two.
std::string tune_key(rsaprng_ctx *c, uint64_t nreq, const rsaprng_id *ids, const uint64_t *counts)
{
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
    uint64_t total = 0, longest = 0;
    double w = 0;
    for (uint64_t i = 0; i < nreq; i++) {
        total += counts[i];
        longest = std::max(longest, counts[i]);
        if (ids[i] < c->count) {
            const InstParams &P = c->h_params[ids[i]];
            w += (double)counts[i] * (double)cost_per_number(std::max(P.e, P.eq));
        }
    }
    auto lg = [](double x) { return x >= 1 ? (int)std::floor(std::log2(x)) : -1; };
    const double mean = nreq ? (double)total / (double)nreq : 0.0;
    const int eclass = total ? (int)(w / (double)total / 2.0) : 0;
    char buf[160];
    snprintf(buf, sizeof buf, "sm%d%d-x%d/req2^%d-mean2^%d-max2^%d/rounding%d/e%d", major, minor,
             c->sms, lg((double)nreq), lg(mean), lg((double)longest), c->cfg.rounding, eclass);
    return buf;
}

void destroy_graph(rsaprng_plan *p)
{
    if (p->exec)
        cudaGraphExecDestroy(p->exec);
    if (p->graph)
        cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

int plan_create_cfg(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nreq, const rsaprng_id *ids,
                    const uint64_t *counts, const uint64_t *offsets, rsaprng_plan **out)
{
    cudaSetDevice(c->device);
    HostPlan hp;
    int rc = build_plan(c, cfg, nreq, ids, counts, offsets, cfg.chunk, hp, 1, 1, true);
    if (rc)
        return rc;
    rsaprng_plan *p = new (std::nothrow) rsaprng_plan();
    if (!p)
        return fail(RSAPRNG_ERR_OOM, "plan alloc");
    p->ctx = c;
    p->cfg = cfg;
    cudaSetDevice(c->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    rc = upload_plan(c, hp, p->dp, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc == RSAPRNG_OK && e != cudaSuccess)
        rc = cuda_fail(e, "plan upload");
    if (rc) {
        free_devplan(p->dp);
        delete p;
        return rc;
    }
    p->launches = (p->dp.nchunks ? 2 : 0) + (p->dp.nitems ? 1 : 0);
    *out = p;
    return RSAPRNG_OK;
}

}  // namespace

extern "C" {

int rsaprng_plan_create(rsaprng_ctx *c, uint64_t nreq, const rsaprng_id *ids,
                        const uint64_t *counts, const uint64_t *out_offsets, rsaprng_plan **out)
{
    if (!c || !out || (nreq && (!ids || !counts || !out_offsets)))
        return fail(RSAPRNG_ERR_ARG, "plan_create: null argument");
    return plan_create_cfg(c, c->cfg, nreq, ids, counts, out_offsets, out);
}

int rsaprng_plan_launch(rsaprng_plan *p, double *d_r, uint64_t *d_c, void *stream)
{
    if (!p || (!d_r && !d_c))
        return fail(RSAPRNG_ERR_ARG, "plan_launch: bad arguments");
    cudaSetDevice(p->ctx->device);
    return launch_plan(p->ctx, p->cfg, p->dp, d_r, d_c, (cudaStream_t)stream, nullptr);
}

int rsaprng_plan_launch_timed(rsaprng_plan *p, double *d_r, uint64_t *d_c, void *stream,
                              void *gen_start, void *gen_end)
{
    if (!p || (!d_r && !d_c) || !gen_start || !gen_end)
        return fail(RSAPRNG_ERR_ARG, "plan_launch_timed: bad arguments");
    cudaSetDevice(p->ctx->device);
    const cudaEvent_t ev[2] = {(cudaEvent_t)gen_start, (cudaEvent_t)gen_end};
    return launch_plan(p->ctx, p->cfg, p->dp, d_r, d_c, (cudaStream_t)stream, nullptr, nullptr,
                       false, ev);
}

int rsaprng_plan_capture(rsaprng_plan *p, double *d_r, uint64_t *d_c, void *stream)
{
    if (!p || (!d_r && !d_c) || !stream)
        return fail(RSAPRNG_ERR_ARG, "plan_capture: needs outputs and a non-default stream");
    cudaSetDevice(p->ctx->device);
    destroy_graph(p);
    cudaStream_t st = (cudaStream_t)stream;
    // Resolve kernel attributes before capture (occupancy queries are not
    // stream work).
    (void)ctx_launch(p->ctx, p->cfg, p->dp.nitems, d_r != nullptr, d_c != nullptr);
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess)
        return cuda_fail(e, "begin capture");
    const uint64_t before = p->ctx->launches;
    int rc = launch_plan(p->ctx, p->cfg, p->dp, d_r, d_c, st, nullptr);
    p->ctx->launches = before;  // recorded, not launched
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (rc)
        return rc;
    if (e != cudaSuccess)
        return cuda_fail(e, "end capture");
    p->graph = g;
    e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e != cudaSuccess) {
        destroy_graph(p);
        return cuda_fail(e, "graph instantiate");
    }
    return RSAPRNG_OK;
}

int rsaprng_plan_replay(rsaprng_plan *p, void *stream)
{
    if (!p || !p->exec)
        return fail(RSAPRNG_ERR_ARG, "plan_replay: no captured graph");
    cudaSetDevice(p->ctx->device);
    cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "graph launch");
    p->ctx->launches += p->launches;
    return RSAPRNG_OK;
}

int rsaprng_plan_info(const rsaprng_plan *p, uint64_t *launches, uint64_t *numbers,
                      uint64_t *chunks)
{
    if (!p)
        return fail(RSAPRNG_ERR_ARG, "null plan");
    if (launches)
        *launches = p->launches;
    if (numbers)
        *numbers = p->dp.numbers;
    if (chunks)
        *chunks = p->dp.nitems;
    return RSAPRNG_OK;
}

int rsaprng_plan_shape(const rsaprng_plan *p, int *grid, int *threads, int *blocks_per_sm,
                       int *persistent)
{
    if (!p)
        return fail(RSAPRNG_ERR_ARG, "null plan");
    if (grid)
        *grid = p->dp.last.grid;
    if (threads)
        *threads = p->dp.last.threads;
    if (blocks_per_sm)
        *blocks_per_sm = p->dp.occupancy;
    if (persistent)
        *persistent = p->dp.last.persistent ? 1 : 0;
    return RSAPRNG_OK;
}

void rsaprng_plan_destroy(rsaprng_plan *p)
{
    if (!p)
        return;
    cudaSetDevice(p->ctx->device);
    cudaDeviceSynchronize();
    destroy_graph(p);
    free_devplan(p->dp);
    delete p;
}

// Host-buffer generation: the requests are cut into slices of about equal
// output size; each slice is generated into one of two device buffers on
// the caller's stream and copied to the host on a second stream, so the copy
// of slice k overlaps the generation of slice k+1.
int rsaprng_generate_batch_host(rsaprng_ctx *c, uint64_t nreq, const rsaprng_id *ids,
                                const uint64_t *counts, const uint64_t *out_offsets, double *h_r,
                                uint64_t *h_c, void *stream)
{
    if (!c || (nreq && (!ids || !counts || !out_offsets)) || (!h_r && !h_c))
        return fail(RSAPRNG_ERR_ARG, "generate_batch_host: bad arguments");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t total = 0;
    for (uint64_t i = 0; i < nreq; i++)
        total += counts[i];
    if (total == 0)
        return RSAPRNG_OK;
    // Page-locked host buffers are mapped into the device's address space: the
    // kernel stores straight into them over the CPU-GPU link (one launch, no
    // staging). Pageable buffers go through device slices and copies below.
    auto mapped = [](void *h) -> void * {
        if (!h)
            return nullptr;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
    };
    void *m_r = mapped(h_r), *m_c = mapped(h_c);
    if ((!h_r || m_r) && (!h_c || m_c)) {
        int rc = rsaprng_generate_batch(c, nreq, ids, counts, out_offsets, (double *)m_r,
                                        (uint64_t *)m_c, stream);
        if (rc)
            return rc;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            return cuda_fail(e, "host-output generation");
        c->d2h_bytes += total * ((h_r ? 8 : 0) + (h_c ? 8 : 0));
        return RSAPRNG_OK;
    }
    const int nslices = (int)std::min<uint64_t>(8, std::max<uint64_t>(1, total >> 22));
    const uint64_t per = (total + nslices - 1) / nslices;
    const size_t width = (h_r ? 8 : 0) + (h_c ? 8 : 0);
    const size_t need = 2 * per * width;
    if (need > c->cap_out_scratch) {
        if (c->d_out_scratch) {
            cudaDeviceSynchronize();
            cudaFree(c->d_out_scratch);
        }
        c->d_out_scratch = nullptr;
        c->cap_out_scratch = 0;
        cudaError_t e = cudaMalloc(&c->d_out_scratch, need);
        if (e != cudaSuccess)
            return fail(RSAPRNG_ERR_OOM, "host-generation staging (%zu B): %s", need,
                        cudaGetErrorString(e));
        c->cap_out_scratch = need;
    }
    cudaStream_t cp;
    cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking);
    cudaEvent_t gen_done[2], copy_done[2];
    for (int k = 0; k < 2; k++) {
        cudaEventCreateWithFlags(&gen_done[k], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&copy_done[k], cudaEventDisableTiming);
    }
    struct Part {
        rsaprng_id id;
        uint64_t count, dev_off, host_off;
    };
    std::vector<Part> parts;
    std::vector<rsaprng_id> sid;
    std::vector<uint64_t> scnt, soff;
    int rc = RSAPRNG_OK;
    uint64_t req = 0, done_in_req = 0;
    bool copy_pending[2] = {false, false};
    for (int k = 0; k < nslices && rc == RSAPRNG_OK; k++) {
        const int buf = k & 1;
        parts.clear();
        uint64_t fill = 0;
        while (req < nreq && fill < per) {
            const uint64_t left = counts[req] - done_in_req;
            const uint64_t take = std::min(left, per - fill);
            if (take)
                parts.push_back({ids[req], take, fill, out_offsets[req] + done_in_req});
            fill += take;
            done_in_req += take;
            if (done_in_req == counts[req]) {
                req++;
                done_in_req = 0;
            }
        }
        if (parts.empty())
            break;
        sid.resize(parts.size());
        scnt.resize(parts.size());
        soff.resize(parts.size());
        for (size_t i = 0; i < parts.size(); i++) {
            sid[i] = parts[i].id;
            scnt[i] = parts[i].count;
            soff[i] = parts[i].dev_off;
        }
        char *base = (char *)c->d_out_scratch + (size_t)buf * per * width;
        double *d_r = h_r ? (double *)base : nullptr;
        uint64_t *d_c = h_c ? (uint64_t *)(base + (h_r ? per * 8 : 0)) : nullptr;
        if (copy_pending[buf])
            cudaStreamWaitEvent(st, copy_done[buf], 0);
        // Chunk the slice so that every SM has work even when it holds few requests.
        const rsaprng_config saved = c->cfg;
        const uint64_t tile = (uint64_t)c->cfg.threads_per_block * c->cfg.numbers_per_thread;
        uint64_t chunk = per / ((uint64_t)c->sms * 8);
        chunk = std::max<uint64_t>(tile, (chunk + tile - 1) / tile * tile);
        c->cfg.chunk = std::min<uint64_t>(chunk, std::max<uint64_t>(saved.chunk, tile));
        rc = rsaprng_generate_batch(c, parts.size(), sid.data(), scnt.data(), soff.data(), d_r, d_c,
                                    stream);
        c->cfg = saved;
        if (rc)
            break;
        cudaEventRecord(gen_done[buf], st);
        cudaStreamWaitEvent(cp, gen_done[buf], 0);
        // One copy per run of parts that is contiguous on the host.
        for (size_t i = 0; i < parts.size();) {
            size_t j = i + 1;
            while (j < parts.size() &&
                   parts[j].host_off == parts[j - 1].host_off + parts[j - 1].count &&
                   parts[j].dev_off == parts[j - 1].dev_off + parts[j - 1].count)
                j++;
            const uint64_t n = parts[j - 1].dev_off + parts[j - 1].count - parts[i].dev_off;
            cudaError_t e = cudaSuccess;
            if (h_r)
                e = cudaMemcpyAsync(h_r + parts[i].host_off, d_r + parts[i].dev_off, n * 8,
                                    cudaMemcpyDeviceToHost, cp);
            if (e == cudaSuccess && h_c)
                e = cudaMemcpyAsync(h_c + parts[i].host_off, d_c + parts[i].dev_off, n * 8,
                                    cudaMemcpyDeviceToHost, cp);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "result copy");
                break;
            }
            c->d2h_bytes += n * width;
            i = j;
        }
        cudaEventRecord(copy_done[buf], cp);
        copy_pending[buf] = true;
    }
    cudaError_t e = cudaStreamSynchronize(cp);
    if (rc == RSAPRNG_OK && e != cudaSuccess)
        rc = cuda_fail(e, "result copy");
    for (int k = 0; k < 2; k++) {
        cudaEventDestroy(gen_done[k]);
        cudaEventDestroy(copy_done[k]);
    }
    cudaStreamDestroy(cp);
    return rc;
}

// Times candidate configurations on the given requests. Instance states are
// saved first and restored after every trial, so tuning does not advance
// any stream.
int rsaprng_autotune(rsaprng_ctx *c, uint64_t nreq, const rsaprng_id *ids, const uint64_t *counts,
                     int reps, rsaprng_config *chosen)
{
    if (!c || !nreq || !ids || !counts)
        return fail(RSAPRNG_ERR_ARG, "autotune: bad arguments");
    if (reps < 1)
        reps = 1;
    cudaSetDevice(c->device);
    std::vector<uint64_t> offs(nreq);
    uint64_t total = 0;
    for (uint64_t i = 0; i < nreq; i++) {
        offs[i] = total;
        total += counts[i];
    }
    double *d_r = nullptr;
    uint64_t *save = nullptr;
    cudaError_t e = cudaMalloc(&d_r, std::max<uint64_t>(total, 1) * 8);
    if (e != cudaSuccess)
        return fail(RSAPRNG_ERR_OOM, "autotune output (%llu numbers)", (unsigned long long)total);
    e = cudaMalloc(&save, c->count * 16);
    if (e != cudaSuccess) {
        cudaFree(d_r);
        return fail(RSAPRNG_ERR_OOM, "autotune state copy");
    }
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaMemcpyAsync(save, c->d_m, c->count * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(save + c->count, c->d_s, c->count * 8, cudaMemcpyDeviceToDevice, st);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto trial = [&](const rsaprng_config &cfg, float *ms) -> int {
        rsaprng_plan *p = nullptr;
        int rc = plan_create_cfg(c, cfg, nreq, ids, counts, offs.data(), &p);
        if (rc)
            return rc;
        rc = launch_plan(c, cfg, p->dp, d_r, nullptr, st, nullptr);  // warm-up
        cudaEventRecord(a, st);
        for (int r = 0; r < reps && rc == RSAPRNG_OK; r++)
            rc = launch_plan(c, cfg, p->dp, d_r, nullptr, st, nullptr);
        cudaEventRecord(b, st);
        cudaError_t ee = cudaEventSynchronize(b);
        cudaEventElapsedTime(ms, a, b);
        cudaMemcpyAsync(c->d_m, save, c->count * 8, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(c->d_s, save + c->count, c->count * 8, cudaMemcpyDeviceToDevice, st);
        cudaStreamSynchronize(st);
        rsaprng_plan_destroy(p);
        if (rc == RSAPRNG_OK && ee != cudaSuccess)
            rc = cuda_fail(ee, "autotune trial");
        return rc;
    };
    rsaprng_config best = c->cfg;
    float best_ms = 1e30f;
    int rc = RSAPRNG_OK;
    // Stage 1: routes at the default tiling. Stage 2: tilings for the best route.
    const int routes[5][2] = {{RSAPRNG_MODEXP_CRT32, RSAPRNG_DIVIDE_INT},
                              {RSAPRNG_MODEXP_CRT32, RSAPRNG_DIVIDE_HYBRID},
                              {RSAPRNG_MODEXP_CRT32, RSAPRNG_DIVIDE_RECIP},
                              {RSAPRNG_MODEXP_MONT64, RSAPRNG_DIVIDE_INT},
                              {RSAPRNG_MODEXP_MONT64, RSAPRNG_DIVIDE_HYBRID}};
    // Instances with CRT exponents run only on the CRT route.
    bool one_exponent = true;
    for (uint64_t i = 0; i < nreq; i++)
        if (ids[i] < c->count && c->h_params[ids[i]].e != c->h_params[ids[i]].eq)
            one_exponent = false;
    for (auto &rt : routes) {
        if (rt[0] == RSAPRNG_MODEXP_MONT64 && !one_exponent)
            continue;
        rsaprng_config cfg = c->cfg;
        if (rt[0] == RSAPRNG_MODEXP_MONT64 && cfg.numbers_per_thread == 16)
            cfg.numbers_per_thread = 8;
        cfg.modexp = rt[0];
        cfg.divide = rt[1];
        float ms;
        if ((rc = trial(cfg, &ms)) != RSAPRNG_OK)
            break;
        if (ms < best_ms) {
            best_ms = ms;
            best = cfg;
        }
    }
    // A candidate replaces the best only when it is faster by more than
    // `margin` (timing noise of a few percent must not move the later, finer
    // knobs away from their defaults).
    auto consider = [&](const rsaprng_config &cfg, float margin) {
        if (rc)
            return;
        float ms;
        if ((rc = trial(cfg, &ms)) != RSAPRNG_OK)
            return;
        if (ms < best_ms * (1.0f - margin)) {
            best_ms = ms;
            best = cfg;
        }
    };
    // Stage 2: tilings (threads per block, numbers per thread) for the best route.
    const int tiles[][2] = {{128, 4},  {128, 8}, {128, 16}, {256, 4}, {256, 8},
                            {256, 16}, {512, 2}, {512, 4},  {512, 8}};
    for (auto &tl : tiles) {
        if (tl[1] == 16 && best.modexp == RSAPRNG_MODEXP_MONT64)
            continue;
        rsaprng_config cfg = best;
        cfg.threads_per_block = tl[0];
        cfg.numbers_per_thread = tl[1];
        consider(cfg, 0.0f);
    }
    // Stage 3: unroll, the chains a thread runs at once (passes of half its numbers).
    {
        const GenLaunch g = ctx_launch(c, best, ~0ULL, true, false);
        if (g.L >= 4 && gen_has_unroll(g.L, g.modexp, g.divide, g.L / 2)) {
            rsaprng_config cfg = best;
            cfg.unroll = g.L / 2;
            consider(cfg, 0.02f);
        }
    }
    // Stage 4: streams per block (instances side by side, whole warps each).
    for (int spb : {2, 4}) {
        if (best.threads_per_block / spb < 32)
            continue;
        rsaprng_config cfg = best;
        cfg.streams_per_block = spb;
        consider(cfg, 0.02f);
    }
    // Stage 5: resident blocks per SM below the occupancy limit.
    {
        int occ = 0;
        (void)ctx_launch(c, best, ~0ULL, true, false, &occ);
        for (int k = 1; k <= 2 && occ - k >= 1; k++) {
            rsaprng_config cfg = best;
            cfg.blocks_per_sm = occ - k;
            consider(cfg, 0.02f);
        }
    }
    // Stage 6: pieces per resident block (load balance against skip-sum work).
    for (int ppb : {2, 4}) {
        rsaprng_config cfg = best;
        cfg.pieces_per_block = ppb;
        consider(cfg, 0.02f);
    }
    // Stage 7: the chunk cap of long streams.
    for (uint64_t ch : {1ULL << 16, 1ULL << 17, 1ULL << 19, 1ULL << 20}) {
        if (ch == best.chunk)
            continue;
        rsaprng_config cfg = best;
        cfg.chunk = ch;
        consider(cfg, 0.02f);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(st);
    cudaFree(save);
    cudaFree(d_r);
    if (rc)
        return rc;
    c->cfg = best;
    if (chosen)
        *chosen = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(c, nreq, ids, counts)] = best;
    return RSAPRNG_OK;
}

int rsaprng_autotune_cached(rsaprng_ctx *c, uint64_t nreq, const rsaprng_id *ids,
                            const uint64_t *counts, int reps, rsaprng_config *chosen,
                            int *from_cache)
{
    if (!c || !nreq || !ids || !counts)
        return fail(RSAPRNG_ERR_ARG, "autotune: bad arguments");
    if (from_cache)
        *from_cache = 0;
    const std::string key = tune_key(c, nreq, ids, counts);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            rsaprng_config cfg = it->second;
            // keep the context's own switches; take the tuned knobs
            cfg.require_safe = c->cfg.require_safe;
            cfg.lookback = c->cfg.lookback;
            cfg.spin_limit = c->cfg.spin_limit;
            cfg.test_flags = c->cfg.test_flags;
            c->cfg = cfg;
            if (chosen)
                *chosen = cfg;
            if (from_cache)
                *from_cache = 1;
            return RSAPRNG_OK;
        }
    }
    return rsaprng_autotune(c, nreq, ids, counts, reps, chosen);
}

uint64_t rsaprng_autotune_cache_size(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune_cache.size();
}

void rsaprng_autotune_cache_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
}

// One line per entry: the key, then the tuned knobs as name=value pairs.
int rsaprng_autotune_cache_save(const char *path)
{
    if (!path)
        return fail(RSAPRNG_ERR_ARG, "autotune cache: null path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE *f = fopen(path, "w");
    if (!f)
        return fail(RSAPRNG_ERR_ARG, "autotune cache: cannot write %s", path);
    for (const auto &kv : g_tune_cache) {
        const rsaprng_config &k = kv.second;
        fprintf(f, "%s modexp=%d divide=%d threads=%d numbers=%d blocks_per_sm=%d chunk=%llu "
                   "streams_per_block=%d unroll=%d pieces_per_block=%d rounding=%d\n",
                kv.first.c_str(), k.modexp, k.divide, k.threads_per_block, k.numbers_per_thread,
                k.blocks_per_sm, (unsigned long long)k.chunk, k.streams_per_block, k.unroll,
                k.pieces_per_block, k.rounding);
    }
    const bool ok = fclose(f) == 0;
    return ok ? RSAPRNG_OK : fail(RSAPRNG_ERR_ARG, "autotune cache: write failed");
}

int rsaprng_autotune_cache_load(const char *path)
{
    if (!path)
        return fail(RSAPRNG_ERR_ARG, "autotune cache: null path");
    FILE *f = fopen(path, "r");
    if (!f)
        return fail(RSAPRNG_ERR_ARG, "autotune cache: cannot read %s", path);
    std::map<std::string, rsaprng_config> got;
    char key[256];
    int modexp, divide, threads, numbers, bps, spb, unroll, ppb, rounding;
    unsigned long long chunk;
    int rc = RSAPRNG_OK;
    for (;;) {
        const int n = fscanf(f, "%255s modexp=%d divide=%d threads=%d numbers=%d blocks_per_sm=%d "
                                "chunk=%llu streams_per_block=%d unroll=%d pieces_per_block=%d "
                                "rounding=%d",
                             key, &modexp, &divide, &threads, &numbers, &bps, &chunk, &spb,
                             &unroll, &ppb, &rounding);
        if (n == EOF)
            break;
        if (n != 11) {
            rc = fail(RSAPRNG_ERR_ARG, "autotune cache: malformed line in %s", path);
            break;
        }
        rsaprng_config k{};
        k.struct_size = sizeof k;
        k.modexp = modexp;
        k.divide = divide;
        k.threads_per_block = threads;
        k.numbers_per_thread = numbers;
        k.blocks_per_sm = bps;
        k.chunk = chunk;
        k.streams_per_block = spb;
        k.unroll = unroll;
        k.pieces_per_block = ppb;
        k.rounding = rounding;
        got[key] = k;
    }
    fclose(f);
    if (rc)
        return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : got)
        g_tune_cache[kv.first] = kv.second;
    return RSAPRNG_OK;
}

}  // extern "C"
