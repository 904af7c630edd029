// Host runtime and C ABI of the generator library (declarations and the
// meaning of every call are in include/rsaprng.h).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rsaprng.h"
#include "api_internal.hpp"
#include "host_params.hpp"
#include "kernels.cuh"

using namespace rsaprng;

namespace rsaprng {

thread_local std::string g_detail;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_detail = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(RSAPRNG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static const rsaprng_config kDefaultConfig = {
    sizeof(rsaprng_config), RSAPRNG_MODEXP_CRT32, RSAPRNG_DIVIDE_RECIP, 128, 16, 0, 1ULL << 18, 0,
    RSAPRNG_ROUND_DEFAULT, RSAPRNG_LOOKBACK_AUTO, 0, 0, 1, 0, 1};

static int check_config(const rsaprng_config &c)
{
    if (c.modexp < 0 || c.modexp > 2 || c.divide < 0 || c.divide > 4)
        return fail(RSAPRNG_ERR_ARG, "config: modexp/divide out of range");
    if (c.threads_per_block && c.threads_per_block != 64 && c.threads_per_block != 128 &&
        c.threads_per_block != 256 && c.threads_per_block != 512)
        return fail(RSAPRNG_ERR_ARG, "config: threads_per_block must be 64, 128, 256 or 512");
    if (c.numbers_per_thread && c.numbers_per_thread != 2 && c.numbers_per_thread != 4 &&
        c.numbers_per_thread != 8 && c.numbers_per_thread != 16)
        return fail(RSAPRNG_ERR_ARG, "config: numbers_per_thread must be 2, 4, 8 or 16");
    if (c.blocks_per_sm < 0 || c.blocks_per_sm > 32)
        return fail(RSAPRNG_ERR_ARG, "config: blocks_per_sm out of range");
    if (c.rounding < 0 || c.rounding > RSAPRNG_ROUND_EXACT)
        return fail(RSAPRNG_ERR_ARG, "config: rounding out of range");
    if (c.lookback < 0 || c.lookback > RSAPRNG_LOOKBACK_CONFIGURED)
        return fail(RSAPRNG_ERR_ARG, "config: lookback out of range");
    if (c.streams_per_block < 0 || c.streams_per_block > 16 ||
        (c.streams_per_block & (c.streams_per_block - 1)))
        return fail(RSAPRNG_ERR_ARG, "config: streams_per_block must be 0, 1, 2, 4, 8 or 16");
    if (c.threads_per_block && c.streams_per_block > 1 &&
        c.threads_per_block / c.streams_per_block < 32)
        return fail(RSAPRNG_ERR_ARG, "config: streams_per_block leaves a stream less than a warp");
    if (c.unroll < 0 || c.unroll > 16 || (c.unroll & (c.unroll - 1)))
        return fail(RSAPRNG_ERR_ARG, "config: unroll must be 0, 1, 2, 4, 8 or 16");
    if (c.pieces_per_block < 0 || c.pieces_per_block > 64)
        return fail(RSAPRNG_ERR_ARG, "config: pieces_per_block out of range");
    return RSAPRNG_OK;
}

static rsaprng_config merged(const rsaprng_config &base, const rsaprng_config *over)
{
    rsaprng_config c = base;
    if (!over)
        return c;
    if (over->modexp)
        c.modexp = over->modexp;
    if (over->divide)
        c.divide = over->divide;
    if (over->threads_per_block)
        c.threads_per_block = over->threads_per_block;
    if (over->numbers_per_thread)
        c.numbers_per_thread = over->numbers_per_thread;
    if (over->blocks_per_sm)
        c.blocks_per_sm = over->blocks_per_sm;
    if (over->chunk)
        c.chunk = over->chunk;
    c.require_safe = over->require_safe;
    if (over->rounding)
        c.rounding = over->rounding;
    if (over->streams_per_block)
        c.streams_per_block = over->streams_per_block;
    if (over->unroll)
        c.unroll = over->unroll;
    if (over->pieces_per_block)
        c.pieces_per_block = over->pieces_per_block;
    c.lookback = over->lookback;
    c.spin_limit = over->spin_limit;
    c.test_flags = over->test_flags;
    return c;
}

DeviceTables ctx_tables(rsaprng_ctx *c)
{
    DeviceTables t;
    t.params = c->d_params;
    t.state_m = c->d_m;
    t.state_s = c->d_s;
    t.pow_lin = c->d_pow_lin;
    t.pow2k = c->d_pow2k;
    return t;
}

GenLaunch ctx_launch(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nitems, bool want_r,
                     bool want_c, int *occupancy)
{
    GenLaunch g;
    g.stride = 1;
    g.threads = cfg.threads_per_block;
    g.L = cfg.numbers_per_thread;
    g.modexp = cfg.modexp == RSAPRNG_MODEXP_MONT64 ? MODEXP_MONT64 : MODEXP_CRT32;
    if (g.modexp == MODEXP_MONT64 && g.L > 8)
        g.L = 8;  // the 64-bit route has no 16-output tiling (register budget)
    g.divide = cfg.rounding == RSAPRNG_ROUND_EXACT   ? DIVIDE_EXACT
               : cfg.divide == RSAPRNG_DIVIDE_FP64   ? DIVIDE_FP64
               : cfg.divide == RSAPRNG_DIVIDE_HYBRID ? DIVIDE_HYBRID
               : cfg.divide == RSAPRNG_DIVIDE_RECIP  ? DIVIDE_RECIP
                                                     : DIVIDE_INT;
    g.unroll = cfg.unroll > 0 && cfg.unroll < g.L ? cfg.unroll : 0;
    if (g.unroll && !gen_has_unroll(g.L, g.modexp, g.divide, g.unroll))
        g.unroll = 0;  // no pass-limited variant: all chains at once
    const size_t smem = gen_smem_bytes(g.threads, g.L, want_r, want_c);
    // Occupancy queries cost microseconds; cache them per kernel and smem size.
    const int ti = g.threads == 64 ? 0 : (g.threads == 128 ? 1 : (g.threads == 256 ? 2 : 3));
    const int li = g.L == 2 ? 0 : (g.L == 4 ? 1 : (g.L == 8 ? 2 : 3));
    const int ui = g.unroll ? 1 : 0;
    int &cached = c->occ_cache[ti][li][g.modexp - 1][g.divide - 1][ui];
    size_t &cached_smem = c->occ_smem[ti][li][g.modexp - 1][g.divide - 1][ui];
    int occ;
    if (cached > 0 && cached_smem == smem) {
        occ = cached;
    } else {
        occ = gen_blocks_per_sm(g, smem);
        cached = occ;
        cached_smem = smem;
    }
    if (occ < 1)
        occ = 1;
    if (occupancy)
        *occupancy = occ;
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < occ)
        occ = cfg.blocks_per_sm;
    const uint64_t resident = (uint64_t)occ * c->sms;
    if (nitems <= resident) {
        g.grid = (int)std::max<uint64_t>(nitems, 1);
        g.persistent = false;
    } else {
        g.grid = (int)resident;
        g.persistent = true;
    }
    return g;
}

static GenLaunch vec_launch(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nvecs, bool want_r,
                            bool want_c, bool packed);

int build_plan(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nreq, const rsaprng_id *ids,
               const uint64_t *counts, const uint64_t *offsets, uint64_t chunk, HostPlan &hp,
               uint64_t tuple, uint64_t stride, bool allow_pack)
{
    // The pieces are sized for the resident blocks and the tiles of the
    // kernel that runs the plan: the vector kernel for the interleaved order
    // and for several streams per block, else the generation kernel.
    const uint64_t pack = allow_pack && stride == 1 && tuple == 1 && cfg.streams_per_block > 1
                              ? (uint64_t)cfg.streams_per_block
                              : 1;
    const GenLaunch full = (stride > 1 || pack > 1)
                               ? vec_launch(c, cfg, ~0ULL, true, false, pack > 1)
                               : ctx_launch(c, cfg, ~0ULL, true, false);
    const PlanGeometry geo{(uint64_t)full.threads, (uint64_t)full.L, (uint64_t)full.grid,
                           (uint64_t)std::max(1, cfg.pieces_per_block)};
    return build_plan_core(c->h_params.data(), c->count, cfg.modexp, geo, nreq, ids, counts,
                           offsets, chunk, hp, tuple, stride, pack);
}

static int grow(void **p, size_t *cap, size_t need)
{
    if (need <= *cap)
        return RSAPRNG_OK;
    size_t n = std::max(need, *cap * 2);
    if (*p)
        cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess)
        return fail(RSAPRNG_ERR_OOM, "cudaMalloc(%zu): %s", n, cudaGetErrorString(e));
    *cap = n;
    return RSAPRNG_OK;
}

static int grow_host(void **p, size_t *cap, size_t need)
{
    if (need <= *cap)
        return RSAPRNG_OK;
    size_t n = std::max(need, *cap * 2);
    if (*p)
        cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMallocHost(p, n);
    if (e != cudaSuccess)
        return fail(RSAPRNG_ERR_OOM, "cudaMallocHost(%zu): %s", n, cudaGetErrorString(e));
    *cap = n;
    return RSAPRNG_OK;
}

// Uploads a host plan into device buffers (through pinned staging) and
// records the launch layout. The buffers are reused; the caller guarantees
// that no earlier launch using them is still pending.
int upload_plan(rsaprng_ctx *c, const HostPlan &hp, DevPlan &dp, cudaStream_t stream)
{
    const size_t b_items = hp.items.size() * sizeof(WorkItem);
    const size_t b_chunks = hp.chunks.size() * sizeof(PrepChunk);
    const size_t b_groups = hp.groups.size() * sizeof(PrepGroup);
    const size_t b_vecs = hp.vecs.size() * sizeof(VecGroup);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t total = al(b_items) + al(b_chunks) + al(b_groups) + al(b_vecs) + 256;
    int rc;
    if ((rc = grow(&dp.d_buf, &dp.cap_buf, total)) != RSAPRNG_OK)
        return rc;
    if ((rc = grow_host(&dp.h_buf, &dp.cap_host, total)) != RSAPRNG_OK)
        return rc;
    const size_t b_sums = hp.chunks.size() * 8 * 2;
    if ((rc = grow(&dp.d_sums, &dp.cap_sums, std::max<size_t>(b_sums, 256))) != RSAPRNG_OK)
        return rc;
    char *h = (char *)dp.h_buf;
    char *d = (char *)dp.d_buf;
    size_t o = 0;
    dp.items = (WorkItem *)(d + o);
    memcpy(h + o, hp.items.data(), b_items);
    o += al(b_items);
    dp.chunks = (PrepChunk *)(d + o);
    memcpy(h + o, hp.chunks.data(), b_chunks);
    o += al(b_chunks);
    dp.groups = (PrepGroup *)(d + o);
    memcpy(h + o, hp.groups.data(), b_groups);
    o += al(b_groups);
    dp.vecs = (VecGroup *)(d + o);
    memcpy(h + o, hp.vecs.data(), b_vecs);
    o += al(b_vecs);
    dp.ticket = (uint32_t *)(d + o);
    memset(h + o, 0, 256);
    o += 256;
    dp.chunk_sum = (uint64_t *)dp.d_sums;
    dp.chunk_s = (uint64_t *)dp.d_sums + hp.chunks.size();
    dp.nitems = (uint32_t)hp.items.size();
    dp.nchunks = (uint32_t)hp.chunks.size();
    dp.ngroups = (uint32_t)hp.groups.size();
    dp.numbers = hp.numbers;
    dp.extent = hp.extent;
    dp.unaligned = hp.unaligned;
    dp.stride = hp.stride;
    dp.nvecs = (uint32_t)hp.vecs.size();
    dp.vec_ts = hp.vec_ts;
    cudaError_t e = cudaMemcpyAsync(dp.d_buf, dp.h_buf, o, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "plan upload");
    c->h2d_bytes += o;
    return RSAPRNG_OK;
}

// Launch shape of the vector kernel (interleaved order) for cfg.
static GenLaunch vec_launch(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nvecs, bool want_r,
                            bool want_c, bool packed)
{
    GenLaunch g = ctx_launch(c, cfg, nvecs, want_r, want_c);
    g.L_wide = g.L;
    g.L = vec_numbers_per_thread(g.L, g.modexp, g.threads);
    g.stride = packed ? 1 : 2;  // selects the packed or the interleaved kernel
    int occ = vec_blocks_per_sm(g, vec_smem_bytes(g.threads, g.L, want_r, want_c));
    if (occ < 1)
        occ = 1;
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < occ)
        occ = cfg.blocks_per_sm;
    const uint64_t resident = (uint64_t)occ * c->sms;
    g.persistent = nvecs > resident;
    g.grid = (int)(g.persistent ? resident : std::max<uint64_t>(nvecs, 1));
    return g;
}

// Launch shape of the histogram consumer for cfg (its own occupancy).
static GenLaunch hist_launch(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nitems)
{
    GenLaunch g = ctx_launch(c, cfg, nitems, true, false);
    int occ = hist_blocks_per_sm(g);
    if (occ < 1)
        occ = 1;
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < occ)
        occ = cfg.blocks_per_sm;
    const uint64_t resident = (uint64_t)occ * c->sms;
    g.persistent = nitems > resident;
    g.grid = (int)(g.persistent ? resident : std::max<uint64_t>(nitems, 1));
    return g;
}

int launch_plan(rsaprng_ctx *c, const rsaprng_config &cfg, DevPlan &dp, double *d_r,
                uint64_t *d_c, cudaStream_t stream, uint64_t *launches, const HistArgs *hist,
                bool fresh, const cudaEvent_t *gen_events)
{
    const DeviceTables t = ctx_tables(c);
    uint64_t nl = 0;
    cudaError_t e;
    const bool vec = !hist && dp.nvecs;  // interleaved order, or packed streams
    GenLaunch g{};
    if (dp.nitems) {
        g = hist  ? hist_launch(c, cfg, dp.nitems)
            : vec ? vec_launch(c, cfg, dp.nvecs, d_r != nullptr, d_c != nullptr, dp.stride == 1)
                  : ctx_launch(c, cfg, dp.nitems, d_r != nullptr, d_c != nullptr, &dp.occupancy);
        g.stride = dp.stride;
        g.out_extent = dp.extent;
        g.out_unaligned = dp.unaligned;
        g.pdl = dp.nchunks > 0;
        dp.last = g;
        // A persistent launch's ticket is reset before the pre-pass, so that the
        // kernels follow one another directly (each a programmatic dependent of
        // the one before).
        if (g.persistent && !fresh) {
            if ((e = cudaMemsetAsync(dp.ticket, 0, sizeof(uint32_t), stream)) != cudaSuccess)
                return cuda_fail(e, "ticket reset");
        }
    }
    if (dp.nchunks) {
        if ((e = launch_prep_sums(t, dp.chunks, dp.nchunks, dp.chunk_sum, dp.chunk_s, stream)) !=
            cudaSuccess)
            return cuda_fail(e, "prep sums launch");
        if ((e = launch_prep_scan(t, dp.groups, dp.ngroups, dp.chunks, dp.chunk_sum, dp.chunk_s,
                                  dp.items, stream)) != cudaSuccess)
            return cuda_fail(e, "prep scan launch");
        nl += 2;
    }
    if (dp.nitems) {
        // An event between the scan and the generation kernel makes the
        // latter an ordinary launch (its griddepcontrol.wait returns at once).
        if (gen_events && (e = cudaEventRecord(gen_events[0], stream)) != cudaSuccess)
            return cuda_fail(e, "timing event");
        if (hist)
            e = launch_histogram(g, t, dp.items, dp.nitems, dp.ticket, *hist, stream);
        else if (vec)
            e = launch_generate_vec(g, t, dp.items, dp.vecs, dp.nvecs, dp.ticket, d_r, d_c,
                                    dp.vec_ts, stream);
        else
            e = launch_generate(g, t, dp.items, dp.nitems, dp.ticket, d_r, d_c, stream);
        if (e != cudaSuccess)
            return cuda_fail(e, hist ? "histogram launch" : "generate launch");
        if (gen_events && (e = cudaEventRecord(gen_events[1], stream)) != cudaSuccess)
            return cuda_fail(e, "timing event");
        nl += 1;
    }
    c->launches += nl;
    if (launches)
        *launches = nl;
    return RSAPRNG_OK;
}

void free_devplan(DevPlan &dp)
{
    if (dp.d_buf)
        cudaFree(dp.d_buf);
    if (dp.d_sums)
        cudaFree(dp.d_sums);
    if (dp.h_buf)
        cudaFreeHost(dp.h_buf);
    if (dp.d_lb)
        cudaFree(dp.d_lb);
    dp = DevPlan{};
}

// Scratch plan slots for one-off generate calls: slot k is reused only after
// the event recorded behind its last launch has completed.
int scratch_slot(rsaprng_ctx *c, ScratchSlot **out)
{
    ScratchSlot &s = c->slots[c->next_slot];
    c->next_slot = (c->next_slot + 1) % kScratchSlots;
    if (s.used) {
        cudaError_t e = cudaEventSynchronize(s.done);
        if (e != cudaSuccess)
            return cuda_fail(e, "scratch slot wait");
    }
    *out = &s;
    return RSAPRNG_OK;
}

}  // namespace rsaprng

namespace rsaprng {
// Runs f(i) for i in [0, count) over all host cores.
template <typename F>
static void parallel_for(uint64_t count, F &&f)
{
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    if (count < 4096 || nt == 1) {
        for (uint64_t i = 0; i < count; i++)
            f(i);
        return;
    }
    std::atomic<uint64_t> next{0};
    std::vector<std::thread> th;
    for (unsigned k = 0; k < nt; k++)
        th.emplace_back([&] {
            for (;;) {
                uint64_t i0 = next.fetch_add(1024);
                if (i0 >= count)
                    break;
                uint64_t i1 = std::min(count, i0 + 1024);
                for (uint64_t i = i0; i < i1; i++)
                    f(i);
            }
        });
    for (auto &x : th)
        x.join();
}

}  // namespace rsaprng

// ============================================================ C ABI

extern "C" {

const char *rsaprng_strerror(int code)
{
    switch (code) {
    case RSAPRNG_OK: return "ok";
    case RSAPRNG_ERR_ARG: return "invalid argument";
    case RSAPRNG_ERR_NOT_PRIME: return "p or q is not prime";
    case RSAPRNG_ERR_RANGE: return "p or q outside [2^31, 2^32)";
    case RSAPRNG_ERR_P_EQ_Q: return "p equals q";
    case RSAPRNG_ERR_E: return "invalid exponent e";
    case RSAPRNG_ERR_ROOT: return "skip multiplier not allowed (or a constant skip split)";
    case RSAPRNG_ERR_OOM: return "out of memory";
    case RSAPRNG_ERR_BUDGET: return "request exceeds the output budget";
    case RSAPRNG_ERR_CUDA: return "CUDA error";
    case RSAPRNG_ERR_TIMEOUT: return "timed out";
    case RSAPRNG_ERR_DEVICE_FLAG: return "device error flag raised";
    case RSAPRNG_ERR_CAPACITY: return "instance table full";
    case RSAPRNG_ERR_CANCELLED: return "request cancelled";
    case RSAPRNG_ERR_STATE: return "state outside its range";
    case RSAPRNG_ERR_ID: return "unknown id";
    case RSAPRNG_ERR_BUSY: return "queue full";
    default: return "unknown error";
    }
}

const char *rsaprng_last_error_detail(void) { return g_detail.c_str(); }

int rsaprng_is_prime(uint64_t x) { return rsaprng::is_prime(x) ? 1 : 0; }

int rsaprng_root_allowed(uint64_t a) { return root_index(a) >= 0 ? 1 : 0; }

int rsaprng_validate_params(uint64_t p, uint64_t q, uint64_t e, int require_safe)
{
    return validate_pqe(p, q, e, require_safe != 0);
}

int rsaprng_params_from_seed(uint64_t seed, int e_rule, uint64_t e_lo, uint64_t e_hi,
                             uint64_t *p, uint64_t *q, uint64_t *e, uint64_t *msg_seed)
{
    if (!p || !q || !e || !msg_seed)
        return fail(RSAPRNG_ERR_ARG, "null output pointer");
    return rsaprng::params_from_seed(seed, e_rule, e_lo, e_hi, *p, *q, *e, *msg_seed);
}

int rsaprng_ctx_create(rsaprng_ctx **out, int device, uint64_t max_instances,
                       const rsaprng_config *cfg)
{
    if (!out || max_instances == 0 || max_instances > 0xFFFFFFF0ULL)
        return fail(RSAPRNG_ERR_ARG, "ctx_create: bad arguments");
    *out = nullptr;
    rsaprng_config conf = merged(kDefaultConfig, cfg);
    int rc = check_config(conf);
    if (rc)
        return rc;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaSetDevice");
    rsaprng_ctx *c = new (std::nothrow) rsaprng_ctx();
    if (!c)
        return fail(RSAPRNG_ERR_OOM, "ctx alloc");
    c->device = device;
    c->cfg = conf;
    c->capacity = max_instances;
    memset(c->occ_cache, 0, sizeof c->occ_cache);
    memset(c->occ_smem, 0, sizeof c->occ_smem);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    auto cleanup = [&](int code) {
        rsaprng_ctx_destroy(c);
        return code;
    };
    if ((e = cudaMalloc(&c->d_params, max_instances * sizeof(InstParams))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_m, max_instances * 8)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_s, max_instances * 8)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_pow_lin, (size_t)kNumRoots * kPowLinRow * 8)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_pow2k, (size_t)kNumRoots * 64 * 8)) != cudaSuccess)
        return cleanup(fail(RSAPRNG_ERR_OOM, "device tables: %s", cudaGetErrorString(e)));
    // Power tables of every allowed root: a^i (i <= kMaxTile) and a^(2^b).
    std::vector<uint64_t> lin((size_t)kNumRoots * kPowLinRow), p2((size_t)kNumRoots * 64);
    for (int r = 0; r < kNumRoots; r++) {
        uint64_t x = 1;
        for (int i = 0; i < kPowLinRow; i++) {
            lin[(size_t)r * kPowLinRow + i] = x;
            x = mulmod(x, kRoots[r], kQ);
        }
        uint64_t y = kRoots[r];
        for (int b = 0; b < 64; b++) {
            p2[(size_t)r * 64 + b] = y;
            y = mulmod(y, y, kQ);
        }
    }
    if ((e = cudaMemcpy(c->d_pow_lin, lin.data(), lin.size() * 8, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(c->d_pow2k, p2.data(), p2.size() * 8, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return cleanup(cuda_fail(e, "power tables"));
    for (auto &s : c->slots) {
        if ((e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess)
            return cleanup(cuda_fail(e, "event create"));
    }
    *out = c;
    return RSAPRNG_OK;
}

void rsaprng_ctx_destroy(rsaprng_ctx *c)
{
    if (!c)
        return;
    cudaSetDevice(c->device);
    for (auto &s : c->slots) {
        if (s.used)
            cudaEventSynchronize(s.done);
        free_devplan(s.plan);
        if (s.done)
            cudaEventDestroy(s.done);
    }
    if (c->d_params)
        cudaFree(c->d_params);
    if (c->d_m)
        cudaFree(c->d_m);
    if (c->d_s)
        cudaFree(c->d_s);
    if (c->d_pow_lin)
        cudaFree(c->d_pow_lin);
    if (c->d_pow2k)
        cudaFree(c->d_pow2k);
    if (c->d_out_scratch)
        cudaFree(c->d_out_scratch);
    if (c->d_err)
        cudaFree(c->d_err);
    delete c;
}

int rsaprng_ctx_configure(rsaprng_ctx *c, const rsaprng_config *cfg)
{
    if (!c || !cfg)
        return fail(RSAPRNG_ERR_ARG, "null");
    rsaprng_config conf = merged(c->cfg, cfg);
    int rc = check_config(conf);
    if (rc)
        return rc;
    c->cfg = conf;
    return RSAPRNG_OK;
}

int rsaprng_ctx_get_config(const rsaprng_ctx *c, rsaprng_config *out)
{
    if (!c || !out)
        return fail(RSAPRNG_ERR_ARG, "null");
    *out = c->cfg;
    return RSAPRNG_OK;
}

uint64_t rsaprng_instance_count(const rsaprng_ctx *c) { return c ? c->count : 0; }

uint64_t rsaprng_launch_count(const rsaprng_ctx *c) { return c ? c->launches : 0; }

int rsaprng_transfer_bytes(const rsaprng_ctx *c, uint64_t *h2d, uint64_t *d2h)
{
    if (!c)
        return fail(RSAPRNG_ERR_ARG, "null");
    if (h2d)
        *h2d = c->h2d_bytes;
    if (d2h)
        *d2h = c->d2h_bytes;
    return RSAPRNG_OK;
}

// Appends validated instances [count .. count+k) and writes them to the device.
static int append_instances(rsaprng_ctx *c, const std::vector<InstParams> &ps,
                            const std::vector<uint64_t> &m0, const std::vector<uint64_t> &s0,
                            rsaprng_id *out_first)
{
    const uint64_t k = ps.size();
    if (c->count + k > c->capacity)
        return fail(RSAPRNG_ERR_CAPACITY, "instance table full (%llu of %llu)",
                    (unsigned long long)c->count, (unsigned long long)c->capacity);
    cudaSetDevice(c->device);
    cudaError_t e;
    if ((e = cudaMemcpy(c->d_params + c->count, ps.data(), k * sizeof(InstParams),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_m + c->count, m0.data(), k * 8, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(c->d_s + c->count, s0.data(), k * 8, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return cuda_fail(e, "instance upload");
    c->h_params.insert(c->h_params.end(), ps.begin(), ps.end());
    if (out_first)
        *out_first = (rsaprng_id)c->count;
    c->count += k;
    return RSAPRNG_OK;
}

int rsaprng_instance_create_ex(rsaprng_ctx *c, uint64_t p, uint64_t q, uint64_t e, uint64_t a,
                               uint64_t m0, uint64_t s0, rsaprng_id *out)
{
    if (!c)
        return fail(RSAPRNG_ERR_ARG, "null ctx");
    int rc = validate_pqe(p, q, e, c->cfg.require_safe != 0);
    if (rc)
        return fail(rc, "instance (p=%llu, q=%llu, e=%llu): %s", (unsigned long long)p,
                    (unsigned long long)q, (unsigned long long)e, rsaprng_strerror(rc));
    if (root_index(a) < 0)
        return fail(RSAPRNG_ERR_ROOT, "a=%llu is not an allowed root", (unsigned long long)a);
    if (m0 >= p * q || s0 == 0 || s0 >= kQ)
        return fail(RSAPRNG_ERR_STATE, "start state out of range");
    std::vector<InstParams> ps(1);
    make_params(p, q, e, a, ps[0]);
    return append_instances(c, ps, {m0}, {s0}, out);
}

int rsaprng_instance_create_crt(rsaprng_ctx *c, uint64_t p, uint64_t q, uint64_t e_p,
                                uint64_t e_q, uint64_t a, uint64_t m0, uint64_t s0,
                                rsaprng_id *out)
{
    if (!c)
        return fail(RSAPRNG_ERR_ARG, "null ctx");
    int rc = validate_crt_exponents(p, q, e_p, e_q, c->cfg.require_safe != 0);
    if (rc)
        return fail(rc, "instance (p=%llu, q=%llu, e_p=%llu, e_q=%llu): %s",
                    (unsigned long long)p, (unsigned long long)q, (unsigned long long)e_p,
                    (unsigned long long)e_q, rsaprng_strerror(rc));
    if (root_index(a) < 0)
        return fail(RSAPRNG_ERR_ROOT, "a=%llu is not an allowed multiplier", (unsigned long long)a);
    if (m0 >= p * q || s0 == 0 || s0 >= kQ)
        return fail(RSAPRNG_ERR_STATE, "start state out of range");
    std::vector<InstParams> ps(1);
    make_params(p, q, e_p, a, ps[0], e_q);
    return append_instances(c, ps, {m0}, {s0}, out);
}

int rsaprng_get_exponents(const rsaprng_ctx *c, rsaprng_id id, uint64_t *e_p, uint64_t *e_q)
{
    if (!c || !e_p || !e_q)
        return fail(RSAPRNG_ERR_ARG, "get_exponents: null argument");
    if (id >= c->count)
        return fail(RSAPRNG_ERR_ID, "unknown id %u", id);
    *e_p = c->h_params[id].e;
    *e_q = c->h_params[id].eq;
    return RSAPRNG_OK;
}

int rsaprng_instance_create(rsaprng_ctx *c, uint64_t p, uint64_t q, uint64_t e, uint64_t seed,
                            rsaprng_id *out)
{
    if (p == 0 || q == 0)
        return fail(RSAPRNG_ERR_RANGE, "p, q must be nonzero");
    return rsaprng_instance_create_ex(c, p, q, e, RSAPRNG_DEFAULT_ROOT, seed % (p * q), 1, out);
}

int rsaprng_instances_create_bulk(rsaprng_ctx *c, uint64_t count, const uint64_t *p,
                                  const uint64_t *q, const uint64_t *e, const uint64_t *seed,
                                  rsaprng_id *out_first)
{
    if (!c || (count && (!p || !q || !e || !seed)))
        return fail(RSAPRNG_ERR_ARG, "null argument");
    std::vector<InstParams> ps(count);
    std::vector<uint64_t> m0(count), s0(count, 1);
    std::vector<int> err(count, 0);
    const bool safe = c->cfg.require_safe != 0;
    parallel_for(count, [&](uint64_t i) {
        err[i] = validate_pqe(p[i], q[i], e[i], safe);
        if (!err[i]) {
            make_params(p[i], q[i], e[i], RSAPRNG_DEFAULT_ROOT, ps[i]);
            m0[i] = seed[i] % (p[i] * q[i]);
        }
    });
    for (uint64_t i = 0; i < count; i++)
        if (err[i])
            return fail(err[i], "entry %llu: %s", (unsigned long long)i, rsaprng_strerror(err[i]));
    return append_instances(c, ps, m0, s0, out_first);
}

int rsaprng_instances_create_seeded(rsaprng_ctx *c, uint64_t count, const uint64_t *seeds,
                                    int e_rule, uint64_t e_lo, uint64_t e_hi,
                                    rsaprng_id *out_first)
{
    if (!c || (count && !seeds))
        return fail(RSAPRNG_ERR_ARG, "null argument");
    std::vector<InstParams> ps(count);
    std::vector<uint64_t> m0(count), s0(count, 1);
    std::vector<int> err(count, 0);
    parallel_for(count, [&](uint64_t i) {
        uint64_t p, q, e, ms;
        err[i] = rsaprng::params_from_seed(seeds[i], e_rule, e_lo, e_hi, p, q, e, ms);
        if (!err[i]) {
            make_params(p, q, e, RSAPRNG_DEFAULT_ROOT, ps[i]);
            m0[i] = ms % (p * q);
        }
    });
    for (uint64_t i = 0; i < count; i++)
        if (err[i])
            return fail(err[i], "seed %llu: %s", (unsigned long long)i, rsaprng_strerror(err[i]));
    return append_instances(c, ps, m0, s0, out_first);
}

int rsaprng_get_state(rsaprng_ctx *c, rsaprng_id id, uint64_t *m, uint64_t *s)
{
    if (!c || !m || !s)
        return fail(RSAPRNG_ERR_ARG, "null");
    if (id >= c->count)
        return fail(RSAPRNG_ERR_ID, "unknown id %u", id);
    cudaSetDevice(c->device);
    cudaError_t e;
    if ((e = cudaMemcpy(m, c->d_m + id, 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(s, c->d_s + id, 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "get_state");
    return RSAPRNG_OK;
}

int rsaprng_set_state(rsaprng_ctx *c, rsaprng_id id, uint64_t m, uint64_t s)
{
    if (!c)
        return fail(RSAPRNG_ERR_ARG, "null");
    if (id >= c->count)
        return fail(RSAPRNG_ERR_ID, "unknown id %u", id);
    if (m >= c->h_params[id].n || s == 0 || s >= kQ)
        return fail(RSAPRNG_ERR_STATE, "state out of range");
    cudaSetDevice(c->device);
    cudaError_t e;
    if ((e = cudaMemcpy(c->d_m + id, &m, 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_s + id, &s, 8, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "set_state");
    return RSAPRNG_OK;
}

int rsaprng_get_params(rsaprng_ctx *c, rsaprng_id id, uint64_t *p, uint64_t *q, uint64_t *e,
                       uint64_t *a)
{
    if (!c)
        return fail(RSAPRNG_ERR_ARG, "null");
    if (id >= c->count)
        return fail(RSAPRNG_ERR_ID, "unknown id %u", id);
    const InstParams &P = c->h_params[id];
    if (p)
        *p = P.p;
    if (q)
        *q = P.q;
    if (e)
        *e = P.e;
    if (a)
        *a = P.a;
    return RSAPRNG_OK;
}

int rsaprng_split(rsaprng_ctx *c, rsaprng_id parent, uint32_t Mv, rsaprng_id *out_children)
{
    if (!c || !out_children || Mv == 0)
        return fail(RSAPRNG_ERR_ARG, "split: bad arguments");
    uint64_t m, s;
    int rc = rsaprng_get_state(c, parent, &m, &s);
    if (rc)
        return rc;
    const InstParams P = c->h_params[parent];
    if (P.a == 1)
        return fail(RSAPRNG_ERR_ROOT, "split: a constant skip (a = 1) has no jump-ahead");
    const uint64_t stride = (kQ - 1) / Mv;
    const uint64_t a_stride = powQ(P.a, stride);
    std::vector<InstParams> ps(Mv, P);
    std::vector<uint64_t> m0(Mv, m), s0(Mv);
    uint64_t x = s;
    for (uint32_t g = 0; g < Mv; g++) {
        s0[g] = x;  // s a^(g stride) mod Q
        x = mulmod(x, a_stride, kQ);
    }
    rsaprng_id first;
    rc = append_instances(c, ps, m0, s0, &first);
    if (rc)
        return rc;
    for (uint32_t g = 0; g < Mv; g++)
        out_children[g] = first + g;
    return RSAPRNG_OK;
}

int rsaprng_generate_batch(rsaprng_ctx *c, uint64_t nreq, const rsaprng_id *ids,
                           const uint64_t *counts, const uint64_t *out_offsets, double *d_r,
                           uint64_t *d_c, void *stream)
{
    if (!c || (nreq && (!ids || !counts || !out_offsets)))
        return fail(RSAPRNG_ERR_ARG, "generate_batch: null argument");
    if (!d_r && !d_c)
        return fail(RSAPRNG_ERR_ARG, "generate_batch: no output buffer");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    HostPlan &hp = c->hp_direct;
    int rc = build_plan(c, c->cfg, nreq, ids, counts, out_offsets, c->cfg.chunk, hp, 1, 1, true);
    if (rc)
        return rc;
    if (hp.items.empty())
        return RSAPRNG_OK;
    ScratchSlot *slot;
    if ((rc = scratch_slot(c, &slot)) != RSAPRNG_OK)
        return rc;
    if ((rc = upload_plan(c, hp, slot->plan, st)) != RSAPRNG_OK)
        return rc;
    rc = launch_plan(c, c->cfg, slot->plan, d_r, d_c, st, nullptr, nullptr, true);
    cudaEventRecord(slot->done, st);
    slot->used = true;
    return rc;
}

int rsaprng_generate_interleaved(rsaprng_ctx *c, uint64_t ngroups, uint32_t Mv,
                                 const rsaprng_id *ids, uint64_t N, double *d_r, uint64_t *d_c,
                                 void *stream)
{
    if (!c || Mv == 0 || (ngroups && !ids))
        return fail(RSAPRNG_ERR_ARG, "generate_interleaved: bad arguments");
    if (!d_r && !d_c)
        return fail(RSAPRNG_ERR_ARG, "generate_interleaved: no output buffer");
    const uint64_t k = ngroups * Mv;
    std::vector<rsaprng_id> sorted(ids, ids + k);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return fail(RSAPRNG_ERR_ARG, "generate_interleaved: an instance appears twice");
    if (N == 0 || k == 0)
        return RSAPRNG_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    // Instance gamma of group g: output k goes to element g N Mv + k Mv + gamma.
    const std::vector<uint64_t> counts(k, N);
    std::vector<uint64_t> offs(k);
    for (uint64_t g = 0; g < ngroups; g++)
        for (uint32_t j = 0; j < Mv; j++)
            offs[g * Mv + j] = g * N * Mv + j;
    HostPlan &hp = c->hp_direct;
    int rc = build_plan(c, c->cfg, k, ids, counts.data(), offs.data(), c->cfg.chunk, hp, 1, Mv);
    if (rc)
        return rc;
    ScratchSlot *slot;
    if ((rc = scratch_slot(c, &slot)) != RSAPRNG_OK)
        return rc;
    if ((rc = upload_plan(c, hp, slot->plan, st)) != RSAPRNG_OK)
        return rc;
    rc = launch_plan(c, c->cfg, slot->plan, d_r, d_c, st, nullptr, nullptr, true);
    cudaEventRecord(slot->done, st);
    slot->used = true;
    return rc;
}

int rsaprng_histogram(rsaprng_ctx *c, uint64_t nreq, const rsaprng_id *ids,
                      const uint64_t *counts, uint32_t D, uint32_t d, int source,
                      uint64_t *d_hist, void *stream)
{
    if (!c || (nreq && (!ids || !counts)) || !d_hist)
        return fail(RSAPRNG_ERR_ARG, "histogram: null argument");
    if (D < 1 || D > 8)
        return fail(RSAPRNG_ERR_ARG, "histogram: D = %u not in [1, 8]", D);
    if (source != RSAPRNG_HIST_HIGH && source != RSAPRNG_HIST_LOW)
        return fail(RSAPRNG_ERR_ARG, "histogram: unknown source %d", source);
    if (d < 2 || (source == RSAPRNG_HIST_LOW && (d & (d - 1))))
        return fail(RSAPRNG_ERR_ARG, "histogram: d = %u (>= 2; a power of two for low bits)", d);
    uint64_t bins = 1;
    for (uint32_t i = 0; i < D; i++) {
        bins *= d;
        if (bins > (1ULL << 32))
            return fail(RSAPRNG_ERR_ARG, "histogram: d^D above 2^32");
    }
    std::vector<rsaprng_id> sorted(ids, ids + nreq);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return fail(RSAPRNG_ERR_ARG, "histogram: an instance appears in two requests");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    // Tuples are counted from each request's start: every request is placed
    // at offset 0, so a piece's offset is its position in its request.
    const std::vector<uint64_t> zero(nreq, 0);
    HostPlan &hp = c->hp_direct;
    int rc = build_plan(c, c->cfg, nreq, ids, counts, zero.data(), c->cfg.chunk, hp, D);
    if (rc)
        return rc;
    if (hp.items.empty())
        return RSAPRNG_OK;
    ScratchSlot *slot;
    if ((rc = scratch_slot(c, &slot)) != RSAPRNG_OK)
        return rc;
    if ((rc = upload_plan(c, hp, slot->plan, st)) != RSAPRNG_OK)
        return rc;
    const HistArgs h{(unsigned long long *)d_hist, d, D, source == RSAPRNG_HIST_LOW ? 1u : 0u, 0u};
    rc = launch_plan(c, c->cfg, slot->plan, nullptr, nullptr, st, nullptr, &h, true);
    cudaEventRecord(slot->done, st);
    slot->used = true;
    return rc;
}

int rsaprng_chi2_uniform(const uint64_t *h_hist, uint64_t bins, double *chi2, uint64_t *total)
{
    if (!h_hist || bins == 0 || !chi2)
        return fail(RSAPRNG_ERR_ARG, "chi2_uniform: null argument or no bins");
    // chi^2 = sum (O - E)^2 / E with E = t / bins equals bins sum O^2 / t - t;
    // t and sum O^2 are exact integers.
    unsigned __int128 s2 = 0;
    uint64_t t = 0;
    for (uint64_t i = 0; i < bins; i++) {
        t += h_hist[i];
        s2 += (unsigned __int128)h_hist[i] * h_hist[i];
    }
    if (t == 0)
        return fail(RSAPRNG_ERR_ARG, "chi2_uniform: empty histogram");
    const long double x = (long double)s2 * (long double)bins / (long double)t - (long double)t;
    *chi2 = (double)x;
    if (total)
        *total = t;
    return RSAPRNG_OK;
}

// Splits one instance's N outputs into chunks sized so that every SM gets
// work, then generates through the batch path.
static int generate_one(rsaprng_ctx *c, rsaprng_id id, uint64_t N, uint64_t *d_c, double *d_r,
                        void *stream)
{
    if (!c)
        return fail(RSAPRNG_ERR_ARG, "null ctx");
    if (id >= c->count)
        return fail(RSAPRNG_ERR_ID, "unknown id %u", id);
    if (N == 0)
        return RSAPRNG_OK;
    cudaSetDevice(c->device);
    bool done = false;
    int rc1 = generate_single_launch(c, id, N, d_c, d_r, (cudaStream_t)stream, &done);
    if (rc1 || done)
        return rc1;
    const uint64_t tile = (uint64_t)c->cfg.threads_per_block * c->cfg.numbers_per_thread;
    const uint64_t target = (uint64_t)c->sms * 8;
    uint64_t chunk = (N + target - 1) / target;
    chunk = std::max<uint64_t>(tile, (chunk + tile - 1) / tile * tile);
    chunk = std::min<uint64_t>(chunk, std::max<uint64_t>(c->cfg.chunk, tile));
    rsaprng_config saved = c->cfg;
    c->cfg.chunk = chunk;
    const uint64_t zero = 0;
    int rc = rsaprng_generate_batch(c, 1, &id, &N, &zero, d_r, d_c, stream);
    c->cfg = saved;
    return rc;
}

int rsaprng_generate_u64(rsaprng_ctx *c, rsaprng_id id, uint64_t N, uint64_t *d_c, void *stream)
{
    if (!d_c)
        return fail(RSAPRNG_ERR_ARG, "null output");
    return generate_one(c, id, N, d_c, nullptr, stream);
}

int rsaprng_generate_f64(rsaprng_ctx *c, rsaprng_id id, uint64_t N, double *d_r, void *stream)
{
    if (!d_r)
        return fail(RSAPRNG_ERR_ARG, "null output");
    return generate_one(c, id, N, nullptr, d_r, stream);
}

int rsaprng_generate_both(rsaprng_ctx *c, rsaprng_id id, uint64_t N, uint64_t *d_c, double *d_r,
                          void *stream)
{
    if (!d_c || !d_r)
        return fail(RSAPRNG_ERR_ARG, "null output");
    return generate_one(c, id, N, d_c, d_r, stream);
}

int rsaprng_unit_f64(rsaprng_ctx *c, rsaprng_id id, uint64_t N, const uint64_t *d_c,
                     double *d_r, int divide, void *stream)
{
    if (!c || (N && (!d_c || !d_r)))
        return fail(RSAPRNG_ERR_ARG, "unit_f64: null argument");
    if (id >= c->count)
        return fail(RSAPRNG_ERR_ID, "unknown id %u", id);
    if (divide == RSAPRNG_DIVIDE_AUTO)
        divide = c->cfg.divide;
    cudaSetDevice(c->device);
    cudaError_t e = launch_unit(ctx_tables(c), id, N, d_c, d_r,
                                c->cfg.rounding == RSAPRNG_ROUND_EXACT ? DIVIDE_EXACT
                                : divide == RSAPRNG_DIVIDE_INT         ? DIVIDE_INT
                                : divide == RSAPRNG_DIVIDE_FP64        ? DIVIDE_FP64
                                : divide == RSAPRNG_DIVIDE_HYBRID      ? DIVIDE_HYBRID
                                                                       : DIVIDE_RECIP,
                                (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "unit launch");
    c->launches += N ? 1 : 0;
    return RSAPRNG_OK;
}

int rsaprng_microbench(rsaprng_ctx *c, int kind, uint64_t bytes, double *result)
{
    if (!c || !result)
        return fail(RSAPRNG_ERR_ARG, "null");
    cudaSetDevice(c->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaError_t e = cudaSuccess;
    if (kind == 0) {
        e = microbench_imad(result, st);
    } else if (kind == 1) {
        e = microbench_ddiv(result, st);
    } else if (kind == 2) {
        void *buf = nullptr;
        if (bytes < (1 << 20))
            bytes = 1 << 20;
        e = cudaMalloc(&buf, bytes);
        if (e == cudaSuccess) {
            e = microbench_write(buf, bytes, result, st);
            cudaFree(buf);
        }
    } else if (kind >= 3 && kind <= 5) {
        e = microbench_mul(kind - 3, result, st);
    } else if (kind >= 6 && kind <= 8) {
        e = microbench_fp64(kind - 6, result, st);
    } else {
        cudaStreamDestroy(st);
        return fail(RSAPRNG_ERR_ARG, "unknown microbenchmark %d", kind);
    }
    cudaStreamDestroy(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "microbenchmark");
    return RSAPRNG_OK;
}

}  // extern "C"
