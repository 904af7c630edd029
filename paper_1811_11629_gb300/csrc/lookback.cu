// Single-launch generation of one stream (the plain call of Sec. V's
// Algorithm over one instance) with a decoupled look-back for the message
// offsets.
//
// Sec. IV: the message before output k is m_0 plus the sum of the skips
// s_1..s_k (mod n), and that sum has no cheap closed form, while the skips
// themselves jump exactly (s_k = s_0 a^k mod Q). Here block b of the launch
// owns tile b of the stream (outputs bS+1 .. bS+S). It jumps to its first
// skip, sums its tile's skips (the tile aggregate) and publishes the
// aggregate; then its threads walk back over the tiles before it, many at
// once, adding their aggregates up to the nearest tile that has published its
// inclusive prefix (Merrill & Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", 2016). The block publishes its own inclusive
// prefix at once and goes on to the messages, the encryption, the division
// and the stores of its tile.
//
// Waiting. A block waits only on tiles with a smaller logical index; logical
// indices are handed out by an atomic ticket in the order blocks start, so
// every tile a block waits on belongs to a block that has started, and every
// started block publishes its aggregate before it waits on anything. Each
// wait is still bounded: after spin_limit empty polls the block raises the
// context's device error flag and returns without writing its tile (the
// host reads the flag with rsaprng_device_status). No wait is unbounded.
//
// Status words carry the call's epoch (a per-context counter, never reused),
// so the status array needs no clearing between calls.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "api_internal.hpp"
#include "device_math.cuh"
#include "kernels.cuh"
#include "tile.cuh"

namespace rsaprng {

namespace {

using dev::addmod;
using dev::mulmodQ;
using tile::FULL;
using tile::sidx;
using tile::to_unit;

// Per-tile status: the tile aggregate and the inclusive prefix, each with the
// epoch of the call that wrote it (written once per call, value before tag).
struct LbStatus {
    u64 agg, agg_tag;
    u64 incl, incl_tag;
};
static_assert(sizeof(LbStatus) == 32, "LbStatus layout");

struct LbArgs {
    u64 N;                    // outputs of the call
    u64 epoch;                // this call's tag
    u64 ticket_base;          // ticket value before this launch's first block
    unsigned long long *ticket;
    LbStatus *status;         // one per tile
    uint32_t *err;            // context device error word
    uint32_t inst;
    uint32_t ntiles;
    uint32_t spin_limit;      // empty polls before a wait gives up
    uint32_t inject;          // bit 0: tile 0 publishes nothing (tests of the error path)
};

__device__ __forceinline__ u64 ld_acquire(const u64 *p)
{
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ u64 ld_relaxed(const u64 *p)
{
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(u64 *p, u64 v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release(u64 *p, u64 v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Run by every thread of the block for tile b > 0, after the block has
// published its own aggregate: the sum (mod n) of the skips of all tiles
// before b. Thread t visits the earlier tiles b-1-t, b-1-t-T, ... nearest
// first, waits at each until it holds its aggregate or its inclusive prefix,
// and stops at the first inclusive prefix it meets (or below the nearest one
// another thread has already met, kept in *sh_near). The nearest inclusive
// prefix J over the block, plus the aggregates of the tiles after J, is the
// result. Every thread polls at most ceil(b / T) tiles at once, so the walk
// costs a few rounds of L2 latency however far back J lies. Returns false in
// every thread when some wait gave up (spin_limit empty polls).
__device__ __forceinline__ bool block_lookback(const LbStatus *st, uint32_t b, u64 epoch, u64 n,
                                               uint32_t spin_limit, int *sh_near, u64 *sh_red,
                                               u64 &excl)
{
    const int t = threadIdx.x, T = blockDim.x;
    bool ok = true;
    long long j = (long long)b - 1 - t;
    for (; j >= 0; j -= T) {
        if (j < *(volatile int *)sh_near)
            break;  // another thread holds a nearer inclusive prefix
        uint32_t empty = 0;
        int kind = 0;
        for (;;) {
            if (ld_acquire(&st[j].incl_tag) == epoch) {
                kind = 2;
                break;
            }
            if (ld_acquire(&st[j].agg_tag) == epoch) {
                kind = 1;
                break;
            }
            if (empty >= spin_limit) {
                ok = false;
                break;
            }
            empty++;
            __nanosleep(64);
        }
        if (!ok)
            break;
        if (kind == 2) {
            atomicMax(sh_near, (int)j);
            break;
        }
    }
    if (__syncthreads_or(!ok))
        return false;
    const long long J = *(volatile int *)sh_near;  // >= 0: tile 0 only ever publishes its prefix
    // The aggregates of this thread's tiles after J (each was seen above with
    // its tag), and the inclusive prefix of J from the thread that owns it.
    u64 sum = 0;
    for (long long k = (long long)b - 1 - t; k > J; k -= T)
        sum = addmod(sum, ld_relaxed(&st[k].agg), n);
    if (J >= 0 && ((long long)b - 1 - J) % T == t)
        sum = addmod(sum, ld_relaxed(&st[J].incl), n);
    excl = tile::block_reduce_mod(sum, n, sh_red);
    return true;
}

template <int L, int MODEXP, int DIV>
__global__ void __launch_bounds__(512) k_generate_lookback(DeviceTables tab, LbArgs A,
                                                         double *__restrict__ out_r,
                                                         u64 *__restrict__ out_c)
{
    extern __shared__ u64 smem[];
    __shared__ u64 sh_scan[32];
    __shared__ u64 sh_m0, sh_s0;
    __shared__ uint32_t sh_b;
    __shared__ int sh_near;
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31;
    const int S = T * L;
    const int slots = S + (S >> 4);
    u64 *st_r = smem;
    u64 *st_c = smem + (out_r ? slots : 0);
    if (t == 0) {
        // Logical tile in start order; the instance state is read before
        // anything is published, so the block that writes the new state
        // (the last tile, after it has seen every earlier tile's prefix
        // chain) cannot overtake a read.
        sh_b = (uint32_t)(atomicAdd(A.ticket, 1ull) - A.ticket_base);
        sh_m0 = tab.state_m[A.inst];
        sh_s0 = tab.state_s[A.inst];
        sh_near = -1;
    }
    __syncthreads();
    const uint32_t b = sh_b;
    if (b >= A.ntiles)
        return;
    const InstParams P = tab.params[A.inst];
    const u64 *plin = tab.pow_lin + (size_t)P.root * kPowLinRow;
    const u64 *p2k = tab.pow2k + (size_t)P.root * 64;
    const u64 base = (u64)b * S;
    const u64 left = A.N - base;
    const int tile_n = left < (u64)S ? (int)left : S;
    const int my0 = t * L;
    const int nvalid = tile_n - my0 < 0 ? 0 : (tile_n - my0 > L ? L : tile_n - my0);

    // The skip before the tile, s_0 a^(bS): lane l multiplies the table
    // powers a^(2^(2l)) and a^(2^(2l+1)) for the set bits of bS, and a
    // butterfly multiplies the lanes' factors (every warp computes it, so no
    // barrier is needed).
    const int b0 = 2 * lane;
    u64 f = ((base >> b0) & 1) ? p2k[b0] : 1;
    if ((base >> (b0 + 1)) & 1)
        f = mulmodQ(f, p2k[b0 + 1]);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1)
        f = mulmodQ(f, __shfl_xor_sync(FULL, f, d));
    const u64 s_thr = mulmodQ(mulmodQ(sh_s0, f), plin[my0]);

    WorkItem W;
    W.inst = A.inst;
    W.flags = b + 1 == A.ntiles ? WI_WRITEBACK : 0u;
    W.count = left;
    W.out_off = base;
    W.m0 = W.s0 = 0;
    bool failed = false;
    u64 carry = 0;
    // The tile's block scan, then the look-back for its carry-in.
    auto scan = [&](u64 v, u64 n, u64 &total) -> u64 {
        const u64 pre = tile::block_exscan_mod(v, n, sh_scan, total);
        LbStatus *me = A.status + b;
        u64 excl = 0;
        bool ok = true;
        if (b > 0) {
            if (t == 0) {
                st_relaxed(&me->agg, total);
                st_release(&me->agg_tag, A.epoch);
            }
            ok = block_lookback(A.status, b, A.epoch, n, A.spin_limit, &sh_near, sh_scan, excl);
        }
        if (t == 0) {
            if (ok && !(b == 0 && (A.inject & 1))) {
                st_relaxed(&me->incl, addmod(excl, total, n));
                st_release(&me->incl_tag, A.epoch);
            }
            if (!ok)
                atomicOr(A.err, 1u);
        }
        failed = !ok;
        carry = excl;
        if (failed)
            W.flags = 0;  // no state write-back after a wait that gave up
        return addmod(carry, pre, n);
    };
    u64 c[L], total;
    tile::tile_ciphertexts_scan<L, MODEXP>(tab, W, P, sh_m0, s_thr, left, my0, nvalid, scan, c,
                                           total);
    if (failed)
        return;
#pragma unroll
    for (int j = 0; j < L; j++) {
        const int i = sidx(my0 + j);
        if (out_r)
            st_r[i] = (u64)__double_as_longlong(to_unit<DIV>(c[j], P, j));
        if (out_c)
            st_c[i] = c[j];
    }
    __syncthreads();
    if (out_r) {
        for (int i = t; i < tile_n; i += T)
            out_r[base + i] = __longlong_as_double((long long)st_r[sidx(i)]);
    }
    if (out_c) {
        for (int i = t; i < tile_n; i += T)
            out_c[base + i] = st_c[sidx(i)];
    }
    if ((W.flags & WI_WRITEBACK) && t == 0)
        tab.state_m[A.inst] = addmod(addmod(sh_m0, carry, P.n), total, P.n);
}

template <int L, int MODEXP, int DIV>
cudaError_t launch_lb_t(int threads, const DeviceTables &tab, const LbArgs &A, double *out_r,
                        u64 *out_c, cudaStream_t stream)
{
    const size_t smem = padded_smem_bytes(threads, L, out_r != nullptr, out_c != nullptr);
    auto kern = k_generate_lookback<L, MODEXP, DIV>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    kern<<<A.ntiles, threads, smem, stream>>>(tab, A, out_r, out_c);
    return cudaGetLastError();
}

// The tilings and routes with a single-launch kernel; others use the chunked
// path. Returns cudaErrorNotSupported when there is none.
cudaError_t launch_lookback(int L, int modexp, int divide, int threads, const DeviceTables &tab,
                            const LbArgs &A, double *out_r, u64 *out_c, cudaStream_t stream)
{
#define RSAPRNG_LB(LL, MM, DD)                                                          \
    if (L == LL && modexp == MM && divide == DD)                                        \
        return launch_lb_t<LL, MM, DD>(threads, tab, A, out_r, out_c, stream);
    RSAPRNG_LB(16, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_LB(16, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_LB(16, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_LB(14, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_LB(13, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_LB(12, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_LB(16, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_LB(16, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_LB(8, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_LB(8, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_LB(8, MODEXP_MONT64, DIVIDE_RECIP)
    RSAPRNG_LB(8, MODEXP_MONT64, DIVIDE_INT)
#undef RSAPRNG_LB
    return cudaErrorNotSupported;
}

// Resident blocks per SM of the latency-mode kernel (512 threads, 16 per
// thread, CRT route), for one output or two; looked up once per process.
std::mutex g_occ_mu;
int g_lat_occ[2][2] = {{-1, -1}, {-1, -1}};  // [rounding exact][both outputs]

int latency_occupancy(bool exact, bool both)
{
    std::lock_guard<std::mutex> lk(g_occ_mu);
    int &o = g_lat_occ[exact][both];
    if (o < 0) {
        const void *k = exact ? (const void *)k_generate_lookback<16, MODEXP_CRT32, DIVIDE_EXACT>
                              : (const void *)k_generate_lookback<16, MODEXP_CRT32, DIVIDE_INT>;
        const size_t smem = padded_smem_bytes(512, 16, true, both);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, 512, smem) != cudaSuccess)
            b = 0;
        o = b;
    }
    return o;
}


// The tile shape of a latency-mode draw of N outputs on sms SMs: threads (a
// multiple of 32, 128 to 512) and outputs per thread L, with at most one tile
// per SM. The four warp schedulers of an SM then share the tile's warps, so
// a scheduler issues the work of ceil(threads / 128) warps of L outputs each
// while every warp runs a chain of L dependent outputs. Of the shapes whose
// tiles cover the draw on one tile per SM, the one that minimises
// L (max(w, 2) + 1), w = ceil(threads / 128), is taken (smaller L on a tie):
// a fit to the measured call time, which grows with the per-scheduler work
// w L and with the chain length L, and which one warp per scheduler does not
// hide. The exact-rational route has only L = 16. When no shape covers the
// draw on one tile per SM, 512 x 16.
void latency_shape(uint64_t N, int sms, bool exact, int *threads, int *L)
{
    static const int kLs[] = {12, 13, 14, 16};
    *threads = 512;
    *L = 16;
    uint64_t best = UINT64_MAX;
    for (int Lc : kLs) {
        if (exact && Lc != 16)
            continue;
        const uint64_t per = (uint64_t)Lc * (uint64_t)sms;
        const uint64_t q = N / per + (N % per != 0);  // threads for one tile per SM
        if (q > 512)
            continue;
        uint64_t T = (q + 31) / 32 * 32;
        if (T < 128)
            T = 128;
        if (T > 512)
            continue;
        const uint64_t w = (T + 127) / 128;
        const uint64_t cost = (uint64_t)Lc * ((w < 2 ? 2 : w) + 1);
        if (cost < best) {
            best = cost;
            *threads = (int)T;
            *L = Lc;
        }
    }
}

// Tiles of one single-launch call at most (the status array of a scratch
// slot holds this many); longer draws take the chunked path.
constexpr uint64_t kLbMaxTiles = 4096;
// Empty poll rounds before a wait gives up when the configuration leaves the
// limit at zero (about a second with the 64 ns pause between rounds).
constexpr uint32_t kLbDefaultSpin = 1u << 23;

int lookback_error_word(rsaprng_ctx *c, uint32_t **out)
{
    if (!c->d_err) {
        cudaError_t e = cudaMalloc(&c->d_err, sizeof(uint32_t));
        if (e != cudaSuccess)
            return cuda_fail(e, "device error word");
        if ((e = cudaMemset(c->d_err, 0, sizeof(uint32_t))) != cudaSuccess)
            return cuda_fail(e, "device error word");
    }
    *out = c->d_err;
    return RSAPRNG_OK;
}

}  // namespace

int generate_single_launch(rsaprng_ctx *c, rsaprng_id id, uint64_t N, uint64_t *d_c,
                           double *d_r, cudaStream_t st, bool *done)
{
    *done = false;
    const rsaprng_config &cfg = c->cfg;
    if (cfg.lookback == RSAPRNG_LOOKBACK_OFF)
        return RSAPRNG_OK;
    GenLaunch g = ctx_launch(c, cfg, 1, d_r != nullptr, d_c != nullptr);
    if (g.modexp == MODEXP_MONT64 && c->h_params[id].e != c->h_params[id].eq)
        return fail(RSAPRNG_ERR_ARG, "instance %u has CRT exponents: the 64-bit route cannot "
                                     "run it", id);
    // Latency mode. A draw that fits one wave of 512-thread blocks of 16
    // outputs per thread runs in a latency shape (latency_shape), on the CRT
    // route with the integer division. Every block then starts at once and
    // runs the same phases at the same time, so the phases add up rather than
    // overlap. The integer division keeps the division phase off the two-lane
    // FP64 pipe, and one tile per SM at most keeps the look-back short. All
    // shapes and routes give the same bits; larger draws keep the configured
    // (throughput) shape.
    if (cfg.lookback != RSAPRNG_LOOKBACK_CONFIGURED) {
        const bool exact = cfg.rounding == RSAPRNG_ROUND_EXACT;
        const uint64_t S_lat = 512 * 16;
        const uint64_t wave = (uint64_t)latency_occupancy(exact, d_r && d_c) * c->sms;
        if ((N + S_lat - 1) / S_lat <= wave) {
            latency_shape(N, c->sms, exact, &g.threads, &g.L);
            g.modexp = MODEXP_CRT32;
            g.divide = exact ? DIVIDE_EXACT : DIVIDE_INT;
        }
    }
    const uint64_t S = (uint64_t)g.threads * g.L;
    const uint64_t ntiles = (N + S - 1) / S;
    if (ntiles > kLbMaxTiles)
        return RSAPRNG_OK;
    uint32_t *err = nullptr;
    int rc = lookback_error_word(c, &err);
    if (rc)
        return rc;
    ScratchSlot *slot;
    if ((rc = scratch_slot(c, &slot)) != RSAPRNG_OK)
        return rc;
    DevPlan &dp = slot->plan;
    const size_t need = 64 + kLbMaxTiles * sizeof(LbStatus);
    if (dp.cap_lb < need) {
        if (dp.d_lb)
            cudaFree(dp.d_lb);
        dp.d_lb = nullptr;
        dp.cap_lb = 0;
        cudaError_t e = cudaMalloc(&dp.d_lb, need);
        if (e != cudaSuccess)
            return fail(RSAPRNG_ERR_OOM, "single-launch status (%zu bytes)", need);
        // zero tags match no epoch (epochs start at 1); the ticket starts at 0
        if ((e = cudaMemsetAsync(dp.d_lb, 0, need, st)) != cudaSuccess)
            return cuda_fail(e, "single-launch status");
        dp.cap_lb = need;
        dp.lb_base = 0;
    }
    LbArgs A;
    A.N = N;
    A.epoch = ++c->lb_epoch;
    A.ticket_base = dp.lb_base;
    A.ticket = (unsigned long long *)dp.d_lb;
    A.status = (LbStatus *)((char *)dp.d_lb + 64);
    A.err = err;
    A.inst = id;
    A.ntiles = (uint32_t)ntiles;
    A.spin_limit = cfg.spin_limit > 0 ? (uint32_t)cfg.spin_limit
                   : cfg.spin_limit < 0 ? 0u
                                        : kLbDefaultSpin;
    A.inject = (uint32_t)cfg.test_flags;
    cudaError_t e = launch_lookback(g.L, g.modexp, g.divide, g.threads, ctx_tables(c), A, d_r,
                                    d_c, st);
    if (e == cudaErrorNotSupported) {
        (void)cudaGetLastError();
        return RSAPRNG_OK;  // no single-launch kernel for this tiling: the chunked path
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "single-launch generation");
    dp.lb_base += ntiles;
    cudaEventRecord(slot->done, st);
    slot->used = true;
    c->launches += 1;
    *done = true;
    return RSAPRNG_OK;
}

}  // namespace rsaprng

extern "C" int rsaprng_latency_shape(uint64_t N, int sms, int rounding_exact, int *threads,
                                     int *numbers_per_thread)
{
    using namespace rsaprng;
    if (!threads || !numbers_per_thread || sms < 1)
        return fail(RSAPRNG_ERR_ARG, "latency_shape: null output or sms < 1");
    latency_shape(N, sms, rounding_exact != 0, threads, numbers_per_thread);
    return RSAPRNG_OK;
}

extern "C" int rsaprng_device_status(rsaprng_ctx *c, void *stream)
{
    using namespace rsaprng;
    if (!c)
        return fail(RSAPRNG_ERR_ARG, "null ctx");
    if (!c->d_err)
        return RSAPRNG_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t flag = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaMemcpy(&flag, c->d_err, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e, "device status");
    if (!flag)
        return RSAPRNG_OK;
    if ((e = cudaMemset(c->d_err, 0, sizeof flag)) != cudaSuccess)
        return cuda_fail(e, "device status");
    return fail(RSAPRNG_ERR_DEVICE_FLAG, "a device-side wait gave up (flags 0x%x)", flag);
}
