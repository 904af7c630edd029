// The vectorised call of Sec. VI (Eq. vectorize) on the tile engine: the
// outputs of Mv instances come back k-major (element k Mv + gamma), so the
// outputs of one instance lie Mv elements apart. Written one instance per
// block, every store would fill one element of a memory sector that other
// blocks complete later, and the memory would read and rewrite each sector.
// Here a block takes G instances of one vector side by side at the same
// positions: TS = T / G threads per instance, each owning L consecutive
// outputs of its instance, so a tile holds K = TS L positions of G
// instances. The skip scan of an instance runs over its TS lanes
// (segmented shuffles, no barrier); the tile is staged instance by instance
// in shared memory and written k-major, as rows of G consecutive elements.
//
// The plan is the ordinary one (pieces, skip-sum pre-pass, start states);
// the host groups up to G work items that cover the same positions of
// consecutive instances of a vector into one block's unit (VecGroup).
//
// The same kernel packs unrelated streams into a block (stride 1): G pieces
// of any instances and lengths, TS = T / G threads each (whole warps, so no
// warp mixes exponents), the group's first piece the longest. The block runs
// the tiles of its longest piece; a segment whose piece has ended computes on
// with nothing valid, and each segment writes its own run contiguously.
#include "device_math.cuh"
#include "kernels.cuh"
#include "tile.cuh"

namespace rsaprng {

namespace {

using dev::addmod;
using dev::mulmodQ;
using tile::sidx;
using tile::to_unit;

// TB > 0: the tuned instance for blocks of exactly TB threads, bounded to
// five resident blocks per SM. MODE 0: the interleaved order with segments
// inside a warp (TS < 32); MODE 1: the interleaved order with segments of
// whole warps (TS >= 32); MODE 2: unrelated streams side by side (stride 1,
// per-segment lengths, segments of whole warps). With whole-warp segments
// the segment index comes from lane 0, so the compiler knows it is the same
// across the warp and keeps the instance's parameters in uniform registers
// (the interleaved 16-per-thread kernel: 96 registers instead of 128).
template <int L, int MODEXP, int DIV, int TB, int MODE>
__global__ void __launch_bounds__(TB ? TB : 512, TB ? 5 : 1)
    k_generate_vec(DeviceTables tab, const WorkItem *__restrict__ items,
                   const VecGroup *__restrict__ vecs, uint32_t nvecs, uint32_t *ticket,
                   double *__restrict__ out_r, u64 *__restrict__ out_c, u64 stride, int TS)
{
    tile::pdl_wait();  // the start states of the pieces, from the start-state scan
    extern __shared__ u64 smem[];
    __shared__ u64 sh_scan[32];
    __shared__ uint32_t sh_item;
    const int T = TB ? TB : (int)blockDim.x, t = threadIdx.x;
    const int tsh = __ffs(TS) - 1, G = T >> tsh, gsh = __ffs(G) - 1;  // both powers of two
    constexpr bool PACKED = MODE == 2;
    const int seg = MODE >= 1 ? __shfl_sync(0xFFFFFFFFu, t >> tsh, 0) : t >> tsh;
    const int lt = t & (TS - 1);
    const int wcol = t & (G - 1), wk0 = t >> gsh;  // this thread's column and first row in stores
    const int K = TS * L;  // positions of each instance per tile
    const int S = K * G;   // = T L outputs per tile
    const int my0 = lt * L;
    // 16-byte column-pair stores of the k-major rows (see below)
    const bool pairs = !PACKED && G >= 2 && (stride & 1) == 0 &&
                       ((uintptr_t)out_r & 15) == 0 && ((uintptr_t)out_c & 15) == 0;
    u64 *st_r = smem;
    u64 *st_c = smem + (out_r ? S + (S >> 4) : 0);

    uint32_t v = blockIdx.x;
    if (ticket) {
        if (t == 0)
            sh_item = atomicAdd(ticket, 1u);
        __syncthreads();
        v = sh_item;
    }
    while (v < nvecs) {
        const VecGroup V = vecs[v];
        const bool on = seg < (int)V.count;
        // Idle segments shadow the first item: they compute alongside (the
        // shuffles need every lane) but store and write back nothing.
        WorkItem W = items[V.first + (on ? seg : 0)];
        if (!on)
            W.flags &= ~(uint32_t)WI_WRITEBACK;
        const InstParams P = tab.params[W.inst];
        const u64 n = P.n;
        const u64 *plin = tab.pow_lin + (size_t)P.root * kPowLinRow;
        u64 m, s;
        if (W.flags & WI_FROM_STATE) {
            m = tab.state_m[W.inst];
            s = tab.state_s[W.inst];
        } else {
            m = W.m0;
            s = W.s0;
        }
        u64 s_thr = mulmodQ(s, plin[my0]);
        const u64 aK = plin[K];
        // This segment's length, and the group's (its first item is the
        // longest); in the interleaved order they are all equal.
        const u64 count = W.count;
        const u64 gcount = PACKED ? items[V.first].count : count;
        const u64 o0 = items[V.first].out_off;
        for (u64 base = 0; base < gcount; base += K) {
            const u64 left = !PACKED || count > base ? count - base : 0;
            const int tile_n = left < (u64)K ? (int)left : K;
            const int nvalid = !on ? 0 : (tile_n - my0 < 0 ? 0 : (tile_n - my0 > L ? L : tile_n - my0));
            u64 c[L], total;
            tile::tile_ciphertexts_scan<L, MODEXP>(
                tab, W, P, m, s_thr, left, my0, nvalid,
                [&](u64 x, u64 nn, u64 &tot) {
                    if constexpr (PACKED) {
                        if (TS > 32)
                            return tile::segment_exscan_mod_warps(x, nn, TS, sh_scan, tot);
                    }
                    return tile::segment_exscan_mod(x, nn, TS, tot);
                },
                c, total);
            // staged by instance: slot seg K + position (padded every 16)
            const int row0 = seg * K + my0;
#pragma unroll
            for (int j = 0; j < L; j++) {
                if (out_r)
                    st_r[sidx(row0 + j)] = (u64)__double_as_longlong(to_unit<DIV>(c[j], P, j));
                if (out_c)
                    st_c[sidx(row0 + j)] = c[j];
            }
            __syncthreads();
            if constexpr (PACKED) {
                // Packed streams: each segment's run is contiguous at its own
                // offset, written by its TS threads.
                if (on) {
                    const u64 o = W.out_off + base;
                    for (int k = lt; k < tile_n; k += TS) {
                        const int slot = sidx(seg * K + k);
                        if (out_r)
                            out_r[o + k] = __longlong_as_double((long long)st_r[slot]);
                        if (out_c)
                            out_c[o + k] = st_c[slot];
                    }
                }
            } else if (pairs && (o0 & 1) == 0) {
                // Written k-major in column pairs: thread t writes columns
                // 2c and 2c + 1 (c = t mod G/2) of rows t / (G/2), ... with
                // one 16-byte store per pair (even stride and first element,
                // 16-byte aligned arrays); a pair whose second column lies
                // past the group's streams stores its first alone.
                const int c2 = 2 * (t & ((G >> 1) - 1));
                const int r0 = t >> (gsh - 1), rstep = 2 * TS;
                if (c2 < (int)V.count) {
                    const bool two = c2 + 1 < (int)V.count;
                    u64 e = o0 + (base + (u64)r0) * stride + (u64)c2;
                    const u64 step = (u64)rstep * stride;
                    for (int k = r0; k < tile_n; k += rstep, e += step) {
                        const int a = sidx(c2 * K + k), b = sidx((c2 + 1) * K + k);
                        if (two) {
                            if (out_r)
                                *reinterpret_cast<ulonglong2 *>(out_r + e) =
                                    make_ulonglong2(st_r[a], st_r[b]);
                            if (out_c)
                                *reinterpret_cast<ulonglong2 *>(out_c + e) =
                                    make_ulonglong2(st_c[a], st_c[b]);
                        } else {
                            if (out_r)
                                out_r[e] = __longlong_as_double((long long)st_r[a]);
                            if (out_c)
                                out_c[e] = st_c[a];
                        }
                    }
                }
            } else if (wcol < (int)V.count) {
                // Written k-major: T is a multiple of G, so thread t always
                // writes column t mod G, at positions t / G, t / G + TS, ...
                u64 e = o0 + (base + (u64)wk0) * stride + (u64)wcol;
                const u64 step = (u64)TS * stride;
                for (int k = wk0; k < tile_n; k += TS, e += step) {
                    const int slot = sidx(wcol * K + k);
                    if (out_r)
                        out_r[e] = __longlong_as_double((long long)st_r[slot]);
                    if (out_c)
                        out_c[e] = st_c[slot];
                }
            }
            __syncthreads();
            m = addmod(m, total, n);
            s_thr = mulmodQ(s_thr, aK);
        }
        if (lt == 0 && (W.flags & WI_WRITEBACK)) {
            tab.state_m[W.inst] = m;
            if (count == 0)
                tab.state_s[W.inst] = s;
        }
        if (ticket) {
            __syncthreads();
            if (t == 0)
                sh_item = atomicAdd(ticket, 1u);
            __syncthreads();
            v = sh_item;
        } else {
            v += gridDim.x;
        }
    }
}

// The tuned tiles of the vector kernel, in blocks of 128 threads on the CRT
// route bounded to five resident blocks per SM: 8 numbers per thread always,
// and 16 when segments are whole warps. Segments inside a warp make every
// thread hold its own instance's parameters, and 16 numbers per thread then
// no longer fit the register budget of five blocks (the compiler spills).
constexpr int kVecTunedThreads = 128;
constexpr int kVecTunedL = 8;
constexpr int kVecWideL = 16;

template <int L, int MODEXP, int MODE>
constexpr bool vec_tuned()
{
    return MODEXP == MODEXP_CRT32 && (L == kVecTunedL || (L == kVecWideL && MODE >= 1));
}

template <int L, int MODEXP, int DIV, int MODE>
auto vec_kernel(int threads)
{
    if constexpr (vec_tuned<L, MODEXP, MODE>())
        if (threads == kVecTunedThreads)
            return k_generate_vec<L, MODEXP, DIV, kVecTunedThreads, MODE>;
    return k_generate_vec<L, MODEXP, DIV, 0, MODE>;
}

// Whole-warp interleaved kernels (MODE 1) exist for the tilings that the
// vector call runs (16 and 8 per thread on the CRT route, 8 on the 64-bit
// route); elsewhere MODE 0 serves every segment width.
template <int L, int MODEXP>
constexpr bool has_warp_mode()
{
    return (MODEXP == MODEXP_CRT32 && (L == 16 || L == 8)) || (MODEXP == MODEXP_MONT64 && L == 8);
}

template <int L, int MODEXP>
int effective_mode(int mode)
{
    return mode == 1 && !has_warp_mode<L, MODEXP>() ? 0 : mode;
}

template <int L, int MODEXP, int DIV>
const void *vec_kernel_any(int threads, int mode)
{
    switch (effective_mode<L, MODEXP>(mode)) {
    case 2: return (const void *)vec_kernel<L, MODEXP, DIV, 2>(threads);
    case 1:
        if constexpr (has_warp_mode<L, MODEXP>())
            return (const void *)vec_kernel<L, MODEXP, DIV, 1>(threads);
        return nullptr;
    default: return (const void *)vec_kernel<L, MODEXP, DIV, 0>(threads);
    }
}

// Every division route gives the same bits, so the vector kernel is
// instantiated for the integer and reciprocal routes (the others map to the
// reciprocal one) and for the exact-rational reading.
template <int DIV>
const void *vec_kernel_ptr_d(int L, int modexp, int threads, int mode)
{
    if (modexp == MODEXP_CRT32) {
        if (L == 16)
            return vec_kernel_any<16, MODEXP_CRT32, DIV>(threads, mode);
        if (L == 8)
            return vec_kernel_any<8, MODEXP_CRT32, DIV>(threads, mode);
        if (L == 4)
            return vec_kernel_any<4, MODEXP_CRT32, DIV>(threads, mode);
        if (L == 2)
            return vec_kernel_any<2, MODEXP_CRT32, DIV>(threads, mode);
    } else {
        if (L == 8)
            return vec_kernel_any<8, MODEXP_MONT64, DIV>(threads, mode);
        if (L == 4)
            return vec_kernel_any<4, MODEXP_MONT64, DIV>(threads, mode);
        if (L == 2)
            return vec_kernel_any<2, MODEXP_MONT64, DIV>(threads, mode);
    }
    return nullptr;
}

int vec_div(int divide)
{
    return divide == DIVIDE_EXACT ? DIVIDE_EXACT : divide == DIVIDE_INT ? DIVIDE_INT : DIVIDE_RECIP;
}

// The launch mode for segments of TS threads (0: unknown width, taken as
// inside a warp).
int vec_mode(const GenLaunch &g, int TS)
{
    return g.stride == 1 ? 2 : (TS >= 32 ? 1 : 0);
}

const void *vec_kernel_ptr(const GenLaunch &g, int mode)
{
    switch (vec_div(g.divide)) {
    case DIVIDE_EXACT: return vec_kernel_ptr_d<DIVIDE_EXACT>(g.L, g.modexp, g.threads, mode);
    case DIVIDE_INT: return vec_kernel_ptr_d<DIVIDE_INT>(g.L, g.modexp, g.threads, mode);
    default: return vec_kernel_ptr_d<DIVIDE_RECIP>(g.L, g.modexp, g.threads, mode);
    }
}

template <int L, int MODEXP, int DIV, int MODE>
cudaError_t launch_vec_p(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                         const VecGroup *vecs, uint32_t nvecs, uint32_t *ticket, double *out_r,
                         uint64_t *out_c, int TS, cudaStream_t stream)
{
    const size_t smem = vec_smem_bytes(g.threads, L, out_r != nullptr, out_c != nullptr);
    auto kern = vec_kernel<L, MODEXP, DIV, MODE>(g.threads);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    return launch_kernel(kern, g.grid, g.threads, smem, stream, g.pdl, t, items, vecs, nvecs,
                         g.persistent ? ticket : nullptr, out_r, out_c, (u64)g.stride, TS);
}

template <int L, int MODEXP, int DIV>
cudaError_t launch_vec_t(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                         const VecGroup *vecs, uint32_t nvecs, uint32_t *ticket, double *out_r,
                         uint64_t *out_c, int TS, cudaStream_t stream)
{
    switch (effective_mode<L, MODEXP>(vec_mode(g, TS))) {
    case 2:
        return launch_vec_p<L, MODEXP, DIV, 2>(g, t, items, vecs, nvecs, ticket, out_r, out_c, TS,
                                               stream);
    case 1:
        if constexpr (has_warp_mode<L, MODEXP>())
            return launch_vec_p<L, MODEXP, DIV, 1>(g, t, items, vecs, nvecs, ticket, out_r, out_c,
                                                   TS, stream);
        return cudaErrorInvalidValue;
    default:
        return launch_vec_p<L, MODEXP, DIV, 0>(g, t, items, vecs, nvecs, ticket, out_r, out_c, TS,
                                               stream);
    }
}

template <int DIV>
cudaError_t launch_vec_d(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                         const VecGroup *vecs, uint32_t nvecs, uint32_t *ticket, double *out_r,
                         uint64_t *out_c, int TS, cudaStream_t stream)
{
#define RSAPRNG_VEC(LL, MM)                                                                   \
    if (g.L == LL && g.modexp == MM)                                                          \
        return launch_vec_t<LL, MM, DIV>(g, t, items, vecs, nvecs, ticket, out_r, out_c, TS, \
                                         stream);
    RSAPRNG_VEC(16, MODEXP_CRT32)
    RSAPRNG_VEC(8, MODEXP_CRT32)
    RSAPRNG_VEC(4, MODEXP_CRT32)
    RSAPRNG_VEC(2, MODEXP_CRT32)
    RSAPRNG_VEC(8, MODEXP_MONT64)
    RSAPRNG_VEC(4, MODEXP_MONT64)
    RSAPRNG_VEC(2, MODEXP_MONT64)
#undef RSAPRNG_VEC
    return cudaErrorInvalidValue;
}

}  // namespace

int vec_numbers_per_thread(int L, int modexp, int threads)
{
    return modexp == MODEXP_CRT32 && threads == kVecTunedThreads && L > kVecTunedL ? kVecTunedL
                                                                                     : L;
}

size_t vec_smem_bytes(int threads, int L, bool want_r, bool want_c)
{
    return padded_smem_bytes(threads, L, want_r, want_c);  // the same padded slots
}

cudaError_t launch_generate_vec(const GenLaunch &g0, const DeviceTables &t, const WorkItem *items,
                                const VecGroup *vecs, uint32_t nvecs, uint32_t *ticket,
                                double *out_r, uint64_t *out_c, int TS, cudaStream_t stream)
{
    // Whole-warp segments take the configured 16 per thread where the plan
    // was cut in tiles of 8 (pieces need not be whole tiles of the kernel).
    GenLaunch g = g0;
    if (vec_mode(g, TS) >= 1 && g.modexp == MODEXP_CRT32 && g.threads == kVecTunedThreads &&
        g.L == kVecTunedL && g.L_wide == kVecWideL)
        g.L = kVecWideL;
    switch (vec_div(g.divide)) {
    case DIVIDE_EXACT:
        return launch_vec_d<DIVIDE_EXACT>(g, t, items, vecs, nvecs, ticket, out_r, out_c, TS,
                                          stream);
    case DIVIDE_INT:
        return launch_vec_d<DIVIDE_INT>(g, t, items, vecs, nvecs, ticket, out_r, out_c, TS,
                                        stream);
    default:
        return launch_vec_d<DIVIDE_RECIP>(g, t, items, vecs, nvecs, ticket, out_r, out_c, TS,
                                          stream);
    }
}

int vec_blocks_per_sm(const GenLaunch &g, size_t smem)
{
    const void *k = vec_kernel_ptr(g, g.stride == 1 ? 2 : 0);
    if (!k)
        return 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, g.threads, smem) != cudaSuccess)
        return 0;
    return blocks;
}

}  // namespace rsaprng
