// Generation kernels for the RSA-exponentiation generator (arXiv:1811.11629).
//
// Tile engine. A block of T threads walks one stream in tiles of S = T L
// outputs; thread t owns the L consecutive outputs tL+1 .. tL+L of a tile:
//   1. skips: its first skip is s_tile a^(tL) (power table), then L steps of
//      s <- a s mod Q with the 32-bit multiplier (Eq. congruentialgenerator1);
//   2. messages: the skips are summed per thread, a block-wide exclusive
//      scan mod n gives each thread the message before its run, and a
//      running carry links the tiles (Sec. IV, m_k = m_{k-1} + s_k); inside
//      a thread's run the messages are 64-bit representatives mod n, not
//      reduced, since step 3 needs only their residues mod p and mod q;
//   3. encryption of the L messages as independent chains (Eq. encrypt2);
//   4. r = c / n (Eq. CodeFloatingPointStep) and the 1.0 guard;
//   5. outputs are staged in shared memory and written with coalesced stores.
// Long streams are cut into chunks; a skip-sum pass over the chunks and a
// scan per instance give every chunk its start state, so no block ever waits
// for another (no inter-block spin).
#include <cstdio>
#include <cstring>

#include "device_math.cuh"
#include "kernels.cuh"
#include "tile.cuh"

namespace rsaprng {

using dev::add_carry_count;
using dev::add_cong;
using dev::mulmod_small_count;
using dev::addmod;
using dev::mulmodQ;
using dev::mulmodQ_small;
using dev::reduce_u64;

namespace {

using tile::bulk_store_rows;
using tile::bulk_wait_all;
using tile::fence_async_shared;
using tile::FULL;
using tile::pdl_trigger;
using tile::put;
using tile::stage_elements;
using tile::stage_run;
using tile::store_elements;
using tile::swz;
using tile::pdl_wait;
using tile::block_exscan_mod;
using tile::block_reduce_mod;
using tile::to_unit;

// The default tile (128 threads x 16 outputs on the CRT route) also has an
// instantiation with a 128-thread, 5-blocks-per-SM launch bound (TB = 128):
// the compiler then plans its registers for exactly that occupancy (measured
// 2 % faster than the generic bound). Other tiles use TB = 0 (up to 512).
constexpr int kTunedThreads = 128;
template <int L, int MODEXP>
constexpr bool tuned_tile()
{
    return L == 16 && MODEXP == MODEXP_CRT32;
}

// U < L: the encryption runs in passes of U chains (the unroll knob).
//
// Output of a tile. Every thread stages its L outputs in the swizzled layout
// of one of nbuf staging buffers per output kind; full tiles leave by bulk
// tensor stores of whole 16-element lines issued by thread 0, other tiles by
// the block's element stores.
//  - With two buffers (stride 1, the SHIFT variant) the staging is shifted
//    by x0 = the item's first output mod 16, so that staging line l holds line (o >> 4) + l of
//    the arrays. The tile's last x0 outputs then fill the first x0 places of
//    the next line, which the tile copies to the head of the other buffer:
//    the next tile stores its first line whole, carried head included. An
//    item's first tile, when x0 != 0, and its ragged last tile use element
//    stores (with the carried head); a last full tile stores its tail by
//    elements. An output written twice is written with the same bits.
//  - Otherwise a tile is stored in bulk when its first output is a multiple
//    of 16 elements into the arrays (the variant without SHIFT carries none
//    of the shift's code: measured 5 % faster at e = 3 with two outputs).
// A buffer is written again only after its bulk stores have read it: with
// two buffers thread 0 waits for the stores of the tile before (which had a
// whole tile of computation to finish) ahead of the barrier that follows the
// staging; with one it waits ahead of an extra barrier before the staging.
// Thread 0 waits for all its bulk stores to complete before the block exits.
template <int L, int MODEXP, int DIV, int TB, int U = L, bool SHIFT = false>
__global__ void __launch_bounds__(TB ? TB : 512, TB ? 5 : 1)
    k_generate(DeviceTables tab, const WorkItem *__restrict__ items, uint32_t nitems,
               uint32_t *ticket, double *__restrict__ out_r, u64 *__restrict__ out_c, u64 stride,
               const __grid_constant__ StoreMaps maps)
{
    static_assert(L % 2 == 0, "a thread stages whole 16-byte chunks");
    pdl_wait();  // the start states of the pieces, from the start-state scan
    extern __shared__ u64 smem[];
    __shared__ u64 sh_scan[32];
    __shared__ uint32_t sh_item;
    const int T = blockDim.x, t = threadIdx.x;
    const int S = T * L;
    // staging buffers, 1024-byte aligned (the swizzle pattern repeats every 1 KB)
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    u64 *const stage = smem + (((sbase + 1023u) & ~1023u) - sbase) / 8;
    const int kinds = (out_r ? 1 : 0) + (out_c ? 1 : 0);
    const int nbuf = maps.nbuf;
    const bool shifted = SHIFT && nbuf == 2 && stride == 1;
    const int SB = stage_elements(S, nbuf);  // elements per staging buffer
    const int rows = S >> 4;
    uint32_t tiles = 0;    // tiles this block has staged
    bool pending = false;  // thread 0: bulk stores issued and not yet waited for

    uint32_t it = blockIdx.x;
    if (ticket) {
        if (t == 0)
            sh_item = atomicAdd(ticket, 1u);
        __syncthreads();
        it = sh_item;
    }
    while (it < nitems) {
        const WorkItem W = items[it];
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
        // Skip at the start of this thread's run in the first tile.
        u64 s_thr = mulmodQ(s, plin[t * L]);
        const u64 aS = plin[S];
        const u64 count = W.count;
        const int x0 = shifted ? (int)(W.out_off & 15) : 0;
        for (u64 base = 0; base < count; base += S) {
            const u64 left = count - base;
            const int tile_n = left < (u64)S ? (int)left : S;
            const int my0 = t * L;
            const int nvalid = tile_n - my0 < 0 ? 0 : (tile_n - my0 > L ? L : tile_n - my0);
            u64 c[L], total;
            tile::tile_ciphertexts<L, MODEXP, U>(tab, W, P, m, s_thr, left, my0, nvalid, sh_scan, c,
                                              total);
            const int b = (int)(tiles % (uint32_t)nbuf);
            u64 *const st_r = stage + (size_t)b * kinds * SB;
            u64 *const st_c = st_r + (out_r ? SB : 0);
            if (nbuf == 1) {
                if (t == 0 && pending)
                    bulk_wait_all<true>();
                __syncthreads();
            }
            if (out_r && x0 == 0) {  // each pair divided as it is staged (fewer live registers)
#pragma unroll
                for (int k = 0; k < L / 2; k++)
                    *reinterpret_cast<ulonglong2 *>(st_r + swz(my0 + 2 * k)) = make_ulonglong2(
                        (u64)__double_as_longlong(to_unit<DIV>(c[2 * k], P, 2 * k)),
                        (u64)__double_as_longlong(to_unit<DIV>(c[2 * k + 1], P, 2 * k + 1)));
            } else if (out_r) {
                u64 v[L];
#pragma unroll
                for (int j = 0; j < L; j++)
                    v[j] = (u64)__double_as_longlong(to_unit<DIV>(c[j], P, j));
                stage_run<L>(st_r, my0, x0, v);
            }
            if (out_c)
                stage_run<L>(st_c, my0, x0, c);
            const u64 o = W.out_off + base * stride;
            const bool first = base == 0, last = left <= (u64)S;
            const bool bulk = maps.extent && stride == 1 && tile_n == S &&
                              (int)(o & 15) == x0 && (x0 == 0 || !first) &&
                              o - x0 + (u64)S <= maps.extent;
            if (bulk)
                fence_async_shared();  // the staging, visible to the bulk copies
            if (nbuf == 2 && t == 0 && pending)
                bulk_wait_all<true>();
            __syncthreads();
            tiles++;
            if (bulk) {
                if (t == 0) {
                    if (out_r)
                        bulk_store_rows(&maps.r, st_r, rows, maps.box_rows, (o - x0) >> 4);
                    if (out_c)
                        bulk_store_rows(&maps.c, st_c, rows, maps.box_rows, (o - x0) >> 4);
                    pending = true;
                }
                if (last && t < x0) {  // the tail beyond the last whole line
                    if (out_r)
                        put(out_r + o + S - x0 + t, st_r[swz(S + t)]);
                    if (out_c)
                        put(out_c + o + S - x0 + t, st_c[swz(S + t)]);
                }
            } else {
                if (out_r)
                    store_elements(out_r + o, st_r, tile_n, x0, stride);
                if (out_c)
                    store_elements(out_c + o, st_c, tile_n, x0, stride);
                if (!first && t < x0) {  // the carried head, which a bulk tile leaves
                    if (out_r)
                        put(out_r + o - x0 + t, st_r[swz(t)]);
                    if (out_c)
                        put(out_c + o - x0 + t, st_c[swz(t)]);
                }
            }
            if (!last && t < x0) {  // carry the tail to the head of the other buffer
                const size_t nb = (size_t)(1 - b) * kinds * SB;
                if (out_r)
                    stage[nb + swz(t)] = st_r[swz(S + t)];
                if (out_c)
                    stage[nb + (out_r ? SB : 0) + swz(t)] = st_c[swz(S + t)];
            }
            m = addmod(m, total, n);
            s_thr = mulmodQ(s_thr, aS);
        }
        if ((W.flags & WI_WRITEBACK) && t == 0) {
            tab.state_m[W.inst] = m;
            if (count == 0)
                tab.state_s[W.inst] = s;
        }
        if (ticket) {
            __syncthreads();
            if (t == 0)
                sh_item = atomicAdd(ticket, 1u);
            __syncthreads();
            it = sh_item;
        } else {
            it += gridDim.x;
        }
    }
    if (t == 0 && pending)
        bulk_wait_all<false>();
}

// Skip sums of chunks: for chunk k with start offset o and length len,
// chunk_s[k] = s a^o mod Q (the skip before its first output) and
// chunk_sum[k] = sum_{x=1..len} (s a^(o+x) mod Q) mod n, where s is the
// instance's current skip. One warp per chunk: the jump a^o is the product
// of the table powers a^(2^b) over the set bits b of o, two bits per lane
// and a butterfly over the lanes; the sum runs in tiles of 32 lanes x 8
// skips and ends in a warp reduction. The last chunk of an instance is
// listed with len = 0: no later chunk needs its sum.
constexpr int kPrepT = 256;
constexpr int kPrepL = 8;
constexpr int kPrepWarps = kPrepT / 32;
__global__ void __launch_bounds__(kPrepT) k_prep_sums(DeviceTables tab,
                                                     const PrepChunk *__restrict__ chunks,
                                                     uint32_t nchunks, u64 *__restrict__ chunk_sum,
                                                     u64 *__restrict__ chunk_s)
{
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const uint32_t nw = gridDim.x * kPrepWarps;
    for (uint32_t k = blockIdx.x * kPrepWarps + (threadIdx.x >> 5); k < nchunks; k += nw) {
        const PrepChunk C = chunks[k];
        const InstParams P = tab.params[C.inst];
        const u64 n = P.n, r64 = P.r64;
        const u32 a = P.a;
        const u64 *plin = tab.pow_lin + (size_t)P.root * kPowLinRow;
        const u64 *p2k = tab.pow2k + (size_t)P.root * 64;
        // a^o: lane l takes bits 2l and 2l + 1 of o
        const int b0 = 2 * lane;
        u64 f = ((C.offset >> b0) & 1) ? p2k[b0] : 1;
        if ((C.offset >> (b0 + 1)) & 1)
            f = mulmodQ(f, p2k[b0 + 1]);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1)
            f = mulmodQ(f, __shfl_xor_sync(FULL, f, d));
        const u64 s0 = mulmodQ(tab.state_s[C.inst], f);
        if (lane == 0)
            chunk_s[k] = s0;
        constexpr int S = 32 * kPrepL;
        u64 s_thr = mulmodQ(s0, plin[lane * kPrepL]);
        const u64 aS = plin[S];
        // the lane's sum is acc + carries 2^64 (2^64 = r64 mod n)
        u64 acc = 0;
        u32 carries = 0;
        const int my0 = lane * kPrepL;
        u64 base = 0;
        for (; base + S <= C.len; base += S) {  // whole tiles
            u64 x = s_thr;
#pragma unroll
            for (int j = 0; j < kPrepL; j++) {
                x = mulmodQ_small(x, a);
                add_carry_count(acc, carries, x);
            }
            s_thr = mulmodQ(s_thr, aS);
        }
        if (base < C.len) {  // the ragged tail
            const int tile_n = (int)(C.len - base);
            const int nvalid = tile_n - my0 < 0 ? 0 : (tile_n - my0 > kPrepL ? kPrepL : tile_n - my0);
            u64 x = s_thr;
#pragma unroll
            for (int j = 0; j < kPrepL; j++) {
                x = mulmodQ_small(x, a);
                if (j < nvalid)
                    add_carry_count(acc, carries, x);
            }
        }
        u64 tot = reduce_u64(acc, n);
        u64 ncarry = carries;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            tot = addmod(tot, __shfl_xor_sync(FULL, tot, d), n);
            ncarry += __shfl_xor_sync(FULL, ncarry, d);
        }
        if (lane == 0)
            chunk_sum[k] = addmod(tot, mulmod_small_count(ncarry, r64, n), n);
    }
}

// Start states of the chunks of each instance: m before chunk j is the
// instance's m plus the skip sums of chunks 0..j-1 (mod n). One block per
// group (grid-stride): each thread takes a contiguous run of chunks, the
// block scans the run totals, and the threads write their chunks' states.
constexpr int kScanT = 128;
__global__ void __launch_bounds__(kScanT) k_prep_scan(DeviceTables tab,
                                                      const PrepGroup *__restrict__ groups,
                                                      uint32_t ngroups,
                                                      const PrepChunk *__restrict__ chunks,
                                                      const u64 *__restrict__ chunk_sum,
                                                      const u64 *__restrict__ chunk_s,
                                                      WorkItem *__restrict__ items)
{
    pdl_wait();  // the chunk sums of the pre-pass
    pdl_trigger();
    __shared__ u64 sh_scan[32];
    const int t = threadIdx.x;
    for (uint32_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const PrepGroup G = groups[g];
        const u64 n = tab.params[G.inst].n;
        const u64 m0 = tab.state_m[G.inst];
        const uint32_t per = (G.count + kScanT - 1) / kScanT;
        const uint32_t j0 = min((uint32_t)t * per, G.count);
        const uint32_t j1 = min(j0 + per, G.count);
        u64 run = 0;
        for (uint32_t j = j0; j < j1; j++)
            run = addmod(run, chunk_sum[G.first + j], n);
        u64 total;
        u64 m = addmod(m0, block_exscan_mod(run, n, sh_scan, total), n);
        for (uint32_t j = j0; j < j1; j++) {
            const uint32_t k = G.first + j;
            const uint32_t it = chunks[k].item;
            if (it != kNoItem) {
                items[it].m0 = m;
                items[it].s0 = chunk_s[k];
            }
            m = addmod(m, chunk_sum[k], n);
        }
        __syncthreads();  // sh_scan is reused by the next group
    }
}

// shift: a launch whose stores may go in bulk with two staging buffers and
// whose items do not all start at multiples of 16 elements (shifted
// staging); the default tile has that variant.
template <int L, int MODEXP, int DIV, int U = L>
auto gen_kernel(int threads, bool shift = false)
{
    if constexpr (tuned_tile<L, MODEXP>()) {
        if constexpr (U == L)
            if (threads == kTunedThreads && shift)
                return k_generate<L, MODEXP, DIV, kTunedThreads, U, true>;
        if (threads == kTunedThreads)
            return k_generate<L, MODEXP, DIV, kTunedThreads, U>;
    }
    return k_generate<L, MODEXP, DIV, 0, U>;
}

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (the library links no driver-API import library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

// The 2-D view [rows][16] of a 64-bit output array, 128-byte swizzled, boxes
// of box_rows lines.
bool encode_view(CUtensorMap *m, void *base, uint64_t rows, int box_rows)
{
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc)
        return false;
    const cuuint64_t dims[2] = {16, rows};
    const cuuint64_t strides[1] = {16 * sizeof(uint64_t)};
    const cuuint32_t box[2] = {16, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Whether p is (null or) memory of the current device: page-locked host
// memory that the kernel writes through its mapping, and another device's
// memory, keep the element stores.
bool device_or_null(const void *p)
{
    if (!p)
        return true;
    // The query enqueues nothing; relaxed capture mode for this thread keeps it
    // legal while a caller captures the stream into a graph.
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaThreadExchangeStreamCaptureMode(&mode);
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    cudaThreadExchangeStreamCaptureMode(&mode);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// The store maps of a launch: bulk stores need the contiguous order, a known
// output extent of at least one tile (and fewer than 2^31 lines, the range of
// a tensor coordinate), and 16-byte aligned arrays in device memory.
StoreMaps store_maps(const GenLaunch &g, int L, double *out_r, uint64_t *out_c)
{
    StoreMaps maps;
    memset(&maps, 0, sizeof maps);
    maps.nbuf = gen_stage_buffers(g.threads, L, out_r != nullptr, out_c != nullptr);
    const int lines = g.threads * L / 16;
    maps.box_rows = lines < 256 ? lines : 256;
    const uint64_t rows = g.out_extent / 16;
    const bool aligned = ((uintptr_t)out_r % 16) == 0 && ((uintptr_t)out_c % 16) == 0;
    if (g.stride != 1 || rows < (uint64_t)lines || rows >= (1ULL << 31) || !aligned ||
        !device_or_null(out_r) || !device_or_null(out_c))
        return maps;
    if (out_r && !encode_view(&maps.r, out_r, rows, maps.box_rows))
        return maps;
    if (out_c && !encode_view(&maps.c, out_c, rows, maps.box_rows))
        return maps;
    maps.extent = rows * 16;
    return maps;
}

template <int L, int MODEXP, int DIV, int U = L>
cudaError_t launch_gen_t(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                         uint32_t nitems, uint32_t *ticket, double *out_r, uint64_t *out_c,
                         cudaStream_t stream)
{
    const size_t smem = gen_smem_bytes(g.threads, L, out_r != nullptr, out_c != nullptr);
    const StoreMaps maps = store_maps(g, L, out_r, out_c);
    auto kern = gen_kernel<L, MODEXP, DIV, U>(g.threads,
                                              maps.extent && maps.nbuf == 2 && g.out_unaligned);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    return launch_kernel(kern, g.grid, g.threads, smem, stream, g.pdl, t, items, nitems,
                         g.persistent ? ticket : nullptr, out_r, out_c, (u64)g.stride, maps);
}

template <int L, int MODEXP, int DIV, int U = L>
const void *gen_kernel_ptr(int threads)
{
    return (const void *)gen_kernel<L, MODEXP, DIV, U>(threads);
}

// The tilings with a pass-limited (unroll) variant: 16 per thread on the CRT
// route (passes of 8) and 8 per thread with reciprocal division (passes of 4).
#define RSAPRNG_UNROLLED(X)                      \
    X(16, MODEXP_CRT32, DIVIDE_RECIP, 8)         \
    X(16, MODEXP_CRT32, DIVIDE_HYBRID, 8)        \
    X(16, MODEXP_CRT32, DIVIDE_INT, 8)           \
    X(8, MODEXP_CRT32, DIVIDE_RECIP, 4)

const void *select_kernel(int L, int modexp, int divide, int threads, int unroll)
{
    if (unroll > 0 && unroll < L) {
#define RSAPRNG_SELU(LL, MM, DD, UU)                                         \
    if (L == LL && modexp == MM && divide == DD && unroll == UU)             \
        return gen_kernel_ptr<LL, MM, DD, UU>(threads);
        RSAPRNG_UNROLLED(RSAPRNG_SELU)
#undef RSAPRNG_SELU
        return nullptr;
    }
#define RSAPRNG_SEL(LL, MM, DD)                                   \
    if (L == LL && modexp == MM && divide == DD)                  \
        return gen_kernel_ptr<LL, MM, DD>(threads);
    RSAPRNG_SEL(2, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_SEL(4, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_SEL(8, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_SEL(16, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_SEL(16, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_SEL(16, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_SEL(16, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_SEL(2, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_SEL(4, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_SEL(8, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_SEL(2, MODEXP_MONT64, DIVIDE_INT)
    RSAPRNG_SEL(4, MODEXP_MONT64, DIVIDE_INT)
    RSAPRNG_SEL(8, MODEXP_MONT64, DIVIDE_INT)
    RSAPRNG_SEL(2, MODEXP_MONT64, DIVIDE_FP64)
    RSAPRNG_SEL(4, MODEXP_MONT64, DIVIDE_FP64)
    RSAPRNG_SEL(8, MODEXP_MONT64, DIVIDE_FP64)
    RSAPRNG_SEL(2, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_SEL(4, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_SEL(8, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_SEL(2, MODEXP_MONT64, DIVIDE_HYBRID)
    RSAPRNG_SEL(4, MODEXP_MONT64, DIVIDE_HYBRID)
    RSAPRNG_SEL(8, MODEXP_MONT64, DIVIDE_HYBRID)
    RSAPRNG_SEL(2, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_SEL(4, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_SEL(8, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_SEL(2, MODEXP_MONT64, DIVIDE_RECIP)
    RSAPRNG_SEL(4, MODEXP_MONT64, DIVIDE_RECIP)
    RSAPRNG_SEL(8, MODEXP_MONT64, DIVIDE_RECIP)
    RSAPRNG_SEL(2, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_SEL(4, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_SEL(8, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_SEL(16, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_SEL(2, MODEXP_MONT64, DIVIDE_EXACT)
    RSAPRNG_SEL(4, MODEXP_MONT64, DIVIDE_EXACT)
    RSAPRNG_SEL(8, MODEXP_MONT64, DIVIDE_EXACT)
#undef RSAPRNG_SEL
    return nullptr;
}

// The output step alone: r[i] = RN(RN(c[i]) / RN(n)) with the 1.0 guard.
// Element i takes the route of output i mod 4 of a thread's run, so the
// hybrid route sends every fourth element through the integer division.
template <int DIV>
__global__ void k_unit(const InstParams *__restrict__ params, uint32_t id,
                       const u64 *__restrict__ c, double *__restrict__ r, u64 N)
{
    const InstParams P = params[id];
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        r[i] = to_unit<DIV>(c[i], P, (int)(i & 3));
}

// ---------------------------------------------------------------- microbenchmarks

// 32-bit integer multiply-add throughput: each thread runs 8 independent
// chains of x <- x * k + c (IMAD) so the pipe, not latency, is the limit.
__global__ void k_mb_imad(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t x[8];
#pragma unroll
    for (int j = 0; j < 8; j++)
        x[j] = seed + threadIdx.x * 8 + j;
    const uint32_t k = 0x9E3779B1u ^ seed;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++)
            x[j] = x[j] * k + (uint32_t)j;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; j++)
        acc ^= x[j];
    if (acc == 0x12345678u)
        sink[0] = acc;
}

// Multiply-instruction shapes: 0 = widening 32x32->64 (IMAD.WIDE), 1 = high
// half (IMAD.HI), 2 = one 32-bit Montgomery product (as in the chains).
template <int S>
__global__ void k_mb_mul(uint32_t iters, uint32_t k, uint32_t p, uint32_t pinv, uint32_t *sink)
{
    uint32_t x[8];
    uint64_t w[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        x[j] = (threadIdx.x * 8 + j + 1) % p;
        w[j] = x[j];
    }
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (S == 0)
                w[j] = (uint64_t)(uint32_t)w[j] * k + (w[j] >> 32);
            else if (S == 1)
                x[j] = __umulhi(x[j], k) ^ (uint32_t)j;
            else
                x[j] = dev::mont32(x[j], x[j], p, pinv);
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; j++)
        acc ^= x[j] ^ (uint32_t)w[j];
    if (acc == 0x12345678u)
        sink[0] = acc;
}

__global__ void k_mb_ddiv(uint32_t iters, double seed, double *sink)
{
    double x[4];
#pragma unroll
    for (int j = 0; j < 4; j++)
        x[j] = seed + threadIdx.x + j;
    const double d = 1.0000001;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++)
            x[j] = __ddiv_rn(x[j], d);
    }
    double acc = x[0] + x[1] + x[2] + x[3];
    if (acc == 1.2345)
        sink[0] = acc;
}

// FP64 pipe shapes, 8 independent chains per thread: 0 = fused multiply-add,
// 1 = unsigned 64-bit integer to double conversion, 2 = the whole reciprocal
// output step (conversion, product, two FMAs and the 1.0 guard) as the
// generation kernels run it. Each result feeds the next input of its chain
// so that nothing is hoisted out of the loop; the integer feedback is a few
// ALU instructions beside the FP64 ones.
template <int S>
__global__ void k_mb_fp64(uint32_t iters, u64 seed, double dn, double y, u64 *sink)
{
    u64 c[8];
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        c[j] = (seed + (u64)(threadIdx.x * 8 + j) * 0x9E3779B97F4A7C15ULL) >> 2;
        x[j] = (double)(threadIdx.x * 8 + j) * 0x1p-20 + 1.0;
    }
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if constexpr (S == 0) {
                x[j] = __fma_rn(x[j], 0.99999999999, 1e-12);
            } else if constexpr (S == 1) {
                c[j] += (u64)__double_as_longlong(__ull2double_rn(c[j])) >> 12;
            } else {
                const double r = dev::unit_recip(c[j], dn, y);
                c[j] = (c[j] + (u64)__double_as_longlong(r)) & 0x3FFFFFFFFFFFFFFFULL;
            }
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int j = 0; j < 8; j++)
        acc ^= c[j] ^ (u64)__double_as_longlong(x[j]);
    if (acc == 0x123456789ULL)
        sink[0] = acc;
}

__global__ void k_mb_write(uint4 *buf, size_t n16)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
        buf[i] = make_uint4((uint32_t)i, 1u, 2u, 3u);
}

int num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <typename F>
cudaError_t time_it(F &&launch, cudaStream_t stream, float *ms)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a, stream);
    launch();
    cudaEventRecord(b, stream);
    cudaError_t e = cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}

}  // namespace

// Two staging buffers per output kind (one barrier per tile fewer) while
// they take at most 40 KB, which keeps five 128-thread blocks of 16 outputs
// per thread on an SM; else one.
int gen_stage_buffers(int threads, int L, bool want_r, bool want_c)
{
    const size_t bytes = (size_t)threads * L * 8 * ((want_r ? 1 : 0) + (want_c ? 1 : 0));
    return 2 * bytes <= 40 * 1024 ? 2 : 1;
}

size_t gen_smem_bytes(int threads, int L, bool want_r, bool want_c)
{
    const int nbuf = gen_stage_buffers(threads, L, want_r, want_c);
    return (size_t)nbuf * stage_elements(threads * L, nbuf) * 8 *
               ((want_r ? 1 : 0) + (want_c ? 1 : 0)) +
           1024;
}

size_t padded_smem_bytes(int threads, int L, bool want_r, bool want_c)
{
    const size_t S = (size_t)threads * L;
    const size_t slots = S + (S >> 4);
    return slots * 8 * ((want_r ? 1 : 0) + (want_c ? 1 : 0));
}

cudaError_t launch_generate(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                            uint32_t nitems, uint32_t *ticket, double *out_r, uint64_t *out_c,
                            cudaStream_t stream)
{
    if (g.unroll > 0 && g.unroll < g.L) {
#define RSAPRNG_DISPATCHU(LL, MM, DD, UU)                                                   \
    if (g.L == LL && g.modexp == MM && g.divide == DD && g.unroll == UU)                    \
        return launch_gen_t<LL, MM, DD, UU>(g, t, items, nitems, ticket, out_r, out_c, stream);
        RSAPRNG_UNROLLED(RSAPRNG_DISPATCHU)
#undef RSAPRNG_DISPATCHU
        return cudaErrorNotSupported;  // no pass-limited kernel for this tiling
    }
#define RSAPRNG_DISPATCH(LL, MM, DD)                                                      \
    if (g.L == LL && g.modexp == MM && g.divide == DD)                                    \
        return launch_gen_t<LL, MM, DD>(g, t, items, nitems, ticket, out_r, out_c, stream);
    RSAPRNG_DISPATCH(2, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_DISPATCH(4, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_DISPATCH(8, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_DISPATCH(16, MODEXP_CRT32, DIVIDE_INT)
    RSAPRNG_DISPATCH(16, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_DISPATCH(16, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_DISPATCH(16, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_DISPATCH(2, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_DISPATCH(4, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_DISPATCH(8, MODEXP_CRT32, DIVIDE_FP64)
    RSAPRNG_DISPATCH(2, MODEXP_MONT64, DIVIDE_INT)
    RSAPRNG_DISPATCH(4, MODEXP_MONT64, DIVIDE_INT)
    RSAPRNG_DISPATCH(8, MODEXP_MONT64, DIVIDE_INT)
    RSAPRNG_DISPATCH(2, MODEXP_MONT64, DIVIDE_FP64)
    RSAPRNG_DISPATCH(4, MODEXP_MONT64, DIVIDE_FP64)
    RSAPRNG_DISPATCH(8, MODEXP_MONT64, DIVIDE_FP64)
    RSAPRNG_DISPATCH(2, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_DISPATCH(4, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_DISPATCH(8, MODEXP_CRT32, DIVIDE_HYBRID)
    RSAPRNG_DISPATCH(2, MODEXP_MONT64, DIVIDE_HYBRID)
    RSAPRNG_DISPATCH(4, MODEXP_MONT64, DIVIDE_HYBRID)
    RSAPRNG_DISPATCH(8, MODEXP_MONT64, DIVIDE_HYBRID)
    RSAPRNG_DISPATCH(2, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_DISPATCH(4, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_DISPATCH(8, MODEXP_CRT32, DIVIDE_RECIP)
    RSAPRNG_DISPATCH(2, MODEXP_MONT64, DIVIDE_RECIP)
    RSAPRNG_DISPATCH(4, MODEXP_MONT64, DIVIDE_RECIP)
    RSAPRNG_DISPATCH(8, MODEXP_MONT64, DIVIDE_RECIP)
    RSAPRNG_DISPATCH(2, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_DISPATCH(4, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_DISPATCH(8, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_DISPATCH(16, MODEXP_CRT32, DIVIDE_EXACT)
    RSAPRNG_DISPATCH(2, MODEXP_MONT64, DIVIDE_EXACT)
    RSAPRNG_DISPATCH(4, MODEXP_MONT64, DIVIDE_EXACT)
    RSAPRNG_DISPATCH(8, MODEXP_MONT64, DIVIDE_EXACT)
#undef RSAPRNG_DISPATCH
    return cudaErrorInvalidValue;
}

bool gen_has_unroll(int L, int modexp, int divide, int unroll)
{
    return select_kernel(L, modexp, divide, 128, unroll) != nullptr;
}

int gen_blocks_per_sm(const GenLaunch &g, size_t smem)
{
    const void *k = select_kernel(g.L, g.modexp, g.divide, g.threads, g.unroll);
    if (!k)
        return 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, g.threads, smem) != cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_prep_sums(const DeviceTables &t, const PrepChunk *chunks, uint32_t nchunks,
                             uint64_t *chunk_sum, uint64_t *chunk_s, cudaStream_t stream)
{
    if (nchunks == 0)
        return cudaSuccess;
    const uint32_t blocks = (nchunks + kPrepWarps - 1) / kPrepWarps;
    const int grid = (int)(blocks < 65535u ? blocks : 65535u);
    k_prep_sums<<<grid, kPrepT, 0, stream>>>(t, chunks, nchunks, chunk_sum, chunk_s);
    return cudaGetLastError();
}

cudaError_t launch_prep_scan(const DeviceTables &t, const PrepGroup *groups, uint32_t ngroups,
                             const PrepChunk *chunks, const uint64_t *chunk_sum,
                             const uint64_t *chunk_s, WorkItem *items, cudaStream_t stream)
{
    if (ngroups == 0)
        return cudaSuccess;
    const int grid = (int)(ngroups < 65535u ? ngroups : 65535u);
    // always right after the pre-pass: a programmatic dependent of it
    return launch_kernel(k_prep_scan, grid, kScanT, 0, stream, true, t, groups, ngroups, chunks,
                         chunk_sum, chunk_s, items);
}

cudaError_t launch_unit(const DeviceTables &t, uint32_t id, uint64_t N, const uint64_t *c,
                        double *r, int divide, cudaStream_t stream)
{
    if (N == 0)
        return cudaSuccess;
    const int grid = num_sms() * 8;
    if (divide == DIVIDE_EXACT)
        k_unit<DIVIDE_EXACT><<<grid, 256, 0, stream>>>(t.params, id, c, r, N);
    else if (divide == DIVIDE_FP64)
        k_unit<DIVIDE_FP64><<<grid, 256, 0, stream>>>(t.params, id, c, r, N);
    else if (divide == DIVIDE_RECIP)
        k_unit<DIVIDE_RECIP><<<grid, 256, 0, stream>>>(t.params, id, c, r, N);
    else if (divide == DIVIDE_HYBRID)
        k_unit<DIVIDE_HYBRID><<<grid, 256, 0, stream>>>(t.params, id, c, r, N);
    else
        k_unit<DIVIDE_INT><<<grid, 256, 0, stream>>>(t.params, id, c, r, N);
    return cudaGetLastError();
}

cudaError_t microbench_imad(double *gops, cudaStream_t stream)
{
    uint32_t *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 64);
    if (e != cudaSuccess)
        return e;
    const int sms = num_sms();
    const int grid = sms * 8, threads = 256;
    const uint32_t iters = 1 << 16;
    float ms = 0;
    e = time_it([&] { k_mb_imad<<<grid, threads, 0, stream>>>(iters, 7u, sink); }, stream, &ms);
    cudaFree(sink);
    *gops = (double)grid * threads * iters * 8 / (ms * 1e-3) / 1e9;
    return e;
}

cudaError_t microbench_mul(int shape, double *gops, cudaStream_t stream)
{
    uint32_t *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 64);
    if (e != cudaSuccess)
        return e;
    const int sms = num_sms();
    const int grid = sms * 8, threads = 256;
    const uint32_t iters = 1 << 12;
    const uint32_t p = 4294967291u;  // the largest prime below 2^32
    uint32_t pinv = p;
    for (int i = 0; i < 4; i++)
        pinv *= 2 - p * pinv;
    float ms = 0;
    if (shape == 0)
        e = time_it([&] { k_mb_mul<0><<<grid, threads, 0, stream>>>(iters, 12345u, p, pinv, sink); },
                    stream, &ms);
    else if (shape == 1)
        e = time_it([&] { k_mb_mul<1><<<grid, threads, 0, stream>>>(iters, 12345u, p, pinv, sink); },
                    stream, &ms);
    else
        e = time_it([&] { k_mb_mul<2><<<grid, threads, 0, stream>>>(iters, 12345u, p, pinv, sink); },
                    stream, &ms);
    cudaFree(sink);
    *gops = (double)grid * threads * iters * 8 / (ms * 1e-3) / 1e9;
    return e;
}

cudaError_t microbench_ddiv(double *gdiv, cudaStream_t stream)
{
    double *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 64);
    if (e != cudaSuccess)
        return e;
    const int sms = num_sms();
    const int grid = sms * 8, threads = 256;
    const uint32_t iters = 1 << 10;
    float ms = 0;
    e = time_it([&] { k_mb_ddiv<<<grid, threads, 0, stream>>>(iters, 3.0, sink); }, stream, &ms);
    cudaFree(sink);
    *gdiv = (double)grid * threads * iters * 4 / (ms * 1e-3) / 1e9;
    return e;
}

cudaError_t microbench_fp64(int shape, double *gops, cudaStream_t stream)
{
    u64 *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 64);
    if (e != cudaSuccess)
        return e;
    const int sms = num_sms();
    const int grid = sms * 8, threads = 256;
    const uint32_t iters = 1 << 10;
    // a modulus just below 2^63 and its correctly rounded reciprocal
    const double dn = 0x1.fffffffffffffp+62, y = 1.0 / dn;
    float ms = 0;
    if (shape == 0)
        e = time_it([&] { k_mb_fp64<0><<<grid, threads, 0, stream>>>(iters, 99, dn, y, sink); },
                    stream, &ms);
    else if (shape == 1)
        e = time_it([&] { k_mb_fp64<1><<<grid, threads, 0, stream>>>(iters, 99, dn, y, sink); },
                    stream, &ms);
    else
        e = time_it([&] { k_mb_fp64<2><<<grid, threads, 0, stream>>>(iters, 99, dn, y, sink); },
                    stream, &ms);
    cudaFree(sink);
    *gops = (double)grid * threads * iters * 8 / (ms * 1e-3) / 1e9;
    return e;
}

cudaError_t microbench_write(void *buf, size_t bytes, double *gbs, cudaStream_t stream)
{
    const int sms = num_sms();
    const size_t n16 = bytes / 16;
    float ms = 0;
    cudaError_t e = time_it(
        [&] { k_mb_write<<<sms * 8, 512, 0, stream>>>((uint4 *)buf, n16); }, stream, &ms);
    *gbs = (double)n16 * 16 / (ms * 1e-3) / 1e9;
    return e;
}

}  // namespace rsaprng
