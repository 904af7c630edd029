// Fused consumer of the generator: the outputs of a batch of streams are
// binned into a histogram inside the generation kernel instead of being
// stored (arXiv:1811.11629 Sec. VII: the one-dimensional frequency test and
// the D-dimensional serial test). The tile engine is the one of k_generate
// (skips, block scan, messages, ciphertexts, division); only step 5 differs:
//   5'. each output becomes a digit in [0, d) -- floor(r d) of its float
//       output r, or c mod d of its ciphertext for d a power of two -- the
//       digits of a tile are staged in shared memory, and every D-tuple of
//       consecutive outputs (r_{kD+1}, ..., r_{kD+D}) of a request that ends
//       in the tile adds one to bin sum_i digit_{kD+i} d^(i-1). Tuples that
//       begin in the previous tile take its last D-1 digits from a carry.
//       When D divides L no tuple leaves a thread's run and the tuples are
//       binned from registers without staging.
// Work items start on tuple boundaries (the planner cuts pieces in multiples
// of D), so no tuple spans two blocks.
#include "device_math.cuh"
#include "kernels.cuh"
#include "tile.cuh"

namespace rsaprng {

namespace {

using dev::addmod;
using dev::mulmodQ;
using tile::to_unit;

// floor(r d), exactly, for a double r in [0, 1) and d < 2^32. A normal r is
// M 2^(E - 1075) with M its 53-bit significand and E its biased exponent, so
// floor(r d) = (M d) >> (1075 - E) with M d < 2^85; subnormal r give 0. For
// d = 2^k it is M >> (1075 - E - k), a shift (the shift is at least 22, so
// the result fits 32 bits), which spares the multiply pipe the product.
__device__ __forceinline__ uint32_t digit_of_unit(double r, uint32_t d)
{
    const u64 b = (u64)__double_as_longlong(r);
    const int E = (int)(b >> 52);
    if (E == 0)
        return 0;
    const u64 M = (b & ((1ULL << 52) - 1)) | (1ULL << 52);
    const int sh = 1075 - E;  // >= 53 since r < 1
    if ((d & (d - 1)) == 0) {
        const int s2 = sh - (__ffs(d) - 1);
        return s2 >= 64 ? 0u : (uint32_t)(M >> s2);
    }
    const u64 lo = M * d, hi = __umul64hi(M, (u64)d);
    if (sh >= 128)
        return 0;
    if (sh >= 64)
        return (uint32_t)(hi >> (sh - 64));
    return (uint32_t)((lo >> sh) | (hi << (64 - sh)));
}

// Bins the whole DD-tuples of one thread's run of L digits (DD divides L;
// the run starts on a tuple boundary); nvalid digits are valid.
template <int L, int DD>
__device__ __forceinline__ void bin_run(const uint32_t (&g)[L], int nvalid, uint32_t d,
                                        unsigned long long *hist)
{
#pragma unroll
    for (int k0 = 0; k0 + DD <= L; k0 += DD) {
        if (k0 + DD <= nvalid) {
            uint32_t bin = 0, w = 1;
#pragma unroll
            for (int i = 0; i < DD; i++) {
                bin += g[k0 + i] * w;
                w *= d;
            }
            atomicAdd(hist + bin, 1ULL);
        }
    }
}

template <int L, int MODEXP, int DIV>
__global__ void __launch_bounds__(512) k_histogram(DeviceTables tab, const WorkItem *__restrict__ items,
                                                   uint32_t nitems, uint32_t *ticket, HistArgs h)
{
    tile::pdl_wait();  // the start states of the pieces, from the start-state scan
    extern __shared__ uint32_t dig[];  // S digits of the tile, then the carry (D - 1 <= 7)
    __shared__ u64 sh_scan[32];
    __shared__ uint32_t sh_item;
    const int T = blockDim.x, t = threadIdx.x;
    const int S = T * L;
    const int my0 = t * L;
    const uint32_t D = h.D, d = h.d;
    uint32_t *carry = dig + S;

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
        u64 s_thr = mulmodQ(s, plin[t * L]);
        const u64 aS = plin[S];
        const u64 count = W.count;
        for (u64 base = 0; base < count; base += S) {
            const u64 left = count - base;
            const int tile_n = left < (u64)S ? (int)left : S;
            const int nvalid = tile_n - my0 < 0 ? 0 : (tile_n - my0 > L ? L : tile_n - my0);
            u64 c[L], total;
            tile::tile_ciphertexts<L, MODEXP>(tab, W, P, m, s_thr, left, my0, nvalid, sh_scan, c,
                                              total);
            uint32_t g[L];
#pragma unroll
            for (int j = 0; j < L; j++)
                g[j] = h.low ? (uint32_t)(c[j] & (d - 1))
                             : digit_of_unit(to_unit<DIV>(c[j], P, j), d);
            // Tuples of D dividing L never cross a thread's run (it starts on
            // a multiple of L, hence of D): bin them from registers.
            if (D == 1 || (D == 2 && L % 2 == 0) || (D == 4 && L % 4 == 0) ||
                (D == 8 && L % 8 == 0)) {
                if (D == 1)
                    bin_run<L, 1>(g, nvalid, d, h.hist);
                else if (D == 2)
                    bin_run<L, 2>(g, nvalid, d, h.hist);
                else if (D == 4)
                    bin_run<L, 4>(g, nvalid, d, h.hist);
                else
                    bin_run<L, 8>(g, nvalid, d, h.hist);
                m = addmod(m, total, n);
                s_thr = mulmodQ(s_thr, aS);
                continue;
            }
#pragma unroll
            for (int j = 0; j < L; j++)
                if (j < nvalid)
                    dig[my0 + j] = g[j];
            __syncthreads();
            // Tuples k (counted from the item's start) whose last output lies
            // in this tile: base <= kD + D - 1 < base + tile_n.
            const u64 k_end = (base + (u64)tile_n) / D;
            for (u64 k = base / D + t; k < k_end; k += T) {
                uint32_t bin = 0, w = 1;
                for (uint32_t i = 0; i < D; i++) {
                    const u64 pos = k * D + i;
                    const uint32_t g = pos >= base ? dig[pos - base] : carry[pos + (D - 1) - base];
                    bin += g * w;
                    w *= d;
                }
                atomicAdd(h.hist + bin, 1ULL);
            }
            __syncthreads();
            if ((uint32_t)t + 1 < D && tile_n >= (int)D - 1)
                carry[t] = dig[tile_n - (int)(D - 1) + t];
            __syncthreads();
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
}

template <int L, int MODEXP, int DIV>
cudaError_t launch_hist_t(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                          uint32_t nitems, uint32_t *ticket, const HistArgs &h, cudaStream_t stream)
{
    const size_t smem = hist_smem_bytes(g.threads, L);
    return launch_kernel(k_histogram<L, MODEXP, DIV>, g.grid, g.threads, smem, stream, g.pdl, t,
                         items, nitems, g.persistent ? ticket : nullptr, h);
}

// The float digits need r itself, which every division route gives bit for
// bit: the integer route and the reciprocal route are instantiated, and the
// other two map to the reciprocal one; the exact-rational reading has its own.
template <int DIV>
const void *hist_kernel_ptr_l(int L, int modexp)
{
    if (modexp == MODEXP_CRT32) {
        if (L == 16)
            return (const void *)k_histogram<16, MODEXP_CRT32, DIV>;
        if (L == 8)
            return (const void *)k_histogram<8, MODEXP_CRT32, DIV>;
        if (L == 4)
            return (const void *)k_histogram<4, MODEXP_CRT32, DIV>;
        if (L == 2)
            return (const void *)k_histogram<2, MODEXP_CRT32, DIV>;
    } else {
        if (L == 8)
            return (const void *)k_histogram<8, MODEXP_MONT64, DIV>;
        if (L == 4)
            return (const void *)k_histogram<4, MODEXP_MONT64, DIV>;
        if (L == 2)
            return (const void *)k_histogram<2, MODEXP_MONT64, DIV>;
    }
    return nullptr;
}

const void *hist_kernel_ptr(const GenLaunch &g)
{
    if (g.divide == DIVIDE_EXACT)
        return hist_kernel_ptr_l<DIVIDE_EXACT>(g.L, g.modexp);
    return g.divide == DIVIDE_INT ? hist_kernel_ptr_l<DIVIDE_INT>(g.L, g.modexp)
                                  : hist_kernel_ptr_l<DIVIDE_RECIP>(g.L, g.modexp);
}

template <int DIV>
cudaError_t launch_hist_div(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                            uint32_t nitems, uint32_t *ticket, const HistArgs &h,
                            cudaStream_t stream)
{
#define RSAPRNG_HIST(LL, MM)                                                     \
    if (g.L == LL && g.modexp == MM)                                             \
        return launch_hist_t<LL, MM, DIV>(g, t, items, nitems, ticket, h, stream);
    RSAPRNG_HIST(16, MODEXP_CRT32)
    RSAPRNG_HIST(8, MODEXP_CRT32)
    RSAPRNG_HIST(4, MODEXP_CRT32)
    RSAPRNG_HIST(2, MODEXP_CRT32)
    RSAPRNG_HIST(8, MODEXP_MONT64)
    RSAPRNG_HIST(4, MODEXP_MONT64)
    RSAPRNG_HIST(2, MODEXP_MONT64)
#undef RSAPRNG_HIST
    return cudaErrorInvalidValue;
}

}  // namespace

size_t hist_smem_bytes(int threads, int L) { return ((size_t)threads * L + 8) * sizeof(uint32_t); }

cudaError_t launch_histogram(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                             uint32_t nitems, uint32_t *ticket, const HistArgs &h,
                             cudaStream_t stream)
{
    if (g.divide == DIVIDE_EXACT)
        return launch_hist_div<DIVIDE_EXACT>(g, t, items, nitems, ticket, h, stream);
    if (g.divide == DIVIDE_INT)
        return launch_hist_div<DIVIDE_INT>(g, t, items, nitems, ticket, h, stream);
    return launch_hist_div<DIVIDE_RECIP>(g, t, items, nitems, ticket, h, stream);
}

int hist_blocks_per_sm(const GenLaunch &g)
{
    const void *k = hist_kernel_ptr(g);
    if (!k)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, g.threads,
                                                      hist_smem_bytes(g.threads, g.L)) !=
        cudaSuccess)
        return 0;
    return blocks;
}

}  // namespace rsaprng
