// Device building blocks of the tile engine shared by the generation kernel
// and the fused consumers (arXiv:1811.11629 Sec. IV-V): the block scan of
// skips mod n, the division route, and steps 1-3 of a tile.
#pragma once
#include <cstdint>

#include "device_math.cuh"
#include "kernels.cuh"

namespace rsaprng {
namespace tile {

using dev::add_cong;
using dev::addmod;
using dev::mulmodQ;
using dev::mulmodQ_small;
using dev::reduce_u64;

constexpr unsigned FULL = 0xFFFFFFFFu;

// Programmatic dependent launch: a kernel launched as a programmatic
// dependent may start while the kernel before it on the stream finishes;
// it waits here, before it reads anything that kernel wrote, until that
// kernel has completed and its writes are visible (a no-op for a kernel
// launched the ordinary way).
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Lets the dependent kernel launch once every block of this kernel has
// started; called at block entry, so the dependent's waiting blocks never
// hold the place of a block of this kernel that has still to run.
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

// Padded shared-memory index: one 8-byte slot of padding every 16 elements
// spreads the stride-L writes of a warp over the banks.
__device__ __forceinline__ int sidx(int i) { return i + (i >> 4); }

// Block-wide exclusive scan of v (mod n). Returns the exclusive prefix and
// the block total. sh must hold 32 entries. Contains two __syncthreads().
__device__ __forceinline__ u64 block_exscan_mod(u64 v, u64 n, u64 *sh, u64 &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    u64 incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const u64 o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d)
            incl = addmod(incl, o, n);
    }
    if (lane == 31)
        sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        u64 w = lane < nwarps ? sh[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const u64 o = __shfl_up_sync(FULL, w, d);
            if (lane >= d)
                w = addmod(w, o, n);
        }
        sh[lane] = w;
    }
    __syncthreads();
    total = sh[nwarps - 1];
    const u64 wpre = warp > 0 ? sh[warp - 1] : 0;
    u64 ex = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0)
        ex = 0;
    return addmod(wpre, ex, n);
}

__device__ __forceinline__ u64 block_reduce_mod(u64 v, u64 n, u64 *sh)
{
    u64 total;
    (void)block_exscan_mod(v, n, sh, total);
    return total;
}

template <int L, int MODEXP>
__device__ __forceinline__ void encrypt(const u64 (&m)[L], u64 (&c)[L], const InstParams &P)
{
    if constexpr (MODEXP == MODEXP_CRT32)
        dev::encrypt_crt<L>(m, c, P);
    else
        dev::encrypt_mont64<L>(m, c, P);
}

// Encryption of a thread's L messages with at most U chains in flight: the
// L outputs run as L / U passes of U, and each pass takes an opaque zero
// computed from the last ciphertext of the pass before it, so the compiler
// cannot start a pass before the previous one has finished (fewer live
// registers, less instruction-level parallelism). U >= L: all at once.
template <int L, int MODEXP, int U>
__device__ __forceinline__ void encrypt_passes(const u64 (&m)[L], u64 (&c)[L], const InstParams &P)
{
    if constexpr (U >= L) {
        encrypt<L, MODEXP>(m, c, P);
    } else {
        static_assert(L % U == 0, "passes of equal size");
        u64 dep = 0;
#pragma unroll
        for (int g = 0; g < L / U; g++) {
            u64 mm[U], cc[U];
#pragma unroll
            for (int j = 0; j < U; j++)
                mm[j] = m[g * U + j] + dep;  // messages are representatives: + 0 changes nothing
            encrypt<U, MODEXP>(mm, cc, P);
#pragma unroll
            for (int j = 0; j < U; j++)
                c[g * U + j] = cc[j];
            asm volatile("and.b64 %0, %1, 0;" : "=l"(dep) : "l"(cc[U - 1]));
        }
    }
}

// Division route for output j of a thread's run.
template <int DIV>
__device__ __forceinline__ double to_unit(u64 c, const InstParams &P, int j)
{
    if constexpr (DIV == DIVIDE_INT)
        return dev::unit_int_fast(c, P);
    else if constexpr (DIV == DIVIDE_FP64)
        return dev::unit_fp64(c, P.dn);
    else if constexpr (DIV == DIVIDE_RECIP)
        return dev::unit_recip(c, P.dn, P.recip);
    else if constexpr (DIV == DIVIDE_EXACT)
        return dev::unit_exact(c, P);
    else
        return (j & 3) == 3 ? dev::unit_int_fast(c, P) : dev::unit_recip(c, P.dn, P.recip);
}

// Exclusive scan of v (mod n) over segments of TS consecutive lanes (TS a
// power of two <= 32, segments aligned in the warp); total receives the
// segment's sum. No barrier: a segment lives in one warp.
__device__ __forceinline__ u64 segment_exscan_mod(u64 v, u64 n, int TS, u64 &total)
{
    const int lt = threadIdx.x & (TS - 1);
    u64 incl = v;
    for (int d = 1; d < TS; d <<= 1) {
        const u64 o = __shfl_up_sync(FULL, incl, d, TS);
        if (lt >= d)
            incl = addmod(incl, o, n);
    }
    total = __shfl_sync(FULL, incl, TS - 1, TS);
    const u64 ex = __shfl_up_sync(FULL, incl, 1, TS);
    return lt == 0 ? 0 : ex;
}

// The same over segments of TS consecutive threads that are whole warps (TS
// a multiple of 32 and a power of two): a warp scan, then the totals of the
// segment's earlier warps from shared memory. sh holds 32 entries; one
// barrier (the caller keeps sh untouched until its next barrier).
__device__ __forceinline__ u64 segment_exscan_mod_warps(u64 v, u64 n, int TS, u64 *sh,
                                                        u64 &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const u64 o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d)
            incl = addmod(incl, o, n);
    }
    if (lane == 31)
        sh[warp] = incl;
    __syncthreads();
    const int wps = TS >> 5, w0 = warp - (warp & (wps - 1));
    u64 wpre = 0, tot = 0;
    for (int w = w0; w < w0 + wps; w++) {
        const u64 x = sh[w];
        if (w < warp)
            wpre = addmod(wpre, x, n);
        tot = addmod(tot, x, n);
    }
    total = tot;
    u64 ex = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0)
        ex = 0;
    return addmod(wpre, ex, n);
}

// Steps 1-3 of a tile for the calling thread, which owns outputs my0+1 ..
// my0+L of its stream's tile: its skips from s_thr (the skip before its run),
// the scan of their sums mod n over the threads of the stream (scan(sum, n,
// total) returns the exclusive prefix), its messages from the carry m (the
// message before the tile), and their L ciphertexts. Entries at or past
// nvalid are computed but meaningless. The thread that owns the stream's last
// output (left = outputs from the tile start to the end of the work item)
// writes the instance's skip back when the item asks for it. total returns
// the tile's skip sum mod n (the carry to the next tile).
template <int L, int MODEXP, class Scan, int U = L>
__device__ __forceinline__ void tile_ciphertexts_scan(const DeviceTables &tab, const WorkItem &W,
                                                      const InstParams &P, u64 m, u64 s_thr,
                                                      u64 left, int my0, int nvalid, Scan &&scan,
                                                      u64 (&c)[L], u64 &total)
{
    const u64 n = P.n, r64 = P.r64;
    const u32 a = P.a;
    u64 sk[L];
    u64 x = s_thr, sum = 0, s_last = 0;
#pragma unroll
    for (int j = 0; j < L; j++) {
        x = mulmodQ_small(x, a);
        sk[j] = x;
        if (j < nvalid) {
            sum = add_cong(sum, x, r64);
            s_last = x;
        }
    }
    sum = reduce_u64(sum, n);
    const u64 pre = scan(sum, n, total);
    u64 msg[L];
    u64 mm = addmod(m, pre, n);
#pragma unroll
    for (int j = 0; j < L; j++) {
        mm = add_cong(mm, sk[j], r64);
        msg[j] = mm;
    }
    if ((W.flags & WI_WRITEBACK) && nvalid > 0 && (u64)(my0 + nvalid) == left)
        tab.state_s[W.inst] = s_last;  // this thread owns the stream's last output
    encrypt_passes<L, MODEXP, U>(msg, c, P);
}

// The same for one stream per block: the block-wide scan (two
// __syncthreads()).
template <int L, int MODEXP, int U = L>
__device__ __forceinline__ void tile_ciphertexts(const DeviceTables &tab, const WorkItem &W,
                                                 const InstParams &P, u64 m, u64 s_thr, u64 left,
                                                 int my0, int nvalid, u64 *sh_scan, u64 (&c)[L],
                                                 u64 &total)
{
    auto scan = [&](u64 v, u64 n, u64 &tot) { return block_exscan_mod(v, n, sh_scan, tot); };
    tile_ciphertexts_scan<L, MODEXP, decltype(scan) &, U>(tab, W, P, m, s_thr, left, my0, nvalid,
                                                       scan, c, total);
}

// ---- bulk tensor stores of staged tiles (the generation kernels)

// Staging of a tile for bulk tensor stores (the layout of a 128-byte
// swizzled tensor map): element i lies in 128-byte line i / 16, and its
// 16-byte chunk (i / 2) % 8 sits at chunk position ((i / 2) % 8) ^ (line % 8).
// A thread writes its run as 16-byte chunks; the eight lanes of one
// shared-memory wavefront then hit eight different chunk positions.
__device__ __forceinline__ int swz(int i)
{
    const int line = i >> 4;
    return (line << 4) | (((((i >> 1) & 7) ^ (line & 7))) << 1) | (i & 1);
}

// Elements per staging buffer: a tile, and with two buffers (shifted
// staging) one more 16-element line, rounded to keep buffers 1 KB aligned.
__host__ __device__ constexpr int stage_elements(int S, int nbuf)
{
    return nbuf == 2 ? S + 128 : S;
}

__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One bulk tensor store per box of rows: rows 16-element lines from the
// swizzled staging src to lines row0 .. row0 + rows - 1 of the view.
__device__ __forceinline__ void bulk_store_rows(const CUtensorMap *map, const u64 *src, int rows,
                                                int box_rows, u64 row0)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(src);
    for (int b = 0; b < rows; b += box_rows)
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     :
                     : "l"((u64)map), "r"(0), "r"((int)(row0 + (u64)b)), "r"(s + (uint32_t)b * 128u)
                     : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// A thread's run of L values to the swizzled staging positions p0 .. p0 +
// L - 1, in 16-byte chunks where the positions allow (p0 even), else as a
// single first and last element around L / 2 - 1 chunks. p0 = my0 (the
// unshifted staging) keeps the positions visible to the compiler.
template <int L>
__device__ __forceinline__ void stage_run(u64 *st, int my0, int shift, const u64 (&v)[L])
{
    if (shift == 0) {
#pragma unroll
        for (int k = 0; k < L / 2; k++)
            *reinterpret_cast<ulonglong2 *>(st + swz(my0 + 2 * k)) =
                make_ulonglong2(v[2 * k], v[2 * k + 1]);
        return;
    }
    const int p0 = my0 + shift;
    if ((p0 & 1) == 0) {
#pragma unroll
        for (int k = 0; k < L / 2; k++)
            *reinterpret_cast<ulonglong2 *>(st + swz(p0 + 2 * k)) =
                make_ulonglong2(v[2 * k], v[2 * k + 1]);
    } else {
        st[swz(p0)] = v[0];
#pragma unroll
        for (int k = 1; k < L / 2; k++)
            *reinterpret_cast<ulonglong2 *>(st + swz(p0 + 2 * k - 1)) =
                make_ulonglong2(v[2 * k - 1], v[2 * k]);
        st[swz(p0 + L - 1)] = v[L - 1];
    }
}

// Element stores of staged outputs i = t, t + T, ... below n from staging
// position shift + i to dst[i * stride]. For T a multiple of 128 the
// swizzled position of shift + t + kT is that of shift + t plus kT (the
// line advances by a multiple of 8), so it is computed once.
__device__ __forceinline__ void put(double *p, u64 bits) { *p = __longlong_as_double((long long)bits); }
__device__ __forceinline__ void put(u64 *p, u64 bits) { *p = bits; }

template <class V>
__device__ __forceinline__ void store_elements(V *dst, const u64 *st, int n, int shift,
                                               u64 stride)
{
    const int T = blockDim.x, t = threadIdx.x;
    if ((T & 127) == 0) {
        for (int i = t, j = swz(shift + t); i < n; i += T, j += T)
            put(dst + (u64)i * stride, st[j]);
    } else {
        for (int i = t; i < n; i += T)
            put(dst + (u64)i * stride, st[swz(shift + i)]);
    }
}

// Waits until the bulk stores issued by this thread have read their source
// (read = true) or have completed.
template <bool READ>
__device__ __forceinline__ void bulk_wait_all()
{
    if constexpr (READ)
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    else
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace tile
}  // namespace rsaprng
