// Kernel interface shared by the kernels and the host runtime.
#pragma once
#include <cstdint>

#include <cuda.h>  // CUtensorMap (the type only; no driver-API link)
#include <cuda_runtime.h>

#include "host_params.hpp"
#include "work.hpp"

namespace rsaprng {

// Largest tile (threads per block x numbers per thread) and the power table
// rows: pow_lin[root][i] = a^i mod Q for i in [0, kMaxTile], pow2k[root][b] =
// a^(2^b) mod Q for b in [0, 63].
constexpr int kMaxThreads = 1024;
constexpr int kMaxL = 16;
constexpr int kMaxTile = kMaxThreads * kMaxL;
constexpr int kPowLinRow = kMaxTile + 1;

enum Modexp { MODEXP_CRT32 = 1, MODEXP_MONT64 = 2 };
// DIVIDE_HYBRID sends three of every four outputs of a thread through the
// FP64 pipe and the fourth through the integer pipes; DIVIDE_RECIP uses the
// reciprocal-and-correction sequence on the FP64 pipe (identical results).
// DIVIDE_EXACT computes the other reading of the division, RN(c / n) of the
// exact rational (selected by the rounding knob, not by the divide route).
enum Divide { DIVIDE_INT = 1, DIVIDE_FP64 = 2, DIVIDE_HYBRID = 3, DIVIDE_RECIP = 4, DIVIDE_EXACT = 5 };

struct DeviceTables {
    const InstParams *params;
    uint64_t *state_m;
    uint64_t *state_s;
    const uint64_t *pow_lin;  // [kNumRoots][kPowLinRow]
    const uint64_t *pow2k;    // [kNumRoots][64]
};

struct GenLaunch {
    int threads;     // threads per block
    int L;           // numbers per thread per tile
    int modexp;      // Modexp
    int divide;      // Divide
    int grid;        // blocks
    bool persistent; // items pulled from *ticket
    uint64_t stride; // element distance between consecutive outputs of a work item
    bool pdl = false;  // launch as a programmatic dependent of the start-state scan
    int unroll = 0;    // 0 or >= L: all L chains at once; else passes of this many
    int L_wide = 0;    // vector kernel: the configured numbers per thread, which
                       // whole-warp segments may run instead of L
    uint64_t out_extent = 0;  // stride 1: elements of the output arrays the launch may
                              // write (0: unknown, no bulk tensor stores)
    bool out_unaligned = false;  // some item starts off a multiple of 16 elements
};

// Bulk tensor stores of the generation kernel's tiles. The output arrays are
// viewed as 2-D tensors [extent / 16][16] of 64-bit elements with 128-byte
// swizzling; a block stages a whole tile in that swizzled layout and one
// thread writes it with cp.async.bulk.tensor, one copy per box of rows.
struct alignas(128) StoreMaps {
    CUtensorMap r;    // view of out_r
    CUtensorMap c;    // view of out_c
    uint64_t extent;  // elements both views cover (a multiple of 16); 0: no bulk stores
    int box_rows;     // 16-element rows per bulk copy (at most 256)
    int nbuf;         // staging buffers per output kind (1 or 2)
};

// Launches kern; with pdl as a programmatic dependent of the kernel before it
// on the stream (kern must wait in griddepcontrol.wait before it reads what
// that kernel wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t stream, bool pdl, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Shared memory bytes the generation kernel needs for a tile: its staging
// buffers (gen_stage_buffers per output kind) and 1 KB to align them.
size_t gen_smem_bytes(int threads, int L, bool want_r, bool want_c);
int gen_stage_buffers(int threads, int L, bool want_r, bool want_c);
// The padded staging of the vector and single-launch kernels: one 8-byte pad
// slot every 16 elements, per output kind.
size_t padded_smem_bytes(int threads, int L, bool want_r, bool want_c);

size_t vec_smem_bytes(int threads, int L, bool want_r, bool want_c);
// Numbers per thread the vector kernel uses for a configured L: the tuned
// tile where it applies, else L itself.
int vec_numbers_per_thread(int L, int modexp, int threads);
cudaError_t launch_generate_vec(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                                const VecGroup *vecs, uint32_t nvecs, uint32_t *ticket,
                                double *out_r, uint64_t *out_c, int TS, cudaStream_t stream);
int vec_blocks_per_sm(const GenLaunch &g, size_t smem);

// Histogram consumer: d^D counters at hist; digits of r (low = 0) or of the
// low bits of c (low = 1, d a power of two); D in [1, 8].
struct HistArgs {
    unsigned long long *hist;
    uint32_t d;
    uint32_t D;
    uint32_t low;
    uint32_t pad;
};
size_t hist_smem_bytes(int threads, int L);
cudaError_t launch_histogram(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                             uint32_t nitems, uint32_t *ticket, const HistArgs &h,
                             cudaStream_t stream);
int hist_blocks_per_sm(const GenLaunch &g);

cudaError_t launch_generate(const GenLaunch &g, const DeviceTables &t, const WorkItem *items,
                            uint32_t nitems, uint32_t *ticket, double *out_r, uint64_t *out_c,
                            cudaStream_t stream);
cudaError_t launch_prep_sums(const DeviceTables &t, const PrepChunk *chunks, uint32_t nchunks,
                             uint64_t *chunk_sum, uint64_t *chunk_s, cudaStream_t stream);
cudaError_t launch_prep_scan(const DeviceTables &t, const PrepGroup *groups, uint32_t ngroups,
                             const PrepChunk *chunks, const uint64_t *chunk_sum,
                             const uint64_t *chunk_s, WorkItem *items, cudaStream_t stream);

cudaError_t launch_unit(const DeviceTables &t, uint32_t id, uint64_t N, const uint64_t *c,
                        double *r, int divide, cudaStream_t stream);

// Microbenchmarks (results in the units documented in rsaprng.h).
cudaError_t microbench_imad(double *gops, cudaStream_t stream);
cudaError_t microbench_ddiv(double *gdiv, cudaStream_t stream);
cudaError_t microbench_mul(int shape, double *gops, cudaStream_t stream);
cudaError_t microbench_fp64(int shape, double *gops, cudaStream_t stream);
cudaError_t microbench_write(void *buf, size_t bytes, double *gbs, cudaStream_t stream);

// Whether the generation kernel has a variant running its chains in passes
// of `unroll` for this tiling and route.
bool gen_has_unroll(int L, int modexp, int divide, int unroll);
// Kernel attribute query for occupancy-based grid sizing.
int gen_blocks_per_sm(const GenLaunch &g, size_t smem);

}  // namespace rsaprng
