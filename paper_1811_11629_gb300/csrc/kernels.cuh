// Kernel interface shared by the kernels and the host runtime.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "host_params.hpp"

namespace rsaprng {

// Largest tile (threads per block x numbers per thread) and the power table
// rows: pow_lin[root][i] = a^i mod Q for i in [0, kMaxTile], pow2k[root][b] =
// a^(2^b) mod Q for b in [0, 63].
constexpr int kMaxThreads = 1024;
constexpr int kMaxL = 16;
constexpr int kMaxTile = kMaxThreads * kMaxL;
constexpr int kPowLinRow = kMaxTile + 1;

// One unit of work for the generation kernel: `count` consecutive outputs of
// instance `inst` written from element `out_off` of the output arrays (one
// element apart, or a launch-wide stride apart for the interleaved order),
// starting from the state (m0, s0) before the first output.
enum : uint32_t {
    WI_FROM_STATE = 1u,  // take (m0, s0) from the instance state table
    WI_WRITEBACK = 2u,   // store the state after the last output
};
struct WorkItem {
    uint32_t inst;
    uint32_t flags;
    uint64_t count;
    uint64_t out_off;
    uint64_t m0, s0;
};
static_assert(sizeof(WorkItem) == 40, "WorkItem layout");

// Chunks of one instance's stream whose start state comes from the skip-sum
// pass: chunk i of the list covers outputs offset+1 .. offset+len of the
// instance's stream in this launch and fills work item `item`.
struct PrepChunk {
    uint32_t inst;
    uint32_t item;
    uint64_t offset;
    uint64_t len;
};
// A run of consecutive PrepChunk entries (in stream order) of one instance.
struct PrepGroup {
    uint32_t inst;
    uint32_t first;
    uint32_t count;
    uint32_t pad;
};

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
};

// Shared memory bytes the generation kernel needs for a tile.
size_t gen_smem_bytes(int threads, int L, bool want_r, bool want_c);

// The interleaved (vector) order: a block takes up to G = threads / TS work
// items that cover the same positions of consecutive instances of a vector
// (items first .. first+count-1, output elements one apart).
struct VecGroup {
    uint32_t first;
    uint32_t count;
};
size_t vec_smem_bytes(int threads, int L, bool want_r, bool want_c);
// Threads per instance (TS) for a block of `threads` and a vector of `stride`
// instances: G = threads / TS instances per block, the smallest power of two
// >= stride between threads / 32 and threads / 4.
int vec_threads_per_instance(int threads, uint64_t stride);
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
cudaError_t microbench_write(void *buf, size_t bytes, double *gbs, cudaStream_t stream);

// Kernel attribute query for occupancy-based grid sizing.
int gen_blocks_per_sm(const GenLaunch &g, size_t smem);

}  // namespace rsaprng
