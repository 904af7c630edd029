// The host planner's interface (plain C++, no CUDA types), shared by the
// library's runtime and the host-only planner tests.
#pragma once
#include <cstdint>
#include <vector>

#include "host_params.hpp"
#include "work.hpp"

namespace rsaprng {

// Work lists of one launch sequence, built on the host.
struct HostPlan {
    std::vector<WorkItem> items;
    std::vector<PrepChunk> chunks;
    std::vector<PrepGroup> groups;
    uint64_t numbers = 0;
    uint64_t stride = 1;  // element distance between consecutive outputs of a request
    uint64_t extent = 0;  // one past the last output element the plan writes
    bool unaligned = false;  // stride 1: a piece starts off a multiple of 16 elements
    std::vector<VecGroup> vecs;  // stride > 1: blocks' units of the vector kernel
    int vec_ts = 0;              // threads per instance in the vector kernel
    // Working storage of the planner, kept so that a plan rebuilt in the same
    // HostPlan reuses its capacity.
    struct Scratch {
        std::vector<uint64_t> order, cost, rank;
        std::vector<uint32_t> perm, where;
        std::vector<WorkItem> sorted;
        std::vector<PrepChunk> chunks;
    } tmp;
};

// Shape of the generation launch the pieces are sized for.
struct PlanGeometry {
    uint64_t threads;     // threads per block
    uint64_t L;           // outputs per thread per tile
    uint64_t grid;        // resident blocks
    uint64_t pieces = 1;  // pieces per resident block the load balance aims for
};

// Error reporting (defined by the runtime; returns code).
int fail(int code, const char *fmt, ...);

// Cost of one output of an instance with exponent e, in Montgomery-product
// units plus a fixed share (the planner's balance weight).
uint64_t cost_per_number(uint32_t e);

// Threads per instance (TS) of the vector kernel for a block of `threads`
// and a vector of `stride` instances: G = threads / TS instances per block,
// the smallest power of two >= stride between threads / 32 and threads / 4.
int vec_threads_per_instance(int threads, uint64_t stride);

// Vector plans: `units` groups of equal cost run on `grid` resident blocks,
// every stream cut into p pieces. The score is the fill of the last round
// over the cost of the skip-sum pass on the (p - 1) / p outputs that need
// it, prep_share being that pass's cost per output relative to generating
// one.
double vec_plan_score(uint64_t units, uint64_t grid, uint64_t p, double prep_share);
// The p in [1, max_pieces] (and at most a few rounds' worth) that scores
// within 3 % of the best, smallest first.
uint64_t vec_pieces_per_stream(uint64_t units, uint64_t grid, uint64_t max_pieces,
                               double prep_share);

// Cuts requests (instance ids[i], counts[i] outputs, written from element
// offsets[i], consecutive outputs `stride` elements apart) into work items:
// requests of one instance continue its stream in array order; a stream is
// cut into pieces of whole tiles (multiples of `tuple` outputs too) so that
// the work spreads over geo.grid blocks, at most `chunk` outputs each (0: no
// cap; with tuple > 1 the cap is rounded down to whole units of tile x tuple,
// at least one unit); pieces after an instance's first get their start state from the
// skip-sum pre-pass (chunks, groups). Items are ordered longest first, or by
// position when stride > 1 (then grouped into VecGroups). With stride 1 and
// pack > 1 (streams per block, geo.threads / pack a whole number of warps)
// pieces are cut in tiles of geo.threads / pack threads, ordered by length
// (longest first) and grouped pack at a time into VecGroups, the groups
// ordered by cost (longest piece times costliest exponent), costliest first.
// params has ninst entries. Errors: RSAPRNG_ERR_ID, RSAPRNG_ERR_ARG.
int build_plan_core(const InstParams *params, uint64_t ninst, int modexp, const PlanGeometry &geo,
                    uint64_t nreq, const uint32_t *ids, const uint64_t *counts,
                    const uint64_t *offsets, uint64_t chunk, HostPlan &hp, uint64_t tuple = 1,
                    uint64_t stride = 1, uint64_t pack = 1);

}  // namespace rsaprng
