// Work lists that the host planner builds and the kernels read (plain
// structs, no CUDA types).
#pragma once
#include <cstdint>

namespace rsaprng {

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
// A chunk entry with item = kNoItem continues the skip-sum range of the
// entry before it (long ranges are cut into segments so that the pre-pass
// spreads over many warps); it starts no work item.
constexpr uint32_t kNoItem = 0xFFFFFFFFu;
// A run of consecutive PrepChunk entries (in stream order) of one instance.
struct PrepGroup {
    uint32_t inst;
    uint32_t first;
    uint32_t count;
    uint32_t pad;
};

// The interleaved (vector) order: a block takes up to G = threads / TS work
// items that cover the same positions of consecutive instances of a vector
// (items first .. first+count-1, output elements one apart).
struct VecGroup {
    uint32_t first;
    uint32_t count;
};

}  // namespace rsaprng
