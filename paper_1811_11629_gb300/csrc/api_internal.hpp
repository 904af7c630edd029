// Internal state of the library's host runtime.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rsaprng.h"
#include "host_params.hpp"
#include "kernels.cuh"
#include "plan_core.hpp"

namespace rsaprng {


// The same lists in device memory (one allocation) plus the skip-sum scratch.
struct DevPlan {
    void *d_buf = nullptr;
    size_t cap_buf = 0;
    void *h_buf = nullptr;  // pinned staging
    size_t cap_host = 0;
    void *d_sums = nullptr;
    size_t cap_sums = 0;
    WorkItem *items = nullptr;
    PrepChunk *chunks = nullptr;
    PrepGroup *groups = nullptr;
    uint32_t *ticket = nullptr;
    uint64_t *chunk_sum = nullptr;
    uint64_t *chunk_s = nullptr;
    uint32_t nitems = 0, nchunks = 0, ngroups = 0;
    uint64_t numbers = 0;
    uint64_t extent = 0;  // one past the last output element the plan writes
    bool unaligned = false;  // a piece starts off a multiple of 16 elements
    uint64_t stride = 1;
    VecGroup *vecs = nullptr;
    uint32_t nvecs = 0;
    int vec_ts = 0;
    GenLaunch last{};  // shape of the most recent generation launch
    int occupancy = 0; // resident blocks per SM of that launch
    // Single-launch calls: a 64-byte ticket word, then the per-tile status
    // array; the ticket only grows, lb_base being its value before the next
    // launch's first block.
    void *d_lb = nullptr;
    size_t cap_lb = 0;
    uint64_t lb_base = 0;
};

constexpr int kScratchSlots = 4;
struct ScratchSlot {
    DevPlan plan;
    cudaEvent_t done = nullptr;
    bool used = false;
};

}  // namespace rsaprng

struct rsaprng_ctx {
    int device = 0;
    int sms = 0;
    uint64_t capacity = 0, count = 0;
    rsaprng::InstParams *d_params = nullptr;
    uint64_t *d_m = nullptr, *d_s = nullptr;
    uint64_t *d_pow_lin = nullptr, *d_pow2k = nullptr;
    std::vector<rsaprng::InstParams> h_params;  // host mirror of the fixed parameters
    rsaprng_config cfg{};
    rsaprng::ScratchSlot slots[rsaprng::kScratchSlots];
    int next_slot = 0;
    uint64_t launches = 0;
    uint64_t h2d_bytes = 0, d2h_bytes = 0;  // host<->device bytes moved by the library
    // blocks/SM by (threads 64/128/256/512, L index, modexp, divide, passes)
    int occ_cache[4][4][2][5][2];
    size_t occ_smem[4][4][2][5][2];
    void *d_out_scratch = nullptr;  // device staging for host-buffer generation
    size_t cap_out_scratch = 0;
    rsaprng::HostPlan hp_direct;  // host plan of the direct calls, rebuilt in place
    uint32_t *d_err = nullptr;    // device error word (bit 0: a device-side wait gave up)
    uint64_t lb_epoch = 0;        // tag of the latest single-launch call
};

namespace rsaprng {

int cuda_fail(cudaError_t e, const char *what);
DeviceTables ctx_tables(rsaprng_ctx *c);
GenLaunch ctx_launch(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nitems, bool want_r,
                     bool want_c, int *occupancy = nullptr);
// Pieces of a stream are whole tiles; with tuple > 1 they are also whole
// multiples of tuple outputs (the histogram consumer's D-tuples). Output k of
// request i goes to element offsets[i] + k stride.
// allow_pack: generation plans may put several streams in a block
// (cfg.streams_per_block); the histogram consumer's plans may not.
int build_plan(rsaprng_ctx *c, const rsaprng_config &cfg, uint64_t nreq, const rsaprng_id *ids,
               const uint64_t *counts, const uint64_t *offsets, uint64_t chunk, HostPlan &hp,
               uint64_t tuple = 1, uint64_t stride = 1, bool allow_pack = false);
int upload_plan(rsaprng_ctx *c, const HostPlan &hp, DevPlan &dp, cudaStream_t stream);
// Launches the pre-pass and the generation kernel, or the histogram
// consumer instead of the generation kernel when hist is given. fresh: the
// plan was uploaded for this launch alone, so its work-queue counter is still
// the zero the upload wrote (a plan launched again, or captured in a graph,
// resets it on the stream). gen_events: two CUDA events recorded on the
// stream right before and after the generation kernel's launch (or null).
int launch_plan(rsaprng_ctx *c, const rsaprng_config &cfg, DevPlan &dp, double *d_r,
                uint64_t *d_c, cudaStream_t stream, uint64_t *launches,
                const HistArgs *hist = nullptr, bool fresh = false,
                const cudaEvent_t *gen_events = nullptr);
void free_devplan(DevPlan &dp);
int scratch_slot(rsaprng_ctx *c, ScratchSlot **out);
// One instance's N outputs in one launch with a decoupled look-back, when the
// configuration and N allow it (*done = true); otherwise nothing is launched
// and the caller takes the chunked path.
int generate_single_launch(rsaprng_ctx *c, rsaprng_id id, uint64_t N, uint64_t *d_c,
                           double *d_r, cudaStream_t st, bool *done);

}  // namespace rsaprng
