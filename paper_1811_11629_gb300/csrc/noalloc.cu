// Generation without any allocation: rsaprng_generate_f64_noalloc.
//
// Some callers cannot allocate device memory at the time they want numbers:
// real-time or latency-critical threads that forbid allocator calls, and hosts
// that hand all device memory to their own pool up front. The regular
// generation calls may grow the context's work-list buffers with cudaMalloc on
// first use; this entry point never does. Its scratch (the chunk work list,
// the per-chunk skip sums and the work queue counter) lives in one file-scope
// device array of fixed size that every GPU loading the library keeps until
// process exit.
#include <cstdio>
#include <mutex>

#include "api_internal.hpp"

using namespace rsaprng;

namespace {

// At most this many chunks per call; a chunk is at most kNoAllocMaxChunkLen outputs.
constexpr uint32_t kNoAllocMaxChunks = 4096;
constexpr uint64_t kNoAllocMaxChunkLen = 1ULL << 24;

struct NoAllocScratch {
    WorkItem items[kNoAllocMaxChunks];
    PrepChunk chunks[kNoAllocMaxChunks];
    uint64_t sums[kNoAllocMaxChunks];
    uint64_t skips[kNoAllocMaxChunks];
    PrepGroup group;
    uint32_t ticket;
};

// The scratch itself (about 330 KB). In host code this name is only a
// host-side stand-in: its device address comes from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_for_device(int dev, NoAllocScratch **out)
{
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_addr[dev] = (NoAllocScratch *)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Writes the chunk list of one instance's next N outputs: chunk i covers
// outputs i*chunk+1 .. min(N, (i+1)*chunk), written at element i*chunk. Also
// clears the work-queue counter.
__global__ void k_noalloc_plan(NoAllocScratch *S, uint32_t inst, uint64_t N, uint64_t chunk,
                               uint32_t nchunks)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        S->group.inst = inst;
        S->group.first = 0;
        S->group.count = nchunks;
        S->group.pad = 0;
        S->ticket = 0;
    }
    if (i >= nchunks)
        return;
    const uint64_t off = (uint64_t)i * chunk;
    const uint64_t len = (N - off < chunk) ? N - off : chunk;
    const bool last = i + 1 == nchunks;
    WorkItem w;
    w.inst = inst;
    w.flags = nchunks == 1 ? (WI_FROM_STATE | WI_WRITEBACK) : (last ? WI_WRITEBACK : 0u);
    w.count = len;
    w.out_off = off;
    w.m0 = 0;
    w.s0 = 0;
    S->items[i] = w;
    PrepChunk c;
    c.inst = inst;
    c.item = i;
    c.offset = off;
    c.len = last ? 0 : len;  // the last chunk's skip sum is needed by no later chunk
    S->chunks[i] = c;
}

}  // namespace

extern "C" {

int rsaprng_generate_f64_noalloc(rsaprng_ctx *c, rsaprng_id id, uint64_t N, double *d_r,
                                 void *stream)
{
    if (!c || (N && !d_r))
        return RSAPRNG_ERR_ARG;
    if (id >= c->count)
        return RSAPRNG_ERR_ID;
    if (N > (uint64_t)kNoAllocMaxChunks * kNoAllocMaxChunkLen)
        return RSAPRNG_ERR_ARG;
    if (c->cfg.modexp == RSAPRNG_MODEXP_MONT64 && c->h_params[id].e != c->h_params[id].eq)
        return RSAPRNG_ERR_ARG;  // CRT exponents need the CRT route
    if (N == 0)
        return RSAPRNG_OK;
    if (c->device < 0 || c->device >= kMaxDevices)
        return RSAPRNG_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess)
        return RSAPRNG_ERR_CUDA;
    NoAllocScratch *S = nullptr;
    if ((e = scratch_for_device(c->device, &S)) != cudaSuccess)
        return RSAPRNG_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // Chunks: enough to give every SM work, each a whole number of tiles and
    // at most kNoAllocMaxChunkLen long, never more than kNoAllocMaxChunks.
    const uint64_t tile = (uint64_t)c->cfg.threads_per_block * c->cfg.numbers_per_thread;
    const uint64_t want = (uint64_t)c->sms * 8;
    uint64_t chunk = (N + want - 1) / want;
    const uint64_t floor_len = (N + kNoAllocMaxChunks - 1) / kNoAllocMaxChunks;
    if (chunk < floor_len)
        chunk = floor_len;
    chunk = (chunk + tile - 1) / tile * tile;
    if (chunk > kNoAllocMaxChunkLen)
        chunk = kNoAllocMaxChunkLen;
    const uint32_t nchunks = (uint32_t)((N + chunk - 1) / chunk);
    if (nchunks > kNoAllocMaxChunks)
        return RSAPRNG_ERR_ARG;
    const DeviceTables t = ctx_tables(c);
    k_noalloc_plan<<<(nchunks + 255) / 256, 256, 0, st>>>(S, id, N, chunk, nchunks);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return RSAPRNG_ERR_CUDA;
    uint64_t nl = 1;
    if (nchunks > 1) {
        if ((e = launch_prep_sums(t, S->chunks, nchunks, S->sums, S->skips, st)) != cudaSuccess)
            return RSAPRNG_ERR_CUDA;
        if ((e = launch_prep_scan(t, &S->group, 1, S->chunks, S->sums, S->skips, S->items, st)) !=
            cudaSuccess)
            return RSAPRNG_ERR_CUDA;
        nl += 2;
    }
    GenLaunch g = ctx_launch(c, c->cfg, nchunks, true, false);
    g.pdl = nchunks > 1;  // right after the start-state scan
    g.out_extent = N;
    if ((e = launch_generate(g, t, S->items, nchunks, &S->ticket, d_r, nullptr, st)) !=
        cudaSuccess)
        return RSAPRNG_ERR_CUDA;
    c->launches += nl + 1;
    return RSAPRNG_OK;
}

}  // extern "C"
