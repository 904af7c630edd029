// The host planner: cuts a batch of requests into work items for the
// persistent generation kernels (plain C++, no CUDA calls; the launch
// geometry comes in as numbers). Sec. IV: a stream's outputs after position
// o start from the state after o outputs, which the skip-sum pre-pass
// provides for every piece but an instance's first.
#include "plan_core.hpp"

#include <algorithm>

#include "../../include/rsaprng.h"

namespace rsaprng {

int vec_threads_per_instance(int threads, uint64_t stride)
{
    int G = threads / 4;  // at most: four threads per instance
    while (G > threads / 32 && (uint64_t)(G / 2) >= stride)
        G /= 2;
    return threads / G;
}

// Cost of one output in Montgomery-product units: squarings + multiplies of
// the exponent chain plus a fixed share for the skip, scan and division.
uint64_t cost_per_number(uint32_t e)
{
    const int bl = 32 - __builtin_clz(e);
    return (uint64_t)(bl + __builtin_popcount(e) + 6);
}

// Pieces per resident block that the load balance aims for: the persistent
// launch hands out items in decreasing cost, and an instance whose work is
// larger than a block's fair share would otherwise finish alone at the end
// of the launch. Every extra piece costs a skip-sum pass over the piece
// before it, so the split is no finer than that.
constexpr uint64_t kPiecesPerBlock = 1;

int build_plan_core(const InstParams *params, uint64_t ninst, int modexp, const PlanGeometry &geo,
                    uint64_t nreq, const uint32_t *ids, const uint64_t *counts,
                    const uint64_t *offsets, uint64_t chunk, HostPlan &hp, uint64_t tuple,
                    uint64_t stride)
{
    hp.items.clear();
    hp.chunks.clear();
    hp.groups.clear();
    hp.numbers = 0;
    hp.stride = stride;
    hp.vecs.clear();
    hp.vec_ts = 0;
    if (chunk == 0)
        chunk = ~0ULL;
    // Group requests by instance, keeping array order inside each instance.
    std::vector<uint64_t> order(nreq);
    uint64_t work = 0;
    for (uint64_t i = 0; i < nreq; i++) {
        if (ids[i] >= ninst)
            return fail(RSAPRNG_ERR_ID, "request %llu: unknown instance id %u",
                        (unsigned long long)i, ids[i]);
        order[i] = i;
        const InstParams &P = params[ids[i]];
        work += counts[i] * cost_per_number(std::max(P.e, P.eq));
        if (P.e != P.eq && modexp == RSAPRNG_MODEXP_MONT64)
            return fail(RSAPRNG_ERR_ARG,
                        "instance %u has CRT exponents; the 64-bit route needs one exponent",
                        ids[i]);
    }
    // Cost of one piece: the work spread over the resident blocks of the
    // launch, kPiecesPerBlock pieces each; pieces are whole tiles.
    uint64_t tile = geo.threads * geo.L * std::max<uint64_t>(1, tuple);
    // The vector kernel puts G instances in a block, each with TS L positions
    // per tile: pieces are whole tiles of it, and there are G times as many
    // pieces to spread over the resident blocks.
    uint64_t per_block = 1;
    if (stride > 1) {
        hp.vec_ts = vec_threads_per_instance((int)geo.threads, stride);
        per_block = geo.threads / (uint64_t)hp.vec_ts;
        tile = (uint64_t)hp.vec_ts * geo.L;
    }
    const uint64_t piece_cost =
        std::max<uint64_t>(1, work / (geo.grid * kPiecesPerBlock * per_block));
    if (tuple > 1 && chunk != ~0ULL)
        chunk = std::max(tile, chunk / tile * tile);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint64_t x, uint64_t y) { return ids[x] < ids[y]; });
    struct Piece {
        uint64_t offset, len, out;
    };
    std::vector<Piece> pieces;
    std::vector<uint64_t> item_cost, item_pos;
    for (uint64_t g0 = 0; g0 < nreq;) {
        uint64_t g1 = g0;
        const uint32_t id = ids[order[g0]];
        while (g1 < nreq && ids[order[g1]] == id)
            g1++;
        pieces.clear();
        const uint64_t w = cost_per_number(std::max(params[id].e, params[id].eq));
        uint64_t total = 0;
        for (uint64_t k = g0; k < g1; k++)
            total += counts[order[k]];
        const uint64_t npieces = (total * w + piece_cost - 1) / piece_cost;
        uint64_t len = npieces > 1 ? (total + npieces - 1) / npieces : total;
        len = (len + tile - 1) / tile * tile;
        const uint64_t cut = std::max<uint64_t>(1, std::min(chunk, len));
        uint64_t off = 0;
        for (uint64_t k = g0; k < g1; k++) {
            const uint64_t r = order[k];
            uint64_t left = counts[r], out = offsets[r];
            while (left > 0) {
                const uint64_t room = cut - (off % cut);
                const uint64_t len = std::min(left, room);
                pieces.push_back({off, len, out});
                off += len;
                out += len * stride;
                left -= len;
            }
        }
        g0 = g1;
        if (pieces.empty())
            continue;
        hp.numbers += off;
        if (pieces.size() == 1) {
            WorkItem it{id, WI_FROM_STATE | WI_WRITEBACK, pieces[0].len, pieces[0].out, 0, 0};
            hp.items.push_back(it);
            item_cost.push_back(pieces[0].len * w);
            item_pos.push_back(0);
            continue;
        }
        PrepGroup grp{id, (uint32_t)hp.chunks.size(), (uint32_t)pieces.size(), 0};
        hp.groups.push_back(grp);
        for (size_t k = 0; k < pieces.size(); k++) {
            const bool last = k + 1 == pieces.size();
            WorkItem it{id, last ? (uint32_t)WI_WRITEBACK : 0u, pieces[k].len, pieces[k].out, 0, 0};
            // The last piece's skip sum is needed by no later piece.
            PrepChunk pc{id, (uint32_t)hp.items.size(), pieces[k].offset, last ? 0 : pieces[k].len};
            hp.chunks.push_back(pc);
            hp.items.push_back(it);
            item_cost.push_back(pieces[k].len * w);
            item_pos.push_back(pieces[k].offset);
        }
    }
    if (hp.items.size() > 0xFFFFFFF0ULL || hp.chunks.size() > 0xFFFFFFF0ULL)
        return fail(RSAPRNG_ERR_ARG, "plan too large");
    // Longest-processing-time-first order for the persistent launch. In the
    // interleaved order (stride > 1) the outputs of different instances at
    // the same position share memory sectors: pieces are ordered by position
    // instead, so those writes happen side by side and merge in L2.
    const bool ordered =
        stride > 1 ? std::is_sorted(item_pos.begin(), item_pos.end())
                   : std::is_sorted(item_cost.begin(), item_cost.end(),
                                    [](uint64_t x, uint64_t y) { return x > y; });
    if (!ordered) {
        std::vector<uint32_t> perm(hp.items.size()), where(hp.items.size());
        for (size_t i = 0; i < perm.size(); i++)
            perm[i] = (uint32_t)i;
        if (stride > 1)
            std::stable_sort(perm.begin(), perm.end(),
                             [&](uint32_t x, uint32_t y) { return item_pos[x] < item_pos[y]; });
        else
            std::stable_sort(perm.begin(), perm.end(),
                             [&](uint32_t x, uint32_t y) { return item_cost[x] > item_cost[y]; });
        std::vector<WorkItem> sorted(hp.items.size());
        for (size_t i = 0; i < perm.size(); i++) {
            sorted[i] = hp.items[perm[i]];
            where[perm[i]] = (uint32_t)i;
        }
        hp.items.swap(sorted);
        for (auto &pc : hp.chunks)
            pc.item = where[pc.item];
    }
    if (stride > 1) {
        // Units of the vector kernel: up to G items in a row with the same
        // length whose outputs are neighbours (consecutive instances of a
        // vector at the same positions).
        const uint32_t G = (uint32_t)(geo.threads / (uint64_t)hp.vec_ts);
        for (uint32_t i = 0; i < (uint32_t)hp.items.size();) {
            uint32_t j = i + 1;
            while (j < hp.items.size() && j - i < G && hp.items[j].count == hp.items[i].count &&
                   hp.items[j].out_off == hp.items[j - 1].out_off + 1)
                j++;
            hp.vecs.push_back({i, j - i});
            i = j;
        }
    }
    return RSAPRNG_OK;
}

}  // namespace rsaprng
