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

// Pieces per resident block that the load balance aims for (geo.pieces,
// default 1): the persistent launch hands out items in decreasing cost, and
// an instance whose work is larger than a block's fair share would otherwise
// finish alone at the end of the launch. Every extra piece costs a skip-sum
// pass over the piece before it, so the split is no finer than asked.

// The vector kernel's units (groups of up to G streams side by side) all
// cost about the same when the streams have one length, so the persistent
// launch runs them in rounds of `grid` blocks and a last round that is only
// partly full idles the rest. Two ways to more units: cutting every stream
// into P pieces (the skip-sum pre-pass then visits (P - 1) / P of the
// outputs once more), and narrower groups (G / 2 streams of TS * 2 threads:
// one more shuffle level in the segmented scan, rows of half the width).
// P stays within a few rounds' worth (kVecRounds).
constexpr uint64_t kVecRounds = 4;
// The skip-sum pass over one output, in the units of cost_per_number: one
// 32-bit-multiplier skip step and one add, measured at 17 % of a whole
// output at e = 3 (cost 10) on GB300.
constexpr double kPrepCostPerNumber = 1.7;
// Score lost per halving of G (the extra scan level, narrower rows).
constexpr double kVecNarrowCost = 0.01;
// Pieces shorter than this many tiles are not worth their start-up.
constexpr uint64_t kVecMinTiles = 8;

// The skip-sum pre-pass runs one warp per chunk entry. A piece's range is
// cut into segments of at most kPrepSegMin outputs, or longer ones when the
// ranges are long enough to give more than kPrepSegPerBlock segments per
// resident generation block (several per resident warp of the pre-pass), so
// that no warp walks a long range alone and the last wave of pre-pass
// blocks is short.
constexpr uint64_t kPrepSegMin = 4096;
constexpr uint64_t kPrepSegPerBlock = 64;

// Units the vector kernel would get from the requests uncut: runs of up to G
// requests (in instance order) of one length whose first outputs are
// neighbours.
static uint64_t vector_units(const std::vector<uint64_t> &order, const uint32_t *ids,
                             const uint64_t *counts, const uint64_t *offsets, uint64_t G)
{
    uint64_t units = 0, run = 0, prev = 0;
    for (uint64_t r : order) {
        if (counts[r] == 0)
            continue;
        const bool join = run > 0 && run < G && counts[r] == counts[prev] &&
                          offsets[r] == offsets[prev] + 1 && ids[r] != ids[prev];
        run = join ? run + 1 : 1;
        units += join ? 0 : 1;
        prev = r;
    }
    return units;
}

double vec_plan_score(uint64_t units, uint64_t grid, uint64_t p, double prep_share)
{
    if (units == 0 || grid == 0 || p == 0)
        return 0.0;
    const uint64_t u = units * p;
    const uint64_t rounds = (u + grid - 1) / grid;
    const double fill = (double)u / (double)(rounds * grid);
    return fill / (1.0 + prep_share * (double)(p - 1) / (double)p);
}

uint64_t vec_pieces_per_stream(uint64_t units, uint64_t grid, uint64_t max_pieces,
                               double prep_share)
{
    if (units == 0 || grid == 0)
        return 1;
    const uint64_t pmax = std::max<uint64_t>(
        1, std::min(max_pieces, kVecRounds * ((grid + units - 1) / units)));
    double best = 0.0;
    for (uint64_t p = 1; p <= pmax; p++)
        best = std::max(best, vec_plan_score(units, grid, p, prep_share));
    // the smallest P within 3 % of the best: fewer pieces, less planning
    for (uint64_t p = 1; p <= pmax; p++)
        if (vec_plan_score(units, grid, p, prep_share) >= 0.97 * best)
            return p;
    return 1;
}

int build_plan_core(const InstParams *params, uint64_t ninst, int modexp, const PlanGeometry &geo,
                    uint64_t nreq, const uint32_t *ids, const uint64_t *counts,
                    const uint64_t *offsets, uint64_t chunk, HostPlan &hp, uint64_t tuple,
                    uint64_t stride, uint64_t pack)
{
    if (stride > 1 || tuple > 1 || pack < 1)
        pack = 1;
    if (pack > 1 && (geo.threads % pack != 0 || geo.threads / pack < 32))
        return fail(RSAPRNG_ERR_ARG, "streams per block: %llu does not divide %llu threads into "
                                     "whole warps", (unsigned long long)pack,
                    (unsigned long long)geo.threads);
    hp.items.clear();
    hp.chunks.clear();
    hp.groups.clear();
    hp.numbers = 0;
    hp.extent = 0;
    hp.unaligned = false;
    hp.stride = stride;
    hp.vecs.clear();
    hp.vec_ts = 0;
    if (chunk == 0)
        chunk = ~0ULL;
    // Group requests by instance, keeping array order inside each instance.
    std::vector<uint64_t> &order = hp.tmp.order;
    order.resize(nreq);
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
    std::stable_sort(order.begin(), order.end(),
                     [&](uint64_t x, uint64_t y) { return ids[x] < ids[y]; });
    // The vector kernel puts G instances in a block, each with TS = T / G
    // threads and TS L positions per tile; pieces are whole tiles of it.
    // Every stream is cut into the same number of pieces; G and the pieces
    // per stream are chosen together for the rounds of vector units.
    uint64_t vec_pieces = 0;
    if (stride > 1) {
        const uint64_t G0 = geo.threads / (uint64_t)vec_threads_per_instance((int)geo.threads, stride);
        const uint64_t Gmin = std::max<uint64_t>(1, geo.threads / 32);
        uint64_t longest = 0, numbers = 0;
        for (uint64_t i = 0; i < nreq; i++) {
            longest = std::max(longest, counts[i]);
            numbers += counts[i];
        }
        const double prep_share =
            numbers ? kPrepCostPerNumber * (double)numbers / (double)std::max<uint64_t>(1, work)
                    : 0.0;
        uint64_t bestG = G0;
        vec_pieces = 1;
        double best = -1.0, narrow = 1.0;
        for (uint64_t G = G0; G >= Gmin; G /= 2, narrow -= kVecNarrowCost) {
            const uint64_t units = vector_units(order, ids, counts, offsets, G);
            const uint64_t tileG = (geo.threads / G) * geo.L;
            const uint64_t p =
                vec_pieces_per_stream(units, geo.grid, longest / (kVecMinTiles * tileG), prep_share);
            const double sc = vec_plan_score(units, geo.grid, p, prep_share) * narrow;
            if (sc > best) {
                best = sc;
                bestG = G;
                vec_pieces = p;
            }
            if (G == 1)
                break;
        }
        hp.vec_ts = (int)(geo.threads / bestG);
        tile = (uint64_t)hp.vec_ts * geo.L;
    }
    if (pack > 1) {  // packed streams: a piece runs on threads / pack threads
        hp.vec_ts = (int)(geo.threads / pack);
        tile = (uint64_t)hp.vec_ts * geo.L;
    }
    const uint64_t piece_cost =
        std::max<uint64_t>(1, work / (geo.grid * std::max<uint64_t>(1, geo.pieces) * pack));
    if (tuple > 1 && chunk != ~0ULL)
        chunk = std::max(tile, chunk / tile * tile);
    struct Piece {
        uint64_t offset, len, out;
    };
    std::vector<Piece> pieces;
    // per item: its cost, and its rank among the pieces of its stream
    std::vector<uint64_t> &item_cost = hp.tmp.cost, &item_rank = hp.tmp.rank;
    item_cost.clear();
    item_rank.clear();
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
        const uint64_t npieces = vec_pieces ? vec_pieces : (total * w + piece_cost - 1) / piece_cost;
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
                hp.extent = std::max(hp.extent, out + (len - 1) * stride + 1);
                hp.unaligned |= stride == 1 && (out & 15) != 0;
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
            item_rank.push_back(0);
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
            item_rank.push_back(k);
        }
    }
    if (hp.items.size() > 0xFFFFFFF0ULL || hp.chunks.size() > 0xFFFFFFF0ULL)
        return fail(RSAPRNG_ERR_ARG, "plan too large");
    // Longest-processing-time-first order for the persistent launch. In the
    // interleaved order (stride > 1) the outputs of different instances at
    // the same position share memory sectors: pieces are ordered by their
    // rank in the stream instead (a stable counting sort; the streams of a
    // vector have one length and are cut alike, so rank is position), and
    // those writes happen side by side and merge in L2.
    const size_t ni = hp.items.size();
    std::vector<uint32_t> &perm = hp.tmp.perm, &where = hp.tmp.where;
    bool ordered = true;
    if (stride > 1) {
        uint64_t ranks = 0;
        for (size_t i = 0; i < ni; i++) {
            ranks = std::max(ranks, item_rank[i] + 1);
            ordered = ordered && (i == 0 || item_rank[i - 1] <= item_rank[i]);
        }
        if (!ordered) {
            std::vector<uint64_t> &start = hp.tmp.order;  // reused: one slot per rank
            start.assign(ranks + 1, 0);
            for (size_t i = 0; i < ni; i++)
                start[item_rank[i] + 1]++;
            for (uint64_t r = 0; r < ranks; r++)
                start[r + 1] += start[r];
            perm.resize(ni);
            for (size_t i = 0; i < ni; i++)
                perm[start[item_rank[i]]++] = (uint32_t)i;
        }
    } else if (pack > 1) {
        // Packed streams share a block's tile loop, which runs as long as the
        // group's longest piece: pieces of one group should be alike in length.
        auto longer = [&](uint32_t x, uint32_t y) {
            return hp.items[x].count != hp.items[y].count ? hp.items[x].count > hp.items[y].count
                                                          : item_cost[x] > item_cost[y];
        };
        perm.resize(ni);
        for (size_t i = 0; i < ni; i++)
            perm[i] = (uint32_t)i;
        ordered = std::is_sorted(perm.begin(), perm.end(), longer);
        if (!ordered)
            std::stable_sort(perm.begin(), perm.end(), longer);
    } else {
        ordered = std::is_sorted(item_cost.begin(), item_cost.end(),
                                 [](uint64_t x, uint64_t y) { return x > y; });
        if (!ordered) {
            perm.resize(ni);
            for (size_t i = 0; i < ni; i++)
                perm[i] = (uint32_t)i;
            std::stable_sort(perm.begin(), perm.end(),
                             [&](uint32_t x, uint32_t y) { return item_cost[x] > item_cost[y]; });
        }
    }
    if (!ordered) {
        std::vector<WorkItem> &sorted = hp.tmp.sorted;
        sorted.resize(ni);
        where.resize(ni);
        for (size_t i = 0; i < ni; i++) {
            sorted[i] = hp.items[perm[i]];
            where[perm[i]] = (uint32_t)i;
        }
        hp.items.swap(sorted);
        for (auto &pc : hp.chunks)
            pc.item = where[pc.item];
        if (stride > 1 || pack > 1) {  // the units below read rank and cost in the new order
            std::vector<uint64_t> &tmp = hp.tmp.order;
            tmp.resize(ni);
            for (size_t i = 0; i < ni; i++)
                tmp[i] = item_rank[perm[i]];
            item_rank.swap(tmp);
            for (size_t i = 0; i < ni; i++)
                tmp[i] = item_cost[perm[i]];
            item_cost.swap(tmp);
        }
    }
    // Skip-sum segments (see kPrepSegMin); the first entry of a piece keeps
    // its item, the others continue its range.
    uint64_t prep_total = 0, prep_longest = 0;
    for (const PrepChunk &pc : hp.chunks) {
        prep_total += pc.len;
        prep_longest = std::max(prep_longest, pc.len);
    }
    const uint64_t seg = std::max<uint64_t>(
        kPrepSegMin,
        (prep_total / std::max<uint64_t>(1, kPrepSegPerBlock * geo.grid) + 255) / 256 * 256);
    if (prep_longest > seg) {
        std::vector<PrepChunk> &out = hp.tmp.chunks;
        out.clear();
        for (PrepGroup &g : hp.groups) {
            const uint32_t first = (uint32_t)out.size();
            for (uint32_t j = g.first; j < g.first + g.count; j++) {
                PrepChunk c = hp.chunks[j];
                uint64_t left = c.len;
                c.len = std::min(left, seg);
                out.push_back(c);
                uint64_t off = c.offset + c.len;
                left -= c.len;
                while (left > 0) {
                    const uint64_t l = std::min(left, seg);
                    out.push_back({c.inst, kNoItem, off, l});
                    off += l;
                    left -= l;
                }
            }
            g.first = first;
            g.count = (uint32_t)(out.size() - first);
        }
        if (out.size() > 0xFFFFFFF0ULL)
            return fail(RSAPRNG_ERR_ARG, "plan too large");
        hp.chunks.swap(out);
    }
    if (pack > 1) {
        // Groups of pack pieces in length order; a group costs its longest
        // piece at its costliest exponent (the segments share the tile loop).
        std::vector<uint64_t> &unit_cost = hp.tmp.order;
        unit_cost.clear();
        for (uint32_t i = 0; i < (uint32_t)hp.items.size(); i += (uint32_t)pack) {
            const uint32_t n = (uint32_t)std::min<uint64_t>(pack, hp.items.size() - i);
            uint64_t w = 0;
            for (uint32_t k = i; k < i + n; k++)
                w = std::max(w, item_cost[k] / std::max<uint64_t>(1, hp.items[k].count));
            hp.vecs.push_back({i, n});
            unit_cost.push_back(hp.items[i].count * w);
        }
        std::vector<uint32_t> &uperm = hp.tmp.perm;
        uperm.resize(hp.vecs.size());
        for (uint32_t u = 0; u < (uint32_t)uperm.size(); u++)
            uperm[u] = u;
        auto costlier = [&](uint32_t x, uint32_t y) { return unit_cost[x] > unit_cost[y]; };
        if (!std::is_sorted(uperm.begin(), uperm.end(), costlier)) {
            std::stable_sort(uperm.begin(), uperm.end(), costlier);
            std::vector<VecGroup> sorted_vecs(uperm.size());
            for (size_t u = 0; u < uperm.size(); u++)
                sorted_vecs[u] = hp.vecs[uperm[u]];
            hp.vecs.swap(sorted_vecs);
        }
    }
    if (stride > 1) {
        // Units of the vector kernel: up to G items in a row with the same
        // length whose outputs are neighbours (consecutive instances of a
        // vector at the same positions).
        const uint32_t G = (uint32_t)(geo.threads / (uint64_t)hp.vec_ts);
        std::vector<uint64_t> &unit_cost = hp.tmp.order;
        unit_cost.clear();
        for (uint32_t i = 0; i < (uint32_t)hp.items.size();) {
            uint32_t j = i + 1;
            uint64_t c = item_cost[i];
            while (j < hp.items.size() && j - i < G && hp.items[j].count == hp.items[i].count &&
                   hp.items[j].out_off == hp.items[j - 1].out_off + 1)
                c = std::max(c, item_cost[j++]);
            hp.vecs.push_back({i, j - i});
            unit_cost.push_back(c);
            i = j;
        }
        // Within a rank (one position range), costliest units first, so that the
        // launch ends on its cheapest units; units of one vector share their
        // exponents and cost, and stay side by side.
        std::vector<uint32_t> &uperm = hp.tmp.perm;
        uperm.resize(hp.vecs.size());
        for (uint32_t u = 0; u < (uint32_t)uperm.size(); u++)
            uperm[u] = u;
        auto unit_before = [&](uint32_t x, uint32_t y) {
            const uint64_t rx = item_rank[hp.vecs[x].first], ry = item_rank[hp.vecs[y].first];
            return rx != ry ? rx < ry : unit_cost[x] > unit_cost[y];
        };
        if (!std::is_sorted(uperm.begin(), uperm.end(), unit_before)) {
            std::stable_sort(uperm.begin(), uperm.end(), unit_before);
            std::vector<VecGroup> sorted_vecs(uperm.size());
            for (size_t u = 0; u < uperm.size(); u++)
                sorted_vecs[u] = hp.vecs[uperm[u]];
            hp.vecs.swap(sorted_vecs);
        }
    }
    return RSAPRNG_OK;
}

}  // namespace rsaprng
