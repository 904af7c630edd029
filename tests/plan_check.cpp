// Host-only checks of the planner (plan_core.cpp) on random request sets and
// launch geometries. Invariants checked for every plan:
//  1. every request's outputs are covered exactly once, at the elements
//     offsets[i] + k * stride, and the outputs of one instance follow its
//     stream (requests of an instance continue one another in array order);
//  2. an instance cut into one piece reads and writes back the state table;
//     cut into several, only its last piece writes back, and its pieces are
//     listed as skip-sum chunks (the last with length 0) in stream order;
//  3. pieces start on tiles (and on multiples of the tuple), respect the
//     chunk cap, and are ordered longest first (or by position for stride > 1);
//  4. vector groups partition the items into runs of neighbours; packed
//     groups (several streams per block) partition them into runs of at most
//     `pack` items in length order, ordered by cost;
//  5. unknown ids and CRT exponents on the 64-bit route are refused.
// Exit status 0 when every case passes.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <string>
#include <vector>

#include "../include/rsaprng.h"
#include "../paper_1811_11629_gb300/csrc/plan_core.hpp"

namespace rsaprng {
int fail(int code, const char *, ...) { return code; }
}  // namespace rsaprng

using namespace rsaprng;

static int failures = 0;
#define CHECK(cond, ...)                                                    \
    do {                                                                    \
        if (!(cond)) {                                                      \
            if (failures < 20) {                                            \
                std::printf("case %d: %s: ", case_no, #cond);               \
                std::printf(__VA_ARGS__);                                   \
                std::printf("\n");                                          \
            }                                                               \
            failures++;                                                     \
            return;                                                         \
        }                                                                   \
    } while (0)

static int case_no = 0;

static void check_case(std::mt19937_64 &rng, bool vector_order)
{
    case_no++;
    const uint64_t threads_opts[] = {64, 128, 256, 512}, L_opts[] = {2, 4, 8, 16};
    PlanGeometry geo{threads_opts[rng() % 4], L_opts[rng() % 4], 1 + rng() % 1200};
    const uint64_t ninst = 1 + rng() % 40;
    std::vector<InstParams> params(ninst);
    for (auto &p : params) {
        p.e = (uint32_t)(3 + 2 * (rng() % 40000));
        p.eq = (rng() % 5 == 0) ? (uint32_t)(3 + 2 * (rng() % 300)) : p.e;
    }
    std::vector<uint32_t> ids;
    std::vector<uint64_t> counts, offsets;
    uint64_t stride = 1, tuple = 1;
    const uint64_t scale = (rng() % 3 == 0) ? 200000 : 3000;
    if (vector_order) {
        // vectors of Mv distinct instances, all of length N, k-major
        const uint64_t Mv = 1 + rng() % std::min<uint64_t>(ninst, 40);
        const uint64_t groups = std::max<uint64_t>(1, ninst / Mv);
        const uint64_t N = rng() % scale;
        stride = Mv;
        std::vector<uint32_t> perm(ninst);
        for (uint32_t i = 0; i < ninst; i++)
            perm[i] = i;
        if (rng() % 2)
            std::shuffle(perm.begin(), perm.end(), rng);
        for (uint64_t g = 0; g < groups; g++)
            for (uint64_t j = 0; j < Mv; j++) {
                ids.push_back(perm[g * Mv + j]);
                counts.push_back(N);
                offsets.push_back(g * N * Mv + j);
            }
    } else {
        const uint64_t nreq = 1 + rng() % 60;
        tuple = (rng() % 4 == 0) ? 1 + rng() % 6 : 1;
        uint64_t off = 0;
        for (uint64_t i = 0; i < nreq; i++) {
            // histogram plans (tuple > 1) take one request per instance
            uint32_t id = (uint32_t)(rng() % ninst);
            if (tuple > 1) {
                if (i >= ninst)
                    break;
                id = (uint32_t)i;
            }
            const uint64_t c = (rng() % 7 == 0) ? 0 : rng() % scale;
            ids.push_back(id);
            counts.push_back(c);
            offsets.push_back(off);
            off += c;
        }
    }
    const uint64_t chunk_opts[] = {0, 1ULL << 12, 1ULL << 16, 5000, 1ULL << 18};
    const uint64_t chunk = chunk_opts[rng() % 5];
    const int modexp = (rng() % 4 == 0) ? RSAPRNG_MODEXP_MONT64 : RSAPRNG_MODEXP_CRT32;
    // streams per block for contiguous plans: whole warps per stream
    uint64_t pack = 1;
    if (stride == 1 && tuple == 1 && rng() % 2)
        pack = std::min<uint64_t>(1ULL << (rng() % 4), geo.threads / 32);
    HostPlan hp;
    const int rc = build_plan_core(params.data(), ninst, modexp, geo, ids.size(), ids.data(),
                                   counts.data(), offsets.data(), chunk, hp, tuple, stride, pack);
    bool split_e = false;
    for (uint32_t id : ids)
        split_e |= params[id].e != params[id].eq;
    if (split_e && modexp == RSAPRNG_MODEXP_MONT64) {
        CHECK(rc == RSAPRNG_ERR_ARG, "rc=%d", rc);
        return;
    }
    CHECK(rc == RSAPRNG_OK, "rc=%d", rc);

    // 1. coverage and stream order: stream position -> element, per instance
    std::map<uint32_t, std::vector<uint64_t>> want;  // instance -> element of each position
    uint64_t total = 0, extent = 0;
    for (size_t i = 0; i < ids.size(); i++) {
        auto &v = want[ids[i]];
        for (uint64_t k = 0; k < counts[i]; k++)
            v.push_back(offsets[i] + k * stride);
        total += counts[i];
        if (counts[i])
            extent = std::max(extent, offsets[i] + (counts[i] - 1) * stride + 1);
    }
    CHECK(hp.numbers == total, "numbers %llu != %llu", (unsigned long long)hp.numbers,
          (unsigned long long)total);
    // the extent bounds the bulk stores' view of the output arrays
    CHECK(hp.extent == extent, "extent %llu != %llu", (unsigned long long)hp.extent,
          (unsigned long long)extent);
    // the shifted staging is chosen when some piece starts off a 16-element line
    bool unaligned = false;
    for (const WorkItem &w : hp.items)
        unaligned |= stride == 1 && (w.out_off & 15) != 0;
    CHECK(hp.unaligned == unaligned, "unaligned flag %d != %d", (int)hp.unaligned, (int)unaligned);
    std::map<uint32_t, std::vector<uint64_t>> got;  // instance -> (position -> element)
    std::map<uint32_t, std::vector<size_t>> items_of;
    uint64_t sum_items = 0;
    for (size_t k = 0; k < hp.items.size(); k++) {
        items_of[hp.items[k].inst].push_back(k);
        sum_items += hp.items[k].count;
        CHECK(hp.items[k].count > 0, "empty item");
    }
    CHECK(sum_items == total, "items cover %llu of %llu", (unsigned long long)sum_items,
          (unsigned long long)total);
    // chunks give each multi-piece item its stream offset
    std::vector<int64_t> item_off(hp.items.size(), -1);
    for (const auto &g : hp.groups) {
        uint64_t expect = 0;
        for (uint32_t j = 0; j < g.count;) {
            const PrepChunk &c = hp.chunks[g.first + j];
            CHECK(c.inst == g.inst && c.item < hp.items.size(), "chunk of another instance");
            const WorkItem &w = hp.items[c.item];
            CHECK(w.inst == g.inst, "chunk item of another instance");
            CHECK(c.offset == expect, "chunk offsets not contiguous");
            // segments without an item continue the piece's skip-sum range
            uint64_t covered = c.len;
            for (j++; j < g.count && hp.chunks[g.first + j].item == kNoItem; j++) {
                const PrepChunk &sg = hp.chunks[g.first + j];
                CHECK(sg.inst == g.inst && sg.len > 0 && sg.offset == expect + covered,
                      "skip-sum segment out of place");
                covered += sg.len;
            }
            const bool last = j == g.count;
            CHECK(covered == (last ? 0 : w.count), "chunk length");
            CHECK(!(w.flags & WI_FROM_STATE), "piece after the first reads the state");
            CHECK(((w.flags & WI_WRITEBACK) != 0) == last, "write-back not on the last piece");
            item_off[c.item] = (int64_t)c.offset;
            expect += w.count;
        }
    }
    for (auto &kv : items_of) {
        const uint32_t inst = kv.first;
        auto &v = got[inst];
        v.assign(want[inst].size(), ~0ULL);
        for (size_t k : kv.second) {
            const WorkItem &w = hp.items[k];
            uint64_t base = 0;
            if (item_off[k] < 0) {
                // 2. a single piece: reads and writes the state table
                CHECK(kv.second.size() == 1, "several items without chunks");
                CHECK(w.flags == (WI_FROM_STATE | WI_WRITEBACK), "single piece flags %u", w.flags);
            } else {
                base = (uint64_t)item_off[k];
            }
            for (uint64_t j = 0; j < w.count; j++) {
                CHECK(base + j < v.size(), "position beyond the instance's outputs");
                CHECK(v[base + j] == ~0ULL, "position covered twice");
                v[base + j] = w.out_off + j * stride;
            }
            // 3. pieces start on tiles (and tuples); all but an instance's last
            // piece hold whole tiles and respect the chunk cap
            if (item_off[k] > 0 && tuple > 1)
                CHECK(base % tuple == 0, "piece off a tuple boundary");
            // with tuples the cap is whole units of tile x tuple, at least one
            const uint64_t unit = geo.threads * geo.L * tuple;
            const uint64_t cap = tuple > 1 ? std::max(unit, chunk / unit * unit) : chunk;
            if (chunk && w.count > cap)
                CHECK(false, "piece of %llu over the chunk cap %llu (tuple %llu stride %llu)",
                      (unsigned long long)w.count, (unsigned long long)cap,
                      (unsigned long long)tuple, (unsigned long long)stride);
        }
        CHECK(v == want[inst], "instance %u: elements differ from the requests", inst);
    }
    // 3. order of the items
    for (size_t k = 1; k < hp.items.size(); k++) {
        if (pack > 1) {
            CHECK(hp.items[k - 1].count >= hp.items[k].count, "packed pieces not by length");
        } else if (stride == 1) {
            auto cost = [&](const WorkItem &w) {
                return w.count *
                       cost_per_number(std::max(params[w.inst].e, params[w.inst].eq));
            };
            CHECK(cost(hp.items[k - 1]) >= cost(hp.items[k]), "not longest first");
        } else {
            const uint64_t a = item_off[k - 1] < 0 ? 0 : (uint64_t)item_off[k - 1];
            const uint64_t b = item_off[k] < 0 ? 0 : (uint64_t)item_off[k];
            CHECK(a <= b, "vector order not by position");
        }
    }
    // 4. vector groups
    if (stride > 1) {
        const uint32_t G = (uint32_t)(geo.threads / (uint64_t)hp.vec_ts);
        CHECK(hp.vec_ts >= 1 && geo.threads % hp.vec_ts == 0 && hp.vec_ts <= 32 && hp.vec_ts >= 4,
              "threads per instance %d", hp.vec_ts);
        // the groups are runs of neighbouring items that together cover every
        // item once; they run by position, costliest first at one position
        std::vector<int> seen(hp.items.size(), 0);
        uint64_t covered = 0, prev_pos = 0, prev_cost = ~0ULL;
        for (const auto &g : hp.vecs) {
            CHECK(g.count >= 1 && g.count <= G && (uint64_t)g.first + g.count <= hp.items.size(),
                  "group layout");
            uint64_t cost = 0;
            for (uint32_t j = 0; j < g.count; j++) {
                CHECK(!seen[g.first + j]++, "item in two groups");
                const WorkItem &b = hp.items[g.first + j];
                cost = std::max(cost, b.count * cost_per_number(std::max(params[b.inst].e,
                                                                         params[b.inst].eq)));
                if (j) {
                    const WorkItem &a = hp.items[g.first + j - 1];
                    CHECK(b.count == a.count && b.out_off == a.out_off + 1,
                          "group members not neighbours");
                }
            }
            const uint64_t pos = item_off[g.first] < 0 ? 0 : (uint64_t)item_off[g.first];
            CHECK(pos >= prev_pos, "vector groups not by position");
            CHECK(pos > prev_pos || cost <= prev_cost, "not costliest first at one position");
            prev_pos = pos;
            prev_cost = cost;
            covered += g.count;
        }
        CHECK(covered == hp.items.size(), "groups cover %llu of %zu items",
              (unsigned long long)covered, hp.items.size());
    } else if (pack > 1) {
        CHECK(hp.vec_ts == (int)(geo.threads / pack), "packed threads per stream %d", hp.vec_ts);
        std::vector<int> seen(hp.items.size(), 0);
        uint64_t covered = 0, prev_cost = ~0ULL;
        for (const auto &g : hp.vecs) {
            CHECK(g.count >= 1 && g.count <= pack && g.first % pack == 0 &&
                      (uint64_t)g.first + g.count <= hp.items.size() &&
                      (g.count == pack || (uint64_t)g.first + g.count == hp.items.size()),
                  "packed group layout");
            uint64_t w = 0;
            for (uint32_t j = 0; j < g.count; j++) {
                CHECK(!seen[g.first + j]++, "item in two groups");
                const WorkItem &b = hp.items[g.first + j];
                w = std::max(w, cost_per_number(std::max(params[b.inst].e, params[b.inst].eq)));
            }
            const uint64_t cost = hp.items[g.first].count * w;
            CHECK(cost <= prev_cost, "packed groups not costliest first");
            prev_cost = cost;
            covered += g.count;
        }
        CHECK(covered == hp.items.size(), "packed groups cover %llu of %zu items",
              (unsigned long long)covered, hp.items.size());
    } else {
        CHECK(hp.vecs.empty(), "vector groups in a contiguous plan");
    }
}

// Planning time for many instances (the split workload's shape): the
// planner must stay linear in the number of pieces.
static double plan_time_ms(int k, uint64_t stride)
{
    std::vector<InstParams> P(k);
    for (auto &p : P)
        p.e = p.eq = 3;
    std::vector<uint32_t> ids(k);
    std::vector<uint64_t> cnt(k, 65536), off(k);
    for (int i = 0; i < k; i++) {
        ids[i] = (uint32_t)i;
        off[i] = stride == 1 ? (uint64_t)i * 65536 : (uint64_t)(i / 32) * 65536 * 32 + (i % 32);
    }
    const PlanGeometry geo{128, 16, 760};
    HostPlan hp;
    // first into a fresh plan, then again into the same one (the library's
    // direct calls keep one per context)
    double ms[2];
    for (double &t : ms) {
        const auto t0 = std::chrono::steady_clock::now();
        build_plan_core(P.data(), k, RSAPRNG_MODEXP_CRT32, geo, k, ids.data(), cnt.data(),
                        off.data(), 0, hp, 1, stride);
        t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return std::max(ms[0], ms[1]);
}

int main(int argc, char **argv)
{
    if (argc > 1 && std::string(argv[1]) == "--time") {
        const double contiguous = plan_time_ms(32768, 1), interleaved = plan_time_ms(32768, 32);
        std::printf("plan_ms %.2f %.2f\n", contiguous, interleaved);
        return 0;
    }
    const int cases = argc > 1 ? std::atoi(argv[1]) : 3000;
    std::mt19937_64 rng(20261203);
    for (int i = 0; i < cases; i++)
        check_case(rng, i % 3 == 2);
    // 5. refusals
    {
        case_no++;
        std::vector<InstParams> params(2);
        params[0].e = params[0].eq = 5;
        params[1].e = 5;
        params[1].eq = 7;
        const PlanGeometry geo{128, 16, 760};
        HostPlan hp;
        const uint32_t bad[1] = {2};
        const uint64_t cnt[1] = {10}, off[1] = {0};
        int rc = build_plan_core(params.data(), 2, RSAPRNG_MODEXP_CRT32, geo, 1, bad, cnt, off, 0, hp);
        if (rc != RSAPRNG_ERR_ID) {
            std::printf("unknown id accepted (rc=%d)\n", rc);
            failures++;
        }
        const uint32_t split[1] = {1};
        rc = build_plan_core(params.data(), 2, RSAPRNG_MODEXP_MONT64, geo, 1, split, cnt, off, 0, hp);
        if (rc != RSAPRNG_ERR_ARG) {
            std::printf("CRT exponents accepted on the 64-bit route (rc=%d)\n", rc);
            failures++;
        }
        rc = build_plan_core(params.data(), 2, RSAPRNG_MODEXP_CRT32, geo, 1, split, cnt, off, 0, hp);
        if (rc != RSAPRNG_OK) {
            std::printf("CRT exponents refused on the CRT route (rc=%d)\n", rc);
            failures++;
        }
    }
    // 6. pieces per stream of the vector kernel: never more than allowed, the
    // last round at least as full as uncut, nearly full where cutting can
    // make it so, and no cut when the pre-pass costs as much as an output
    for (double share : {0.0, 0.05, 0.2, 1e9}) {
        for (uint64_t grid : {1ULL, 7ULL, 152ULL, 608ULL, 760ULL, 1216ULL}) {
            for (uint64_t units = 1; units < 5000; units += 1 + units / 7) {
                for (uint64_t maxp : {0ULL, 1ULL, 3ULL, 100ULL, 100000ULL}) {
                    case_no++;
                    const uint64_t p = vec_pieces_per_stream(units, grid, maxp, share);
                    auto fill = [&](uint64_t q) {
                        const uint64_t u = units * q;
                        return (double)u / (double)(((u + grid - 1) / grid) * grid);
                    };
                    // within kVecRounds (4) rounds' worth of pieces
                    const uint64_t cap = 4 * ((grid + units - 1) / units);
                    const bool bad =
                        p < 1 || p > std::max<uint64_t>(1, std::min<uint64_t>(cap, maxp)) ||
                        fill(p) + 1e-12 < fill(1) || (units % grid == 0 && p != 1) ||
                        (share <= 0.2 && maxp >= cap && fill(p) < 0.75) ||
                        (share > 1e6 && p != 1) ||
                        vec_plan_score(units, grid, p, share) + 1e-12 <
                            0.97 * vec_plan_score(units, grid, 1, share);
                    if (bad) {
                        std::printf("vec pieces: units %llu grid %llu max %llu share %g -> %llu "
                                    "(fill %.3f)\n",
                                    (unsigned long long)units, (unsigned long long)grid,
                                    (unsigned long long)maxp, share, (unsigned long long)p,
                                    fill(p));
                        failures++;
                    }
                }
            }
        }
    }
    // 7. the split workload's shapes (parents x 32 substreams x 2^16, 128 x 8 tiles, 760
    // resident blocks): the vector units' last round is nearly full
    for (uint32_t parents : {8u, 32u, 256u, 1024u, 4096u}) {
        case_no++;
        const uint32_t k = parents * 32;
        std::vector<InstParams> P(k);
        for (uint32_t i = 0; i < k; i++)
            P[i].e = P[i].eq = 3 + 2 * ((i / 32) % 3);
        std::vector<uint32_t> ids(k);
        std::vector<uint64_t> cnt(k, 65536), off(k);
        for (uint32_t i = 0; i < k; i++) {
            ids[i] = i;
            off[i] = (uint64_t)(i / 32) * 65536 * 32 + (i % 32);
        }
        const PlanGeometry geo{128, 8, 760};
        HostPlan hp;
        if (build_plan_core(P.data(), k, RSAPRNG_MODEXP_CRT32, geo, k, ids.data(), cnt.data(),
                            off.data(), 0, hp, 1, 32) != RSAPRNG_OK) {
            failures++;
            continue;
        }
        const uint64_t u = hp.vecs.size(), rounds = (u + geo.grid - 1) / geo.grid;
        const double fill = (double)u / (double)(rounds * geo.grid);
        if (fill < 0.85) {
            std::printf("split shape %u parents: %llu units, last round fill %.3f\n", parents,
                        (unsigned long long)u, fill);
            failures++;
        }
    }
    std::printf("%d cases, %d failures\n", case_no, failures);
    return failures ? 1 : 0;
}
