// Continuous-batching request server over a context's instances.
//
// Clients submit (instance, count) requests. A worker thread admits them in
// FIFO order while their outputs (8 B per number) fit in the server's device
// arena, then repeatedly gathers the admitted work into one batched launch
// sequence (skip-sum pre-pass + generation, as rsaprng_generate_batch) on one
// of several CUDA streams, so iterations overlap on the device. Each request's
// numbers are the instance's next outputs in admission order: an instance
// appears in at most one in-flight iteration, and its requests are scheduled
// strictly in FIFO order, so a result does not depend on what else is in the
// mix. Large requests are cut into pieces per iteration.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.hpp"

using namespace rsaprng;

namespace {

using clk = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

// First-fit allocator over [0, capacity) elements with coalescing frees.
// Allocations are whole 16-element (128-byte) lines, so every result starts
// on a line and the iterations' full tiles leave by bulk tensor stores
// without a staging shift.
static uint64_t whole_lines(uint64_t n) { return (n + 15) & ~15ULL; }

class Arena {
  public:
    explicit Arena(uint64_t cap) : cap_(cap) { free_[0] = cap; }
    bool alloc(uint64_t n, uint64_t *off)
    {
        if (n == 0) {
            *off = 0;
            return true;
        }
        n = whole_lines(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest)
                    free_[at] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n)
    {
        if (n == 0)
            return;
        n = whole_lines(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }

  private:
    uint64_t cap_, used_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

enum ReqState { RQ_QUEUED, RQ_ACTIVE, RQ_DONE, RQ_CANCELLED };

struct Request {
    rsaprng_id id;
    uint64_t count;
    uint64_t arena_off = 0;
    uint64_t scheduled = 0;  // numbers handed to iterations
    uint64_t done = 0;       // numbers completed
    int state = RQ_QUEUED;
    bool auto_release = false;
    double t_submit = 0, t_done = 0;
};

struct Piece {
    uint64_t ticket;
    uint64_t count;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr;  // recorded before the iteration's upload
    cudaEvent_t done = nullptr;
    DevPlan plan;
    bool busy = false;
    uint64_t iter = 0;
    std::vector<Piece> pieces;
    std::vector<rsaprng_id> insts;
    double t_launch = 0;
};

}  // namespace

struct rsaprng_server {
    rsaprng_ctx *ctx = nullptr;
    uint64_t budget_numbers = 0;
    double *d_arena = nullptr;
    Arena *arena = nullptr;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::unordered_map<uint64_t, Request> reqs;
    std::deque<uint64_t> queue;   // waiting for admission
    std::deque<uint64_t> active;  // admitted, not fully scheduled
    std::vector<uint64_t> busy;   // per instance: in-flight iteration (0 = free)
    std::vector<uint64_t> stamp;  // per instance: iteration that blocked it
    uint64_t next_ticket = 1, iter_counter = 0;
    // An iteration carries at most per_iter_cap numbers and at most
    // per_req_cap of one request, so small requests are not queued behind a
    // large one for long.
    uint64_t per_req_cap = 1ULL << 22, per_iter_cap = 1ULL << 24;
    // statistics
    uint64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, cancelled = 0;
    uint64_t numbers_done = 0, iterations = 0;
    uint64_t max_inflight = 0, overlapped = 0;
    // Device intervals (ms after t_ref) of the most recently retired
    // iterations, to count the iterations that ran beside another one.
    cudaEvent_t t_ref = nullptr;
    std::deque<std::pair<float, float>> recent;
    std::vector<double> lat_ms;
    double t_first = 0, t_last = 0, busy_s = 0;
    int error = RSAPRNG_OK;
    std::string error_detail;
};

namespace {

void admit_locked(rsaprng_server *S)
{
    while (!S->queue.empty()) {
        const uint64_t t = S->queue.front();
        auto it = S->reqs.find(t);
        if (it == S->reqs.end() || it->second.state != RQ_QUEUED) {
            S->queue.pop_front();
            continue;
        }
        Request &r = it->second;
        uint64_t off;
        if (!S->arena->alloc(r.count, &off))
            break;  // FIFO: later requests wait behind the head
        r.arena_off = off;
        r.state = RQ_ACTIVE;
        S->queue.pop_front();
        S->active.push_back(t);
        S->admitted++;
    }
}

void complete_locked(rsaprng_server *S, Request &r, uint64_t ticket, double t)
{
    r.state = RQ_DONE;
    r.t_done = t;
    S->completed++;
    S->lat_ms.push_back((t - r.t_submit) * 1e3);
    S->t_last = t;
    if (r.auto_release) {
        S->arena->release(r.arena_off, r.count);
        S->reqs.erase(ticket);
    }
}

// Retires finished iterations; returns true if any finished.
bool retire(rsaprng_server *S, bool block_oldest)
{
    bool any = false;
    for (auto &sl : S->slots) {
        if (!sl.busy)
            continue;
        cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady)
            continue;
        if (q != cudaSuccess) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->error = RSAPRNG_ERR_CUDA;
            S->error_detail = cudaGetErrorString(q);
        }
        const double t = now_s();
        float d0 = 0, d1 = 0;
        const bool timed = cudaEventElapsedTime(&d0, S->t_ref, sl.start) == cudaSuccess &&
                           cudaEventElapsedTime(&d1, S->t_ref, sl.done) == cudaSuccess;
        std::lock_guard<std::mutex> lk(S->mu);
        if (timed) {
            // Retired in any order: compare with every recent interval.
            for (const auto &iv : S->recent)
                if (d0 < iv.second && iv.first < d1) {
                    S->overlapped++;
                    break;
                }
            S->recent.emplace_back(d0, d1);
            if (S->recent.size() > 64)
                S->recent.pop_front();
        }
        S->busy_s += t - sl.t_launch;
        for (rsaprng_id id : sl.insts)
            if (S->busy[id] == sl.iter)
                S->busy[id] = 0;
        for (const Piece &p : sl.pieces) {
            auto it = S->reqs.find(p.ticket);
            if (it == S->reqs.end())
                continue;
            Request &r = it->second;
            r.done += p.count;
            S->numbers_done += p.count;
            if (r.done == r.count)
                complete_locked(S, r, p.ticket, t);
        }
        sl.busy = false;
        sl.pieces.clear();
        sl.insts.clear();
        any = true;
    }
    (void)block_oldest;
    if (any) {
        S->cv_done.notify_all();
    }
    return any;
}

// Builds and launches one iteration on slot `sl`. Returns false if there was
// nothing to schedule.
bool launch_iteration(rsaprng_server *S, Slot &sl)
{
    std::vector<rsaprng_id> ids;
    std::vector<uint64_t> counts, offs;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        admit_locked(S);
        if (S->active.empty())
            return false;
        const uint64_t iter = ++S->iter_counter;
        uint64_t budget = S->per_iter_cap;
        std::deque<uint64_t> keep;
        for (uint64_t t : S->active) {
            auto it = S->reqs.find(t);
            if (it == S->reqs.end())
                continue;
            Request &r = it->second;
            if (r.state != RQ_ACTIVE)
                continue;
            if (r.scheduled == r.count) {
                continue;  // fully scheduled, waiting for completion
            }
            const rsaprng_id id = r.id;
            if (budget == 0 || (S->busy[id] && S->busy[id] != iter) || S->stamp[id] == iter) {
                S->stamp[id] = iter;  // later requests of this instance wait too
                keep.push_back(t);
                continue;
            }
            const uint64_t take = std::min({r.count - r.scheduled, S->per_req_cap, budget});
            ids.push_back(id);
            counts.push_back(take);
            offs.push_back(r.arena_off + r.scheduled);
            sl.pieces.push_back({t, take});
            r.scheduled += take;
            budget -= take;
            if (!S->busy[id]) {
                S->busy[id] = iter;
                sl.insts.push_back(id);
            }
            if (r.scheduled < r.count) {
                S->stamp[id] = iter;
                keep.push_back(t);
            }
        }
        S->active.swap(keep);
        sl.iter = iter;
        if (ids.empty()) {
            sl.pieces.clear();
            sl.insts.clear();
            return false;
        }
    }
    // Outside the lock: plan, upload, launch. Chunks are sized so that the
    // iteration spreads over all SMs.
    uint64_t numbers = 0;
    for (uint64_t x : counts)
        numbers += x;
    const uint64_t tile =
        (uint64_t)S->ctx->cfg.threads_per_block * S->ctx->cfg.numbers_per_thread;
    uint64_t chunk = numbers / ((uint64_t)S->ctx->sms * 8);
    chunk = std::max<uint64_t>(tile, (chunk + tile - 1) / tile * tile);
    chunk = std::min<uint64_t>(chunk, std::max<uint64_t>(S->ctx->cfg.chunk, tile));
    HostPlan hp;
    cudaEventRecord(sl.start, sl.stream);
    // The iteration sizes its pieces itself (the chunk above); the load-balance
    // split for long launches would only add skip-sum work to short ones.
    rsaprng_config cfg = S->ctx->cfg;
    cfg.pieces_per_block = 1;
    int rc = build_plan(S->ctx, cfg, ids.size(), ids.data(), counts.data(), offs.data(),
                        chunk, hp, 1, 1, true);
    if (rc == RSAPRNG_OK)
        rc = upload_plan(S->ctx, hp, sl.plan, sl.stream);
    if (rc == RSAPRNG_OK)
        rc = launch_plan(S->ctx, cfg, sl.plan, S->d_arena, nullptr, sl.stream, nullptr,
                         nullptr, true);
    cudaEventRecord(sl.done, sl.stream);
    sl.t_launch = now_s();
    sl.busy = true;
    uint64_t in_flight = 0;
    for (auto &o : S->slots)
        in_flight += o.busy ? 1 : 0;
    std::lock_guard<std::mutex> lk(S->mu);
    S->max_inflight = std::max(S->max_inflight, in_flight);
    S->iterations++;
    if (rc != RSAPRNG_OK) {
        S->error = rc;
        S->error_detail = rsaprng_last_error_detail();
    }
    return true;
}

void worker_main(rsaprng_server *S)
{
    cudaSetDevice(S->ctx->device);
    for (;;) {
        retire(S, false);
        bool launched = false;
        for (auto &sl : S->slots) {
            if (sl.busy)
                continue;
            if (!launch_iteration(S, sl))
                break;
            launched = true;
        }
        bool inflight = false;
        for (auto &sl : S->slots)
            inflight = inflight || sl.busy;
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stop && !inflight)
            return;
        if (launched)
            continue;
        if (!inflight) {
            // idle, or the queue head waits for arena space: sleep until a
            // submit or release wakes us (bounded, to re-check `stop`)
            S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        } else {
            lk.unlock();
            std::this_thread::yield();
        }
    }
}

}  // namespace

extern "C" {

int rsaprng_server_create(rsaprng_ctx *c, uint64_t out_budget_bytes, int nstreams,
                          rsaprng_server **out)
{
    if (!c || !out || out_budget_bytes < 8 || nstreams < 1 || nstreams > 16)
        return fail(RSAPRNG_ERR_ARG, "server_create: bad arguments");
    *out = nullptr;
    rsaprng_server *S = new (std::nothrow) rsaprng_server();
    if (!S)
        return fail(RSAPRNG_ERR_OOM, "server alloc");
    S->ctx = c;
    S->budget_numbers = out_budget_bytes / 8;
    cudaSetDevice(c->device);
    // whole lines: a request of the whole budget still fits after rounding
    const uint64_t cap = whole_lines(S->budget_numbers);
    cudaError_t e = cudaMalloc(&S->d_arena, cap * 8);
    if (e != cudaSuccess) {
        delete S;
        return fail(RSAPRNG_ERR_OOM, "server arena (%llu B): %s",
                    (unsigned long long)out_budget_bytes, cudaGetErrorString(e));
    }
    S->arena = new Arena(cap);
    S->slots.resize(nstreams);
    for (auto &sl : S->slots) {
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        cudaEventCreate(&sl.start);
        cudaEventCreate(&sl.done);
    }
    cudaEventCreate(&S->t_ref);
    cudaEventRecord(S->t_ref, S->slots[0].stream);
    cudaEventSynchronize(S->t_ref);
    S->busy.assign(c->capacity, 0);
    S->stamp.assign(c->capacity, 0);
    S->t_first = now_s();
    S->worker = std::thread(worker_main, S);
    *out = S;
    return RSAPRNG_OK;
}

static int submit_impl(rsaprng_server *S, rsaprng_id id, uint64_t count, uint64_t *ticket,
                       bool auto_release, double t_submit)
{
    if (!S || !ticket)
        return fail(RSAPRNG_ERR_ARG, "server_submit: null argument");
    if (id >= S->ctx->count)
        return fail(RSAPRNG_ERR_ID, "unknown instance %u", id);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error)
        return fail(S->error, "server failed earlier: %s", S->error_detail.c_str());
    if (count > S->budget_numbers) {
        S->rejected++;
        return fail(RSAPRNG_ERR_BUDGET, "request of %llu numbers exceeds the %llu-number arena",
                    (unsigned long long)count, (unsigned long long)S->budget_numbers);
    }
    const uint64_t t = S->next_ticket++;
    Request r;
    r.id = id;
    r.count = count;
    r.auto_release = auto_release;
    r.t_submit = t_submit;
    S->reqs.emplace(t, r);
    S->submitted++;
    if (count == 0) {
        auto &rr = S->reqs[t];
        rr.state = RQ_ACTIVE;
        S->admitted++;
        complete_locked(S, rr, t, t_submit);
    } else {
        S->queue.push_back(t);
    }
    *ticket = t;
    S->cv_work.notify_one();
    return RSAPRNG_OK;
}

int rsaprng_server_submit(rsaprng_server *S, rsaprng_id id, uint64_t count, uint64_t *ticket)
{
    return submit_impl(S, id, count, ticket, false, now_s());
}

int rsaprng_server_poll(rsaprng_server *S, uint64_t ticket, int *done)
{
    if (!S || !done)
        return fail(RSAPRNG_ERR_ARG, "null");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return fail(RSAPRNG_ERR_ID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state == RQ_CANCELLED)
        return fail(RSAPRNG_ERR_CANCELLED, "ticket cancelled");
    *done = it->second.state == RQ_DONE ? 1 : 0;
    return S->error ? fail(S->error, "server failed: %s", S->error_detail.c_str()) : RSAPRNG_OK;
}

int rsaprng_server_wait(rsaprng_server *S, uint64_t ticket, uint64_t timeout_ns)
{
    if (!S)
        return fail(RSAPRNG_ERR_ARG, "null");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = clk::now() + std::chrono::nanoseconds(timeout_ns);
    for (;;) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end())
            return fail(RSAPRNG_ERR_ID, "unknown ticket %llu", (unsigned long long)ticket);
        if (it->second.state == RQ_DONE)
            return RSAPRNG_OK;
        if (it->second.state == RQ_CANCELLED)
            return fail(RSAPRNG_ERR_CANCELLED, "ticket cancelled");
        if (S->error)
            return fail(S->error, "server failed: %s", S->error_detail.c_str());
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = S->reqs.find(ticket);
            if (it2 != S->reqs.end() && it2->second.state == RQ_DONE)
                return RSAPRNG_OK;
            return fail(RSAPRNG_ERR_TIMEOUT, "ticket %llu not done within %llu ns",
                        (unsigned long long)ticket, (unsigned long long)timeout_ns);
        }
    }
}

int rsaprng_server_result(rsaprng_server *S, uint64_t ticket, const double **d_r, uint64_t *count)
{
    if (!S || !d_r || !count)
        return fail(RSAPRNG_ERR_ARG, "null");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return fail(RSAPRNG_ERR_ID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state != RQ_DONE)
        return fail(RSAPRNG_ERR_ARG, "ticket %llu not complete", (unsigned long long)ticket);
    *d_r = S->d_arena + it->second.arena_off;
    *count = it->second.count;
    return RSAPRNG_OK;
}

int rsaprng_server_copy(rsaprng_server *S, uint64_t ticket, double *d_dst, void *stream)
{
    const double *src;
    uint64_t n;
    int rc = rsaprng_server_result(S, ticket, &src, &n);
    if (rc)
        return rc;
    if (n == 0)
        return RSAPRNG_OK;
    if (!d_dst)
        return fail(RSAPRNG_ERR_ARG, "null destination");
    cudaError_t e = cudaMemcpyAsync(d_dst, src, n * 8, cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "server_copy");
    return RSAPRNG_OK;
}

int rsaprng_server_release(rsaprng_server *S, uint64_t ticket)
{
    if (!S)
        return fail(RSAPRNG_ERR_ARG, "null");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return fail(RSAPRNG_ERR_ID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state == RQ_DONE)
        S->arena->release(it->second.arena_off, it->second.count);
    else if (it->second.state != RQ_CANCELLED)
        return fail(RSAPRNG_ERR_ARG, "ticket %llu still in progress", (unsigned long long)ticket);
    S->reqs.erase(it);
    S->cv_work.notify_one();
    return RSAPRNG_OK;
}

int rsaprng_server_cancel(rsaprng_server *S, uint64_t ticket)
{
    if (!S)
        return fail(RSAPRNG_ERR_ARG, "null");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return fail(RSAPRNG_ERR_ID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state != RQ_QUEUED)
        return fail(RSAPRNG_ERR_ARG, "ticket %llu already admitted", (unsigned long long)ticket);
    it->second.state = RQ_CANCELLED;
    S->cancelled++;
    S->cv_done.notify_all();
    return RSAPRNG_OK;
}

int rsaprng_server_stats(rsaprng_server *S, rsaprng_stats *out)
{
    if (!S || !out)
        return fail(RSAPRNG_ERR_ARG, "null");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof *out);
    out->submitted = S->submitted;
    out->admitted = S->admitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->cancelled = S->cancelled;
    out->queued_now = S->queue.size();
    uint64_t infl = 0;
    for (auto &kv : S->reqs)
        infl += kv.second.state == RQ_ACTIVE;
    out->inflight_now = infl;
    out->numbers_done = S->numbers_done;
    out->iterations = S->iterations;
    out->max_inflight_iterations = S->max_inflight;
    out->overlapped_iterations = S->overlapped;
    out->busy_s = S->busy_s;
    out->wall_s = (S->t_last > S->t_first ? S->t_last : now_s()) - S->t_first;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t k = (size_t)std::min<double>(v.size() - 1, std::ceil(p * v.size()) - 1);
            return v[k];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double x : v)
            s += x;
        out->mean_ms = s / v.size();
        out->max_ms = v.back();
    }
    return RSAPRNG_OK;
}

// Open-loop trace replay for load measurements: request i is submitted at
// arrival_ns[i] (nanoseconds after the call starts) with its outputs released
// as soon as they complete. Returns when every request has completed (or
// timeout_ns passes). Latencies (ms) go to lat_ms_out[i] when non-NULL.
static int replay_impl(rsaprng_server *S, uint64_t n, const rsaprng_id *ids,
                       const uint64_t *counts, const uint64_t *arrival_ns, uint64_t timeout_ns,
                       double *lat_ms_out, uint64_t *tickets_out)
{
    if (!S || (n && (!ids || !counts || !arrival_ns)))
        return fail(RSAPRNG_ERR_ARG, "server_replay: null argument");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->lat_ms.clear();
        S->numbers_done = 0;
        S->submitted = S->admitted = S->completed = S->rejected = 0;
        S->iterations = 0;
        S->busy_s = 0;
        S->max_inflight = S->overlapped = 0;
        S->recent.clear();
    }
    std::vector<uint64_t> tickets(n, 0);
    const auto t0 = clk::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->t_first = now_s();
    }
    for (uint64_t i = 0; i < n; i++) {
        const auto due = t0 + std::chrono::nanoseconds(arrival_ns[i]);
        while (clk::now() < due) {
            const auto left = due - clk::now();
            if (left > std::chrono::microseconds(200))
                std::this_thread::sleep_for(left - std::chrono::microseconds(100));
        }
        const double ts = std::chrono::duration<double>(due.time_since_epoch()).count();
        int rc = submit_impl(S, ids[i], counts[i], &tickets[i], tickets_out == nullptr, ts);
        if (rc)
            return rc;
        if (tickets_out)
            tickets_out[i] = tickets[i];
    }
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = clk::now() + std::chrono::nanoseconds(timeout_ns);
    while (S->completed < n && !S->error) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && S->completed < n)
            return fail(RSAPRNG_ERR_TIMEOUT, "replay: %llu of %llu requests done",
                        (unsigned long long)S->completed, (unsigned long long)n);
    }
    if (S->error)
        return fail(S->error, "server failed: %s", S->error_detail.c_str());
    if (lat_ms_out)
        for (uint64_t i = 0; i < n && i < S->lat_ms.size(); i++)
            lat_ms_out[i] = S->lat_ms[i];
    return RSAPRNG_OK;
}

int rsaprng_server_replay(rsaprng_server *S, uint64_t n, const rsaprng_id *ids,
                          const uint64_t *counts, const uint64_t *arrival_ns, uint64_t timeout_ns,
                          double *lat_ms_out)
{
    return replay_impl(S, n, ids, counts, arrival_ns, timeout_ns, lat_ms_out, nullptr);
}

int rsaprng_server_replay_keep(rsaprng_server *S, uint64_t n, const rsaprng_id *ids,
                               const uint64_t *counts, const uint64_t *arrival_ns,
                               uint64_t timeout_ns, uint64_t *tickets_out)
{
    if (!tickets_out)
        return fail(RSAPRNG_ERR_ARG, "server_replay_keep: null tickets");
    return replay_impl(S, n, ids, counts, arrival_ns, timeout_ns, nullptr, tickets_out);
}

void rsaprng_server_destroy(rsaprng_server *S)
{
    if (!S)
        return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // drop work that has not started
        S->queue.clear();
        for (uint64_t t : S->active) {
            auto it = S->reqs.find(t);
            if (it != S->reqs.end())
                it->second.scheduled = it->second.count;
        }
        S->active.clear();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable())
        S->worker.join();
    cudaSetDevice(S->ctx->device);
    for (auto &sl : S->slots) {
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
        free_devplan(sl.plan);
        if (sl.done)
            cudaEventDestroy(sl.done);
        if (sl.start)
            cudaEventDestroy(sl.start);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
    }
    if (S->t_ref)
        cudaEventDestroy(S->t_ref);
    if (S->d_arena)
        cudaFree(S->d_arena);
    delete S->arena;
    delete S;
}

}  // extern "C"
