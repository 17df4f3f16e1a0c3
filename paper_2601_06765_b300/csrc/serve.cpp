// serve.cpp -- batching and continuous-batching serving of independent systems on one GPU.
//
// Every system owns a CUDA stream, so the device work of different systems overlaps whenever
// their host control runs concurrently.  gb_batch_groebner drives a fixed set of systems with a
// pool of host workers.  gb_server admits submitted systems into slots while the summed device
// footprint estimate of the admitted systems stays under the cap; a slot that finishes frees its
// footprint and the next queued system is admitted at once, while the others keep running.
#include <algorithm>
#include <condition_variable>
#include <unordered_map>

#include "internal.hpp"

namespace gb {
gb_status groebner(gb_system *S, gb_run_stats *stats);
}

using namespace gb;

namespace {

gb_status run_one(gb_system *S, gb_run_stats *st) {
    try {
        GB_CUDA(cudaSetDevice(S->ctx->device));
        return groebner(S, st);
    } catch (const gb::Error &e) {
        set_last_error(e.what());
        return e.st;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return GB_EDEVICE;
    }
}

unsigned default_workers(uint32_t count) {
    unsigned hw = std::thread::hardware_concurrency();
    if (!hw) hw = 4;
    return std::max(1u, std::min<unsigned>(count, std::min(hw, 32u)));
}

}  // namespace

struct gb_server {
    gb_ctx *ctx = nullptr;
    gb_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<std::pair<uint64_t, gb_system *>> queue;
    std::unordered_map<uint64_t, std::pair<gb_system *, gb_status>> done;
    std::unordered_map<uint64_t, bool> known;
    size_t admitted_bytes = 0;
    uint32_t running = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

static void server_worker(gb_server *srv) {
    for (;;) {
        std::pair<uint64_t, gb_system *> job;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            // admission: a slot is free and the head of the queue fits under the cap (a system
            // larger than the whole cap is still admitted when nothing else runs)
            srv->cv.wait(lk, [&] {
                if (srv->stop) return true;
                if (srv->queue.empty()) return false;
                const size_t need = srv->queue.front().second->footprint;
                return srv->running == 0 || srv->admitted_bytes + need <= srv->opts.hbm_cap_bytes;
            });
            if (srv->stop && srv->queue.empty()) return;
            if (srv->queue.empty()) continue;
            job = srv->queue.front();
            srv->queue.pop_front();
            srv->admitted_bytes += job.second->footprint;
            srv->running++;
        }
        const gb_status st = run_one(job.second, nullptr);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->admitted_bytes -= job.second->footprint;
            srv->running--;
            srv->done[job.first] = {job.second, st};
        }
        srv->cv.notify_all();
        srv->done_cv.notify_all();
    }
}

extern "C" {

gb_status gb_batch_groebner(gb_ctx *ctx, uint32_t count, gb_system *const *systems,
                            gb_run_stats *per_system) {
    if (!ctx || (count && !systems)) return GB_EINVAL;
    for (uint32_t i = 0; i < count; ++i)
        if (!systems[i] || systems[i]->ctx != ctx) return GB_EINVAL;
    std::atomic<uint32_t> next{0};
    std::vector<gb_status> st(count, GB_OK);
    auto work = [&] {
        for (uint32_t i; (i = next.fetch_add(1)) < count;)
            st[i] = run_one(systems[i], per_system ? &per_system[i] : nullptr);
    };
    std::vector<std::thread> pool;
    const unsigned w = default_workers(count);
    for (unsigned t = 1; t < w; ++t) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
    for (uint32_t i = 0; i < count; ++i)
        if (st[i] != GB_OK) return st[i];
    return GB_OK;
}

gb_status gb_server_create(gb_ctx *ctx, const gb_server_opts *opts, gb_server **out) {
    if (!ctx || !out) return GB_EINVAL;
    auto *srv = new (std::nothrow) gb_server();
    if (!srv) return GB_ENOMEM;
    srv->ctx = ctx;
    if (opts) srv->opts = *opts;
    if (!srv->opts.max_slots) srv->opts.max_slots = 64;
    if (!srv->opts.hbm_cap_bytes) srv->opts.hbm_cap_bytes = ctx->arena.capacity();
    for (uint32_t i = 0; i < srv->opts.max_slots; ++i) srv->workers.emplace_back(server_worker, srv);
    *out = srv;
    return GB_OK;
}

gb_status gb_server_submit(gb_server *srv, gb_system *sys, uint64_t *ticket) {
    if (!srv || !sys || !ticket || sys->ctx != srv->ctx) return GB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return GB_EINVAL;
        *ticket = srv->next_ticket++;
        srv->known[*ticket] = true;
        srv->queue.emplace_back(*ticket, sys);
    }
    srv->cv.notify_all();
    return GB_OK;
}

gb_status gb_server_poll(gb_server *srv, uint64_t ticket, gb_system **done, gb_status *result) {
    if (!srv || !done) return GB_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (!srv->known.count(ticket)) return GB_EINVAL;
    auto it = srv->done.find(ticket);
    if (it == srv->done.end()) return GB_EBUSY;
    *done = it->second.first;
    if (result) *result = it->second.second;
    srv->done.erase(it);
    srv->known.erase(ticket);
    return GB_OK;
}

gb_status gb_server_destroy(gb_server *srv) {
    if (!srv) return GB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    for (auto &t : srv->workers) t.join();
    // systems still queued or finished but never polled are destroyed with the server
    for (auto &q : srv->queue) gb_system_destroy(q.second);
    for (auto &d : srv->done) gb_system_destroy(d.second.first);
    delete srv;
    return GB_OK;
}

}  // extern "C"
