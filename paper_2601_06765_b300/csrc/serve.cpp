// serve.cpp -- batching and continuous-batching serving of independent systems on one GPU.
//
// Both run systems in lockstep: one iteration takes one F4 step of every running system with
// pairs left (one launch of each pipeline kernel covers all of their rows) and builds the reduced
// basis of every running system without pairs.  gb_batch_groebner iterates over a fixed set until
// all are finished.  gb_server's scheduler thread admits queued systems between iterations while
// a slot is free and the summed device footprint estimate of the running systems stays under the
// cap, so a request that arrives joins the very next iteration and one that finishes leaves at
// once (iteration-level continuous batching).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <unordered_map>
#include <unordered_set>

#include "internal.hpp"

namespace gb {
void f4_steps(const std::vector<gb_system *> &Ss, std::vector<gb_step_stats> *stats);
void finish_batch(const std::vector<gb_system *> &Ss);
void groebner_batch(const std::vector<gb_system *> &Ss);
}  // namespace gb

using namespace gb;

struct gb_server {
    gb_ctx *ctx = nullptr;
    gb_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::pair<uint64_t, gb_system *>> queue;
    std::unordered_map<uint64_t, std::pair<gb_system *, gb_status>> done;
    std::unordered_map<uint64_t, bool> known;
    std::unordered_set<const gb_system *> held;  // submitted and not yet polled back
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread scheduler;
    gb_server_stats stats{};
};

namespace {

struct Running {
    uint64_t ticket;
    gb_system *sys;
    uint32_t waited = 0;  // iterations spent out of pairs, waiting for the final reduction
};

// take queued systems while a slot is free and the footprint fits (a system larger than the whole
// cap is still admitted when nothing else runs); called with srv->mu held
void admit(gb_server *srv, std::vector<Running> &run, size_t &bytes) {
    const size_t wave = std::max<uint32_t>(srv->opts.admit_min, 1);
    if (!run.empty() && srv->opts.max_slots - run.size() < std::min<size_t>(wave, srv->opts.max_slots)) return;
    while (!srv->queue.empty() && run.size() < srv->opts.max_slots) {
        gb_system *S = srv->queue.front().second;
        if (!run.empty() && bytes + S->footprint > srv->opts.hbm_cap_bytes) break;
        run.push_back(Running{srv->queue.front().first, S});
        bytes += S->footprint;
        srv->queue.pop_front();
        srv->stats.admitted++;
    }
}

void scheduler_loop(gb_server *srv) {
    std::vector<Running> run;
    size_t bytes = 0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (run.empty()) srv->cv.wait(lk, [&] { return srv->stop || !srv->queue.empty(); });
            if (srv->stop) {  // running and queued systems are destroyed with the server
                for (auto &r : run) srv->done[r.ticket] = {r.sys, GB_EBUSY};
                return;
            }
            admit(srv, run, bytes);
        }
        // one lockstep iteration: a step for every system with pairs left, and the final reduction
        // of the systems out of pairs -- now, or (finish_min > 1) once enough of them are ready
        std::vector<gb_system *> Ss, step, fin;
        for (auto &r : run) {
            Ss.push_back(r.sys);
            if (r.sys->finished) continue;
            if (!r.sys->pairs.empty()) step.push_back(r.sys);
        }
        {
            size_t ready = 0;
            bool due = step.empty();
            for (auto &r : run)
                if (!r.sys->finished && r.sys->pairs.empty()) {
                    ++ready;
                    due = due || r.waited >= 4;
                }
            due = due || ready >= std::max<uint32_t>(srv->opts.finish_min, 1);
            for (auto &r : run)
                if (!r.sys->finished && r.sys->pairs.empty()) {
                    if (due) fin.push_back(r.sys);
                    else ++r.waited;
                }
        }
        gb_status st = GB_OK;
        double fin_ms = 0.0;
        const auto t0 = std::chrono::steady_clock::now();
        try {
            std::lock_guard<std::recursive_mutex> g(srv->ctx->mu);
            GB_CUDA(cudaSetDevice(srv->ctx->device));
            if (!fin.empty()) {
                finish_batch(fin);
                fin_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            }
            if (!step.empty()) f4_steps(step, nullptr);
        } catch (const gb::Error &e) {
            set_last_error(e.what());
            st = e.st;
        } catch (const std::bad_alloc &) {
            st = GB_ENOMEM;
        } catch (const std::exception &e) {
            set_last_error(e.what());
            st = GB_EDEVICE;
        }
        // a failed iteration leaves its systems in an undefined state: all of them finish with the
        // error (the pipeline runs them together, so the failing one is not singled out)
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stats.iterations++;
        srv->stats.system_steps += Ss.size();
        srv->stats.busy_ms += ms;
        srv->stats.finish_ms += fin_ms;
        if (!fin.empty()) srv->stats.finish_passes++;
        srv->stats.max_running = std::max<uint32_t>(srv->stats.max_running, (uint32_t)Ss.size());
        size_t w = 0;
        for (auto &r : run) {
            if (st != GB_OK || r.sys->finished) {
                srv->done[r.ticket] = {r.sys, st};
                bytes -= r.sys->footprint;
                srv->stats.finished++;
            } else {
                run[w++] = r;
            }
        }
        run.resize(w);
    }
}

}  // namespace

extern "C" {

gb_status gb_batch_groebner(gb_ctx *ctx, uint32_t count, gb_system *const *systems,
                            gb_run_stats *per_system) {
    try {
        if (!ctx || (count && !systems)) return GB_EINVAL;
        std::vector<gb_system *> Ss;
        for (uint32_t i = 0; i < count; ++i) {
            if (!systems[i] || systems[i]->ctx != ctx) return GB_EINVAL;
            if (std::find(Ss.begin(), Ss.end(), systems[i]) != Ss.end()) {
                set_last_error("a system appears twice in the batch");
                return GB_EINVAL;
            }
            Ss.push_back(systems[i]);
        }
        {
            std::lock_guard<std::recursive_mutex> g(ctx->mu);
            GB_CUDA(cudaSetDevice(ctx->device));
            groebner_batch(Ss);
        }
        for (uint32_t i = 0; per_system && i < count; ++i) per_system[i] = Ss[i]->run;
        return GB_OK;
    } catch (const gb::Error &e) {
        set_last_error(e.what());
        return e.st;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return GB_ENOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return GB_EDEVICE;
    }
}

gb_status gb_server_create(gb_ctx *ctx, const gb_server_opts *opts, gb_server **out) {
    if (!ctx || !out) return GB_EINVAL;
    auto *srv = new (std::nothrow) gb_server();
    if (!srv) return GB_ENOMEM;
    srv->ctx = ctx;
    if (opts) srv->opts = *opts;
    if (!srv->opts.max_slots) srv->opts.max_slots = 64;
    if (!srv->opts.hbm_cap_bytes) srv->opts.hbm_cap_bytes = ctx->arena.capacity();
    try {
        srv->scheduler = std::thread(scheduler_loop, srv);
    } catch (const std::exception &e) {
        set_last_error(e.what());
        delete srv;
        return GB_EDEVICE;
    }
    *out = srv;
    return GB_OK;
}

gb_status gb_server_submit(gb_server *srv, gb_system *sys, uint64_t *ticket) {
    if (!srv || !sys || !ticket || sys->ctx != srv->ctx) return GB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return GB_EINVAL;
        if (!srv->held.insert(sys).second) {  // already queued, running or finished unpolled
            set_last_error("gb_server_submit: this system is already held by the server");
            return GB_EINVAL;
        }
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
    srv->held.erase(it->second.first);
    srv->done.erase(it);
    srv->known.erase(ticket);
    return GB_OK;
}

gb_status gb_server_stats_get(gb_server *srv, gb_server_stats *out) {
    if (!srv || !out) return GB_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->queued = (uint32_t)srv->queue.size();
    return GB_OK;
}

gb_status gb_server_destroy(gb_server *srv) {
    if (!srv) return GB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->scheduler.joinable()) srv->scheduler.join();
    // systems that were submitted and never polled (queued, running or finished) go with the server
    std::vector<gb_system *> owned;
    for (auto &q : srv->queue) owned.push_back(q.second);
    for (auto &d : srv->done) owned.push_back(d.second.first);
    delete srv;
    for (gb_system *S : owned) gb_system_destroy(S);
    return GB_OK;
}

}  // extern "C"
