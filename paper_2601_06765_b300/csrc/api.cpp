// api.cpp -- the extern "C" entry points of include/gb.h: argument checks, handle lifetime,
// exports to host arrays, error mapping, and the device arena.
#include <algorithm>
#include <chrono>
#include <cstdio>

#include "internal.hpp"

namespace gb {
void modp_apply(int op, uint32_t p, uint64_t n, uint32_t window, const uint32_t *a, const uint32_t *b,
                const uint32_t *c, uint32_t *out, cudaStream_t st);
void reduce_rows_noalloc(uint32_t p, uint32_t N, uint32_t nA, uint32_t nC, uint32_t nb,
                         const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                         const uint32_t *pcols, const uint32_t *nonpiv, uint32_t *dprime,
                         cudaStream_t st);
void f4_steps(const std::vector<gb_system *> &Ss, std::vector<gb_step_stats> *stats);
void groebner_batch(const std::vector<gb_system *> &Ss);
void system_init(gb_system *S, uint32_t nvars, uint32_t p, const gb_polys *F);
void autotune(gb_ctx *ctx, const std::vector<gb_system *> &Ss, gb_tune_report *rep);
void tune_save(const gb_ctx *ctx, const char *path);
void tune_load(gb_ctx *ctx, const char *path);

static thread_local std::string t_last_error;
std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_graph_launches{0};
thread_local bool t_capturing = false;
thread_local unsigned t_captured = 0;

void set_last_error(const std::string &msg) { t_last_error = msg; }

void fail(gb_status s, const std::string &msg) { throw Error(s, msg); }

void cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        throw Error(GB_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    throw Error(GB_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

void opt_in_smem(const void *kernel) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, bool> done;
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if (done.count({dev, kernel})) return;
    int optin = 0;
    GB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    GB_CUDA(cudaFuncGetAttributes(&fa, kernel));
    GB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes));
    done[{dev, kernel}] = true;
}

// ---- page-locked staging of the batch in flight --------------------------------------------------

// A bump allocator over one page-locked area: a region stays valid until the next ctx_sync, which
// (after the stream has drained, so no copy still reads or writes the area) starts over at zero.
void *ctx_pinned(gb_ctx *ctx, size_t bytes) {
    const size_t need = (std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
    if (ctx->stage_off + need > ctx->stage_bytes) {
        ctx_sync(ctx);
        if (need > ctx->stage_bytes) {
            if (ctx->stage) GB_CUDA(cudaFreeHost(ctx->stage));
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
            const size_t sz = std::max<size_t>({need, 2 * ctx->stage_bytes, size_t(8) << 20});
            GB_CUDA(cudaHostAlloc(&ctx->stage, sz, cudaHostAllocDefault));
            ctx->stage_bytes = sz;
        }
    }
    void *p = static_cast<char *>(ctx->stage) + ctx->stage_off;
    ctx->stage_off += need;
    return p;
}

// GB_TRACE=1 in the environment: per-stage wall times of the final reduction on stderr
bool trace_on() {
    static const bool on = [] {
        const char *e = std::getenv("GB_TRACE");
        return e && *e && *e != '0';
    }();
    return on;
}

void ctx_sync(gb_ctx *ctx) {
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->arena.flush(ctx->stream);
    ctx->stage_off = 0;
}

void Stage::upload(gb_ctx *ctx, DBuf<char> &d) {
    d.alloc(ctx->arena, h.size() + 16, ctx->stream);
    char *hp = static_cast<char *>(ctx_pinned(ctx, h.size() + 16));
    std::memcpy(hp, h.data(), h.size());
    GB_CUDA(cudaMemcpyAsync(d.p, hp, h.size(), cudaMemcpyHostToDevice, ctx->stream));
}

// ---- arena ------------------------------------------------------------------------------------

void Arena::init(void *base, size_t bytes, bool owned) {
    std::lock_guard<std::mutex> g(mu_);
    base_ = static_cast<char *>(base);
    cap_ = bytes & ~size_t(255);
    owned_ = owned;
    used_ = 0;
    free_.clear();
    live_.clear();
    pending_.clear();
    if (cap_) free_[0] = cap_;
}

void Arena::release() {
    std::lock_guard<std::mutex> g(mu_);
    if (owned_ && base_) cudaFree(base_);
    base_ = nullptr;
    cap_ = used_ = 0;
    free_.clear();
    live_.clear();
    pending_.clear();
}

void *Arena::alloc(size_t bytes) {
    const size_t need = (std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
    std::lock_guard<std::mutex> g(mu_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > need) free_[off + need] = sz - need;
        live_[off] = need;
        used_ += need;
        peak_ = std::max(peak_, used_);
        return base_ + off;
    }
    char msg[160];
    std::snprintf(msg, sizeof msg, "device arena exhausted: %zu bytes requested, %zu of %zu in use",
                  need, used_, cap_);
    throw Error(GB_ENOMEM, msg);
}

void Arena::free_locked(size_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return;
    size_t sz = it->second;
    live_.erase(it);
    used_ -= sz;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + sz == nx->first) {
        sz += nx->second;
        nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
            pv->second += sz;
            return;
        }
    }
    free_[off] = sz;
}

void Arena::defer_free(void *p, cudaStream_t s) {
    if (!p || !base_) return;
    std::lock_guard<std::mutex> g(mu_);
    pending_.emplace(s, (size_t)(static_cast<char *>(p) - base_));
}

void Arena::flush(cudaStream_t s) {
    std::lock_guard<std::mutex> g(mu_);
    auto range = pending_.equal_range(s);
    for (auto it = range.first; it != range.second; ++it) free_locked(it->second);
    pending_.erase(range.first, range.second);
}

}  // namespace gb

using namespace gb;

#define GB_API_BEGIN try {
#define GB_API_END                                      \
    }                                                   \
    catch (const gb::Error &e) {                        \
        set_last_error(e.what());                       \
        return e.st;                                    \
    }                                                   \
    catch (const std::bad_alloc &) {                    \
        set_last_error("host allocation failed");       \
        return GB_ENOMEM;                               \
    }                                                   \
    catch (const std::exception &e) {                   \
        set_last_error(e.what());                       \
        return GB_EDEVICE;                              \
    }

static void use_device(const gb_ctx *ctx) { GB_CUDA(cudaSetDevice(ctx->device)); }

// Systems run on their context's stream, so work the caller queued there comes first.  Every
// call that touches the stream holds the context's lock for its duration.
namespace {
struct Enter {
    std::lock_guard<std::recursive_mutex> g;
    explicit Enter(gb_ctx *ctx) : g(ctx->mu) { use_device(ctx); }
};
}  // namespace

extern "C" {

const char *gb_status_str(gb_status s) {
    switch (s) {
        case GB_OK: return "GB_OK";
        case GB_DONE: return "GB_DONE";
        case GB_EINVAL: return "GB_EINVAL";
        case GB_ENOMEM: return "GB_ENOMEM";
        case GB_EOVERFLOW: return "GB_EOVERFLOW";
        case GB_ETIMEOUT: return "GB_ETIMEOUT";
        case GB_EDEVICE: return "GB_EDEVICE";
        case GB_EUNSUPPORTED: return "GB_EUNSUPPORTED";
        case GB_EBUSY: return "GB_EBUSY";
    }
    return "unknown gb_status";
}

const char *gb_last_error(void) { return t_last_error.c_str(); }

uint64_t gb_kernel_launches(void) { return g_launches.load(); }

uint64_t gb_graph_launches(void) { return g_graph_launches.load(); }

gb_status gb_ctx_create(int device, const gb_ctx_opts *opts, gb_ctx **out) {
    GB_API_BEGIN
    if (!out) fail(GB_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    GB_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) fail(GB_EINVAL, "no such CUDA device");
    auto ctx = std::make_unique<gb_ctx>();
    ctx->device = device;
    GB_CUDA(cudaSetDevice(device));
    gb_ctx_opts o{};
    if (opts) o = *opts;
    ctx->flags = o.flags;
    if (o.stream) {
        ctx->stream = static_cast<cudaStream_t>(o.stream);
        ctx->own_stream = false;
    } else {
        GB_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    if (o.arena) {
        if (!o.arena_bytes) fail(GB_EINVAL, "arena given without arena_bytes");
        ctx->arena.init(o.arena, o.arena_bytes, false);
    } else {
        const size_t bytes = o.arena_bytes ? o.arena_bytes : (size_t(2) << 30);
        void *p = nullptr;
        GB_CUDA(cudaMalloc(&p, bytes));
        ctx->arena.init(p, bytes, true);
    }
    for (auto &e : ctx->ev) GB_CUDA(cudaEventCreate(&e));
    *out = ctx.release();
    return GB_OK;
    GB_API_END
}

gb_status gb_ctx_destroy(gb_ctx *ctx) {
    GB_API_BEGIN
    if (!ctx) return GB_EINVAL;
    use_device(ctx);
    cudaDeviceSynchronize();
    ctx->arena.release();
    if (ctx->stage) cudaFreeHost(ctx->stage);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->mm_ev) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
    delete ctx;
    return GB_OK;
    GB_API_END
}

gb_status gb_ctx_memory(const gb_ctx *ctx, size_t *used, size_t *capacity) {
    if (!ctx) return GB_EINVAL;
    if (used) *used = ctx->arena.used();
    if (capacity) *capacity = ctx->arena.capacity();
    return GB_OK;
}

gb_status gb_ctx_memory_peak(gb_ctx *ctx, size_t *peak, int reset) {
    if (!ctx || !peak) return GB_EINVAL;
    *peak = ctx->arena.peak();
    if (reset) ctx->arena.reset_peak();
    return GB_OK;
}

gb_status gb_system_create(gb_ctx *ctx, uint32_t nvars, uint32_t p, gb_order order,
                           const gb_polys *F, gb_system **out) {
    GB_API_BEGIN
    if (!ctx || !out) fail(GB_EINVAL, "null context or out");
    *out = nullptr;
    if (order != GB_GREVLEX && order != GB_DEGLEX) fail(GB_EINVAL, "unknown term order");
    if (F && F->npolys && (!F->poly_off || ((!F->exps || !F->coeffs) && F->poly_off[F->npolys])))
        fail(GB_EINVAL, "null arrays in the input system");
    // host work only: the input reaches the device with the system's first step
    auto S = std::make_unique<gb_system>();
    S->ctx = ctx;
    S->stream = ctx->stream;
    S->deglex = order == GB_DEGLEX;
    system_init(S.get(), nvars, p, F);
    *out = S.release();
    return GB_OK;
    GB_API_END
}

gb_status gb_system_destroy(gb_system *S) {
    GB_API_BEGIN
    if (!S) return GB_EINVAL;
    // The system's device blocks go to the arena's deferred list (no work that is still queued uses
    // them: a system is destroyed only when no step of it runs).  They are reclaimed at the
    // context's next synchronisation; done here at once unless another thread is using the
    // context, so a destroy never waits for a server's iteration.
    gb_ctx *ctx = S->ctx;
    delete S;
    std::unique_lock<std::recursive_mutex> lk(ctx->mu, std::try_to_lock);
    if (lk.owns_lock()) {
        GB_CUDA(cudaSetDevice(ctx->device));
        ctx_sync(ctx);
    }
    return GB_OK;
    GB_API_END
}

gb_status gb_symbolic_preprocess(gb_system *S, uint32_t r, const uint8_t *t_exps, const uint32_t *k,
                                 int closure, gb_macaulay **out) {
    GB_API_BEGIN
    if (!S || !out || (r && (!t_exps || !k))) fail(GB_EINVAL, "null argument");
    *out = nullptr;
    Enter entered(S->ctx);
    make_resident({S});
    std::vector<std::pair<Mono, uint32_t>> tk(r);
    for (uint32_t i = 0; i < r; ++i) {
        Mono t{};
        std::memcpy(t.e, t_exps + (size_t)i * S->n, S->n);
        tk[i] = {t, k[i]};
    }
    std::vector<SpTask> tasks(1);
    tasks[0].S = S;
    tasks[0].rows = order_rows(S, std::move(tk));
    tasks[0].closure = closure != 0;
    for (uint32_t g = 0; g < S->redundant.size(); ++g)
        if (!S->redundant[g]) tasks[0].nonred.push_back(g);
    symbolic_preprocess(tasks);
    *out = tasks[0].out.release();
    return GB_OK;
    GB_API_END
}

static void d2h(gb_system *S, void *dst, const void *src, size_t bytes) {
    if (bytes) GB_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, S->stream));
}

gb_status gb_macaulay_stats_get(const gb_macaulay *M, gb_macaulay_stats *out) {
    GB_API_BEGIN
    if (!M || !out) fail(GB_EINVAL, "null argument");
    *out = gb_macaulay_stats{};
    out->nrows = M->nrows;
    out->ndict = M->ndict;
    out->npivot = M->nA;
    out->closure_rounds = M->closure_rounds;
    out->nnz = M->nnz;
    out->ms_sp = M->ms_sp;
    out->ms_dict = M->ms_dict;
    out->ms_assemble = M->ms_sp - M->ms_dict;
    return GB_OK;
    GB_API_END
}

gb_status gb_macaulay_export(const gb_macaulay *M, gb_macaulay_host *h) {
    GB_API_BEGIN
    if (!M || !h) fail(GB_EINVAL, "null argument");
    gb_system *S = M->sys;
    Enter entered(S->ctx);
    h->nvars = M->n;
    h->nrows = M->nrows;
    h->ndict = M->ndict;
    h->npivot = M->nA;
    h->nnz = M->nnz;
    const uint32_t n = M->n;
    if (h->row_ptr) d2h(S, h->row_ptr, M->row_ptr.p, 4ull * (M->nrows + 1));
    if (h->col_ind) d2h(S, h->col_ind, M->col.p, 4ull * M->nnz);
    if (h->val) d2h(S, h->val, M->val.p, 4ull * M->nnz);
    if (h->row_k) d2h(S, h->row_k, M->row_k.p, 4ull * M->nrows);
    std::vector<uint4> dict, rt;
    std::vector<uint8_t> fl;
    if (h->dict_exps) { dict.resize(M->ndict); d2h(S, dict.data(), M->dict.p, 16ull * M->ndict); }
    if (h->row_t) { rt.resize(M->nrows); d2h(S, rt.data(), M->row_t.p, 16ull * M->nrows); }
    if (h->row_flags) { fl.resize(M->nrows); d2h(S, fl.data(), M->row_flags.p, M->nrows); }
    ctx_sync(S->ctx);
    for (uint32_t i = 0; h->dict_exps && i < M->ndict; ++i)
        std::memcpy(h->dict_exps + (size_t)i * n, &dict[i], n);
    for (uint32_t i = 0; h->row_t && i < M->nrows; ++i) std::memcpy(h->row_t + (size_t)i * n, &rt[i], n);
    for (uint32_t i = 0; h->row_flags && i < M->nrows; ++i) h->row_flags[i] = fl[i] & 3u;
    return GB_OK;
    GB_API_END
}

gb_status gb_macaulay_destroy(gb_macaulay *M) {
    GB_API_BEGIN
    if (!M) return GB_EINVAL;
    delete M;
    return GB_OK;
    GB_API_END
}

gb_status gb_reduce_macaulay(gb_macaulay *M, gb_echelon **out) {
    GB_API_BEGIN
    if (!M || !out) fail(GB_EINVAL, "null argument");
    *out = nullptr;
    Enter entered(M->sys->ctx);
    auto Es = reduce_rows({M}, true);
    *out = Es[0].release();
    return GB_OK;
    GB_API_END
}

gb_status gb_echelon_export(const gb_echelon *E, gb_echelon_host *h) {
    GB_API_BEGIN
    if (!E || !h) fail(GB_EINVAL, "null argument");
    gb_system *S = E->mac->sys;
    Enter entered(S->ctx);
    h->nC = E->nC;
    h->nb = E->nb;
    h->rank = E->rank;
    if (h->nonpiv) d2h(S, h->nonpiv, E->mac->nonpiv.p, 4ull * E->nb);
    if (h->dprime) d2h(S, h->dprime, E->dprime.p, 4ull * E->nC * E->nb);
    if (h->rref_piv) d2h(S, h->rref_piv, E->rpiv.p, 4ull * E->rank);
    if (h->rref) d2h(S, h->rref, E->rref.p, 4ull * E->rank * E->nb);
    ctx_sync(S->ctx);
    return GB_OK;
    GB_API_END
}

gb_status gb_echelon_destroy(gb_echelon *E) {
    GB_API_BEGIN
    if (!E) return GB_EINVAL;
    delete E;
    return GB_OK;
    GB_API_END
}

gb_status gb_f4_step(gb_system *S, gb_step_stats *stats) {
    GB_API_BEGIN
    if (!S) fail(GB_EINVAL, "null system");
    if (S->finished || S->pairs.empty()) return GB_DONE;
    Enter entered(S->ctx);
    std::vector<gb_step_stats> st;
    f4_steps({S}, &st);
    if (stats) *stats = st[0];
    return GB_OK;
    GB_API_END
}

gb_status gb_sig_filter(gb_ctx *ctx, uint32_t index, uint32_t e, uint32_t ncand, const uint32_t *forbidden,
                        uint64_t *keys, uint32_t *count) {
    GB_API_BEGIN
    if (!ctx || !count || (ncand && !keys)) fail(GB_EINVAL, "null argument");
    Enter entered(ctx);
    *count = sig_filter(ctx, index, e, ncand, forbidden, reinterpret_cast<unsigned long long *>(keys));
    return GB_OK;
    GB_API_END
}

gb_status gb_f5_groebner(gb_system *S, uint32_t dmax, uint32_t flags, gb_f5_block *blocks, uint32_t blocks_cap,
                         uint32_t *nblocks, gb_f5_stats *stats) {
    GB_API_BEGIN
    if (!S || (blocks_cap && !blocks)) fail(GB_EINVAL, "null argument");
    if (flags & ~GB_F5_NO_CRITERION) fail(GB_EINVAL, "unknown flags");
    Enter entered(S->ctx);
    std::vector<gb_f5_block> out;
    f5_groebner(S, dmax, flags, &out, stats);
    const size_t k = std::min<size_t>(out.size(), blocks_cap);
    if (k) std::memcpy(blocks, out.data(), k * sizeof(gb_f5_block));
    if (nblocks) *nblocks = (uint32_t)out.size();
    return GB_OK;
    GB_API_END
}

gb_status gb_groebner(gb_system *S, gb_run_stats *stats) {
    GB_API_BEGIN
    if (!S) fail(GB_EINVAL, "null system");
    Enter entered(S->ctx);
    groebner_batch({S});
    if (stats) *stats = S->run;
    return GB_OK;
    GB_API_END
}

gb_status gb_autotune(gb_ctx *ctx, uint32_t count, gb_system *const *systems, gb_tune_report *report) {
    GB_API_BEGIN
    if (!ctx || (count && !systems)) fail(GB_EINVAL, "null context or systems");
    Enter entered(ctx);
    autotune(ctx, std::vector<gb_system *>(systems, systems + count), report);
    return GB_OK;
    GB_API_END
}

gb_status gb_tune_save(const gb_ctx *ctx, const char *path) {
    GB_API_BEGIN
    if (!ctx || !path) fail(GB_EINVAL, "null context or path");
    tune_save(ctx, path);
    return GB_OK;
    GB_API_END
}

gb_status gb_tune_load(gb_ctx *ctx, const char *path) {
    GB_API_BEGIN
    if (!ctx || !path) fail(GB_EINVAL, "null context or path");
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    tune_load(ctx, path);
    return GB_OK;
    GB_API_END
}

gb_status gb_basis_export(const gb_system *S, int reduced, gb_polys_host *h) {
    GB_API_BEGIN
    if (!S || !h) fail(GB_EINVAL, "null argument");
    const uint32_t n = S->n;
    if (reduced) {
        if (!S->finished) fail(GB_EINVAL, "the reduced basis exists after gb_groebner");
        h->npolys = (uint32_t)S->fin_off.size() - 1;
        h->nterms = S->fin_terms;
        if (h->poly_off) std::memcpy(h->poly_off, S->fin_off.data(), 4 * S->fin_off.size());
        if ((h->exps || h->coeffs) && S->fin_terms) {
            // the terms stay on the device after gb_groebner: one copy into the caller's arrays
            Enter entered(S->ctx);
            cudaStream_t st = S->ctx->stream;
            if (h->exps)
                GB_CUDA(cudaMemcpyAsync(h->exps, S->fin_exps.p, (size_t)S->fin_terms * n, cudaMemcpyDeviceToHost, st));
            if (h->coeffs)
                GB_CUDA(cudaMemcpyAsync(h->coeffs, S->fin_cf.p, 4ull * S->fin_terms, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
        }
        return GB_OK;
    }
    gb_system *Sm = const_cast<gb_system *>(S);
    Enter entered(S->ctx);
    make_resident({Sm});
    const uint32_t ng = (uint32_t)S->lm.size();
    uint64_t T = 0;
    for (uint32_t l : S->len) T += l;
    h->npolys = ng;
    h->nterms = T;
    if (!h->poly_off && !h->exps && !h->coeffs) return GB_OK;
    std::vector<uint4> mon(S->nterms);
    std::vector<uint32_t> cf(S->nterms);
    d2h(Sm, mon.data(), S->bmon.p, 16ull * S->nterms);
    d2h(Sm, cf.data(), S->bcf.p, 4ull * S->nterms);
    ctx_sync(Sm->ctx);
    uint64_t o = 0;
    for (uint32_t g = 0; g < ng; ++g) {
        if (h->poly_off) h->poly_off[g] = (uint32_t)o;
        for (uint32_t j = 0; j < S->len[g]; ++j, ++o) {
            if (h->exps) std::memcpy(h->exps + o * n, &mon[S->off[g] + j], n);
            if (h->coeffs) h->coeffs[o] = cf[S->off[g] + j];
        }
    }
    if (h->poly_off) h->poly_off[ng] = (uint32_t)o;
    return GB_OK;
    GB_API_END
}

gb_status gb_basis_redundant(const gb_system *S, uint32_t *count, uint8_t *flags) {
    if (!S || !count) return GB_EINVAL;
    *count = (uint32_t)S->redundant.size();
    if (flags) std::memcpy(flags, S->redundant.data(), S->redundant.size());
    return GB_OK;
}

gb_status gb_reduce_rows_noalloc(uint32_t p, uint32_t ndict, uint32_t npivot, uint32_t nnonpivot,
                                 uint32_t nb, const uint32_t *row_ptr, const uint32_t *col_ind,
                                 const uint32_t *val, const uint32_t *pivot_cols,
                                 const uint32_t *nonpivot_cols, uint32_t *dprime, void *stream) {
    GB_API_BEGIN
    reduce_rows_noalloc(p, ndict, npivot, nnonpivot, nb, row_ptr, col_ind, val, pivot_cols, nonpivot_cols,
                        dprime, static_cast<cudaStream_t>(stream));
    return GB_OK;
    GB_API_END
}

gb_status gb_block_wiedemann(const gb_macaulay *mac, uint32_t b, const uint32_t *X, const uint32_t *Z,
                             const uint32_t *delta, uint32_t *seq, uint32_t *W, uint32_t wcap,
                             gb_krylov_stats *stats) {
    GB_API_BEGIN
    if (!mac || !mac->sys) fail(GB_EINVAL, "null matrix handle");
    gb_ctx *ctx = mac->sys->ctx;
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    use_device(ctx);
    block_wiedemann(mac, b, X, Z, delta, seq, W, wcap, stats);
    return GB_OK;
    GB_API_END
}

gb_status gb_modp_apply(gb_modp_op op, uint32_t p, uint64_t n, uint32_t window, const uint32_t *a,
                        const uint32_t *b, const uint32_t *c, uint32_t *out, void *stream) {
    GB_API_BEGIN
    modp_apply((int)op, p, n, window, a, b, c, out, static_cast<cudaStream_t>(stream));
    return GB_OK;
    GB_API_END
}

gb_status gb_pair_update_replay(uint32_t n, uint32_t nelem, const uint8_t *lms, uint32_t ngroups,
                                const uint32_t *group_sizes, const uint8_t *select_before, uint32_t cap,
                                uint32_t *pairs, uint32_t *npairs, uint8_t *in_basis) {
    GB_API_BEGIN
    if (!n || n > 16) fail(GB_EINVAL, "n must be 1..16");
    if ((nelem && (!lms || !in_basis)) || (ngroups && !group_sizes) || !npairs || (cap && !pairs))
        fail(GB_EINVAL, "null pointer");
    uint64_t total = 0;
    for (uint32_t g = 0; g < ngroups; ++g) total += group_sizes[g];
    if (total != nelem) fail(GB_EINVAL, "group sizes do not add up to nelem");
    gb_system S;
    S.n = n;
    uint32_t e = 0;
    for (uint32_t g = 0; g < ngroups; ++g) {
        if (select_before && select_before[g] && !S.pairs.empty()) {  // the normal strategy
            uint32_t d = UINT32_MAX;
            for (const PairL &q : S.pairs) d = std::min(d, q.deg);
            size_t w = 0;
            for (const PairL &q : S.pairs)
                if (q.deg != d) S.pairs[w++] = q;
            S.pairs.resize(w);
        }
        const uint32_t h0 = e;
        for (uint32_t k = 0; k < group_sizes[g]; ++k, ++e) {
            Mono m{};
            std::memcpy(m.e, lms + (size_t)e * n, n);
            push_lm(&S, m);
        }
        if (e > h0) update_pairs_host(&S, h0);
    }
    *npairs = (uint32_t)S.pairs.size();
    if (S.pairs.size() > cap) fail(GB_EINVAL, "more pairs than cap (npairs holds the count)");
    for (size_t q = 0; q < S.pairs.size(); ++q) {
        pairs[2 * q] = std::min(S.pairs[q].i, S.pairs[q].j);
        pairs[2 * q + 1] = std::max(S.pairs[q].i, S.pairs[q].j);
    }
    for (uint32_t k = 0; k < nelem; ++k) in_basis[k] = S.redundant[k] ? 0 : 1;
    return GB_OK;
    GB_API_END
}

gb_status gb_matmul_modp(gb_ctx *ctx, uint32_t p, uint32_t m, uint32_t n, uint32_t k, const uint32_t *A,
                         uint64_t lda, const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc,
                         int subtract) {
    GB_API_BEGIN
    if (!ctx) fail(GB_EINVAL, "null context");
    if (p < 3 || p >= (1u << 31) || !is_prime32(p)) fail(GB_EINVAL, "p must be an odd prime below 2^31");
    if (!m || !n) return GB_OK;
    if (!C || (k && (!A || !B))) fail(GB_EINVAL, "null device pointer");
    if (lda < k || ldb < n || ldc < n) fail(GB_EINVAL, "row pitch below the matrix width");
    if (!k) return GB_OK;
    Enter entered(ctx);
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    DBuf<uint32_t> err;
    err.alloc(ar, 1, st);
    GB_CUDA(cudaMemsetAsync(err.p, 0, 4, st));
    matmul_dev(ar, make_fp(p), m, n, k, A, lda, B, ldb, C, ldc, subtract != 0, err.p, st);
    uint32_t *h = static_cast<uint32_t *>(ctx_pinned(ctx, 16));
    GB_CUDA(cudaMemcpyAsync(h, err.p, 4, cudaMemcpyDeviceToHost, st));
    ctx_sync(ctx);
    if (*h) fail(GB_ETIMEOUT, "gb_matmul_modp: a bounded wait in the tensor-core kernel gave up");
    return GB_OK;
    GB_API_END
}

gb_status gb_system_last_step(const gb_system *S, const gb_macaulay **mac, const gb_echelon **ech) {
    if (!S) return GB_EINVAL;
    if (!S->last_mac || !S->last_ech) {
        set_last_error("no step kept: create the context with GB_CTX_KEEP_STEP and run a step");
        return GB_EINVAL;
    }
    if (mac) *mac = S->last_mac.get();
    if (ech) *ech = S->last_ech.get();
    return GB_OK;
}

}  // extern "C"
