// tune.cpp -- the autotuner of the reduction schedules.
//
// The reduction of a Macaulay matrix (Sec. 9.2) has schedules with identical results: the sparse
// row-by-row reduction against the dense blocked elimination on the tensor cores, and for
// RREF(D') the panel updates on CUDA cores with host-launched rounds, the same rounds as one CUDA
// graph, or tensor-core panel updates inside the graph.  Which one is fastest depends on the
// matrix shape and the device, so the tuner measures: it runs copies of the caller's systems to
// completion once per candidate, reads each step's device times (the CUDA events of the step
// statistics), and keeps per shape bucket the schedule with the least total time.  Every run
// builds the same matrices, step for step, because the F4 trajectory does not depend on how a
// matrix is reduced.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <sstream>

#include "internal.hpp"

namespace gb {

void f4_steps(const std::vector<gb_system *> &Ss, std::vector<gb_step_stats> *stats);
gb_system *system_clone_fresh(const gb_system *S);
void ctx_sync(gb_ctx *ctx);

uint64_t tune_key(uint32_t kind, uint32_t p, uint32_t a, uint32_t b, uint32_t c) {
    auto lg = [](uint32_t x) -> uint64_t { return 63u - (uint64_t)__builtin_clzll((uint64_t)x + 1u); };
    return ((uint64_t)kind << 40) | ((uint64_t)(p >= 65536u) << 32) | (lg(a) << 16) | (lg(b) << 8) | lg(c);
}

namespace {

// the candidate runs: (reduction schedule, RREF schedule); the sparse reduction runs twice, and
// each bucket keeps the smaller of its two times, which damps one-off noise on that side
struct Run {
    int reduce, rref;
};
constexpr Run RUNS[3] = {{0, 0}, {1, 2}, {0, 1}};

struct ForceGuard {
    gb_ctx *ctx;
    ~ForceGuard() {
        ctx->tune.force_reduce = -1;
        ctx->tune.force_rref = -1;
    }
};

// The prefix-sum tile per size bucket: each candidate timed on device arrays of n = 2^b values
// (b = 8..24; a scan's cost depends on n only), best of three launches after a warm-up.
void tune_scans(gb_ctx *ctx) {
    constexpr int B0 = 8, B1 = 24;
    constexpr int ITEMS[3] = {4, 8, 16};
    cudaStream_t st = ctx->stream;
    DBuf<uint32_t> in, out;
    in.alloc(ctx->arena, (size_t(1) << B1) + 1, st);
    out.alloc(ctx->arena, (size_t(1) << B1) + 1, st);
    GB_CUDA(cudaMemsetAsync(in.p, 1, 4ull << B1, st));
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    for (int b = B0; b <= B1; ++b) {
        const size_t n = size_t(1) << b;
        TuneEntry e;
        for (int c = 0; c < 3; ++c) {
            float best = 1e30f;
            for (int r = 0; r < 4; ++r) {
                GB_CUDA(cudaEventRecord(e0, st));
                exclusive_scan_items(ctx, ITEMS[c], in.p, out.p, n, st);
                GB_CUDA(cudaEventRecord(e1, st));
                GB_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (r) best = std::min(best, ms);
                ctx_sync(ctx);  // the scan's tile buffers are free again
            }
            e.ms[c] = best;
            if (best < e.ms[e.choice]) e.choice = (uint8_t)c;
        }
        ctx->tune.table[tune_key(TUNE_SCAN, 0, (uint32_t)n, 0, 0)] = e;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

}  // namespace

void autotune(gb_ctx *ctx, const std::vector<gb_system *> &Ss, gb_tune_report *rep) {
    for (const gb_system *S : Ss) {
        if (!S || S->ctx != ctx) fail(GB_EINVAL, "gb_autotune: a system is null or belongs to another context");
        if (S->steps || S->resident) fail(GB_EINVAL, "gb_autotune: a system has already run a step");
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::map<uint64_t, std::array<double, 3>> red, rr;  // per run / per RREF schedule, ms
    uint32_t steps = 0;
    {
        ForceGuard guard{ctx};
        for (int r = 0; r < 3; ++r) {
            ctx->tune.force_reduce = RUNS[r].reduce;
            ctx->tune.force_rref = RUNS[r].rref;
            for (const gb_system *S : Ss) {
                std::unique_ptr<gb_system> C(system_clone_fresh(S));
                while (!C->finished && !C->pairs.empty()) {
                    std::vector<gb_step_stats> st;
                    f4_steps({C.get()}, &st);
                    const gb_step_stats &s = st[0];
                    ++steps;
                    if (!s.nC || !s.nb) continue;
                    auto &a = red.try_emplace(tune_key(TUNE_REDUCE, C->p, s.npivot, s.nC, s.nb),
                                              std::array<double, 3>{0, 0, 0}).first->second;
                    a[r] += s.ms_reduce;
                    auto &b = rr.try_emplace(tune_key(TUNE_RREF, C->p, s.nC, s.nb, 0),
                                             std::array<double, 3>{0, 0, 0}).first->second;
                    b[RUNS[r].rref] += s.ms_rref;
                }
                C.reset();
                ctx_sync(ctx);  // the copy's device blocks are free again
            }
        }
    }
    for (const auto &kv : red) {
        TuneEntry e;
        const double sparse = std::min(kv.second[0], kv.second[2]), dense = kv.second[1];
        e.ms[0] = (float)sparse;
        e.ms[1] = (float)dense;
        e.choice = dense < sparse ? 1 : 0;
        ctx->tune.table[kv.first] = e;
    }
    tune_scans(ctx);
    for (const auto &kv : rr) {
        TuneEntry e;
        for (int i = 0; i < 3; ++i) e.ms[i] = (float)kv.second[i];
        e.choice = 0;
        for (int i = 1; i < 3; ++i)
            if (kv.second[i] < kv.second[e.choice]) e.choice = (uint8_t)i;
        ctx->tune.table[kv.first] = e;
    }
    if (rep) {
        *rep = gb_tune_report{};
        rep->runs = 3;
        rep->steps = steps;
        for (const auto &kv : ctx->tune.table) {
            if ((kv.first >> 40) == TUNE_REDUCE) {
                ++rep->buckets_reduce;
                rep->dense_buckets += kv.second.choice == 1;
            } else if ((kv.first >> 40) == TUNE_RREF) {
                ++rep->buckets_rref;
            } else {
                ++rep->buckets_scan;
            }
        }
        rep->ms_wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
}

// One line per bucket: kind prime_class lg_a lg_b lg_c choice ms_0 ms_1 ms_2
void tune_save(const gb_ctx *ctx, const char *path) {
    std::ofstream f(path);
    if (!f) fail(GB_EINVAL, std::string("gb_tune_save: cannot open ") + path);
    cudaDeviceProp prop{};
    GB_CUDA(cudaGetDeviceProperties(&prop, ctx->device));
    f << "# reduction schedule table, measured on " << prop.name << " (" << prop.multiProcessorCount
      << " SMs)\n"
      << "# kind prime(0: p < 2^16, 1: p < 2^31) lg_a lg_b lg_c choice ms_0 ms_1 ms_2\n"
      << "# lg_x = floor(log2(x + 1)); reduce: a pivots, b non-pivot rows, c non-pivot columns,\n"
      << "#   choice 0 sparse, 1 dense (tensor cores); rref: a rows, b columns of D',\n"
      << "#   choice 0 CUDA cores + host rounds, 1 CUDA cores + graph, 2 tensor cores + graph;\n"
      << "#   scan: a values, choice 0, 1, 2 = tiles of 4, 8, 16 values per thread\n";
    char line[160];
    for (const auto &kv : ctx->tune.table) {
        const uint64_t k = kv.first;
        const TuneEntry &e = kv.second;
        const uint64_t kind = k >> 40;
        std::snprintf(line, sizeof line, "%s %u %u %u %u %u %.4f %.4f %.4f\n",
                      kind == TUNE_REDUCE ? "reduce" : kind == TUNE_RREF ? "rref" : "scan", (unsigned)((k >> 32) & 0xFF),
                      (unsigned)((k >> 16) & 0xFF), (unsigned)((k >> 8) & 0xFF), (unsigned)(k & 0xFF),
                      (unsigned)e.choice, e.ms[0], e.ms[1], e.ms[2]);
        f << line;
    }
    if (!f) fail(GB_EINVAL, std::string("gb_tune_save: write failed on ") + path);
}

void tune_load(gb_ctx *ctx, const char *path) {
    std::ifstream f(path);
    if (!f) fail(GB_EINVAL, std::string("gb_tune_load: cannot open ") + path);
    std::map<uint64_t, TuneEntry> add;
    std::string line;
    int no = 0;
    while (std::getline(f, line)) {
        ++no;
        if (line.empty() || line[0] == '#') continue;
        std::istringstream in(line);
        std::string kind;
        unsigned cls, a, b, c, choice;
        float ms[3];
        if (!(in >> kind >> cls >> a >> b >> c >> choice >> ms[0] >> ms[1] >> ms[2]))
            fail(GB_EINVAL, "gb_tune_load: malformed line " + std::to_string(no));
        std::string rest;
        const bool red = kind == "reduce", scan = kind == "scan";
        if ((!red && !scan && kind != "rref") || (in >> rest) || cls > 1 || a > 32 || b > 32 || c > 32 ||
            choice > (red ? 1u : 2u) || (!red && c != 0) || (scan && (b != 0 || cls != 0)))
            fail(GB_EINVAL, "gb_tune_load: malformed line " + std::to_string(no));
        TuneEntry e;
        e.choice = (uint8_t)choice;
        for (int i = 0; i < 3; ++i) e.ms[i] = ms[i];
        const uint64_t key = ((uint64_t)(red ? TUNE_REDUCE : scan ? TUNE_SCAN : TUNE_RREF) << 40) | ((uint64_t)cls << 32) |
                             ((uint64_t)a << 16) | ((uint64_t)b << 8) | c;
        add[key] = e;
    }
    for (const auto &kv : add) ctx->tune.table[kv.first] = kv.second;
}

}  // namespace gb
