// internal.hpp -- host-side structures of the library behind include/gb.h.
#pragma once
#include <cuda_runtime.h>

#if defined(__SSE2__)
#include <emmintrin.h>
#endif
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gb.h"
#include "device.cuh"

namespace gb {

// ---- errors ---------------------------------------------------------------------------------
struct Error : std::runtime_error {
    gb_status st;
    Error(gb_status s, const std::string &m) : std::runtime_error(m), st(s) {}
};
[[noreturn]] void fail(gb_status s, const std::string &msg);
void cuda_check(cudaError_t e, const char *what);
#define GB_CUDA(x) ::gb::cuda_check((x), #x)
void set_last_error(const std::string &msg);

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum, once per kernel and
// device.  The limit is a per-kernel attribute shared by every thread of the process, so it is
// only ever raised: a thread lowering it while another launches with more would fail the launch.
void opt_in_smem(const void *kernel);

// every kernel launch site calls counted() right after its <<<...>>>.  While this thread records
// a CUDA graph (t_capturing), the launches only become graph nodes: they are tallied in
// t_captured, and the code that launches the graph counts them once per execution.
extern std::atomic<unsigned long long> g_launches;
extern std::atomic<unsigned long long> g_graph_launches;
extern thread_local bool t_capturing;
extern thread_local unsigned t_captured;
inline void counted(unsigned k = 1) {
    if (t_capturing) t_captured += k;
    else g_launches.fetch_add(k, std::memory_order_relaxed);
    GB_CUDA(cudaGetLastError());
}

// ---- device memory: a first-fit arena over one device allocation ------------------------------
// The arena is either caller-owned device memory (for instance a torch tensor) or one cudaMalloc
// made when the context is created.  Blocks are 256-byte aligned.  Thread-safe.
// A block is only ever used by work on the stream that allocated it.  Freeing is deferred: a
// block freed on stream s becomes reusable after flush(s), which callers invoke right after
// synchronising s, so no kernel still queued on s can touch a block handed out again.
class Arena {
  public:
    void init(void *base, size_t bytes, bool owned);
    void release();
    void *alloc(size_t bytes);  // throws Error(GB_ENOMEM)
    void defer_free(void *p, cudaStream_t s);
    void flush(cudaStream_t s);  // s has been synchronised: its deferred blocks are free again
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }
    size_t peak() const { return peak_; }
    void reset_peak() {
        std::lock_guard<std::mutex> g(mu_);
        peak_ = used_;
    }

  private:
    void free_locked(size_t off);
    char *base_ = nullptr;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
    bool owned_ = false;
    std::map<size_t, size_t> free_;  // offset -> size
    std::map<size_t, size_t> live_;  // offset -> size
    std::multimap<cudaStream_t, size_t> pending_;
    std::mutex mu_;
};

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    Arena *a = nullptr;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept { *this = std::move(o); }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            reset();
            p = o.p; n = o.n; a = o.a; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { reset(); }
    void alloc(Arena &ar, size_t count, cudaStream_t stream) {
        reset();
        a = &ar;
        s = stream;
        n = count;
        p = static_cast<T *>(ar.alloc(sizeof(T) * (count ? count : 1)));
    }
    // grow to at least `count` elements, keeping the first `keep` elements (stream-ordered copy)
    void grow(Arena &ar, size_t count, size_t keep, cudaStream_t stream) {
        if (count <= n && p) return;
        DBuf<T> nb;
        nb.alloc(ar, count, stream);
        if (keep && p)
            GB_CUDA(cudaMemcpyAsync(nb.p, p, sizeof(T) * keep, cudaMemcpyDeviceToDevice, stream));
        *this = std::move(nb);
    }
    void reset() {
        if (p && a) a->defer_free(p, s);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return sizeof(T) * n; }
};

// ---- host monomials (same packing as the device: byte i = exponent of x_{i+1}) ---------------
struct Mono {
    uint8_t e[16];
};
inline bool operator==(const Mono &a, const Mono &b) { return std::memcmp(a.e, b.e, 16) == 0; }
int mono_deg(const Mono &a, int n);
int mono_cmp(const Mono &a, const Mono &b, int n, bool deglex = false);  // +1 a > b, -1 a < b, 0 equal
Mono mono_mul(const Mono &a, const Mono &b, int n);
Mono mono_div(const Mono &b, const Mono &a, int n);
Mono mono_lcm(const Mono &a, const Mono &b, int n);
bool mono_divides(const Mono &a, const Mono &b, int n);
bool mono_coprime(const Mono &a, const Mono &b, int n);
inline uint4 to_u4(const Mono &m) {
    uint4 r;
    std::memcpy(&r, m.e, 16);
    return r;
}

Fp make_fp(uint32_t p);
uint32_t host_inv(uint32_t a, uint32_t p);
bool is_prime32(uint32_t q);

// ---- rows handed to symbolic preprocessing -------------------------------------------------
struct RowSpec {
    Mono t;
    uint32_t k;
    uint8_t pivot;  // chosen pivot among given rows sharing a leading monomial
    uint8_t skip;   // 1: the first term of g_k is left out (tail rows of the final reduction)
};

struct Pair {
    uint32_t i, j;
};

// Monomials as two 64-bit words of eight 8-bit exponents.  While every exponent is below 128,
// bytewise comparisons run without carries between bytes (SWAR):
//   (b | H) - a has the high bit of byte i set  iff  b_i >= a_i   (no borrow leaves a byte)
struct M16 {
    uint64_t lo, hi;
};
inline M16 m16(const Mono &m) {
    M16 r;
    std::memcpy(&r, m.e, 16);
    return r;
}
inline bool operator==(const M16 &a, const M16 &b) { return a.lo == b.lo && a.hi == b.hi; }
constexpr uint64_t SWAR_H = 0x8080808080808080ull, SWAR_L = 0x7F7F7F7F7F7F7F7Full;
#if defined(__SSE2__)
// byte-wise monomial tests with SSE2 (every x86-64 host has it): one vector per monomial
inline __m128i v16(const M16 &a) { return _mm_set_epi64x((long long)a.hi, (long long)a.lo); }
inline bool divides16(const M16 &a, const M16 &b) {  // a | b: every byte of a at most b's
    const __m128i x = v16(a), y = v16(b);
    return _mm_movemask_epi8(_mm_cmpeq_epi8(_mm_max_epu8(x, y), y)) == 0xFFFF;
}
inline M16 lcm16(const M16 &a, const M16 &b) {
    const __m128i m = _mm_max_epu8(v16(a), v16(b));
    M16 r;
    _mm_storeu_si128(reinterpret_cast<__m128i *>(&r), m);
    return r;
}
inline bool coprime16(const M16 &a, const M16 &b) {
    return _mm_movemask_epi8(_mm_cmpeq_epi8(_mm_min_epu8(v16(a), v16(b)), _mm_setzero_si128())) == 0xFFFF;
}
inline uint32_t deg16(const M16 &a) {
    const __m128i s = _mm_sad_epu8(v16(a), _mm_setzero_si128());  // two 64-bit byte sums
    return (uint32_t)(_mm_cvtsi128_si64(s) + _mm_cvtsi128_si64(_mm_unpackhi_epi64(s, s)));
}
#else
// the same with 64-bit SWAR words (exponents below 128)
inline bool ge_all(uint64_t b, uint64_t a) { return (((b | SWAR_H) - a) & SWAR_H) == SWAR_H; }
inline bool divides16(const M16 &a, const M16 &b) { return ge_all(b.lo, a.lo) && ge_all(b.hi, a.hi); }
inline uint64_t max8(uint64_t a, uint64_t b) {
    const uint64_t ge = ((a | SWAR_H) - b) & SWAR_H;  // bytes where a >= b
    const uint64_t mask = (ge >> 7) * 0xFFull;
    return (a & mask) | (b & ~mask);
}
inline M16 lcm16(const M16 &a, const M16 &b) { return M16{max8(a.lo, b.lo), max8(a.hi, b.hi)}; }
inline uint64_t nonzero8(uint64_t x) { return (((x & SWAR_L) + SWAR_L) | x) & SWAR_H; }
inline bool coprime16(const M16 &a, const M16 &b) {
    return !(nonzero8(a.lo) & nonzero8(b.lo)) && !(nonzero8(a.hi) & nonzero8(b.hi));
}
inline uint32_t deg16(const M16 &a) {
    uint64_t s = (a.lo & 0x00FF00FF00FF00FFull) + ((a.lo >> 8) & 0x00FF00FF00FF00FFull) +
                 (a.hi & 0x00FF00FF00FF00FFull) + ((a.hi >> 8) & 0x00FF00FF00FF00FFull);
    s = (s & 0x0000FFFF0000FFFFull) + ((s >> 16) & 0x0000FFFF0000FFFFull);
    return (uint32_t)((s & 0xFFFFFFFFull) + (s >> 32));
}
#endif

struct PairL {  // a critical pair with its lcm cached
    uint32_t i, j, deg, pad;
    M16 lcm;
};

}  // namespace gb

// ---- handles ---------------------------------------------------------------------------------
namespace gb {
struct HostPool;

// Autotuning of the interchangeable schedules of the reduction (tune.cpp).  All of them give the
// same D' and RREF(D'):
//   reduction (TUNE_REDUCE): 0 sparse row-by-row, 1 dense blocked elimination on the tensor cores;
//   RREF (TUNE_RREF): 0 panel updates on CUDA cores, rounds launched from the host;
//                     1 the same rounds as one CUDA graph with the loop on the device;
//                     2 panel updates on the tensor cores, rounds as one graph;
//   prefix sums (TUNE_SCAN, bucket floor(log2(n + 1))): 0, 1, 2 = 4, 8, 16 values per thread.
constexpr uint32_t TUNE_REDUCE = 0, TUNE_RREF = 1, TUNE_SCAN = 2;
struct TuneEntry {
    uint8_t choice = 0;
    float ms[3] = {-1.f, -1.f, -1.f};  // measured total per schedule, -1 where not measured
};
struct TuneState {
    int force_reduce = -1, force_rref = -1;  // >= 0: every matrix takes this schedule (tuning runs)
    std::map<uint64_t, TuneEntry> table;     // bucket key -> the fastest schedule measured
};
// bucket of a shape: the kind, the prime's class (below 2^16 or not) and floor(log2(x + 1)) of
// up to three sizes (reduction: pivots, non-pivot rows, non-pivot columns; RREF: rows, columns)
uint64_t tune_key(uint32_t kind, uint32_t p, uint32_t a, uint32_t b, uint32_t c);
}

struct gb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;  // every system of the context runs on this stream
    bool own_stream = false;
    cudaStream_t capture = nullptr;  // private stream that CUDA graphs are recorded on (lazily created)
    uint32_t flags = 0;
    gb::Arena arena;
    cudaEvent_t ev[8] = {};         // stage timing of the batch in flight
    std::vector<cudaEvent_t> mm_ev; // pairs around the tensor-core launches of one reduction
    void *stage = nullptr;          // page-locked staging of the batch in flight
    size_t stage_bytes = 0;
    size_t stage_off = 0;           // bump offset, back to 0 at every ctx_sync
    // host worker threads for per-system host control of a batch (pair updates, selection)
    std::unique_ptr<gb::HostPool> pool;
    // held by every call that queues work on the stream or uses the staging area, so that a
    // server's scheduler thread and the caller's own calls on the same context do not interleave
    std::recursive_mutex mu;
    gb::TuneState tune;
    gb_ctx();
    ~gb_ctx();
};

// The materialised plan Pi of one batch (Def. 5.2) on the device.
struct gb_macaulay {
    gb_system *sys = nullptr;
    uint32_t n = 0, degree = 0, nrows = 0, ndict = 0, nA = 0, nC = 0, nb = 0;
    uint32_t closure_rounds = 0;
    uint32_t sp_redo = 0;  // symbolic preprocessing ran again (hash table growth or a key clash)
    uint64_t nnz = 0;
    gb::DBuf<uint32_t> row_ptr, col, val;  // CSR, val in [0, p)
    gb::DBuf<uint4> dict;                  // descending monomials
    gb::DBuf<uint4> row_t;
    gb::DBuf<uint32_t> row_k;
    gb::DBuf<uint8_t> row_flags;           // bit0 pivot, bit1 reducer, bit2 tail row
    gb::DBuf<uint32_t> pcols;              // nA pivot columns ascending (pivot row i has lm pcols[i])
    gb::DBuf<uint32_t> nonpiv;             // nb non-pivot columns ascending
    gb::DBuf<uint32_t> colpos;             // ndict: pivot index | 0x80000000 for a pivot column,
                                           // else the position among the non-pivot columns
    float ms_sp = 0.f;
    float ms_dict = 0.f;  // of ms_sp: up to the finished dictionary (expansion, closure, ranks, emit)
};

// D' and RREF(D') on the device.
struct gb_echelon {
    gb_macaulay *mac = nullptr;
    uint32_t nC = 0, nb = 0, rank = 0;
    gb::DBuf<uint32_t> dprime;  // nC x nb
    gb::DBuf<uint32_t> rref;    // rank x nb, rows in pivot order
    gb::DBuf<uint32_t> rpiv;    // rank pivot positions (ascending)
    uint64_t work[2] = {0, 0};  // pivot-row applications, mod-p multiply-adds of the reduction
    float ms_reduce = 0.f, ms_rref = 0.f, ms_reduce_kernel = 0.f;
    double ms_mm = 0.0, mm_flops = 0.0;  // tensor-core product launches (MmTimer)
    uint64_t mm_launches = 0;
    uint32_t sketched = 0;  // RREF(D') from a random sketch of D' (checked exactly)
};

struct gb_system {
    gb_ctx *ctx = nullptr;
    uint32_t n = 0, p = 0;
    gb::Fp fp{};
    cudaStream_t stream = nullptr;  // the context's stream
    // host mirror of the basis metadata
    std::vector<gb::Mono> lm;
    std::vector<uint32_t> off, len;
    std::vector<uint8_t> redundant;
    std::vector<gb::PairL> pairs;
    std::vector<gb::M16> lm16;     // leading monomials, SWAR form
    bool swar = true;              // every exponent so far below 128
    bool deglex = false;           // term order: deglex, else grevlex
    // device basis: terms of element k are [off[k], off[k] + len[k]) of bmon / bcf
    gb::DBuf<uint4> bmon;
    gb::DBuf<unsigned long long> bkey;  // mono_key of every basis term (the hash dictionary's keys)
    gb::DBuf<uint32_t> bcf;
    gb::DBuf<uint32_t> boff, blen;
    uint64_t nterms = 0;
    uint32_t last_ndict = 0;  // dictionary size of the last step (sizes the next hash table)
    // the normalised input until its upload with the first step (SWAR monomials, coefficients)
    bool resident = false;
    std::vector<uint4> in_mon;
    std::vector<uint32_t> in_cf;
    // kept objects of the last step (GB_CTX_KEEP_STEP)
    std::unique_ptr<gb_macaulay> last_mac;
    std::unique_ptr<gb_echelon> last_ech;
    // progress
    uint32_t steps = 0;
    bool unit = false;       // a constant input or element: the ideal is R
    bool finished = false;
    gb_run_stats run{};
    // the reduced basis after gb_groebner: element offsets on the host, the terms on the device
    // (read by gb_basis_export straight into the caller's arrays)
    std::vector<uint32_t> fin_off;
    gb::DBuf<uint8_t> fin_exps;  // fin_terms x n exponent bytes
    gb::DBuf<uint32_t> fin_cf;   // fin_terms coefficients
    uint64_t fin_terms = 0;
    // estimate of the device footprint (server admission)
    size_t footprint = 0;
};

namespace gb {

// many small host arrays staged for one host-to-device copy through the context's pinned area
struct Stage {
    std::vector<char> h;
    size_t put(const void *src, size_t bytes) {
        const size_t at = (h.size() + 15) & ~size_t(15);
        h.resize(at + bytes);
        if (bytes && src) std::memcpy(h.data() + at, src, bytes);
        return at;
    }
    // stream-ordered copy into a new device block d (no synchronisation)
    void upload(gb_ctx *ctx, DBuf<char> &d);
};

// prefix table of per-job block counts appended to a stage; returns the total
inline uint32_t plan(Stage &sg, const std::vector<uint32_t> &per_job, size_t &at) {
    std::vector<uint32_t> pre(per_job.size() + 1, 0);
    for (size_t j = 0; j < per_job.size(); ++j) pre[j + 1] = pre[j] + per_job[j];
    at = sg.put(pre.data(), 4 * pre.size());
    return pre.back();
}

// one job of symbolic preprocessing: the rows of one system's batch
struct SpTask {
    gb_system *S = nullptr;
    std::vector<RowSpec> rows;
    bool closure = true;
    std::vector<uint32_t> nonred;  // non-redundant basis indices, ascending
    uint64_t cap = 0;              // frontier capacity (0: estimate)
    uint64_t hcap = 0;             // hash-dictionary slots, a power of two (0: estimate)
    bool ranks = false;            // dense-rank bitmap for every term instead of the hash dictionary
    std::unique_ptr<gb_macaulay> out;
};
// mono_key of n basis terms (after an upload of input terms)
void basis_keys(const uint4 *mon, unsigned long long *key, uint64_t n, cudaStream_t st);

// pipeline stages for many systems of one context at once (sp.cu, reduce.cu)
void symbolic_preprocess(std::vector<SpTask> &tasks);
std::vector<std::unique_ptr<gb_echelon>> reduce_rows(const std::vector<gb_macaulay *> &Ms, bool echelon);
// RREF of each dense matrix Es[j]->dprime (nC x nb) into Es[j]->rank / rref / rpiv (reduce.cu);
// bounded waits of the tensor-core updates that give up are flagged in derr
void echelon_stage(gb_ctx *ctx, const std::vector<gb_echelon *> &Es, const std::vector<Fp> &fps, uint32_t *derr);
// the block Wiedemann path of gb_block_wiedemann (krylov.cu)
void block_wiedemann(const gb_macaulay *mac, uint32_t b, const uint32_t *X, const uint32_t *Z, const uint32_t *delta,
                     uint32_t *seq, uint32_t *W, uint32_t wcap, gb_krylov_stats *stats);
// host side of the F4 driver (f4.cpp): a new leading monomial in the host mirrors; rows (t, k) in
// pivot order; the inputs of fresh systems onto the device; the reduced basis of finished systems
void push_lm(gb_system *S, const Mono &m);
// the Gebauer-Moeller update of S's pairs for its elements h0 .. lm.size() - 1, all at once (f4.cpp)
void update_pairs_host(gb_system *S, uint32_t h0);
std::vector<RowSpec> order_rows(const gb_system *S, std::vector<std::pair<Mono, uint32_t>> tk);
void make_resident(const std::vector<gb_system *> &Ss);
void finish_batch(const std::vector<gb_system *> &Ss);
// the F5 criterion over one block of candidates (sig.cu): the admissible candidates' packed keys,
// compacted into keys (device); returns their number
uint32_t sig_filter(gb_ctx *ctx, uint32_t index, uint32_t e, uint32_t ncand, const uint32_t *forbidden,
                    unsigned long long *keys);
// gb_f5_groebner (f5.cpp)
void f5_groebner(gb_system *S, uint32_t dmax, uint32_t flags, std::vector<gb_f5_block> *blocks, gb_f5_stats *stats);
// append each job's echelon rows as new basis elements on the device; returns their LMs
void append_echelon(const std::vector<gb_echelon *> &Es, std::vector<std::vector<Mono>> &lms);
// final reduction: element elems[j][i] of job j becomes LM + row i of its D' (writes fin_*)
void replace_tails(const std::vector<gb_echelon *> &Es, const std::vector<std::vector<uint32_t>> &elems);
// a region of the context's page-locked staging area, valid until the next ctx_sync
void *ctx_pinned(gb_ctx *ctx, size_t bytes);
void ctx_sync(gb_ctx *ctx);
bool trace_on();  // GB_TRACE set in the environment: stage timings on stderr                     // synchronise the stream, release deferred blocks
// run fn(i) for i in [0, n) on the context's host workers and the calling thread
void parallel_for(gb_ctx *ctx, size_t n, const std::function<void(size_t)> &fn);
// exclusive scan of n u32 values on the stream; out has n + 1 entries (out[n] = total)
void exclusive_scan(gb_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s);
// the same with a given tile (ITEMS = 4, 8 or 16 values per thread), for the autotuner
void exclusive_scan_items(gb_ctx *ctx, int items, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s);

// ---- exact dense update over F_p on the tensor cores (mm.cu) --------------------------------
// Digit planes of a matrix: [L][rows][kpad] BF16 bit patterns of the balanced base-256 digits of
// its residues (L = 2 for p < 2^16, 4 for p < 2^31), K-major: row r holds the K values of one
// row of A, or of one column of B (B^T).
struct DigitPlanes {
    uint32_t L = 0;
    uint64_t rows = 0, K = 0, kpad = 0;
    uint16_t *p = nullptr;
    DBuf<uint16_t> buf;
    void alloc(Arena &ar, uint32_t L, uint64_t rows, uint64_t K, cudaStream_t st);
};
int sm_count();  // SMs of the current device
uint32_t digits_for(uint32_t p);
uint32_t mm_kmax(uint32_t p);  // longest K one exact tensor-core accumulation covers
// digit planes of the R x K matrix whose element (r, k) is src[r * rs + k * ks]
void to_digits(const uint32_t *src, uint64_t rs, uint64_t ks, const DigitPlanes &D, uint32_t p, cudaStream_t st);
// Updates C[cy + m][cx + n] <- C -/+ (A B)[m][n] mod p (m < M, n < N, K <= mm_kmax(p)) on the
// tensor cores (mm.cu), with A and B^T given by digit planes and C (crows x ccols, row pitch ldc,
// 16-byte aligned, ldc a multiple of 4) by TMA.  The tensor maps are encoded once per plan; each
// update's region ends the C tensor on the right and bottom.  err collects device error flags.
// Device time of the tensor-core product launches of one reduction: while a reduction runs on
// this thread, MmPlan::update records a pair of the context's events around each launch made
// outside graph capture; the reduction reads them after its stream synchronises.
struct MmTimer {
    gb_ctx *ctx = nullptr;
    size_t used = 0;  // events taken from ctx->mm_ev (two per launch, or two per span)
    double flops = 0.0;
    uint64_t launches = 0;
    // a span: one event pair around a run of consecutive k_mm launches with nothing else between
    // them, in place of a pair per launch (events between launches would keep each launch from
    // overlapping the one before, see launch_mm)
    cudaEvent_t span_end = nullptr;
    void begin_span(cudaStream_t st);
    void end_span(cudaStream_t st);
    double elapsed_ms() const;  // after the stream has synchronised
};
extern thread_local MmTimer *t_mm_timer;

struct MmPlan {
    MmPlan(const DigitPlanes &A, const DigitPlanes &B, uint32_t *C, uint64_t ldc, uint32_t crows, uint32_t ccols,
           const Fp &fp);
    ~MmPlan();
    MmPlan(const MmPlan &) = delete;
    MmPlan &operator=(const MmPlan &) = delete;
    // dig (optional): the digit planes of the updated region's first dig_cols columns are also
    // written there (row m, K index n), dig_cols a multiple of 16.  pdl: a programmatic dependent
    // launch (for a run of consecutive k_mm launches; see launch_mm in mm.cu)
    void update(uint32_t ax, uint32_t ay, uint32_t bx, uint32_t by, uint32_t cx, uint32_t cy, uint32_t M, uint32_t N,
                uint32_t K, bool sub, uint32_t *err, cudaStream_t st, const DigitPlanes *dig = nullptr,
                uint32_t dig_cols = 0, bool pdl = false) const;
    const DigitPlanes *A, *B;
    uint32_t *C;
    uint64_t ldc;
    uint32_t rows, cols;
    Fp fp;
    struct Maps;
    Maps *maps;
};

// C <- C -/+ A B mod p on the tensor cores (A m x k, B k x n, C m x n; row pitches in elements),
// enqueued on st; digit planes and any staging come from the arena (mm.cu)
void matmul_dev(Arena &ar, const Fp &fp, uint32_t m, uint32_t n, uint32_t k, const uint32_t *A, uint64_t lda,
                const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc, bool subtract, uint32_t *err,
                cudaStream_t st);

// ---- dense blocked reduction of the non-pivot rows (dense.cu) --------------------------------
struct DenseJob {
    const uint32_t *row_ptr, *col, *val, *colpos;  // CSR (pivot rows first) and column map
    const uint32_t *pcols;                         // dictionary column of each pivot, ascending
    const uint32_t *Uinv;                          // 32 x 32 chunk-triangle inverses
    uint32_t N, nA, nC, nb;
    Fp fp;
    unsigned long long *work;                      // [0] pivot rows, [1] dense multiply-adds
    // set by reduce_dense: block size, pivots padded to 64, padded width, row pitches
    uint32_t bs, nAp, Np;
    uint64_t ldm, wkpad, fkpad;
    uint32_t *M, *Ub;
    uint16_t *WT, *F;
};
// whether the dense schedule is expected to beat the sparse one for a matrix of this shape
bool dense_pays(uint32_t p, uint32_t N, uint32_t nA, uint32_t nC);
// device bytes reduce_dense takes from the arena for one matrix
size_t dense_bytes(uint32_t p, uint32_t N, uint32_t nA, uint32_t nC);
// D' (nC x nb) of one matrix by dense blocked elimination (the chunk inverses must be ready)
void reduce_dense(DenseJob J, uint32_t *dprime, Arena &ar, uint32_t *err, cudaStream_t st);
}  // namespace gb
