// f4.cpp -- host control of the F4 loop (Sec. 4.2, "algebraic control"): input normalisation,
// critical pairs with the Gebauer-Moeller update, degree-driven selection, and the driver that
// runs the device pipeline (sp.cu, reduce.cu) once per step.
//
// The choices the paper leaves open are fixed as follows (the CPU oracle fixes the same ones in
// its own code):
//   grevlex with x1 > ... > xn; inputs normalised (merged mod p, zeros dropped, monic, sorted) and
//   inserted in input order through UPDATE; every pair of minimal lcm degree selected (normal
//   strategy); reducer = the oldest non-redundant element whose leading monomial divides; new
//   elements appended in echelon-row order; final basis minimalised (an element goes when another
//   one's leading monomial divides its own, the older one staying on equality), tails fully
//   reduced, sorted by leading monomial descending.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <numeric>

#include "internal.hpp"

namespace gb {

// ---- monomials (grevlex, x1 > ... > xn) ---------------------------------------------------------

int mono_deg(const Mono &a, int n) {
    int d = 0;
    for (int i = 0; i < n; ++i) d += a.e[i];
    return d;
}

int mono_cmp(const Mono &a, const Mono &b, int n, bool deglex) {
    // grevlex, equal degrees: the last differing exponent decides, the smaller one giving the
    // larger monomial.  With byte i = exponent of x_{i+1} (bytes >= n zero), the last differing
    // byte is the most significant differing byte of the 128-bit little-endian word, so the words
    // compare in reverse.  deglex, equal degrees: the first differing exponent decides, the larger
    // one giving the larger monomial (bytewise lexicographic comparison).
    const M16 x = m16(a), y = m16(b);
    const uint32_t da = deg16(x), db = deg16(y);
    if (da != db) return da > db ? 1 : -1;
    if (deglex) {
        const int c = std::memcmp(a.e, b.e, (size_t)n);
        return c > 0 ? 1 : c < 0 ? -1 : 0;
    }
    if (x.hi != y.hi) return x.hi < y.hi ? 1 : -1;
    if (x.lo != y.lo) return x.lo < y.lo ? 1 : -1;
    return 0;
}

Mono mono_mul(const Mono &a, const Mono &b, int n) {
    Mono r{};
    for (int i = 0; i < n; ++i) {
        const int s = a.e[i] + b.e[i];
        if (s > 255) fail(GB_EOVERFLOW, "exponent above 255");
        r.e[i] = (uint8_t)s;
    }
    return r;
}

Mono mono_div(const Mono &b, const Mono &a, int n) {
    Mono r{};
    for (int i = 0; i < n; ++i) r.e[i] = (uint8_t)(b.e[i] - a.e[i]);
    return r;
}

Mono mono_lcm(const Mono &a, const Mono &b, int n) {
    Mono r{};
    for (int i = 0; i < n; ++i) r.e[i] = std::max(a.e[i], b.e[i]);
    return r;
}

bool mono_divides(const Mono &a, const Mono &b, int n) {
    for (int i = 0; i < n; ++i)
        if (a.e[i] > b.e[i]) return false;
    return true;
}

bool mono_coprime(const Mono &a, const Mono &b, int n) {
    for (int i = 0; i < n; ++i)
        if (a.e[i] && b.e[i]) return false;
    return true;
}

// ---- F_p constants ----------------------------------------------------------------------------

Fp make_fp(uint32_t p) {
    Fp f{};
    f.p = p;
    uint32_t x = p;  // Newton iteration for p^{-1} mod 2^32 (p odd): 5 steps double 3 correct bits
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    f.pinv_neg = 0u - x;
    f.mu = UINT64_MAX / p;  // = floor(2^64 / p) since p does not divide 2^64
    const unsigned __int128 R = (unsigned __int128)1 << 64;
    f.r2 = (uint32_t)(R % p);
    f.small = p < 65536u ? 1u : 0u;
    f.mu32 = (uint32_t)(0xFFFFFFFFu / p);  // = floor(2^32 / p) since p does not divide 2^32
    return f;
}

uint32_t host_inv(uint32_t a, uint32_t p) {
    int64_t r0 = p, r1 = a % p, s0 = 0, s1 = 1;
    while (r1) {
        const int64_t q = r0 / r1;
        int64_t t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    s0 %= (int64_t)p;
    return (uint32_t)(s0 < 0 ? s0 + p : s0);
}

// ---- host workers ----------------------------------------------------------------------------
//
// The per-system host control of a batch (pair updates, selection, minimalisation) is independent
// across systems, so it runs on a small persistent pool; the calling thread takes part.

struct HostPool {
    explicit HostPool(unsigned nthreads) {
        for (unsigned t = 0; t < nthreads; ++t) th.emplace_back([this] { loop(); });
    }
    ~HostPool() {
        {
            std::lock_guard<std::mutex> g(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto &t : th) t.join();
    }
    void run(size_t n, const std::function<void(size_t)> &f) {
        {
            std::lock_guard<std::mutex> g(mu);
            fn = &f;
            count = n;
            next = 0;
            err = nullptr;
            pending = (unsigned)th.size();
            ++gen;
        }
        cv.notify_all();
        work();
        std::unique_lock<std::mutex> lk(mu);
        done_cv.wait(lk, [&] { return pending == 0; });
        fn = nullptr;
        if (err) std::rethrow_exception(err);
    }

   private:
    void work() {
        for (size_t i; (i = next.fetch_add(1)) < count;) {
            try {
                (*fn)(i);
            } catch (...) {
                std::lock_guard<std::mutex> g(mu);
                if (!err) err = std::current_exception();
            }
        }
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || gen != seen; });
                if (stop) return;
                seen = gen;
            }
            work();
            std::lock_guard<std::mutex> g(mu);
            if (--pending == 0) done_cv.notify_all();
        }
    }
    std::vector<std::thread> th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    const std::function<void(size_t)> *fn = nullptr;
    size_t count = 0;
    std::atomic<size_t> next{0};
    uint64_t gen = 0;
    unsigned pending = 0;
    bool stop = false;
    std::exception_ptr err;
};

void parallel_for(gb_ctx *ctx, size_t n, const std::function<void(size_t)> &fn) {
    if (n <= 1) {
        for (size_t i = 0; i < n; ++i) fn(i);
        return;
    }
    if (!ctx->pool) {
        unsigned hw = std::thread::hardware_concurrency();
        if (!hw) hw = 4;
        ctx->pool = std::make_unique<HostPool>(std::min(hw, 16u) - 1);
    }
    ctx->pool->run(n, fn);
}

// ---- critical pairs: UPDATE of Becker and Weispfenning (Gebauer-Moeller criteria) --------------
//
// Leading monomials are compared as SWAR words (internal.hpp) while every exponent is below 128;
// beyond that the bytewise routines above are used.  Pair lcms are cached with the pair.

namespace {
// leading-monomial arithmetic of one system
struct LmOps {
    const gb_system *S;
    int n;
    bool swar;
    explicit LmOps(const gb_system *s) : S(s), n((int)s->n), swar(s->swar) {}
    M16 lcm(uint32_t a, uint32_t b) const {
        if (swar) return lcm16(S->lm16[a], S->lm16[b]);
        return m16(mono_lcm(S->lm[a], S->lm[b], n));
    }
    bool divides(const M16 &a, const M16 &b) const {
        if (swar) return divides16(a, b);
        Mono x, y;
        std::memcpy(x.e, &a, 16);
        std::memcpy(y.e, &b, 16);
        return mono_divides(x, y, n);
    }
    bool coprime(uint32_t a, uint32_t b) const {
        return swar ? coprime16(S->lm16[a], S->lm16[b]) : mono_coprime(S->lm[a], S->lm[b], n);
    }
    // the second loop of UPDATE: the waiting pair pr goes when h arrives iff LM(h) divides its
    // lcm while lcm(LM(i), LM(h)) and lcm(LM(j), LM(h)) both differ from it
    bool dropped_by(const PairL &pr, uint32_t h) const {
        return divides(S->lm16[h], pr.lcm) && !(lcm(pr.i, h) == pr.lcm) && !(lcm(pr.j, h) == pr.lcm);
    }
};

// The first loop of UPDATE for one new element h: the pairs (g, h), g in C (the elements older
// than h that are not redundant when h arrives, oldest first), that it keeps, appended to out
// without those of coprime leading monomials (Buchberger's product criterion).
void new_pairs(const LmOps &o, uint32_t h, const std::vector<uint32_t> &C, std::vector<PairL> &out) {
    // per-thread scratch, reused across calls
    struct Scratch {
        std::vector<uint32_t> Ld, ord, cnt, und, slot;
        std::vector<M16> L, mins;
        std::vector<char> kept, cop, dom;
    };
    static thread_local Scratch z;
    const size_t c = C.size();
    z.L.resize(c);
    z.Ld.resize(c);
    z.kept.assign(c, 0);
    z.cop.assign(c, 0);
    z.dom.assign(c, 0);
    std::vector<M16> &L = z.L;
    std::vector<uint32_t> &Ld = z.Ld;
    std::vector<char> &kept = z.kept, &cop = z.cop, &dom = z.dom;
    uint32_t dmax = 0;
    for (size_t a = 0; a < c; ++a) {
        L[a] = o.lcm(h, C[a]);
        Ld[a] = deg16(L[a]);
        dmax = std::max(dmax, Ld[a]);
        cop[a] = o.coprime(h, C[a]);
    }
    // The new pairs (h, g) are taken oldest g first: one is kept when its leading monomials are
    // coprime, or when no pair still waiting and no pair already kept has an lcm dividing its lcm.
    // That sequential rule has a closed form (by induction over the order, following a chain of
    // divisors down to a minimal lcm): a non-coprime pair is kept iff no new pair's lcm strictly
    // divides its lcm, no later pair has the same lcm, and no coprime pair has the same lcm.  A
    // strict divisor has lower degree, and when there is one, one of the minimal lcms of lower
    // degree divides too; so the pairs are visited by degree against the minimal lcms found so far.
    // Visit order: by degree, then index (a counting sort: degrees are small).
    std::vector<uint32_t> &ord = z.ord, &cnt = z.cnt;
    cnt.assign(dmax + 2, 0);
    for (size_t a = 0; a < c; ++a) ++cnt[Ld[a] + 1];
    for (uint32_t d = 0; d <= dmax; ++d) cnt[d + 1] += cnt[d];
    ord.resize(c);
    for (uint32_t a = 0; a < c; ++a) ord[cnt[Ld[a]]++] = a;
    std::vector<M16> &mins = z.mins;
    mins.clear();
    for (size_t s0 = 0; s0 < c;) {
        size_t e = s0;
        while (e < c && Ld[ord[e]] == Ld[ord[s0]]) ++e;
        for (size_t q = s0; q < e; ++q)
            for (const M16 &m : mins)
                if (o.divides(m, L[ord[q]])) {
                    dom[ord[q]] = 1;
                    break;
                }
        for (size_t q = s0; q < e; ++q) {
            if (dom[ord[q]]) continue;
            bool have = false;
            for (size_t t = mins.size(); t-- > 0 && Ld[ord[q]] == deg16(mins[t]);)
                if (mins[t] == L[ord[q]]) {
                    have = true;
                    break;
                }
            if (!have) mins.push_back(L[ord[q]]);
        }
        s0 = e;
    }
    // equal lcms among the undominated pairs: an open-addressing table keyed by the lcm keeps, per
    // lcm, its largest index and whether a coprime pair has it
    std::vector<uint32_t> &und = z.und, &slot = z.slot;
    und.clear();
    for (uint32_t a = 0; a < c; ++a)
        if (!dom[a]) und.push_back(a);
    size_t cap = 16;
    while (cap < 2 * und.size()) cap <<= 1;
    slot.assign(cap, UINT32_MAX);  // index of the group's largest member (flags in cop/kept below)
    std::vector<char> &anyc = dom;   // reused: dom is no longer needed for undominated indices
    for (uint32_t a : und) anyc[a] = 0;
    for (uint32_t a : und) {
        const uint64_t hsh = (L[a].lo * 0x9E3779B97F4A7C15ull) ^ (L[a].hi * 0xC2B2AE3D27D4EB4Full);
        size_t k = (size_t)(hsh >> 20) & (cap - 1);
        while (slot[k] != UINT32_MAX && !(L[slot[k]] == L[a])) k = (k + 1) & (cap - 1);
        if (slot[k] == UINT32_MAX) {
            slot[k] = a;
            anyc[a] = cop[a];
        } else {
            const uint32_t b0 = slot[k];
            const char any = anyc[b0] || cop[a];
            slot[k] = std::max(b0, a);
            anyc[slot[k]] = any;
        }
    }
    for (size_t k = 0; k < cap; ++k)
        if (slot[k] != UINT32_MAX && !anyc[slot[k]]) kept[slot[k]] = 1;  // the last of its lcm
    for (size_t a = 0; a < c; ++a)
        if (kept[a] && !cop[a]) out.push_back(PairL{C[a], h, Ld[a], 0, L[a]});
}
}  // namespace

// UPDATE (Becker and Weispfenning) for the new elements h0, h0 + 1, ..., lm.size() - 1 of each
// system, whose leading monomials are already recorded: the same pairs, in the same order, and the
// same redundant elements as UPDATE called on them one at a time, computed in parallel.  One at a
// time, h_i (= h0 + i) first takes its new pairs against C_i, the older elements not yet
// redundant; then drops the waiting pairs its leading monomial rules out; then marks redundant the
// older elements whose leading monomial it divides.  So:
//   - e is redundant when h_i arrives iff it was before the step, or some h_f with e < h_f, f < i
//     has LM(h_f) | LM(e): with first(e) the least such f (k when there is none), C_i is the set
//     of g < h_i not redundant before the step with first(g) >= i;
//   - a pair waiting at the step's start survives iff no h_i drops it, and a new pair of h_i
//     survives iff no later h_j drops it (the test looks at the pair and h_j only);
//   - the survivors come in the sequential order: the waiting ones, then those of h_0, h_1, ...
// first(), the new pairs of each h_i and the survivor tests are independent work items.
static void update_steps(gb_ctx *ctx, const std::vector<gb_system *> &Ss, const std::vector<uint32_t> &h0) {
    const size_t nj = Ss.size();
    auto run = [&](size_t n, const std::function<void(size_t)> &f) {
        if (ctx) parallel_for(ctx, n, f);
        else for (size_t i = 0; i < n; ++i) f(i);
    };
    struct Sys {
        std::vector<uint32_t> first;         // per element: the least f as above, k if none
        std::vector<std::vector<PairL>> fresh;  // per new element: its surviving new pairs
        std::vector<uint8_t> keep;           // per waiting pair: whether it survives
        uint32_t k = 0;
    };
    std::vector<Sys> W(nj);
    struct Item {
        uint32_t j, a, b;  // system, range [a, b) of elements or pairs, or (a = new element, b = ~0u)
    };
    constexpr uint32_t CHUNK = 1024, PCHUNK = 8192;
    std::vector<Item> items;
    for (size_t j = 0; j < nj; ++j) {
        const uint32_t nt = (uint32_t)Ss[j]->lm.size();
        W[j].k = nt - h0[j];
        W[j].first.assign(nt, W[j].k);
        if (W[j].k)
            for (uint32_t a = 0; a < nt; a += CHUNK) items.push_back(Item{(uint32_t)j, a, std::min(nt, a + CHUNK)});
    }
    run(items.size(), [&](size_t t) {
        const Item it = items[t];
        const gb_system *S = Ss[it.j];
        const LmOps o(S);
        Sys &w = W[it.j];
        const uint32_t base = h0[it.j];
        for (uint32_t e = it.a; e < it.b; ++e) {
            if (S->redundant[e]) continue;
            for (uint32_t f = e < base ? 0 : e - base + 1; f < w.k; ++f)
                if (o.divides(S->lm16[base + f], S->lm16[e])) {
                    w.first[e] = f;
                    break;
                }
        }
    });
    items.clear();
    for (size_t j = 0; j < nj; ++j) {
        if (!W[j].k) continue;
        W[j].fresh.resize(W[j].k);
        W[j].keep.assign(Ss[j]->pairs.size(), 1);
        for (uint32_t i = W[j].k; i-- > 0;) items.push_back(Item{(uint32_t)j, i, ~0u});  // largest C first
        const uint32_t np = (uint32_t)Ss[j]->pairs.size();
        for (uint32_t a = 0; a < np; a += PCHUNK) items.push_back(Item{(uint32_t)j, a, std::min(np, a + PCHUNK)});
    }
    run(items.size(), [&](size_t t) {
        const Item it = items[t];
        const gb_system *S = Ss[it.j];
        const LmOps o(S);
        Sys &w = W[it.j];
        const uint32_t base = h0[it.j];
        if (it.b == ~0u) {
            const uint32_t i = it.a, h = base + i;
            static thread_local std::vector<uint32_t> C;
            C.clear();
            for (uint32_t g = 0; g < h; ++g)
                if (!S->redundant[g] && w.first[g] >= i) C.push_back(g);
            std::vector<PairL> &out = w.fresh[i];
            new_pairs(o, h, C, out);
            size_t n = 0;
            for (const PairL &pr : out) {
                bool drop = false;
                for (uint32_t f = i + 1; f < w.k && !drop; ++f) drop = o.dropped_by(pr, base + f);
                if (!drop) out[n++] = pr;
            }
            out.resize(n);
        } else {
            for (uint32_t q = it.a; q < it.b; ++q) {
                const PairL &pr = S->pairs[q];
                for (uint32_t f = 0; f < w.k; ++f)
                    if (o.dropped_by(pr, base + f)) {
                        w.keep[q] = 0;
                        break;
                    }
            }
        }
    });
    run(nj, [&](size_t j) {
        gb_system *S = Ss[j];
        Sys &w = W[j];
        if (!w.k) return;
        size_t n = 0;
        for (size_t q = 0; q < S->pairs.size(); ++q)
            if (w.keep[q]) S->pairs[n++] = S->pairs[q];
        S->pairs.resize(n);
        for (const auto &v : w.fresh) S->pairs.insert(S->pairs.end(), v.begin(), v.end());
        for (size_t e = 0; e < S->lm.size(); ++e)
            if (w.first[e] < w.k) S->redundant[e] = 1;
    });
}

// the critical-pair update of one system for its elements h0.. (host only)
void update_pairs_host(gb_system *S, uint32_t h0) { update_steps(nullptr, {S}, {h0}); }

// record a new leading monomial (SWAR form, and whether the fast comparisons still apply)
void push_lm(gb_system *S, const Mono &m) {
    S->lm.push_back(m);
    S->lm16.push_back(m16(m));
    for (uint32_t i = 0; i < S->n; ++i)
        if (m.e[i] >= 128) S->swar = false;
    S->redundant.push_back(0);
}

static std::vector<uint32_t> nonredundant(const gb_system *S) {
    std::vector<uint32_t> r;
    for (uint32_t g = 0; g < S->redundant.size(); ++g)
        if (!S->redundant[g]) r.push_back(g);
    return r;
}

// given rows -> RowSpec list: equal (t, k) collapse; ordered by (LM descending, k ascending); the
// first row of each leading monomial is its pivot
std::vector<RowSpec> order_rows(const gb_system *S, std::vector<std::pair<Mono, uint32_t>> tk) {
    const int n = (int)S->n;
    struct R {
        Mono t, lm;
        uint32_t k;
    };
    std::vector<R> rows;
    rows.reserve(tk.size());
    for (auto &x : tk) {
        if (x.second >= S->lm.size()) fail(GB_EINVAL, "row refers to a basis element that does not exist");
        rows.push_back(R{x.first, mono_mul(x.first, S->lm[x.second], n), x.second});
    }
    const bool dl = S->deglex;
    std::sort(rows.begin(), rows.end(), [n, dl](const R &a, const R &b) {
        const int c = mono_cmp(a.lm, b.lm, n, dl);
        if (c) return c > 0;
        if (a.k != b.k) return a.k < b.k;
        return mono_cmp(a.t, b.t, n, dl) < 0;
    });
    std::vector<RowSpec> out;
    for (size_t i = 0; i < rows.size(); ++i) {
        if (i && rows[i].k == rows[i - 1].k && rows[i].t == rows[i - 1].t) continue;
        const bool first = out.empty() || !(rows[i].lm == mono_mul(out.back().t, S->lm[out.back().k], n));
        out.push_back(RowSpec{rows[i].t, rows[i].k, (uint8_t)(first ? 1 : 0), 0});
    }
    return out;
}

// register one normalised polynomial as a new basis element (its terms already sit at the end of
// the device basis) and run UPDATE
static void append_host_poly(gb_system *S, const Mono &lm, uint32_t len) {
    S->off.push_back((uint32_t)S->nterms);
    S->len.push_back(len);
    S->nterms += len;
    push_lm(S, lm);
    if (mono_deg(lm, (int)S->n) == 0) S->unit = true;
    update_steps(nullptr, {S}, {(uint32_t)(S->lm.size() - 1)});
}

bool is_prime32(uint32_t q) {
    if (q < 2) return false;
    for (uint32_t d : {2u, 3u, 5u, 7u, 11u, 13u})
        if (q % d == 0) return q == d;
    // deterministic Miller-Rabin: bases 2, 3, 5, 7 are exact below 3,215,031,751
    uint32_t d = q - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; ++s; }
    for (uint64_t a : {2ull, 3ull, 5ull, 7ull}) {
        uint64_t x = 1, b = a % q;
        for (uint32_t e = d; e; e >>= 1) {
            if (e & 1) x = x * b % q;
            b = b * b % q;
        }
        if (x == 1 || x == q - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = x * x % q;
            if (x == q - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

void system_init(gb_system *S, uint32_t nvars, uint32_t p, const gb_polys *F) {
    if (nvars < 1 || nvars > 16) fail(GB_EINVAL, "nvars must be in [1, 16]");
    if (p < 3 || p >= (1u << 31) || !is_prime32(p)) fail(GB_EINVAL, "p must be an odd prime below 2^31");
    S->n = nvars;
    S->p = p;
    S->fp = make_fp(p);
    const int n = (int)nvars;
    std::vector<std::vector<Mono>> mons;
    std::vector<std::vector<uint32_t>> cfs;
    uint64_t total = 0;
    for (uint32_t i = 0; F && i < F->npolys; ++i) {
        const uint32_t a = F->poly_off[i], b = F->poly_off[i + 1];
        if (b < a) fail(GB_EINVAL, "poly_off must be non-decreasing");
        std::vector<std::pair<Mono, uint32_t>> t;
        for (uint32_t q = a; q < b; ++q) {
            Mono m{};
            std::memcpy(m.e, F->exps + (size_t)q * n, n);
            t.emplace_back(m, F->coeffs[q] % p);
        }
        const bool dl = S->deglex;
        std::sort(t.begin(), t.end(), [n, dl](const auto &x, const auto &y) { return mono_cmp(x.first, y.first, n, dl) > 0; });
        std::vector<Mono> mon;
        std::vector<uint32_t> cf;
        for (size_t q = 0; q < t.size();) {
            size_t r = q;
            uint64_t c = 0;
            while (r < t.size() && t[r].first == t[q].first) c = (c + t[r++].second) % p;
            if (c) { mon.push_back(t[q].first); cf.push_back((uint32_t)c); }
            q = r;
        }
        if (mon.empty()) continue;
        const uint32_t inv = host_inv(cf[0], p);
        for (auto &c : cf) c = (uint32_t)((uint64_t)c * inv % p);
        total += mon.size();
        mons.push_back(std::move(mon));
        cfs.push_back(std::move(cf));
    }
    if (total >= (1ull << 32)) fail(GB_EUNSUPPORTED, "input above 2^32 terms");
    const uint32_t ng = (uint32_t)mons.size();
    S->in_mon.reserve(total);
    S->in_cf.reserve(total);
    for (uint32_t g = 0; g < ng; ++g) {
        for (const Mono &m : mons[g]) S->in_mon.push_back(to_u4(m));
        S->in_cf.insert(S->in_cf.end(), cfs[g].begin(), cfs[g].end());
    }
    for (uint32_t g = 0; g < ng; ++g) append_host_poly(S, mons[g][0], (uint32_t)mons[g].size());
    // Device footprint estimate for admission control.  The peak arena use of a whole run grows
    // geometrically with n, faster for higher input degree: measured high-water marks of systems
    // run alone (n = 5..11, degree 2 and 3, 10-66 terms per polynomial) follow
    // log2(peak / MiB) ~ 1.7 (d - 1) n - 8.5 - 3.5 (d - 1) for input degree d, within a factor
    // of about 1.5.  The estimate is twice that, plus 8 MiB.
    uint32_t dmax = 1;
    for (const Mono &m : S->lm) dmax = std::max<uint32_t>(dmax, (uint32_t)mono_deg(m, n));
    const double d1 = (double)std::max<uint32_t>(dmax, 2) - 1.0;
    const double log2_mib = std::min(40.0, 1.7 * d1 * nvars - 8.5 - 3.5 * d1);
    S->footprint = (size_t)((8.0 + 2.0 * std::exp2(log2_mib)) * 1048576.0);
}

// A new system with the same normalised input as S, which must not have run a step: its input
// polynomials are then in_mon / in_cf, element g holding len[g] terms in order.
gb_system *system_clone_fresh(const gb_system *S) {
    if (S->steps || S->resident) fail(GB_EINVAL, "the system has already run a step");
    const uint32_t n = S->n, ng = (uint32_t)S->len.size();
    std::vector<uint32_t> po(ng + 1, 0);
    for (uint32_t g = 0; g < ng; ++g) po[g + 1] = po[g] + S->len[g];
    if (po[ng] != S->in_mon.size() || S->in_cf.size() != S->in_mon.size())
        fail(GB_EDEVICE, "system copy: input arrays do not match the element lengths");
    std::vector<uint8_t> ex((size_t)po[ng] * n);
    for (size_t q = 0; q < S->in_mon.size(); ++q) {
        Mono m{};
        std::memcpy(m.e, &S->in_mon[q], 16);
        std::memcpy(ex.data() + q * n, m.e, n);
    }
    gb_polys F{};
    F.npolys = ng;
    F.poly_off = po.data();
    F.exps = ex.data();
    F.coeffs = S->in_cf.data();
    auto C = std::make_unique<gb_system>();
    C->ctx = S->ctx;
    C->stream = S->stream;
    C->deglex = S->deglex;
    system_init(C.get(), n, S->p, &F);
    return C.release();
}

// the inputs of systems not yet on the device, in one staged copy: terms, coefficients, offsets
// and lengths (no step has run yet, so the host mirrors off / len describe exactly the input)
void make_resident(const std::vector<gb_system *> &Ss) {
    std::vector<gb_system *> todo;
    for (gb_system *S : Ss)
        if (!S->resident) todo.push_back(S);
    if (todo.empty()) return;
    gb_ctx *ctx = todo[0]->ctx;
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    Stage sg;
    struct At { size_t m, c, o, l; };
    std::vector<At> at(todo.size());
    for (size_t j = 0; j < todo.size(); ++j) {
        gb_system *S = todo[j];
        const uint64_t T = S->nterms;
        const size_t ng = S->off.size();
        S->bmon.alloc(ar, std::max<uint64_t>(T, 1024), st);
        S->bkey.alloc(ar, std::max<uint64_t>(T, 1024), st);
        S->bcf.alloc(ar, std::max<uint64_t>(T, 1024), st);
        S->boff.alloc(ar, std::max<size_t>(ng, 64), st);
        S->blen.alloc(ar, std::max<size_t>(ng, 64), st);
        at[j] = At{sg.put(S->in_mon.data(), 16ull * T), sg.put(S->in_cf.data(), 4ull * T),
                   sg.put(S->off.data(), 4ull * ng), sg.put(S->len.data(), 4ull * ng)};
    }
    DBuf<char> d;
    sg.upload(ctx, d);
    for (size_t j = 0; j < todo.size(); ++j) {
        gb_system *S = todo[j];
        const uint64_t T = S->nterms;
        const size_t ng = S->off.size();
        if (T) {
            GB_CUDA(cudaMemcpyAsync(S->bmon.p, d.p + at[j].m, 16ull * T, cudaMemcpyDeviceToDevice, st));
            GB_CUDA(cudaMemcpyAsync(S->bcf.p, d.p + at[j].c, 4ull * T, cudaMemcpyDeviceToDevice, st));
            basis_keys(S->bmon.p, S->bkey.p, T, st);
        }
        if (ng) {
            GB_CUDA(cudaMemcpyAsync(S->boff.p, d.p + at[j].o, 4ull * ng, cudaMemcpyDeviceToDevice, st));
            GB_CUDA(cudaMemcpyAsync(S->blen.p, d.p + at[j].l, 4ull * ng, cudaMemcpyDeviceToDevice, st));
        }
        S->resident = true;
        std::vector<uint4>().swap(S->in_mon);
        std::vector<uint32_t>().swap(S->in_cf);
    }
}

// ---- lockstep F4 steps of many systems ------------------------------------------------------------
//
// One step of every system: each selects its pairs of minimal degree (normal strategy) on the host
// workers, then one symbolic preprocessing, one sparse reduction and one RREF run over all of the
// systems' matrices together (each kernel launch covers every system's rows), and the new basis
// elements go through UPDATE on the host workers again.

namespace {
using Clock = std::chrono::steady_clock;
double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}
}  // namespace

void f4_steps(const std::vector<gb_system *> &Ss, std::vector<gb_step_stats> *stats) {
    const size_t nj = Ss.size();
    if (stats) stats->assign(nj, gb_step_stats{});
    if (!nj) return;
    gb_ctx *ctx = Ss[0]->ctx;
    const auto t0 = Clock::now();
    make_resident(Ss);
    std::vector<SpTask> tasks(nj);
    std::vector<uint32_t> dmin(nj, UINT32_MAX), npairs(nj, 0);
    parallel_for(ctx, nj, [&](size_t j) {
        gb_system *S = Ss[j];
        const int n = (int)S->n;
        for (const PairL &q : S->pairs) dmin[j] = std::min(dmin[j], q.deg);
        if (dmin[j] > 255) fail(GB_EOVERFLOW, "step degree above 255");
        std::vector<std::pair<Mono, uint32_t>> tk;
        std::vector<PairL> rest;
        for (const PairL &q : S->pairs) {
            if (q.deg != dmin[j]) { rest.push_back(q); continue; }
            ++npairs[j];
            Mono l;
            std::memcpy(l.e, &q.lcm, 16);
            tk.emplace_back(mono_div(l, S->lm[q.i], n), q.i);
            tk.emplace_back(mono_div(l, S->lm[q.j], n), q.j);
        }
        S->pairs.swap(rest);
        tasks[j].S = S;
        tasks[j].rows = order_rows(S, std::move(tk));
        tasks[j].closure = true;
        tasks[j].nonred = nonredundant(S);
    });
    const auto ts = Clock::now();
    symbolic_preprocess(tasks);
    std::vector<gb_macaulay *> Ms(nj);
    for (size_t j = 0; j < nj; ++j) Ms[j] = tasks[j].out.get();
    auto Es = reduce_rows(Ms, true);
    const auto t1 = Clock::now();
    std::vector<gb_echelon *> Ep(nj);
    for (size_t j = 0; j < nj; ++j) Ep[j] = Es[j].get();
    std::vector<std::vector<Mono>> lms;
    append_echelon(Ep, lms);
    const auto tp = Clock::now();
    std::vector<uint32_t> h0(nj);
    for (size_t j = 0; j < nj; ++j) {
        gb_system *S = Ss[j];
        h0[j] = (uint32_t)S->lm.size();
        for (const Mono &m : lms[j]) {
            push_lm(S, m);
            if (mono_deg(m, (int)S->n) == 0) S->unit = true;
        }
    }
    update_steps(ctx, Ss, h0);
    const auto t2 = Clock::now();
    for (size_t j = 0; j < nj; ++j) {
        gb_system *S = Ss[j];
        gb_macaulay *mac = Ms[j];
        gb_echelon *ech = Ep[j];
        S->steps++;
        gb_step_stats st{};
        st.step = S->steps;
        st.degree = dmin[j];
        st.npairs = npairs[j];
        st.nrows = mac->nrows;
        st.ndict = mac->ndict;
        st.npivot = mac->nA;
        st.nC = mac->nC;
        st.nb = mac->nb;
        st.rank = ech->rank;
        st.nbasis = (uint32_t)S->lm.size();
        st.closure_rounds = mac->closure_rounds;
        st.sp_redo = mac->sp_redo;
        st.nnz = mac->nnz;
        st.axpy_rows = ech->work[0];
        st.axpy_fma = ech->work[1];
        // device stages are timed once for the whole batch
        st.ms_sp = mac->ms_sp;
        st.ms_reduce = ech->ms_reduce;
        st.ms_rref = ech->ms_rref;
        st.ms_reduce_kernel = ech->ms_reduce_kernel;
        st.ms_update = (float)ms_between(t1, tp);
        st.ms_pairs = (float)ms_between(tp, t2);
        st.ms_select = (float)ms_between(t0, ts);
        st.ms_wall = ms_between(t0, t2);
        st.ms_mm = ech->ms_mm;
        st.mm_flops = ech->mm_flops;
        st.mm_launches = ech->mm_launches;
        st.rref_sketched = ech->sketched;
        S->run.steps = S->steps;
        S->run.nnz_total += st.nnz;
        S->run.nnz_steps += st.nnz;
        S->run.ms_mm += st.ms_mm;
        S->run.mm_flops += st.mm_flops;
        S->run.mm_launches += st.mm_launches;
        S->run.axpy_rows += st.axpy_rows;
        S->run.axpy_fma += st.axpy_fma;
        S->run.ms_sp += st.ms_sp;
        S->run.ms_reduce += st.ms_reduce;
        S->run.ms_rref += st.ms_rref;
        S->run.ms_reduce_kernel += st.ms_reduce_kernel;
        S->run.ms_update += st.ms_update;
        S->run.ms_pairs += st.ms_pairs;
        S->run.ms_select += st.ms_select;
        S->run.ms_wall += st.ms_wall;
        if (stats) (*stats)[j] = st;
        if (ctx->flags & GB_CTX_KEEP_STEP) {
            S->last_ech = std::move(Es[j]);
            S->last_mac = std::move(tasks[j].out);
        }
    }
}

// ---- the reduced basis ------------------------------------------------------------------------


void finish_batch(const std::vector<gb_system *> &Ss) {
    const size_t nj = Ss.size();
    if (!nj) return;
    gb_ctx *ctx = Ss[0]->ctx;
    const auto t0 = Clock::now();
    make_resident(Ss);
    // minimalisation: an element goes when another one's leading monomial divides its own (the
    // older one staying on equality); the rest in leading-monomial order, descending
    std::vector<std::vector<uint32_t>> keep(nj);
    parallel_for(ctx, nj, [&](size_t j) {
        gb_system *S = Ss[j];
        const int n = (int)S->n;
        const uint32_t ng = (uint32_t)S->lm.size();
        std::vector<uint32_t> live;
        for (uint32_t i = 0; i < ng; ++i)
            if (!S->redundant[i]) live.push_back(i);
        for (uint32_t i : live) {
            bool drop = false;
            for (uint32_t g : live) {
                if (g == i) continue;
                const bool div = S->swar ? divides16(S->lm16[g], S->lm16[i]) : mono_divides(S->lm[g], S->lm[i], n);
                if (div && (!(S->lm[g] == S->lm[i]) || g < i)) { drop = true; break; }
            }
            if (!drop) keep[j].push_back(i);
        }
        std::sort(keep[j].begin(), keep[j].end(),
                  [&](uint32_t a, uint32_t b) { return mono_cmp(S->lm[a], S->lm[b], n, S->deglex) > 0; });
    });
    // the tails t(g) = g - LM(g), reduced by the minimal basis with the same pipeline: the closure
    // supplies reducer rows for every tail monomial a leading monomial divides, and the sparse
    // reduction leaves each tail with non-pivot (standard) monomials only
    std::vector<SpTask> tasks;
    std::vector<std::vector<uint32_t>> elems;
    std::vector<gb_system *> owners;
    for (size_t j = 0; j < nj; ++j) {
        gb_system *S = Ss[j];
        if (keep[j].empty()) {
            S->fin_off.assign(1, 0);
            S->fin_exps.reset();
            S->fin_cf.reset();
            S->fin_terms = 0;
            continue;
        }
        SpTask t;
        t.S = S;
        for (uint32_t g : keep[j]) t.rows.push_back(RowSpec{Mono{}, g, 0, 1});
        t.closure = true;
        t.nonred = keep[j];
        tasks.push_back(std::move(t));
        elems.push_back(keep[j]);
        owners.push_back(S);
    }
    const auto tm = Clock::now();
    if (!tasks.empty()) {
        symbolic_preprocess(tasks);
        const auto ts = Clock::now();
        std::vector<gb_macaulay *> Ms;
        for (auto &t : tasks) Ms.push_back(t.out.get());
        auto Es = reduce_rows(Ms, false);
        const auto tr = Clock::now();
        std::vector<gb_echelon *> Ep;
        for (auto &e : Es) Ep.push_back(e.get());
        replace_tails(Ep, elems);
        if (trace_on())
            std::fprintf(stderr, "[gb] finish: %zu systems, minimalise %.3f ms, SP %.3f ms, reduce %.3f ms, tails %.3f ms\n",
                         nj, ms_between(t0, tm), ms_between(tm, ts), ms_between(ts, tr), ms_between(tr, Clock::now()));
        for (size_t k = 0; k < owners.size(); ++k) {
            gb_system *S = owners[k];
            S->run.ms_sp += Ms[k]->ms_sp;
            S->run.ms_reduce += Ep[k]->ms_reduce;
            S->run.ms_reduce_kernel += Ep[k]->ms_reduce_kernel;
            S->run.nnz_total += Ms[k]->nnz;
            S->run.ms_mm += Ep[k]->ms_mm;
            S->run.mm_flops += Ep[k]->mm_flops;
            S->run.mm_launches += Ep[k]->mm_launches;
            S->run.axpy_rows += Ep[k]->work[0];
            S->run.axpy_fma += Ep[k]->work[1];
        }
    }
    const double ms = ms_between(t0, Clock::now());
    for (size_t j = 0; j < nj; ++j) {
        gb_system *S = Ss[j];
        S->finished = true;
        S->run.nbasis = (uint32_t)keep[j].size();
        S->run.ms_wall += ms;
        S->run.ms_finish += ms;
    }
}

// One lockstep iteration over a set of running systems: those without pairs left get their reduced
// basis, the others take one F4 step together.
void advance(const std::vector<gb_system *> &Ss) {
    std::vector<gb_system *> step, fin;
    for (gb_system *S : Ss) {
        if (S->finished) continue;
        (S->pairs.empty() ? fin : step).push_back(S);
    }
    if (!fin.empty()) finish_batch(fin);
    if (!step.empty()) f4_steps(step, nullptr);
}

void groebner_batch(const std::vector<gb_system *> &Ss) {
    for (;;) {
        bool any = false;
        for (gb_system *S : Ss) any = any || !S->finished;
        if (!any) return;
        advance(Ss);
    }
}

}  // namespace gb

gb_ctx::gb_ctx() = default;
gb_ctx::~gb_ctx() = default;
