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
#include <chrono>
#include <numeric>

#include "internal.hpp"

namespace gb {

// ---- monomials (grevlex, x1 > ... > xn) ---------------------------------------------------------

int mono_deg(const Mono &a, int n) {
    int d = 0;
    for (int i = 0; i < n; ++i) d += a.e[i];
    return d;
}

int mono_cmp(const Mono &a, const Mono &b, int n) {
    // equal degrees: the last differing exponent decides, the smaller one giving the larger
    // monomial.  With byte i = exponent of x_{i+1} (bytes >= n zero), the last differing byte is
    // the most significant differing byte of the 128-bit little-endian word, so the words compare
    // in reverse.
    const M16 x = m16(a), y = m16(b);
    const uint32_t da = deg16(x), db = deg16(y);
    (void)n;
    if (da != db) return da > db ? 1 : -1;
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

// ---- small host helpers -----------------------------------------------------------------------

void *pinned(gb_system *S, size_t bytes) {
    if (bytes > S->pinned_bytes) {
        if (S->pinned) {
            sync(S);
            GB_CUDA(cudaFreeHost(S->pinned));
            S->pinned = nullptr;
        }
        // page-locked allocations cost about a millisecond each: start at 1 MiB, grow 4x
        const size_t sz = std::max<size_t>({bytes, 4 * S->pinned_bytes, size_t(1) << 20});
        GB_CUDA(cudaHostAlloc(&S->pinned, sz, cudaHostAllocDefault));
        S->pinned_bytes = sz;
    }
    return S->pinned;
}

void sync(gb_system *S) {
    GB_CUDA(cudaStreamSynchronize(S->stream));
    S->ctx->arena.flush(S->stream);
}

// ---- critical pairs: UPDATE of Becker and Weispfenning (Gebauer-Moeller criteria) --------------
//
// Leading monomials are compared as SWAR words (internal.hpp) while every exponent is below 128;
// beyond that the bytewise routines above are used.  Pair lcms are cached with the pair.

namespace {
struct MonoOps {
    int n;
    bool swar;
    bool divides(const M16 &a, const M16 &b, const Mono &ma, const Mono &mb) const {
        return swar ? divides16(a, b) : mono_divides(ma, mb, n);
    }
};
}  // namespace

static void gm_update(gb_system *S, uint32_t h) {
    const int n = (int)S->n;
    const Mono &lh = S->lm[h];
    const M16 lh16 = S->lm16[h];
    const bool swar = S->swar;
    auto lcm_of = [&](uint32_t a, uint32_t b) -> M16 {
        if (swar) return lcm16(S->lm16[a], S->lm16[b]);
        return m16(mono_lcm(S->lm[a], S->lm[b], n));
    };
    auto divides = [&](const M16 &a, const M16 &b) -> bool {
        if (swar) return divides16(a, b);
        Mono x, y;
        std::memcpy(x.e, &a, 16);
        std::memcpy(y.e, &b, 16);
        return mono_divides(x, y, n);
    };
    auto coprime = [&](uint32_t a) -> bool {
        return swar ? coprime16(lh16, S->lm16[a]) : mono_coprime(lh, S->lm[a], n);
    };
    std::vector<uint32_t> C;
    C.reserve(h);
    for (uint32_t g = 0; g < h; ++g)
        if (!S->redundant[g]) C.push_back(g);
    std::vector<M16> L(C.size());
    for (size_t a = 0; a < C.size(); ++a) L[a] = lcm_of(h, C[a]);
    // pairs (h, g), oldest g first: keep one when its leading monomials are coprime, or when no
    // pair still waiting or already kept has an lcm dividing its lcm
    std::vector<char> kept(C.size(), 0), cop(C.size(), 0);
    for (size_t a = 0; a < C.size(); ++a) {
        cop[a] = coprime(C[a]);
        bool keep = true;
        if (!cop[a]) {
            for (size_t b = a + 1; b < C.size() && keep; ++b)
                if (divides(L[b], L[a])) keep = false;
            for (size_t b = 0; b < a && keep; ++b)
                if (kept[b] && divides(L[b], L[a])) keep = false;
        }
        kept[a] = keep;
    }
    // old pairs whose lcm LM(h) divides, with both lcm(g1, h) and lcm(g2, h) different, go
    size_t w = 0;
    for (size_t q = 0; q < S->pairs.size(); ++q) {
        const PairL &pr = S->pairs[q];
        bool drop = divides(lh16, pr.lcm);
        if (drop) drop = !(lcm_of(pr.i, h) == pr.lcm) && !(lcm_of(pr.j, h) == pr.lcm);
        if (!drop) S->pairs[w++] = pr;
    }
    S->pairs.resize(w);
    // kept new pairs, except those with coprime leading monomials (Buchberger's product criterion)
    for (size_t a = 0; a < C.size(); ++a)
        if (kept[a] && !cop[a]) {
            PairL pr{C[a], h, 0, 0, L[a]};
            Mono l;
            std::memcpy(l.e, &L[a], 16);
            pr.deg = (uint32_t)mono_deg(l, n);
            S->pairs.push_back(pr);
        }
    for (uint32_t g = 0; g < h; ++g)
        if (!S->redundant[g] && divides(lh16, S->lm16[g])) S->redundant[g] = 1;
}

// record a new leading monomial (SWAR form, and whether the fast comparisons still apply)
static void push_lm(gb_system *S, const Mono &m) {
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
    std::sort(rows.begin(), rows.end(), [n](const R &a, const R &b) {
        const int c = mono_cmp(a.lm, b.lm, n);
        if (c) return c > 0;
        if (a.k != b.k) return a.k < b.k;
        return mono_cmp(a.t, b.t, n) < 0;
    });
    std::vector<RowSpec> out;
    for (size_t i = 0; i < rows.size(); ++i) {
        if (i && rows[i].k == rows[i - 1].k && rows[i].t == rows[i - 1].t) continue;
        const bool first = out.empty() || !(rows[i].lm == mono_mul(out.back().t, S->lm[out.back().k], n));
        out.push_back(RowSpec{rows[i].t, rows[i].k, (uint8_t)(first ? 1 : 0), 0});
    }
    return out;
}

// upload one normalised polynomial (host terms) as a new basis element and run UPDATE
static void append_host_poly(gb_system *S, const std::vector<Mono> &mon, const std::vector<uint32_t> &cf) {
    Arena &ar = S->ctx->arena;
    cudaStream_t st = S->stream;
    const uint32_t len = (uint32_t)mon.size();
    const uint64_t base = S->nterms;
    const size_t ng0 = S->off.size();
    if (base + len > S->bmon.n) {
        S->bmon.grow(ar, std::max<size_t>(base + len, std::max<size_t>(1024, 2 * S->bmon.n)), base, st);
        S->bcf.grow(ar, std::max<size_t>(base + len, std::max<size_t>(1024, 2 * S->bcf.n)), base, st);
    }
    if (ng0 + 1 > S->boff.n) {
        S->boff.grow(ar, std::max<size_t>(ng0 + 1, std::max<size_t>(64, 2 * S->boff.n)), ng0, st);
        S->blen.grow(ar, std::max<size_t>(ng0 + 1, std::max<size_t>(64, 2 * S->blen.n)), ng0, st);
    }
    char *h = static_cast<char *>(pinned(S, 20ull * len + 64));
    sync(S);  // earlier uploads from the staging buffer have landed
    std::vector<uint4> m4(len);
    for (uint32_t j = 0; j < len; ++j) m4[j] = to_u4(mon[j]);
    std::memcpy(h, m4.data(), 16ull * len);
    std::memcpy(h + 16ull * len, cf.data(), 4ull * len);
    uint32_t *ol = reinterpret_cast<uint32_t *>(h + 20ull * len);
    ol[0] = (uint32_t)base;
    ol[1] = len;
    GB_CUDA(cudaMemcpyAsync(S->bmon.p + base, h, 16ull * len, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaMemcpyAsync(S->bcf.p + base, h + 16ull * len, 4ull * len, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaMemcpyAsync(S->boff.p + ng0, ol, 4, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaMemcpyAsync(S->blen.p + ng0, ol + 1, 4, cudaMemcpyHostToDevice, st));
    sync(S);
    S->nterms = base + len;
    S->off.push_back((uint32_t)base);
    S->len.push_back(len);
    push_lm(S, mon[0]);
    if (mono_deg(mon[0], (int)S->n) == 0) S->unit = true;
    gm_update(S, (uint32_t)(S->lm.size() - 1));
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
    for (uint32_t i = 0; F && i < F->npolys; ++i) {
        const uint32_t a = F->poly_off[i], b = F->poly_off[i + 1];
        if (b < a) fail(GB_EINVAL, "poly_off must be non-decreasing");
        std::vector<std::pair<Mono, uint32_t>> t;
        for (uint32_t q = a; q < b; ++q) {
            Mono m{};
            std::memcpy(m.e, F->exps + (size_t)q * n, n);
            t.emplace_back(m, F->coeffs[q] % p);
        }
        std::sort(t.begin(), t.end(), [n](const auto &x, const auto &y) { return mono_cmp(x.first, y.first, n) > 0; });
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
        append_host_poly(S, mon, cf);
    }
    // footprint estimate for admission control: the basis plus a few dense step matrices
    uint64_t terms = 0;
    for (uint32_t l : S->len) terms += l;
    const uint64_t N = [&] {
        uint64_t r = 1;
        for (uint32_t i = 1; i <= nvars; ++i) r = r * (nvars + 2 + i) / i;  // C(n + 3, n)
        return r;
    }();
    S->footprint = (size_t)(64ull << 20) + (size_t)(terms * 20 * 64) + (size_t)(N * N / 4);
}

// ---- one F4 step ------------------------------------------------------------------------------

gb_status f4_step(gb_system *S, gb_step_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    if (S->pairs.empty()) return GB_DONE;
    const int n = (int)S->n;
    // normal strategy: every pair of minimal lcm degree
    uint32_t dmin = UINT32_MAX;
    for (const PairL &q : S->pairs) dmin = std::min(dmin, q.deg);
    if (dmin > 255) fail(GB_EOVERFLOW, "step degree above 255");
    std::vector<std::pair<Mono, uint32_t>> tk;
    std::vector<PairL> rest;
    uint32_t npairs = 0;
    for (const PairL &q : S->pairs) {
        if (q.deg != dmin) { rest.push_back(q); continue; }
        ++npairs;
        Mono l;
        std::memcpy(l.e, &q.lcm, 16);
        tk.emplace_back(mono_div(l, S->lm[q.i], n), q.i);
        tk.emplace_back(mono_div(l, S->lm[q.j], n), q.j);
    }
    S->pairs.swap(rest);
    std::vector<RowSpec> rows = order_rows(S, std::move(tk));
    const auto ts = std::chrono::steady_clock::now();
    auto mac = symbolic_preprocess(S, rows, true, nonredundant(S));
    auto ech = reduce_rows(mac.get(), true);
    const auto t1 = std::chrono::steady_clock::now();
    std::vector<Mono> lms;
    std::vector<uint32_t> lens;
    append_echelon(S, ech.get(), lms, lens);
    const auto tp = std::chrono::steady_clock::now();
    for (size_t e = 0; e < lms.size(); ++e) {
        push_lm(S, lms[e]);
        if (mono_deg(lms[e], n) == 0) S->unit = true;
        gm_update(S, (uint32_t)(S->lm.size() - 1));
    }
    const auto t2 = std::chrono::steady_clock::now();
    S->steps++;
    gb_step_stats st{};
    st.step = S->steps;
    st.degree = (uint32_t)dmin;
    st.npairs = npairs;
    st.nrows = mac->nrows;
    st.ndict = mac->ndict;
    st.npivot = mac->nA;
    st.nC = mac->nC;
    st.nb = mac->nb;
    st.rank = ech->rank;
    st.nbasis = (uint32_t)S->lm.size();
    st.closure_rounds = mac->closure_rounds;
    st.nnz = mac->nnz;
    st.axpy_rows = ech->work[0];
    st.axpy_fma = ech->work[1];
    st.ms_sp = mac->ms_sp;
    st.ms_reduce = ech->ms_reduce;
    st.ms_rref = ech->ms_rref;
    st.ms_update = (float)std::chrono::duration<double, std::milli>(tp - t1).count();
    st.ms_pairs = (float)std::chrono::duration<double, std::milli>(t2 - tp).count();
    st.ms_select = (float)std::chrono::duration<double, std::milli>(ts - t0).count();
    st.ms_wall = std::chrono::duration<double, std::milli>(t2 - t0).count();
    S->run.steps = S->steps;
    S->run.nnz_total += st.nnz;
    S->run.axpy_rows += st.axpy_rows;
    S->run.axpy_fma += st.axpy_fma;
    S->run.ms_sp += st.ms_sp;
    S->run.ms_reduce += st.ms_reduce;
    S->run.ms_rref += st.ms_rref;
    S->run.ms_update += st.ms_update;
    S->run.ms_pairs += st.ms_pairs;
    S->run.ms_select += st.ms_select;
    S->run.ms_wall += st.ms_wall;
    if (stats) *stats = st;
    if (S->ctx->flags & GB_CTX_KEEP_STEP) {
        S->last_ech = std::move(ech);
        S->last_mac = std::move(mac);
    }
    return GB_OK;
}

// ---- the reduced basis ------------------------------------------------------------------------

void finish(gb_system *S) {
    const auto t0 = std::chrono::steady_clock::now();
    const int n = (int)S->n;
    const uint32_t ng = (uint32_t)S->lm.size();
    std::vector<uint32_t> keep;
    for (uint32_t i = 0; i < ng; ++i) {
        if (S->redundant[i]) continue;
        bool drop = false;
        for (uint32_t j = 0; j < ng && !drop; ++j) {
            if (j == i || S->redundant[j]) continue;
            if (mono_divides(S->lm[j], S->lm[i], n) && (!(S->lm[j] == S->lm[i]) || j < i)) drop = true;
        }
        if (!drop) keep.push_back(i);
    }
    // final order: leading monomials descending
    std::sort(keep.begin(), keep.end(), [&](uint32_t a, uint32_t b) { return mono_cmp(S->lm[a], S->lm[b], n) > 0; });
    std::vector<uint32_t> off{0};
    std::vector<uint8_t> exps;
    std::vector<uint32_t> cf;
    if (!keep.empty()) {
        // the tails t(g) = g - LM(g), reduced by the minimal basis with the same pipeline: the
        // closure supplies reducer rows for every tail monomial a leading monomial divides, and the
        // sparse reduction leaves each tail with non-pivot (standard) monomials only
        std::vector<RowSpec> rows;
        for (uint32_t g : keep) rows.push_back(RowSpec{Mono{}, g, 0, 1});
        auto mac = symbolic_preprocess(S, rows, true, keep);
        auto ech = reduce_rows(mac.get(), false);
        replace_tails(S, ech.get(), keep, off, exps, cf);
        S->run.ms_sp += mac->ms_sp;
        S->run.ms_reduce += ech->ms_reduce;
        S->run.nnz_total += mac->nnz;
        S->run.axpy_rows += ech->work[0];
        S->run.axpy_fma += ech->work[1];
    }
    S->fin_off.swap(off);
    S->fin_exps.swap(exps);
    S->fin_cf.swap(cf);
    S->finished = true;
    S->run.nbasis = (uint32_t)keep.size();
    S->run.ms_wall += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

gb_status groebner(gb_system *S, gb_run_stats *stats) {
    if (!S->finished) {
        while (f4_step(S, nullptr) == GB_OK) {
        }
        finish(S);
    }
    if (stats) *stats = S->run;
    return GB_OK;
}

}  // namespace gb
