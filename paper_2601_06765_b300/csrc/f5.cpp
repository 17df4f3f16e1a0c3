// f5.cpp -- Groebner bases of homogeneous systems through signature-filtered Macaulay matrices:
// the signature regime of the paper (Thm. signature-sound; Sec. 14, "GPU-facing reformulation")
// with the F5 criterion as the admissibility predicate, degree by degree.
//
// For d = least input degree .. dmax and each generator i (input order) with d_i <= d, block
// (d, i) is one pass of the ordinary pipeline:
//   candidates   x^a f_i for every monomial x^a of degree e = d - d_i (signature x^a e_i);
//   Adm          on the device (sig.cu): x^a must not be a leading monomial of the degree-e part
//                of <f_1 .. f_{i-1}>, the set L(i-1, e) kept from the blocks of degree e as a
//                bitmap over the candidate positions; the survivors are compacted by a scan;
//   rows         the echelon rows of degree d so far (basis elements, or shifted inputs whose
//                leading monomial was new) and the admissible candidates;
//   SP           symbolic preprocessing without closure: every row is given, and the rows of
//                degree d already span the earlier generators' part of degree d;
//   reduction    A6 and the RREF of D' (A7); the new elements join the device basis (A8).
// L(i, d) then holds the leading monomials of the block's rows and of its new elements.  The
// criterion removes only rows that rows of smaller signature span: if x^a = LM(h) with
// h = sum_{j<i} q_j f_j, then LC(h) x^a f_i = sum_j q_j f_i f_j - (h - LC(h) x^a) f_i.  So the
// rows of degree d span the degree-d part of <f_1 .. f_i> after block (d, i), and for a regular
// sequence no admissible row reduces to zero (F5's theorem).  After the last degree the elements
// whose leading monomials are minimal go through the reduction of tails (finish_batch), as at the
// end of an F4 run.
#include <chrono>
#include <unordered_map>

#include "internal.hpp"

namespace gb {

namespace {

struct MonoHash {
    size_t operator()(const Mono &m) const {
        uint64_t a, b;
        std::memcpy(&a, m.e, 8);
        std::memcpy(&b, m.e + 8, 8);
        return (size_t)((a * 0x9E3779B97F4A7C15ull) ^ (b + 0x632BE59BD9B4E019ull + (a >> 29)));
    }
};

// the monomials of one degree in descending grevlex order, and their positions
struct DegreeTable {
    std::vector<Mono> mons;
    std::unordered_map<Mono, uint32_t, MonoHash> at;
};

void compositions(int n, int k, int left, Mono &cur, std::vector<Mono> &out) {
    if (k == n - 1) {
        cur.e[k] = (uint8_t)left;
        out.push_back(cur);
        return;
    }
    for (int a = left; a >= 0; --a) {
        cur.e[k] = (uint8_t)a;
        compositions(n, k + 1, left - a, cur, out);
    }
    cur.e[k] = 0;
}

struct Bits {
    std::vector<uint32_t> w;
    explicit Bits(size_t n = 0) : w((n + 31) / 32, 0u) {}
    bool test(uint32_t j) const { return (w[j >> 5] >> (j & 31u)) & 1u; }
    void set(uint32_t j) { w[j >> 5] |= 1u << (j & 31u); }
};

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point a) { return std::chrono::duration<double, std::milli>(Clock::now() - a).count(); }

}  // namespace

void f5_groebner(gb_system *S, uint32_t dmax, uint32_t flags, std::vector<gb_f5_block> *blocks, gb_f5_stats *stats) {
    if (S->steps || S->resident || S->finished) fail(GB_EINVAL, "the signature-filtered run needs a fresh system");
    if (S->deglex) fail(GB_EUNSUPPORTED, "the signature-filtered run is for grevlex");
    if (dmax > 255) fail(GB_EINVAL, "dmax above 255");
    gb_ctx *ctx = S->ctx;
    const int n = (int)S->n;
    const auto t_run = Clock::now();
    const uint32_t m = (uint32_t)S->lm.size();
    std::vector<uint32_t> dg(m);
    uint32_t dmin = 255;
    for (uint32_t g = 0; g < m; ++g) {
        dg[g] = (uint32_t)mono_deg(S->lm[g], n);
        for (uint32_t q = S->off[g]; q < S->off[g] + S->len[g]; ++q) {
            Mono t;
            std::memcpy(t.e, &S->in_mon[q], 16);
            if ((uint32_t)mono_deg(t, n) != dg[g]) fail(GB_EINVAL, "the signature-filtered run takes homogeneous inputs");
        }
        dmin = std::min(dmin, dg[g]);
    }
    if (m && dmax < dmin) fail(GB_EINVAL, "dmax below the least input degree");
    make_resident({S});
    // the inputs' critical pairs and redundancy belong to the F4 loop; here redundancy means a
    // leading monomial that is not a minimal generator of the leading-monomial ideal
    S->pairs.clear();
    std::fill(S->redundant.begin(), S->redundant.end(), 0);
    const bool criterion = !(flags & GB_F5_NO_CRITERION);
    std::vector<DegreeTable> tables(m ? dmax + 1 : 0);
    std::vector<bool> built(tables.size(), false);
    auto table = [&](uint32_t e) -> const DegreeTable & {
        if (!built[e]) {
            Mono cur{};
            if (n == 1) {
                cur.e[0] = (uint8_t)e;
                tables[e].mons.push_back(cur);
            } else {
                compositions(n, 0, (int)e, cur, tables[e].mons);
            }
            std::sort(tables[e].mons.begin(), tables[e].mons.end(),
                      [n](const Mono &a, const Mono &b) { return mono_cmp(a, b, n, false) > 0; });
            for (uint32_t j = 0; j < tables[e].mons.size(); ++j) tables[e].at.emplace(tables[e].mons[j], j);
            built[e] = true;
        }
        return tables[e];
    };
    // L[e][i]: leading monomials of the degree-e part of <f_1 .. f_i> (bit j: the j-th monomial)
    std::vector<std::vector<Bits>> L(tables.size());
    // a leading monomial t of degree d is a minimal generator unless t / x_v lies in L[d-1][m]
    auto minimal = [&](const Mono &t, uint32_t d) {
        if (d == 0 || d - 1 < dmin) return true;
        const DegreeTable &T = table(d - 1);
        for (int v = 0; v < n; ++v) {
            if (!t.e[v]) continue;
            Mono q = t;
            --q.e[v];
            if (L[d - 1][m].test(T.at.at(q))) return false;
        }
        return true;
    };
    gb_f5_stats st{};
    Arena &ar = ctx->arena;
    cudaStream_t s = ctx->stream;
    for (uint32_t d = dmin; m && d <= dmax; ++d) {
        const DegreeTable &T = table(d);
        L[d].assign(m + 1, Bits(T.mons.size()));
        Bits cur(T.mons.size());
        std::vector<std::pair<Mono, uint32_t>> E;  // echelon rows of degree d: (shift, element)
        for (uint32_t i = 1; i <= m; ++i) {
            if (dg[i - 1] > d) {
                L[d][i] = cur;
                continue;
            }
            const uint32_t e = d - dg[i - 1];
            const DegreeTable &C = table(e);
            const uint32_t ncand = (uint32_t)C.mons.size();
            gb_f5_block b{};
            b.degree = d;
            b.index = i;
            b.candidates = ncand;
            // the admissibility filter on the device
            const auto tf = Clock::now();
            DBuf<uint32_t> forb;
            DBuf<unsigned long long> keys;
            const uint32_t *df = nullptr;
            if (criterion && e >= dmin) {
                const Bits &F = L[e][i - 1];
                forb.alloc(ar, F.w.size(), s);
                void *h = ctx_pinned(ctx, 4 * F.w.size());
                std::memcpy(h, F.w.data(), 4 * F.w.size());
                GB_CUDA(cudaMemcpyAsync(forb.p, h, 4 * F.w.size(), cudaMemcpyHostToDevice, s));
                df = forb.p;
            }
            keys.alloc(ar, std::max<uint32_t>(ncand, 1), s);
            const uint32_t nadm = sig_filter(ctx, i, e, ncand, df, keys.p);
            std::vector<unsigned long long> hk(nadm);
            if (nadm) {
                void *h = ctx_pinned(ctx, 8ull * nadm);
                GB_CUDA(cudaMemcpyAsync(h, keys.p, 8ull * nadm, cudaMemcpyDeviceToHost, s));
                ctx_sync(ctx);
                std::memcpy(hk.data(), h, 8ull * nadm);
            }
            b.admissible = nadm;
            b.ms_filter = (float)ms_since(tf);
            // the block's rows; candidates whose leading monomial is new at this degree stay as
            // echelon rows of degree d (the first row of a leading monomial is its pivot)
            std::vector<std::pair<Mono, uint32_t>> rows(E);
            std::vector<uint32_t> fresh;  // positions (degree d) of the candidates' new leading monomials
            std::vector<std::pair<Mono, uint32_t>> fresh_rows;
            bool input_new = false, input_adm = false;
            for (unsigned long long k : hk) {
                const uint32_t j = (uint32_t)(k & 0xFFFFFFFFull);
                rows.emplace_back(C.mons[j], i - 1);
                const uint32_t at = T.at.at(mono_mul(C.mons[j], S->lm[i - 1], n));
                if (e == 0) input_adm = true;
                if (!cur.test(at)) {
                    fresh.push_back(at);
                    fresh_rows.emplace_back(C.mons[j], i - 1);
                    if (e == 0) input_new = true;
                }
            }
            b.rows = (uint32_t)rows.size();
            uint32_t added = 0;
            if (nadm) {
                std::vector<SpTask> tasks(1);
                tasks[0].S = S;
                tasks[0].rows = order_rows(S, std::move(rows));
                tasks[0].closure = false;
                for (uint32_t g = 0; g < S->redundant.size(); ++g)
                    if (!S->redundant[g]) tasks[0].nonred.push_back(g);
                symbolic_preprocess(tasks);
                gb_macaulay *mac = tasks[0].out.get();
                b.ndict = mac->ndict;
                b.npivot = mac->nA;
                b.nC = mac->nC;
                b.ms_sp = mac->ms_sp;
                st.nnz += mac->nnz;
                if (mac->nC) {
                    auto Es = reduce_rows({mac}, true);
                    gb_echelon *ech = Es[0].get();
                    b.ms_reduce = ech->ms_reduce;
                    b.ms_rref = ech->ms_rref;
                    std::vector<std::vector<Mono>> lms;
                    append_echelon({ech}, lms);
                    for (const Mono &t : lms[0]) {
                        push_lm(S, t);
                        const uint32_t g = (uint32_t)S->lm.size() - 1;
                        const uint32_t at = T.at.at(t);
                        cur.set(at);
                        E.emplace_back(Mono{}, g);
                        if (!minimal(t, d)) S->redundant[g] = 1;
                        ++added;
                    }
                }
            }
            for (size_t q = 0; q < fresh.size(); ++q) {
                cur.set(fresh[q]);
                E.push_back(fresh_rows[q]);
            }
            // the input itself: needed only when its leading monomial was new and is minimal
            if (e == 0 && !(input_adm && input_new && minimal(S->lm[i - 1], d))) S->redundant[i - 1] = 1;
            b.rank = added;
            b.zero_reductions = nadm - (uint32_t)(added + fresh.size());
            L[d][i] = cur;
            st.blocks++;
            st.candidates += b.candidates;
            st.admissible += b.admissible;
            st.zero_reductions += b.zero_reductions;
            st.ms_filter += b.ms_filter;
            st.ms_sp += b.ms_sp;
            st.ms_reduce += b.ms_reduce;
            st.ms_rref += b.ms_rref;
            if (blocks) blocks->push_back(b);
        }
    }
    const auto tfin = Clock::now();
    finish_batch({S});
    st.ms_finish = ms_since(tfin);
    st.nbasis = S->run.nbasis;
    st.ms_wall = ms_since(t_run);
    if (stats) *stats = st;
}

}  // namespace gb
