/*
 * f4_oracle.c -- THE ORACLE.  Test infrastructure only.
 *
 * A plain, slow, single-threaded CPU implementation of the F4 method over F_p in the graded
 * reverse lexicographic order (x1 > x2 > ... > xn).  Only tests/, the package's smoke check and
 * bench.py's CPU-baseline leg may load it.  It shares no code, header, table or helper with the
 * CUDA path; the two meet only in the seeded input systems.
 *
 * It follows the paper step by step, in the paper's notation:
 *   - batch reduction by a Macaulay matrix whose rows are shifted reducers t*g (Sec. 2.3, Def. 3.1);
 *   - symbolic preprocessing SP : batch -> (T, R, Pi) with the one-step reduction closure
 *     (Def. 5.2, Rem. 3.3, the support-closure definition of Sec. 11) and the dictionary
 *     T = Sort(Set(M(R))) (Sec. 5.1);
 *   - CSR layout Pi = (row_ptr, col_ind, val, dict_keys, row_meta) (Def. 5.2, the FBSP algorithm (Sec. 10));
 *   - structured elimination: pivot / non-pivot split, row reduction of the non-pivot rows by the
 *     pivot rows, then reduced echelon form of the remaining block (Sec. 9.2);
 *   - reconstruction of new basis elements and the basis update (Sec. 4.2, step 4).
 * Arithmetic is the plain definition: (a*b) % p in 64-bit integers, inverses by the extended
 * Euclidean algorithm.  No Montgomery or Barrett form (Sec. 8 describes those for the GPU side).
 *
 * Readings of points the paper leaves open (each is fixed identically, but independently, in the
 * CUDA path's host control):
 *   R1 grevlex with x1 > ... > xn: x^a > x^b iff deg a > deg b, or the degrees agree and the last
 *      nonzero entry of a - b is negative.  With the flag OR_DEGLEX the other graded order of
 *      Sec. 7.3, deglex: the same degree comparison, ties broken lexicographically (the first
 *      nonzero entry of a - b is positive).
 *   R2 inputs are normalised: duplicate monomials merged mod p, zero terms and zero polynomials
 *      dropped, each polynomial made monic, terms sorted descending.
 *   R3 pairs are created and pruned with the Gebauer-Moeller update (Becker-Weispfenning 1993,
 *      UPDATE), inserting inputs in input order and new elements in echelon-row order.
 *   R4 selection: every pair of minimal lcm degree (the normal strategy).
 *   R5 reducer for a monomial m: the oldest (smallest index) non-redundant g with LM(g) | m.
 *   R6 dictionary descending, 0-based columns (column 0 = largest monomial).
 *   R7 row order: pivot rows first by leading column, then the other rows by (leading column, k).
 *      For a leading monomial with no reducer row, the pair row with the smallest k is the pivot.
 *   R8 new elements: the rows of the reduced echelon form of the reduced non-pivot block, in order.
 *   R9 final basis: minimalised, tails fully reduced, monic, sorted by leading monomial descending.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORN 16 /* maximum number of variables */

typedef struct { uint8_t e[ORN]; } omono;

typedef struct {
    int len;
    omono *mon;   /* descending */
    uint32_t *cf; /* in [0, p) */
} opoly;

typedef struct { int i, j; } opair;

typedef struct {
    omono t;     /* shift */
    int k;       /* basis index */
    int reducer; /* 1: added by the closure, 0: half of a selected pair */
    int lm_col;  /* dictionary column of LM(t*g_k) */
    int pivot;   /* 1: pivot row */
} orow;

typedef struct {
    int n;
    uint32_t p;
    int flags;
    /* basis */
    int ng, capg;
    opoly *g;
    uint8_t *redundant;
    /* pairs */
    int np, capp;
    opair *pairs;
    /* progress */
    int steps;
    int finished;
    /* last step (row order as in R7) */
    int last_degree, last_npairs;
    int nrows, ndict, nA, nC, nb, rank;
    int64_t nnz;
    omono *dict;
    orow *rows;
    uint32_t *row_ptr, *col, *val;
    uint32_t *nonpiv; /* nb dictionary columns */
    uint32_t *dprime; /* nC x nb */
    uint32_t *rref;   /* rank x nb */
    uint32_t *rpiv;   /* rank positions in [0, nb) */
    uint8_t *red_snapshot; /* redundant flags when the step's rows were chosen */
    int ng_snapshot;
    /* final reduced basis */
    int nfinal;
    opoly *fin;
} osys;

enum { OR_ONE_PAIR = 1, OR_NEWEST_REDUCER = 2, OR_DEGLEX = 4 };

/* R1: the term order of the system being worked on, set from its flags by every entry point that
   compares monomials (the oracle is single-threaded) */
static int g_deglex;

/* ---------------- monomials (R1) ---------------- */

static int m_deg(const omono *a, int n) {
    int d = 0;
    for (int i = 0; i < n; ++i) d += a->e[i];
    return d;
}

/* +1 if a > b, -1 if a < b, 0 if equal, in grevlex (or deglex) with x1 > ... > xn */
static int m_cmp(const omono *a, const omono *b, int n) {
    int da = m_deg(a, n), db = m_deg(b, n);
    if (da != db) return da > db ? 1 : -1;
    if (g_deglex) {
        for (int i = 0; i < n; ++i)
            if (a->e[i] != b->e[i]) return a->e[i] > b->e[i] ? 1 : -1;
        return 0;
    }
    for (int i = n - 1; i >= 0; --i)
        if (a->e[i] != b->e[i]) return a->e[i] < b->e[i] ? 1 : -1;
    return 0;
}

static int m_eq(const omono *a, const omono *b, int n) { return memcmp(a->e, b->e, (size_t)n) == 0; }

static omono m_mul(const omono *a, const omono *b, int n) {
    omono r;
    memset(&r, 0, sizeof r);
    for (int i = 0; i < n; ++i) r.e[i] = (uint8_t)(a->e[i] + b->e[i]);
    return r;
}

static int m_divides(const omono *a, const omono *b, int n) { /* a | b */
    for (int i = 0; i < n; ++i)
        if (a->e[i] > b->e[i]) return 0;
    return 1;
}

static omono m_div(const omono *b, const omono *a, int n) { /* b / a, a | b */
    omono r;
    memset(&r, 0, sizeof r);
    for (int i = 0; i < n; ++i) r.e[i] = (uint8_t)(b->e[i] - a->e[i]);
    return r;
}

static omono m_lcm(const omono *a, const omono *b, int n) {
    omono r;
    memset(&r, 0, sizeof r);
    for (int i = 0; i < n; ++i) r.e[i] = a->e[i] > b->e[i] ? a->e[i] : b->e[i];
    return r;
}

static int m_coprime(const omono *a, const omono *b, int n) {
    for (int i = 0; i < n; ++i)
        if (a->e[i] && b->e[i]) return 0;
    return 1;
}

/* ---------------- F_p (plain definitions) ---------------- */

static uint32_t f_mul(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }

static uint32_t f_inv(uint32_t a, uint32_t p) { /* extended Euclid, a != 0 */
    int64_t r0 = p, r1 = a, s0 = 0, s1 = 1;
    while (r1) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    s0 %= (int64_t)p;
    if (s0 < 0) s0 += p;
    return (uint32_t)s0;
}

/* ---------------- small containers ---------------- */

static void *xrealloc(void *ptr, size_t bytes) {
    void *q = realloc(ptr, bytes ? bytes : 1);
    if (!q) abort();
    return q;
}

static void poly_free(opoly *f) {
    free(f->mon);
    free(f->cf);
    f->mon = NULL;
    f->cf = NULL;
    f->len = 0;
}

typedef struct { omono m; uint32_t c; } oterm;

static int term_cmp_desc(const void *x, const void *y, void *ctx) {
    int n = *(const int *)ctx;
    return -m_cmp(&((const oterm *)x)->m, &((const oterm *)y)->m, n);
}

/* R2: sort descending, merge equal monomials mod p, drop zeros, make monic. */
static opoly poly_normalise(oterm *t, int len, int n, uint32_t p) {
    opoly f = {0, NULL, NULL};
    qsort_r(t, (size_t)len, sizeof(oterm), term_cmp_desc, &n);
    oterm *w = (oterm *)xrealloc(NULL, sizeof(oterm) * (size_t)(len ? len : 1));
    int k = 0;
    for (int i = 0; i < len;) {
        uint64_t c = 0;
        int j = i;
        while (j < len && m_eq(&t[j].m, &t[i].m, n)) c = (c + t[j++].c) % p;
        if (c) { w[k].m = t[i].m; w[k].c = (uint32_t)c; ++k; }
        i = j;
    }
    if (k) {
        uint32_t inv = f_inv(w[0].c, p);
        f.len = k;
        f.mon = (omono *)xrealloc(NULL, sizeof(omono) * (size_t)k);
        f.cf = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)k);
        for (int i = 0; i < k; ++i) { f.mon[i] = w[i].m; f.cf[i] = f_mul(w[i].c, inv, p); }
    }
    free(w);
    return f;
}

/* ---------------- monomial hash set (a plain set, for T and Done) ---------------- */

typedef struct {
    omono *key;
    uint8_t *used;
    size_t cap, cnt;
    int n;
} oset;

static uint64_t m_hash(const omono *a, int n) { /* FNV-1a */
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < n; ++i) { h ^= a->e[i]; h *= 1099511628211ull; }
    return h;
}

static void set_init(oset *s, int n, size_t cap) {
    size_t c = 64;
    while (c < 2 * cap) c <<= 1;
    s->cap = c;
    s->cnt = 0;
    s->n = n;
    s->key = (omono *)xrealloc(NULL, sizeof(omono) * c);
    s->used = (uint8_t *)calloc(c, 1);
    if (!s->used) abort();
}

static void set_free(oset *s) { free(s->key); free(s->used); }

static int set_insert(oset *s, const omono *m); /* returns 1 if new */

static void set_grow(oset *s) {
    oset t;
    set_init(&t, s->n, s->cap);
    for (size_t i = 0; i < s->cap; ++i)
        if (s->used[i]) set_insert(&t, &s->key[i]);
    set_free(s);
    *s = t;
}

static int set_insert(oset *s, const omono *m) {
    if (2 * (s->cnt + 1) > s->cap) set_grow(s);
    size_t mask = s->cap - 1, h = (size_t)m_hash(m, s->n) & mask;
    while (s->used[h]) {
        if (m_eq(&s->key[h], m, s->n)) return 0;
        h = (h + 1) & mask;
    }
    s->used[h] = 1;
    s->key[h] = *m;
    s->cnt++;
    return 1;
}

static int set_has(const oset *s, const omono *m) {
    size_t mask = s->cap - 1, h = (size_t)m_hash(m, s->n) & mask;
    while (s->used[h]) {
        if (m_eq(&s->key[h], m, s->n)) return 1;
        h = (h + 1) & mask;
    }
    return 0;
}

/* ---------------- basis and the Gebauer-Moeller update (R3) ---------------- */

static void add_pair(osys *S, int i, int j) {
    if (S->np == S->capp) {
        S->capp = S->capp ? 2 * S->capp : 64;
        S->pairs = (opair *)xrealloc(S->pairs, sizeof(opair) * (size_t)S->capp);
    }
    S->pairs[S->np].i = i;
    S->pairs[S->np].j = j;
    S->np++;
}

/* UPDATE(G, B, h) of Becker-Weispfenning: h = g[hidx] is already stored in the basis array. */
static void gm_update(osys *S, int hidx) {
    int n = S->n;
    const omono *lh = &S->g[hidx].mon[0];
    /* C: pairs (h, g) for the non-redundant g, oldest first */
    int nc = 0;
    int *C = (int *)xrealloc(NULL, sizeof(int) * (size_t)(hidx + 1));
    for (int g = 0; g < hidx; ++g)
        if (!S->redundant[g]) C[nc++] = g;
    omono *L = (omono *)xrealloc(NULL, sizeof(omono) * (size_t)(nc + 1));
    for (int a = 0; a < nc; ++a) L[a] = m_lcm(lh, &S->g[C[a]].mon[0], n);
    uint8_t *keepD = (uint8_t *)calloc((size_t)nc + 1, 1);
    /* first loop: keep (h,g1) if coprime, or if its lcm is divisible by no lcm of a pair still
       waiting in C or already accepted into D */
    for (int a = 0; a < nc; ++a) {
        int keep = 1;
        if (!m_coprime(lh, &S->g[C[a]].mon[0], n)) {
            for (int b = a + 1; b < nc && keep; ++b)
                if (m_divides(&L[b], &L[a], n)) keep = 0;
            for (int b = 0; b < a && keep; ++b)
                if (keepD[b] && m_divides(&L[b], &L[a], n)) keep = 0;
        }
        keepD[a] = (uint8_t)keep;
    }
    /* old pairs: drop (g1,g2) when LM(h) | lcm(g1,g2) and both lcm(g1,h), lcm(g2,h) differ */
    int w = 0;
    for (int q = 0; q < S->np; ++q) {
        const omono *a = &S->g[S->pairs[q].i].mon[0], *b = &S->g[S->pairs[q].j].mon[0];
        omono l12 = m_lcm(a, b, n), l1h = m_lcm(a, lh, n), l2h = m_lcm(b, lh, n);
        int drop = m_divides(lh, &l12, n) && !m_eq(&l1h, &l12, n) && !m_eq(&l2h, &l12, n);
        if (!drop) S->pairs[w++] = S->pairs[q];
    }
    S->np = w;
    /* second loop (product criterion): accepted pairs with coprime leading monomials are dropped */
    for (int a = 0; a < nc; ++a)
        if (keepD[a] && !m_coprime(lh, &S->g[C[a]].mon[0], n)) add_pair(S, C[a], hidx);
    /* basis: elements whose LM is divisible by LM(h) become redundant */
    for (int g = 0; g < hidx; ++g)
        if (!S->redundant[g] && m_divides(lh, &S->g[g].mon[0], n)) S->redundant[g] = 1;
    free(C);
    free(L);
    free(keepD);
}

static void basis_append(osys *S, opoly f) {
    if (S->ng == S->capg) {
        S->capg = S->capg ? 2 * S->capg : 64;
        S->g = (opoly *)xrealloc(S->g, sizeof(opoly) * (size_t)S->capg);
        S->redundant = (uint8_t *)xrealloc(S->redundant, (size_t)S->capg);
    }
    S->g[S->ng] = f;
    S->redundant[S->ng] = 0;
    S->ng++;
    gm_update(S, S->ng - 1);
}

/* ---------------- one F4 step ---------------- */

static int row_cmp_kt(const void *x, const void *y, void *ctx) {
    const orow *a = (const orow *)x, *b = (const orow *)y;
    int n = *(const int *)ctx;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    return m_cmp(&a->t, &b->t, n);
}

static int mono_cmp_desc(const void *x, const void *y, void *ctx) {
    return -m_cmp((const omono *)x, (const omono *)y, *(const int *)ctx);
}

typedef struct { const omono *dict; int N, n; } dict_ctx;

static int dict_index(const dict_ctx *D, const omono *m) { /* binary search, descending order */
    int lo = 0, hi = D->N - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2, c = m_cmp(m, &D->dict[mid], D->n);
        if (c == 0) return mid;
        if (c > 0) hi = mid - 1; else lo = mid + 1;
    }
    abort(); /* every row monomial is in T (the dictionary-correctness theorem of Sec. 11) */
}

static int row_cmp_final(const void *x, const void *y) {
    const orow *a = (const orow *)x, *b = (const orow *)y;
    if (a->pivot != b->pivot) return a->pivot ? -1 : 1;
    if (a->lm_col != b->lm_col) return a->lm_col < b->lm_col ? -1 : 1;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    return 0;
}

static void free_last(osys *S) {
    free(S->dict); free(S->rows); free(S->row_ptr); free(S->col); free(S->val);
    free(S->nonpiv); free(S->dprime); free(S->rref); free(S->rpiv); free(S->red_snapshot);
    S->dict = NULL; S->rows = NULL; S->row_ptr = S->col = S->val = NULL;
    S->nonpiv = S->dprime = S->rref = S->rpiv = NULL;
    S->red_snapshot = NULL;
}

static int find_reducer(const osys *S, const omono *m) { /* R5 */
    if (S->flags & OR_NEWEST_REDUCER) {
        for (int g = S->ng - 1; g >= 0; --g)
            if (!S->redundant[g] && m_divides(&S->g[g].mon[0], m, S->n)) return g;
    } else {
        for (int g = 0; g < S->ng; ++g)
            if (!S->redundant[g] && m_divides(&S->g[g].mon[0], m, S->n)) return g;
    }
    return -1;
}

static void push_row(orow **rows, int *nr, int *cap, omono t, int k, int reducer) {
    if (*nr == *cap) {
        *cap = *cap ? 2 * *cap : 256;
        *rows = (orow *)xrealloc(*rows, sizeof(orow) * (size_t)*cap);
    }
    orow *r = &(*rows)[(*nr)++];
    r->t = t; r->k = k; r->reducer = reducer; r->lm_col = -1; r->pivot = 0;
}

/* Returns 1 if a step ran, 0 if no pairs remain. */
/* One non-pivot row of the structured elimination (Sec. 9.2): the row is reduced by the monic
   pivot rows (piv_of_col[c]: the pivot row whose leading column is c, or -1), pivot columns in
   ascending order from the row's leading column `start`; the result is read at the non-pivot
   columns.  acc holds N zeros on entry and on return. */
static void reduce_row(uint32_t p, int N, const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                       const int *piv_of_col, uint64_t *acc, int start, const uint32_t *rcol, const uint32_t *rval,
                       uint32_t rlen, int nb, const uint32_t *nonpiv, uint32_t *out) {
    for (uint32_t q = 0; q < rlen; ++q) acc[rcol[q]] = rval[q];
    for (int c = start; c < N; ++c) {
        uint32_t f = (uint32_t)(acc[c] % p);
        acc[c] = f;
        int pr = piv_of_col[c];
        if (pr < 0 || f == 0) continue;
        uint32_t mf = p - f; /* v <- v - f * pivot row */
        for (uint32_t q = row_ptr[pr]; q < row_ptr[pr + 1]; ++q)
            acc[col[q]] = (acc[col[q]] + (uint64_t)mf * val[q]) % p;
    }
    for (int j = 0; j < nb; ++j) out[j] = (uint32_t)(acc[nonpiv[j]] % p);
    memset(acc, 0, sizeof(uint64_t) * (size_t)N);
}

int or_step(osys *S) {
    int n = S->n;
    uint32_t p = S->p;
    g_deglex = (S->flags & OR_DEGLEX) != 0;
    if (S->np == 0) return 0;
    free_last(S);

    /* R4: selection, all pairs of minimal lcm degree (or one pair in the Buchberger variant) */
    int dmin = 1 << 30;
    for (int q = 0; q < S->np; ++q) {
        omono l = m_lcm(&S->g[S->pairs[q].i].mon[0], &S->g[S->pairs[q].j].mon[0], n);
        int d = m_deg(&l, n);
        if (d < dmin) dmin = d;
    }
    int nr = 0, capr = 0, nsel = 0, w = 0;
    orow *rows = NULL;
    for (int q = 0; q < S->np; ++q) {
        opair pr = S->pairs[q];
        omono l = m_lcm(&S->g[pr.i].mon[0], &S->g[pr.j].mon[0], n);
        int take = m_deg(&l, n) == dmin && !((S->flags & OR_ONE_PAIR) && nsel == 1);
        if (!take) { S->pairs[w++] = pr; continue; }
        nsel++;
        push_row(&rows, &nr, &capr, m_div(&l, &S->g[pr.i].mon[0], n), pr.i, 0);
        push_row(&rows, &nr, &capr, m_div(&l, &S->g[pr.j].mon[0], n), pr.j, 0);
    }
    S->np = w;
    /* duplicate (t, k) rows collapse */
    qsort_r(rows, (size_t)nr, sizeof(orow), row_cmp_kt, &n);
    int u = 0;
    for (int a = 0; a < nr; ++a)
        if (u == 0 || rows[u - 1].k != rows[a].k || !m_eq(&rows[u - 1].t, &rows[a].t, n)) rows[u++] = rows[a];
    nr = u;

    /* Symbolic preprocessing with the one-step reduction closure (Rem. 3.3, the support-closure definition of Sec. 11):
       T = supports of the rows, Done = LMs of the pair rows; every m in T \ Done gets the
       reducer row (m / LM(g), g) of R5, whose support joins T. */
    oset T, Done;
    set_init(&T, n, 1024);
    set_init(&Done, n, 1024);
    int nstack = 0, capstack = 1024;
    omono *stack = (omono *)xrealloc(NULL, sizeof(omono) * (size_t)capstack);
    for (int a = 0; a < nr; ++a) {
        omono lm = m_mul(&rows[a].t, &S->g[rows[a].k].mon[0], n);
        set_insert(&Done, &lm);
    }
    for (int a = 0;; ++a) {
        /* rows grows while we walk it: process every row's support once */
        while (a >= nr && nstack) {
            omono m = stack[--nstack];
            if (set_has(&Done, &m)) continue;
            set_insert(&Done, &m);
            int g = find_reducer(S, &m);
            if (g >= 0) push_row(&rows, &nr, &capr, m_div(&m, &S->g[g].mon[0], n), g, 1);
        }
        if (a >= nr) break;
        const opoly *f = &S->g[rows[a].k];
        for (int j = 0; j < f->len; ++j) {
            omono m = m_mul(&rows[a].t, &f->mon[j], n);
            if (set_insert(&T, &m) && !set_has(&Done, &m)) {
                if (nstack == capstack) {
                    capstack *= 2;
                    stack = (omono *)xrealloc(stack, sizeof(omono) * (size_t)capstack);
                }
                stack[nstack++] = m;
            }
        }
    }
    free(stack);

    /* Dictionary T = Sort(Set(M(R))) descending (Sec. 5.1, R6) */
    int N = (int)T.cnt;
    omono *dict = (omono *)xrealloc(NULL, sizeof(omono) * (size_t)N);
    int d = 0;
    for (size_t i = 0; i < T.cap; ++i)
        if (T.used[i]) dict[d++] = T.key[i];
    qsort_r(dict, (size_t)N, sizeof(omono), mono_cmp_desc, &n);
    set_free(&T);
    set_free(&Done);
    dict_ctx D = {dict, N, n};

    /* Row order (R7) */
    for (int a = 0; a < nr; ++a) {
        omono lm = m_mul(&rows[a].t, &S->g[rows[a].k].mon[0], n);
        rows[a].lm_col = dict_index(&D, &lm);
        rows[a].pivot = rows[a].reducer;
    }
    /* among pair rows sharing a leading column the smallest k is the pivot (no reducer row can
       share it: pair-row LMs start in Done) */
    int *best = (int *)xrealloc(NULL, sizeof(int) * (size_t)N);
    for (int c = 0; c < N; ++c) best[c] = -1;
    for (int a = 0; a < nr; ++a)
        if (!rows[a].reducer) {
            int c = rows[a].lm_col;
            if (best[c] < 0 || rows[a].k < rows[best[c]].k) best[c] = a;
        }
    for (int c = 0; c < N; ++c)
        if (best[c] >= 0) rows[best[c]].pivot = 1;
    free(best);
    qsort(rows, (size_t)nr, sizeof(orow), row_cmp_final);
    int nA = 0;
    while (nA < nr && rows[nA].pivot) ++nA;
    int nC = nr - nA;

    /* CSR in the row order: Pass 1 lengths and exclusive prefix sums, Pass 2 fill (the FBSP algorithm (Sec. 10)) */
    uint32_t *row_ptr = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)(nr + 1));
    row_ptr[0] = 0;
    for (int a = 0; a < nr; ++a) row_ptr[a + 1] = row_ptr[a] + (uint32_t)S->g[rows[a].k].len;
    int64_t M = row_ptr[nr];
    uint32_t *col = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)(M ? M : 1));
    uint32_t *val = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)(M ? M : 1));
    for (int a = 0; a < nr; ++a) {
        const opoly *f = &S->g[rows[a].k];
        for (int j = 0; j < f->len; ++j) {
            omono m = m_mul(&rows[a].t, &f->mon[j], n);
            col[row_ptr[a] + j] = (uint32_t)dict_index(&D, &m);
            val[row_ptr[a] + j] = f->cf[j];
        }
    }

    /* Structured elimination (Sec. 9.2): pivot columns are the leading columns of the pivot rows.
       Each non-pivot row is reduced by the pivot rows, pivot columns in ascending order. */
    int *piv_of_col = (int *)xrealloc(NULL, sizeof(int) * (size_t)N);
    for (int c = 0; c < N; ++c) piv_of_col[c] = -1;
    for (int a = 0; a < nA; ++a) piv_of_col[rows[a].lm_col] = a;
    int nb = 0;
    for (int c = 0; c < N; ++c) nb += piv_of_col[c] < 0;
    uint32_t *nonpiv = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)(nb ? nb : 1));
    int *pos_of_col = (int *)xrealloc(NULL, sizeof(int) * (size_t)N);
    nb = 0;
    for (int c = 0; c < N; ++c) {
        pos_of_col[c] = -1;
        if (piv_of_col[c] < 0) { pos_of_col[c] = nb; nonpiv[nb++] = (uint32_t)c; }
    }
    uint32_t *dprime = (uint32_t *)calloc((size_t)nC * (size_t)nb + 1, sizeof(uint32_t));
    uint64_t *acc = (uint64_t *)calloc((size_t)(N ? N : 1), sizeof(uint64_t));
    for (int i = 0; i < nC; ++i) {
        int a = nA + i;
        reduce_row(p, N, row_ptr, col, val, piv_of_col, acc, rows[a].lm_col, col + row_ptr[a], val + row_ptr[a],
                   row_ptr[a + 1] - row_ptr[a], nb, nonpiv, dprime + (size_t)i * nb);
    }
    free(acc);
    free(piv_of_col);
    free(pos_of_col);

    /* Reduced row echelon form of D' (Gauss-Jordan, column order kept, pivots scaled to 1) */
    uint32_t *R = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * ((size_t)nC * nb + 1));
    memcpy(R, dprime, sizeof(uint32_t) * (size_t)nC * nb);
    uint32_t *rpiv = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)(nC + 1));
    int rank = 0;
    for (int c = 0; c < nb && rank < nC; ++c) {
        int sel = -1;
        for (int i = rank; i < nC; ++i)
            if (R[(size_t)i * nb + c]) { sel = i; break; }
        if (sel < 0) continue;
        if (sel != rank)
            for (int j = 0; j < nb; ++j) {
                uint32_t t = R[(size_t)sel * nb + j];
                R[(size_t)sel * nb + j] = R[(size_t)rank * nb + j];
                R[(size_t)rank * nb + j] = t;
            }
        uint32_t inv = f_inv(R[(size_t)rank * nb + c], p);
        for (int j = c; j < nb; ++j) R[(size_t)rank * nb + j] = f_mul(R[(size_t)rank * nb + j], inv, p);
        for (int i = 0; i < nC; ++i) {
            if (i == rank) continue;
            uint32_t f = R[(size_t)i * nb + c];
            if (!f) continue;
            uint32_t mf = p - f;
            for (int j = c; j < nb; ++j)
                R[(size_t)i * nb + j] = (uint32_t)((R[(size_t)i * nb + j] + (uint64_t)mf * R[(size_t)rank * nb + j]) % p);
        }
        rpiv[rank++] = (uint32_t)c;
    }

    /* keep the step's dumps */
    S->red_snapshot = (uint8_t *)xrealloc(NULL, (size_t)S->ng + 1);
    memcpy(S->red_snapshot, S->redundant, (size_t)S->ng);
    S->ng_snapshot = S->ng;
    S->last_degree = dmin;
    S->last_npairs = nsel;
    S->nrows = nr; S->ndict = N; S->nA = nA; S->nC = nC; S->nb = nb; S->rank = rank; S->nnz = M;
    S->dict = dict; S->rows = rows; S->row_ptr = row_ptr; S->col = col; S->val = val;
    S->nonpiv = nonpiv; S->dprime = dprime; S->rref = R; S->rpiv = rpiv;

    /* Reconstruction (R8): each echelon row is a new monic element, then UPDATE */
    for (int i = 0; i < rank; ++i) {
        int cnt = 0;
        for (int j = 0; j < nb; ++j) cnt += R[(size_t)i * nb + j] != 0;
        opoly f;
        f.len = cnt;
        f.mon = (omono *)xrealloc(NULL, sizeof(omono) * (size_t)cnt);
        f.cf = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)cnt);
        int q = 0;
        for (int j = 0; j < nb; ++j) {
            uint32_t c = R[(size_t)i * nb + j];
            if (c) { f.mon[q] = dict[nonpiv[j]]; f.cf[q] = c; ++q; }
        }
        basis_append(S, f);
    }
    S->steps++;
    return 1;
}

/* ---------------- final reduced basis (R9) ---------------- */

/* Full reduction of f by the set B (a Groebner basis): plain multivariate division, every term. */
static opoly full_reduce(const osys *S, const opoly *f, const int *B, int nB) {
    int n = S->n;
    uint32_t p = S->p;
    int cap = f->len + 16, len = f->len, pos = 0;
    oterm *cur = (oterm *)xrealloc(NULL, sizeof(oterm) * (size_t)cap);
    for (int i = 0; i < len; ++i) { cur[i].m = f->mon[i]; cur[i].c = f->cf[i]; }
    int rlen = 0, rcap = 16;
    oterm *rem = (oterm *)xrealloc(NULL, sizeof(oterm) * (size_t)rcap);
    while (pos < len) {
        oterm lt = cur[pos];
        int h = -1;
        for (int b = 0; b < nB; ++b)
            if (m_divides(&S->g[B[b]].mon[0], &lt.m, n)) { h = B[b]; break; }
        if (h < 0) {
            if (rlen == rcap) { rcap *= 2; rem = (oterm *)xrealloc(rem, sizeof(oterm) * (size_t)rcap); }
            rem[rlen++] = lt;
            ++pos;
            continue;
        }
        /* cur <- cur - lt.c * (lt.m / LM(h)) * h, merging two descending term lists */
        const opoly *g = &S->g[h];
        omono t = m_div(&lt.m, &g->mon[0], n);
        uint32_t mf = p - lt.c;
        int ncap = (len - pos) + g->len + 1;
        oterm *nx = (oterm *)xrealloc(NULL, sizeof(oterm) * (size_t)ncap);
        int a = pos, b = 0, k = 0;
        while (a < len || b < g->len) {
            omono gm;
            int c;
            if (b < g->len) gm = m_mul(&t, &g->mon[b], n);
            if (a >= len) c = -1;
            else if (b >= g->len) c = 1;
            else c = m_cmp(&cur[a].m, &gm, n);
            if (c > 0) { nx[k++] = cur[a++]; }
            else if (c < 0) { nx[k].m = gm; nx[k].c = f_mul(mf, g->cf[b], p); ++k; ++b; }
            else {
                uint32_t v = (uint32_t)((cur[a].c + (uint64_t)mf * g->cf[b]) % p);
                if (v) { nx[k].m = cur[a].m; nx[k].c = v; ++k; }
                ++a; ++b;
            }
        }
        free(cur);
        cur = nx;
        len = k;
        pos = 0;
        cap = ncap;
    }
    free(cur);
    opoly r;
    r.len = rlen;
    r.mon = (omono *)xrealloc(NULL, sizeof(omono) * (size_t)(rlen ? rlen : 1));
    r.cf = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)(rlen ? rlen : 1));
    for (int i = 0; i < rlen; ++i) { r.mon[i] = rem[i].m; r.cf[i] = rem[i].c; }
    free(rem);
    return r;
}

static int fin_cmp(const void *x, const void *y, void *ctx) {
    return -m_cmp(&((const opoly *)x)->mon[0], &((const opoly *)y)->mon[0], *(const int *)ctx);
}

int or_finish(osys *S) {
    int n = S->n;
    g_deglex = (S->flags & OR_DEGLEX) != 0;
    if (S->finished) return 0;
    /* minimalise: drop g_i when another element's LM divides LM(g_i) (older wins on equality) */
    int *B = (int *)xrealloc(NULL, sizeof(int) * (size_t)(S->ng + 1));
    int nB = 0;
    for (int i = 0; i < S->ng; ++i) {
        if (S->redundant[i]) continue;
        int drop = 0;
        for (int j = 0; j < S->ng && !drop; ++j) {
            if (j == i || S->redundant[j]) continue;
            if (m_divides(&S->g[j].mon[0], &S->g[i].mon[0], n) &&
                (!m_eq(&S->g[j].mon[0], &S->g[i].mon[0], n) || j < i))
                drop = 1;
        }
        if (!drop) B[nB++] = i;
    }
    S->fin = (opoly *)xrealloc(NULL, sizeof(opoly) * (size_t)(nB ? nB : 1));
    for (int b = 0; b < nB; ++b) {
        const opoly *g = &S->g[B[b]];
        opoly tail = {g->len - 1, g->mon + 1, g->cf + 1};
        opoly r = full_reduce(S, &tail, B, nB);
        opoly h;
        h.len = r.len + 1;
        h.mon = (omono *)xrealloc(NULL, sizeof(omono) * (size_t)h.len);
        h.cf = (uint32_t *)xrealloc(NULL, sizeof(uint32_t) * (size_t)h.len);
        h.mon[0] = g->mon[0];
        h.cf[0] = 1;
        for (int i = 0; i < r.len; ++i) { h.mon[i + 1] = r.mon[i]; h.cf[i + 1] = r.cf[i]; }
        poly_free(&r);
        S->fin[b] = h;
    }
    S->nfinal = nB;
    qsort_r(S->fin, (size_t)nB, sizeof(opoly), fin_cmp, &n);
    free(B);
    S->finished = 1;
    return 0;
}

/* ---------------- exported interface (ctypes) ---------------- */

osys *or_new(int n, uint32_t p, int m, const uint32_t *poly_off, const uint8_t *exps,
             const uint32_t *coeffs, int flags) {
    if (n < 1 || n > ORN || p < 3) return NULL;
    osys *S = (osys *)calloc(1, sizeof(osys));
    if (!S) return NULL;
    S->n = n;
    S->p = p;
    S->flags = flags;
    g_deglex = (flags & OR_DEGLEX) != 0;
    int unit = 0;
    for (int i = 0; i < m; ++i) {
        int len = (int)(poly_off[i + 1] - poly_off[i]);
        oterm *t = (oterm *)xrealloc(NULL, sizeof(oterm) * (size_t)(len ? len : 1));
        for (int j = 0; j < len; ++j) {
            memset(&t[j].m, 0, sizeof(omono));
            memcpy(t[j].m.e, exps + (size_t)(poly_off[i] + j) * n, (size_t)n);
            t[j].c = coeffs[poly_off[i] + j] % p;
        }
        opoly f = poly_normalise(t, len, n, p);
        free(t);
        if (f.len == 0) continue;
        if (m_deg(&f.mon[0], n) == 0) unit = 1;
        basis_append(S, f);
    }
    (void)unit; /* a constant input makes every other LM redundant; R9 then yields {1} */
    return S;
}

/* D' of one non-pivot row of a Macaulay matrix given as CSR (the nA pivot rows first, each monic
   with its leading column first; columns ascending within a row): the row (rcol, rval) reduced by
   the pivot rows and read at the nb non-pivot columns, exactly as or_step reduces its own rows. */
void or_reduce_row(uint32_t p, int N, int nA, const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                   const uint32_t *rcol, const uint32_t *rval, uint32_t rlen, int nb, const uint32_t *nonpiv,
                   uint32_t *out) {
    int *piv_of_col = (int *)xrealloc(NULL, sizeof(int) * (size_t)(N ? N : 1));
    for (int c = 0; c < N; ++c) piv_of_col[c] = -1;
    for (int a = 0; a < nA; ++a) piv_of_col[col[row_ptr[a]]] = a;
    uint64_t *acc = (uint64_t *)calloc((size_t)(N ? N : 1), sizeof(uint64_t));
    reduce_row(p, N, row_ptr, col, val, piv_of_col, acc, rlen ? (int)rcol[0] : N, rcol, rval, rlen, nb, nonpiv, out);
    free(acc);
    free(piv_of_col);
}

void or_free(osys *S) {
    if (!S) return;
    for (int i = 0; i < S->ng; ++i) poly_free(&S->g[i]);
    for (int i = 0; i < S->nfinal; ++i) poly_free(&S->fin[i]);
    free(S->g); free(S->redundant); free(S->pairs); free(S->fin);
    free_last(S);
    free(S);
}

int or_run(osys *S) {
    while (or_step(S)) {}
    return or_finish(S);
}

int or_npairs(const osys *S) { return S->np; }

/* stats: steps, degree, npairs, rows, N, nnz, nA, nC, nb, rank, ng */
void or_stats(const osys *S, int64_t *o) {
    o[0] = S->steps; o[1] = S->last_degree; o[2] = S->last_npairs; o[3] = S->nrows;
    o[4] = S->ndict; o[5] = S->nnz; o[6] = S->nA; o[7] = S->nC; o[8] = S->nb; o[9] = S->rank;
    o[10] = S->ng;
}

void or_dict(const osys *S, uint8_t *out) {
    for (int i = 0; i < S->ndict; ++i) memcpy(out + (size_t)i * S->n, S->dict[i].e, (size_t)S->n);
}

void or_rows(const osys *S, uint8_t *t, uint32_t *k, uint8_t *piv, uint8_t *reducer) {
    for (int a = 0; a < S->nrows; ++a) {
        memcpy(t + (size_t)a * S->n, S->rows[a].t.e, (size_t)S->n);
        k[a] = (uint32_t)S->rows[a].k;
        piv[a] = (uint8_t)S->rows[a].pivot;
        reducer[a] = (uint8_t)S->rows[a].reducer;
    }
}

void or_csr(const osys *S, uint32_t *row_ptr, uint32_t *col, uint32_t *val) {
    memcpy(row_ptr, S->row_ptr, sizeof(uint32_t) * (size_t)(S->nrows + 1));
    memcpy(col, S->col, sizeof(uint32_t) * (size_t)S->nnz);
    memcpy(val, S->val, sizeof(uint32_t) * (size_t)S->nnz);
}

void or_nonpiv(const osys *S, uint32_t *out) { memcpy(out, S->nonpiv, sizeof(uint32_t) * (size_t)S->nb); }

void or_dprime(const osys *S, uint32_t *out) {
    memcpy(out, S->dprime, sizeof(uint32_t) * (size_t)S->nC * S->nb);
}

void or_rref(const osys *S, uint32_t *pivpos, uint32_t *out) {
    memcpy(pivpos, S->rpiv, sizeof(uint32_t) * (size_t)S->rank);
    memcpy(out, S->rref, sizeof(uint32_t) * (size_t)S->rank * S->nb);
}

/* redundant flags of the basis as it was when the last step chose its rows */
int or_snapshot(const osys *S, uint8_t *red) {
    if (red) memcpy(red, S->red_snapshot, (size_t)S->ng_snapshot);
    return S->ng_snapshot;
}

int or_ng(const osys *S) { return S->ng; }
int or_poly_len(const osys *S, int i) { return S->g[i].len; }
void or_poly(const osys *S, int i, uint8_t *exps, uint32_t *cf) {
    for (int j = 0; j < S->g[i].len; ++j) {
        memcpy(exps + (size_t)j * S->n, S->g[i].mon[j].e, (size_t)S->n);
        cf[j] = S->g[i].cf[j];
    }
}
void or_redundant(const osys *S, uint8_t *red) { memcpy(red, S->redundant, (size_t)S->ng); }
void or_pairs(const osys *S, int32_t *ij) {
    for (int q = 0; q < S->np; ++q) { ij[2 * q] = S->pairs[q].i; ij[2 * q + 1] = S->pairs[q].j; }
}

/* final basis: returns the number of elements, fills the total term count */
int or_final_size(const osys *S, int64_t *terms) {
    int64_t t = 0;
    for (int i = 0; i < S->nfinal; ++i) t += S->fin[i].len;
    if (terms) *terms = t;
    return S->nfinal;
}

void or_final(const osys *S, uint32_t *poly_off, uint8_t *exps, uint32_t *cf) {
    uint32_t o = 0;
    for (int i = 0; i < S->nfinal; ++i) {
        poly_off[i] = o;
        for (int j = 0; j < S->fin[i].len; ++j) {
            memcpy(exps + (size_t)(o + j) * S->n, S->fin[i].mon[j].e, (size_t)S->n);
            cf[o + j] = S->fin[i].cf[j];
        }
        o += (uint32_t)S->fin[i].len;
    }
    poly_off[S->nfinal] = o;
}
