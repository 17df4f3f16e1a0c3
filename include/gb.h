/*
 * gb.h -- C ABI of the B300 F4 library (sm_103a).
 *
 * Problem (Sec. 1): R = F_p[x1..xn] with a term order, I = <f1..fm>; compute a Groebner basis of I.
 * The library runs the data-parallel hot path of the F4 method on one GPU:
 *   - symbolic preprocessing SP : batch -> (T, R, Pi) (Def. 5.2), realised as the two-pass FBSP
 *     pipeline of the FBSP algorithm (Sec. 10) with the one-step reduction closure (Rem. 3.3;
 *     the support-closure definition of Sec. 11);
 *   - exact structured elimination of the Macaulay matrix A (Def. 3.1) over F_p: pivot / non-pivot
 *     split, sparse row reduction, reduced echelon form of the remaining block (Sec. 9.2), with
 *     Barrett / Montgomery modular arithmetic (Sec. 8);
 *   - reconstruction of new basis elements and the basis update (Sec. 4.2).
 *
 * Conventions for every entry point:
 *   - Every call returns gb_status.  Outputs are written only on GB_OK (or GB_DONE).  Nothing
 *     throws across this boundary.  gb_last_error() gives a human-readable detail for the calling
 *     thread's last failure.
 *   - Pointers in argument lists are HOST pointers unless the name says otherwise.  Input arrays
 *     are owned by the caller and copied during the call.
 *   - Handles (gb_ctx, gb_system, gb_macaulay, gb_echelon, gb_server) are owned by the library and
 *     released by the matching *_destroy call.
 *   - Exports use a two-call pattern: call with NULL array pointers to learn the sizes (the size
 *     fields are filled), then call again with caller-allocated arrays of at least those sizes.
 *   - Coefficients cross the boundary as standard residues in [0, p).
 *   - Term order, per system (gb_order): grevlex with x1 > x2 > ... > xn (x^a > x^b iff
 *     deg a > deg b, or equal degrees and the last nonzero entry of a - b is negative), or deglex
 *     (equal degrees: the first nonzero entry of a - b is positive), the two graded orders of the
 *     monomial keys of Sec. 7.3.  Monomials are exponent vectors of n bytes.
 *   - p must be an odd prime below 2^31 (GB_EINVAL otherwise), 1 <= n <= 16.
 *   - A context and everything created from it is used by one host thread at a time, except the
 *     server, whose submit/poll calls may come from any thread.
 */
#ifndef GB_H
#define GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GB_OK = 0,
    GB_DONE = 1,           /* gb_f4_step: no critical pairs remain */
    GB_EINVAL = -1,        /* bad argument (null handle, bad prime, n out of range, ...) */
    GB_ENOMEM = -2,        /* device arena or host memory exhausted */
    GB_EOVERFLOW = -3,     /* an exponent above 255 or a monomial space too large for the keys */
    GB_ETIMEOUT = -4,      /* a bounded device wait gave up */
    GB_EDEVICE = -5,       /* a CUDA error */
    GB_EUNSUPPORTED = -6,  /* valid but outside what the library handles */
    GB_EBUSY = -7          /* server: the ticket is still running */
} gb_status;

typedef enum { GB_GREVLEX = 0, GB_DEGLEX = 1 } gb_order;

typedef struct gb_ctx gb_ctx;
typedef struct gb_system gb_system;
typedef struct gb_macaulay gb_macaulay;
typedef struct gb_echelon gb_echelon;
typedef struct gb_server gb_server;

/* Context options.  All fields may be zero. */
typedef struct {
    void *stream;        /* cudaStream_t to run on; NULL: the context creates its own stream */
    void *arena;         /* DEVICE memory the caller owns (e.g. a torch tensor), or NULL */
    size_t arena_bytes;  /* size of `arena`; when arena is NULL, bytes the context allocates
                            with cudaMalloc at creation (0: 2 GiB) */
    uint32_t flags;      /* GB_CTX_KEEP_STEP: keep the last F4 step's matrix and echelon form
                            of each system for gb_system_last_step (costs memory);
                            GB_CTX_REDUCE_SPARSE / GB_CTX_REDUCE_DENSE: reduce every matrix
                            row by row (sparse), or by dense blocked elimination on the tensor
                            cores whenever the arena has room (DENSE also runs every panel
                            update of the echelon form of D' on the tensor cores); neither:
                            chosen per matrix by its shape.  All give the same (unique) D' and
                            RREF(D');
                            GB_CTX_NO_GRAPHS: launch the rounds of the echelon form of D' one
                            by one from the host instead of as one CUDA graph whose loop runs
                            on the device (same results);
                            GB_CTX_SP_HASH: symbolic preprocessing setifies through a hash
                            dictionary keyed by an additive monomial key instead of ranking every
                            term into a bitmap; a key shared by two monomials is detected and the
                            step rebuilt on the rank path (same results);
                            GB_CTX_SKETCH: the echelon form of a tall D' (at least 2048 rows)
                            through a random sketch first: RREF(R D') for a random R of 512 rows,
                            checked exactly against D', the full echelon form when the check fails
                            (same results). */
    uint32_t reserved;
} gb_ctx_opts;

#define GB_CTX_KEEP_STEP 1u
#define GB_CTX_REDUCE_SPARSE 2u
#define GB_CTX_REDUCE_DENSE 4u
#define GB_CTX_NO_GRAPHS 8u
#define GB_CTX_SP_HASH 16u
#define GB_CTX_SKETCH 32u

/* A polynomial system on the host: polynomial i has the terms [poly_off[i], poly_off[i+1]). */
typedef struct {
    uint32_t npolys;
    const uint32_t *poly_off; /* npolys + 1 */
    const uint8_t *exps;      /* poly_off[npolys] * nvars, row-major */
    const uint32_t *coeffs;   /* poly_off[npolys]; reduced mod p on input */
} gb_polys;

/* Host export of polynomials (two-call pattern on npolys / nterms). */
typedef struct {
    uint32_t npolys;
    uint64_t nterms;
    uint32_t *poly_off; /* npolys + 1 */
    uint8_t *exps;      /* nterms * nvars */
    uint32_t *coeffs;   /* nterms */
} gb_polys_host;

/* Host export of Pi = (row_ptr, col_ind, val, dict_keys, row_meta) (Def. 5.2). */
typedef struct {
    uint32_t nvars, nrows, ndict, npivot;
    uint64_t nnz;
    uint32_t *row_ptr;  /* nrows + 1 */
    uint32_t *col_ind;  /* nnz, 0-based dictionary columns, ascending within a row */
    uint32_t *val;      /* nnz */
    uint8_t *dict_exps; /* ndict * nvars, monomials in descending order (column 0 = largest) */
    uint8_t *row_t;     /* nrows * nvars: the shift t_i of row i */
    uint32_t *row_k;    /* nrows: the basis index k_i of row i */
    uint8_t *row_flags; /* nrows: bit 0 pivot row, bit 1 added by the closure (reducer row) */
} gb_macaulay_host;

/* Host export of the elimination: D' and its reduced row echelon form (Sec. 9.2). */
typedef struct {
    uint32_t nC, nb, rank;
    uint32_t *nonpiv;   /* nb: dictionary columns of D', ascending */
    uint32_t *dprime;   /* nC * nb: the non-pivot rows after reduction by the pivot rows */
    uint32_t *rref_piv; /* rank: pivot positions in [0, nb), ascending */
    uint32_t *rref;     /* rank * nb: RREF(D') */
} gb_echelon_host;

typedef struct {
    uint32_t step, degree, npairs, nrows, ndict, npivot, nC, nb, rank, nbasis;
    uint32_t closure_rounds;
    uint32_t sp_redo;    /* times the step's symbolic preprocessing ran again: its frontier queue
                            or (GB_CTX_SP_HASH) hash dictionary needed more room, or two monomials
                            shared a hash key (then the rank path built it) */
    uint64_t nnz;
    uint64_t axpy_rows;  /* pivot rows applied by the sparse reduction (eq. 8.1 row updates) */
    uint64_t axpy_fma;   /* modular multiply-adds a <- a + b c of the sparse reduction */
    float ms_sp;       /* device time: symbolic preprocessing (DictBuild + RowAssemble) */
    float ms_reduce;   /* device time: sparse reduction of the non-pivot rows */
    float ms_rref;     /* device time: reduced echelon form of D' */
    float ms_update;   /* wall time: reconstruction of the new elements on the device */
    float ms_pairs;    /* host time: critical-pair update (Gebauer-Moeller) for the new elements */
    float ms_select;   /* host time: pair selection and ordering of the step's rows */
    float ms_reduce_kernel; /* device time of the row-reduction kernel launches alone (a part of
                               ms_reduce, which also covers their setup) */
    double ms_wall;    /* host wall time of the step */
    double ms_mm;      /* device time of the tensor-core product launches (the dense blocked
                          reduction and RREF updates), CUDA events around each launch made outside
                          a CUDA graph; for a batch, the whole batch's */
    double mm_flops;   /* BF16 digit-product FLOPs of those launches: 2 L^2 per mod-p multiply-add
                          (L = 2 digits for p < 2^16, 4 otherwise) */
    uint64_t mm_launches; /* the launches ms_mm covers */
    uint32_t rref_sketched; /* 1: RREF(D') came from a random sketch, checked exactly */
    uint32_t reserved;
} gb_step_stats;

typedef struct {
    uint32_t steps, nbasis;
    uint64_t nnz_total;
    uint64_t axpy_rows, axpy_fma;
    double ms_sp, ms_reduce, ms_rref, ms_update, ms_pairs, ms_select, ms_wall;
    double ms_reduce_kernel;
    double ms_finish;  /* wall time of the final minimalisation and tail reduction */
    uint64_t nnz_steps; /* sum of nnz(A) over the F4 steps only (nnz_total also counts the matrix
                           of the final tail reduction) */
    double ms_mm, mm_flops;  /* as in gb_step_stats, summed over the run */
    uint64_t mm_launches;
} gb_run_stats;

/* ---- context -------------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  opts may be NULL. */
gb_status gb_ctx_create(int device, const gb_ctx_opts *opts, gb_ctx **out);
gb_status gb_ctx_destroy(gb_ctx *ctx);
/* Device bytes currently allocated from the context's arena, and its size. */
gb_status gb_ctx_memory(const gb_ctx *ctx, size_t *used, size_t *capacity);
/* High-water mark of the arena's allocated bytes; reset != 0 restarts it at the current use. */
gb_status gb_ctx_memory_peak(gb_ctx *ctx, size_t *peak, int reset);

/* ---- systems -------------------------------------------------------------------------------- */

/* Create a system <f1..fm> in F_p[x1..xn] (Sec. 1).  The inputs are normalised: equal monomials
   merged mod p, zero terms and zero polynomials dropped, each polynomial made monic, terms sorted
   descending.  The normalised inputs become the first basis elements, inserted in input order with
   the Gebauer-Moeller pair update.  GB_EOVERFLOW: an exponent above 255. */
gb_status gb_system_create(gb_ctx *ctx, uint32_t nvars, uint32_t p, gb_order order,
                           const gb_polys *F, gb_system **out);
gb_status gb_system_destroy(gb_system *sys);

/* ---- the hot path --------------------------------------------------------------------------- */

/* Symbolic preprocessing (Def. 5.2, the FBSP algorithm (Sec. 10)) of the r shifted rows (t_i, g_{k_i}) of the
   system's current basis.  t_exps: r * nvars host bytes; k: r basis indices.  Equal (t, k) rows
   collapse.  closure != 0 adds, for every dictionary monomial m that is not the leading monomial of
   a given row and is divisible by the leading monomial of a non-redundant basis element, the
   reducer row (m / LM(g), g) for the oldest such g, until closed (Rem. 3.3).  Row order: pivot rows
   (one per leading column; reducer rows, else the given row of smallest k) by leading column,
   then the other rows by (leading column, k).  The result lives on the device. */
gb_status gb_symbolic_preprocess(gb_system *sys, uint32_t r, const uint8_t *t_exps,
                                 const uint32_t *k, int closure, gb_macaulay **out);
gb_status gb_macaulay_export(const gb_macaulay *mac, gb_macaulay_host *inout);
gb_status gb_macaulay_destroy(gb_macaulay *mac);

/* Sizes and stage times of one materialised plan (the per-run record of Sec. 12: N, M, nnz(A),
   and the DictBuild / RowAssemble split of the kernel decomposition of Sec. 12).  Every nonzero is
   one expanded term t m (t m is injective within a row), so the key volume M equals nnz.  The
   times are device times of the symbolic-preprocessing call that built the matrix (for a batch,
   the batch's). */
typedef struct {
    uint32_t nrows, ndict, npivot, closure_rounds;
    uint64_t nnz;          /* = M, the expanded terms */
    float ms_sp;           /* the whole stage */
    float ms_dict;         /* DictBuild: expansion, closure rounds, dense ranks, the dictionary emitted */
    float ms_assemble;     /* RowAssemble: pivot split, row lengths, the fill of col_ind / val */
    uint32_t reserved;
} gb_macaulay_stats;
gb_status gb_macaulay_stats_get(const gb_macaulay *mac, gb_macaulay_stats *out);

/* Structured elimination of Pi (Sec. 9.2): each non-pivot row is reduced by the pivot rows
   (pivot columns in ascending order) to D', zero on every pivot column, then D' is brought to its
   reduced row echelon form.  Both are unique. */
gb_status gb_reduce_macaulay(gb_macaulay *mac, gb_echelon **out);
gb_status gb_echelon_export(const gb_echelon *ech, gb_echelon_host *inout);
gb_status gb_echelon_destroy(gb_echelon *ech);

/* One F4 step (Sec. 4.2): select every critical pair of minimal lcm degree, build the rows of both
   halves of each pair, run symbolic preprocessing with closure and the elimination, append the
   echelon rows as new basis elements and update the pairs.  GB_DONE when no pair remains (nothing
   is changed).  stats may be NULL. */
gb_status gb_f4_step(gb_system *sys, gb_step_stats *stats);

/* F4 steps until no pair remains, then the reduced Groebner basis of the ideal <f1..fm> in
   F_p[x1..xn] under the system's term order (the problem statement of Sec. 1; the reduced basis
   and Buchberger's criterion of Sec. 2.1; the F4 loop of Sec. 2.3 and Sec. 4.2): redundant
   elements dropped, tails fully reduced, monic, sorted by leading monomial descending.  The basis stays in the
   context's device arena (held by the system) until gb_basis_export copies it out or the system
   is destroyed.  stats may be NULL. */
gb_status gb_groebner(gb_system *sys, gb_run_stats *stats);

/* The reduced basis after gb_groebner (reduced != 0; the unique reduced Groebner basis of
   Sec. 2.1, each element monic with the leading monomial first), or the running basis in
   insertion order, redundant elements included (reduced == 0).  Two-call pattern: with null arrays only npolys
   and nterms are written; the terms then come from the device in one copy per array. */
gb_status gb_basis_export(const gb_system *sys, int reduced, gb_polys_host *inout);
/* Redundancy flags of the running basis (one byte per element; two-call pattern on *count). */
gb_status gb_basis_redundant(const gb_system *sys, uint32_t *count, uint8_t *flags);

/* With GB_CTX_KEEP_STEP: borrowed handles to the last step's matrix and echelon form (valid until
   the next step or the system's destruction). */
gb_status gb_system_last_step(const gb_system *sys, const gb_macaulay **mac,
                              const gb_echelon **ech);

/* ---- batching and serving ------------------------------------------------------------------- */

/* Run gb_groebner on `count` independent systems of one context in lockstep: each iteration takes
   one F4 step of every system with pairs left (each pipeline kernel is launched once for all of
   their matrices) and builds the reduced basis of every system without pairs; per-system host
   control runs on the context's worker threads.  The results are those of gb_groebner on each
   system alone.  Each stage of an iteration allocates for all of its systems together, so the
   arena must hold the batch's steps side by side: a batch of large systems is split by the caller
   (or goes through the server, which admits by estimated footprint); GB_ENOMEM otherwise.  A
   failing iteration fails the whole call (the systems are left unusable).  per_system may be
   NULL. */
gb_status gb_batch_groebner(gb_ctx *ctx, uint32_t count, gb_system *const *systems,
                            gb_run_stats *per_system);

typedef struct {
    size_t hbm_cap_bytes;  /* admission cap on the summed device footprint of admitted systems */
    uint32_t max_slots;    /* systems running at once (0: 64) */
    uint32_t finish_min;   /* systems out of pairs wait for their final reduction until at least
                              this many are ready, for at most 4 iterations, or until no other
                              system takes a step (0 or 1: at once); one final-reduction pass then
                              serves them all */
    uint32_t admit_min;    /* queued systems are admitted only while at least this many slots are
                              free, or when nothing runs (0 or 1: into any free slot), so that they
                              join in waves and take their steps in phase */
    uint32_t reserved;
} gb_server_opts;

/* A continuous-batching server: one scheduler thread runs lockstep iterations (as in
   gb_batch_groebner) over the admitted systems, and between iterations admits queued systems into
   free slots while their summed device footprint estimate fits under the cap.  A submitted system
   thus joins the next iteration and a finished one leaves at once.  Ownership of a submitted
   system moves to the server until it is returned by poll; submitting a system the server still
   holds (queued, running, or finished and not yet polled) gives GB_EINVAL.  An iteration that
   fails finishes all of its systems with its error status. */
gb_status gb_server_create(gb_ctx *ctx, const gb_server_opts *opts, gb_server **out);
gb_status gb_server_submit(gb_server *srv, gb_system *sys, uint64_t *ticket);
/* GB_OK and *done = the system when finished (ownership returns to the caller, with its status in
   *result); GB_EBUSY while it is queued or running. */
gb_status gb_server_poll(gb_server *srv, uint64_t ticket, gb_system **done, gb_status *result);
gb_status gb_server_destroy(gb_server *srv);

typedef struct {
    uint64_t iterations;    /* lockstep iterations run */
    uint64_t system_steps;  /* sum over iterations of the systems in the iteration */
    uint64_t admitted, finished;
    double busy_ms;         /* wall time inside iterations */
    uint32_t max_running;   /* most systems in one iteration */
    uint32_t queued;        /* systems waiting for admission now */
    uint64_t finish_passes; /* final-reduction passes run */
    double finish_ms;       /* wall time inside them (a part of busy_ms) */
} gb_server_stats;

/* Counters of the server since its creation. */
gb_status gb_server_stats_get(gb_server *srv, gb_server_stats *out);

/* ---- dense update over F_p on the tensor cores ------------------------------------------------ */

/* C <- C - A B (subtract != 0) or C <- C + A B (subtract == 0), mod p, exactly: the GEMM-like
   block update of the panel-structured elimination (Sec. 9.2), with the modular multiply-add of
   Sec. 8 taken out of the inner loop.  The product runs on the tensor cores: each residue is split
   into balanced base-256 digits (two for p < 2^16, four for p < 2^31), the digit products are
   accumulated in FP32 (exact: every partial sum is an integer below 2^24 in magnitude) and the
   digit sums are recombined mod p.
   All matrix pointers are DEVICE pointers on the context's device, row-major with the given row
   pitches (in elements): A is m x k, B is k x n, C is m x n; entries in [0, p).  A and B are
   read, C is updated in place.  The work runs on the context's stream and the call returns when
   it is done.  Scratch (the digit planes) comes from the context's arena.
   GB_EINVAL: null handle or pointer, p not an odd prime below 2^31, a pitch below the width.
   GB_ENOMEM: the arena cannot hold the digit planes (2 (m + n) k digits of 2 bytes, times 2 for
   p >= 2^16).  GB_ETIMEOUT: a bounded device wait gave up. */
gb_status gb_matmul_modp(gb_ctx *ctx, uint32_t p, uint32_t m, uint32_t n, uint32_t k, const uint32_t *A,
                         uint64_t lda, const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc,
                         int subtract);

/* ---- sparse reduction without device allocation --------------------------------------------- */

/* Limits of gb_reduce_rows_noalloc: its scratch is a fixed array compiled into the library. */
#define GB_NOALLOC_MAX_DICT 51200u    /* ndict for p < 2^16 (25600 for larger p) */
#define GB_NOALLOC_MAX_PIVOTS 16384u  /* pivot rows */

/* The sparse row reduction of gb_reduce_macaulay (D' only, no echelon form), for callers that
   cannot allocate device memory.  Examples: a process whose device memory is owned by another
   allocator (a framework's caching allocator, a fixed pool sized at start-up) that must not see
   the device's free memory change behind its back between its own calls; or a host thread with a
   latency budget that must not take the driver's allocation path.  This entry point allocates
   nothing: it works on the caller's buffers plus one scratch array of about 2.3 MB that is part
   of the library image (each GPU that loads the library holds it until the process exits).  It
   has no counterpart in the paper.
   All pointers are DEVICE pointers on the current device:
     row_ptr[npivot + nnonpivot + 1], col_ind, val: CSR of the matrix, the npivot pivot rows first
       (row i monic with leading column pivot_cols[i], pivot_cols ascending), then the non-pivot
       rows; columns ascending within a row and below ndict, values in [0, p); row_ptr must be
       non-decreasing and col_ind / val must hold row_ptr[npivot + nnonpivot] entries;
     nonpivot_cols[nb]: the columns that are no pivot's leading column, ascending;
     dprime[nnonpivot * nb] (output): the non-pivot rows reduced by the pivot rows, restricted to
       nonpivot_cols -- the D' of gb_echelon_export.
   stream: a cudaStream_t of the current device (NULL: the legacy default stream).  The call only
   enqueues work; it returns before the work finishes.  The job description reaches the device
   as a kernel parameter, so no host memory is read after the call returns.
   The kernels check every index that becomes an address (row pointers non-decreasing, columns
   ascending and below ndict, each pivot row opening at its pivot column, pivot and non-pivot
   columns below ndict).  If one fails, nothing outside dprime and the scratch array is written
   and every entry of dprime is set to 0xFFFFFFFF, which no residue mod p < 2^31 can be: test
   dprime[0] after the stream has finished.
   The first call on each device looks up the scratch array's device address (no allocation); make
   that first call before any stream capture.  Every call uses the same scratch array and leaves
   its contents there; each call clears what it needs at zero.  Calls whose work overlaps on the
   GPU (several streams, several host threads) race on that array: serialise them.
   GB_EINVAL: p not an odd prime below 2^31, a size above the limits above, D' above 2^31 entries,
   or a null pointer.  GB_EDEVICE: a launch was refused. */
gb_status gb_reduce_rows_noalloc(uint32_t p, uint32_t ndict, uint32_t npivot, uint32_t nnonpivot,
                                 uint32_t nb, const uint32_t *row_ptr, const uint32_t *col_ind,
                                 const uint32_t *val, const uint32_t *pivot_cols,
                                 const uint32_t *nonpivot_cols, uint32_t *dprime, void *stream);

/* ---- kernel vectors by the block Wiedemann method ---------------------------------------------- */

typedef struct {
    uint32_t b, d, nterms;       /* block width, Hankel blocks d = ceil(r / b) + 1, sequence terms 2d */
    uint32_t hankel_rank;        /* rank of the block Hankel matrix */
    uint32_t free_columns;       /* its free columns: the generator vectors tried */
    uint32_t found;              /* dimension of the span of the vectors found (rows of W) */
    uint32_t verified;           /* rows w of W with w^T A = 0 checked on the device */
    uint32_t reserved;
    uint64_t spmm_products;      /* mod-p multiply-adds of the sparse products (32 lanes per entry) */
    double ms_sequence, ms_hankel, ms_vectors, ms_total;  /* device time of the stages */
} gb_krylov_stats;

/* Relations among the rows of one step's Macaulay matrix A (r rows, N columns): vectors v with
   v^T A = 0, i.e. sum_i v_i t_i g_{k_i} = 0 (Prop. 3.2), by the block Wiedemann method of
   Sec. 9.3 (the Krylov alternative to elimination, Sec. 13.4): with M = A diag(delta) A^T, the
   sequence S_i = X^T M^(i+1) Z (i < 2d, d = ceil(r / b) + 1) is computed with sparse products
   of A and A^T with blocks of b vectors; the right kernel of the block Hankel matrix
   H[i b + a][j b + c] = S_{i+j}[a][c] (i < d, j <= d) gives, one vector c per free column of
   RREF(H), y(c) = sum_j M^j Z c_j in ker M; W is the reduced row echelon form of the y(c).
   With random X, Z, delta, W spans min(b, dim ker A^T) dimensions of the left kernel.
   mac: a matrix from gb_symbolic_preprocess or gb_system_last_step (not modified).
   b: block width, 1..32.  X, Z: HOST arrays r x b row-major, entries in [0, p); delta: HOST N
   entries in [1, p); all copied at the call (the caller draws them: they are the method's random
   choices).  seq (HOST, may be NULL): 2d x b x b, the sequence S_i row-major.  W (HOST, may be
   NULL): wcap x r, the first min(wcap, found) rows of W.  stats (may be NULL).  Runs on the
   context's stream; returns when done.
   GB_EINVAL: null handle or input, b out of range, an entry out of range, an empty matrix.
   GB_ENOMEM: the arena cannot hold the block Hankel system (about 3 (d b)^2 4-byte words) and its
   work.  GB_EUNSUPPORTED: a Hankel system above 2^34 entries.  GB_ETIMEOUT: a bounded device
   wait gave up. */
gb_status gb_block_wiedemann(const gb_macaulay *mac, uint32_t b, const uint32_t *X, const uint32_t *Z,
                             const uint32_t *delta, uint32_t *seq, uint32_t *W, uint32_t wcap,
                             gb_krylov_stats *stats);

/* ---- signature-filtered Macaulay matrices (F5 criterion) ------------------------------------------ */

/* The admissibility predicate over packed signature keys, and the compaction of the survivors
   (Sec. 14, "GPU-facing reformulation": a signature key per candidate row, the predicate evaluated
   over row metadata in bulk, the survivors compacted by a scan).  The candidates are the
   signatures x^a e_index, x^a running over the monomials of degree e in descending grevlex order;
   candidate j (0 <= j < ncand) is admissible iff bit j of forbidden is clear (bit j % 32 of word
   j / 32; forbidden is a DEVICE array of ceil(ncand / 32) words, or NULL: every candidate is
   admissible).  The admissible candidates' packed keys (index << 40) | (e << 32) | j go to keys
   (DEVICE, room for ncand) in increasing j, and their number to *count (HOST).  Runs on the
   context's stream; returns when the count is on the host.
   GB_EINVAL: null context or count, null keys with ncand > 0, index >= 2^24 or e > 255. */
gb_status gb_sig_filter(gb_ctx *ctx, uint32_t index, uint32_t e, uint32_t ncand, const uint32_t *forbidden,
                        uint64_t *keys, uint32_t *count);

typedef struct {
    uint32_t degree, index;      /* block (d, i): degree d, generator i (1-based, in input order) */
    uint32_t candidates;         /* candidate rows x^a f_i: the monomials x^a of degree d - d_i */
    uint32_t admissible;         /* those the F5 criterion keeps (all of them with GB_F5_NO_CRITERION) */
    uint32_t rows;               /* rows of the block's matrix: the echelon rows of degree d, then the admissible candidates */
    uint32_t ndict, npivot, nC;  /* its columns, pivot rows and other rows (0 when no candidate is admissible) */
    uint32_t rank;               /* new basis elements: the reduced echelon rows of the non-pivot part */
    uint32_t zero_reductions;    /* admissible rows that did not enlarge the row space */
    float ms_filter, ms_sp, ms_reduce, ms_rref;  /* the filter (host clock, with its copies), device stages */
} gb_f5_block;

typedef struct {
    uint32_t blocks, nbasis;     /* blocks run; elements of the reduced basis */
    uint64_t candidates, admissible, zero_reductions;
    uint64_t nnz;                /* nonzeros of the blocks' matrices */
    double ms_wall, ms_filter, ms_sp, ms_reduce, ms_rref, ms_finish;
} gb_f5_stats;

#define GB_F5_NO_CRITERION 1u /* every candidate admissible: the unfiltered Macaulay matrices */

/* The Groebner basis of a homogeneous system degree by degree through signature-filtered Macaulay
   matrices (the signature regime of Thm. signature-sound, with F5's criterion as the predicate
   Adm, position over term, e_1 < e_2 < ...).  For d from the least input degree to dmax and each
   generator i with d_i <= d: the candidate rows x^a f_i (deg x^a = d - d_i) go through
   gb_sig_filter with the leading monomials of the degree-(d - d_i) part of <f_1 .. f_{i-1}>
   as the forbidden set; the admissible rows and the echelon rows of degree d found so far go
   through symbolic preprocessing (without closure), the reduction and the RREF of D' on the
   device, and the new elements join the basis.  Then the reduced basis of the elements whose
   leading monomials are minimal, as gb_groebner leaves it (gb_basis_export).  It is the reduced
   Groebner basis of the ideal when dmax reaches that basis's largest degree; for a regular
   sequence no admissible row reduces to zero.  sys: a fresh system (no step run), grevlex, every
   input homogeneous.  blocks (HOST, may be NULL): the first blocks_cap block records in order;
   *nblocks (may be NULL): the number of blocks run.  stats may be NULL.
   GB_EINVAL: a system that has run, an inhomogeneous input, dmax above 255 or below the least
   input degree, an unknown flag.  GB_EUNSUPPORTED: deglex.  Otherwise as gb_groebner. */
gb_status gb_f5_groebner(gb_system *sys, uint32_t dmax, uint32_t flags, gb_f5_block *blocks, uint32_t blocks_cap,
                         uint32_t *nblocks, gb_f5_stats *stats);

/* ---- the mod-p primitives, one at a time ------------------------------------------------------ */

/* Each operation applies one of the device's F_p primitives elementwise: the same functions, with
   the same precomputed constants, that the reduction kernels use.  It exists so that each
   primitive can be checked on its own against plain integer arithmetic. */
typedef enum {
    GB_MODP_REDUCE64 = 0,  /* out = (a 2^32 + b) mod p: Barrett with k = 64 (Sec. 8.3), any 64-bit x */
    GB_MODP_REDUCE32 = 1,  /* out = a mod p: Barrett with k = 32, p < 2^16, any 32-bit a */
    GB_MODP_MULADD = 2,    /* out = (a b + c) mod p through the 64-bit Barrett step (Sec. 8.1) */
    GB_MODP_REDC = 3,      /* out = redc(t), t = a 2^32 + b < p 2^32: t 2^-32 mod p, in [0, 2p)
                              (Montgomery, R = 2^32, Sec. 8.4) */
    GB_MODP_TO_MONT = 4,   /* out = a 2^32 mod p (the Montgomery domain of Sec. 8.4), a < p */
    GB_MODP_MONT_MUL = 5,  /* out = redc((a 2^32 mod p) b): a b mod p, in [0, 2p) -- the product of
                              the sparse update, multiplier in Montgomery form, entry standard */
    GB_MODP_INV = 6,       /* out = a^-1 mod p (binary extended Euclid), 0 < a < p */
    GB_MODP_INV_SMALL = 7, /* out = a^(p-2) mod p (Fermat), p < 2^16, 0 < a < p */
    GB_MODP_LAZY32 = 8,    /* out[i] = (c[i] + sum_j (a b mod p)) mod p over a window of `window`
                              terms a[i*window + j] b[i*window + j], summed in 32 bits without
                              reduction between terms (the lazy window of Rem. 8.1), p < 2^16,
                              window < 2^16, c[i] < p */
    GB_MODP_LAZY_MONT = 9, /* the same with 64-bit sums of GB_MODP_MONT_MUL terms (each below 2p) */
    GB_MODP_CHAIN_BARRETT = 10, /* x <- (x b[i] + c[i]) mod p, `window` times from x = a[i], in registers:
                                   the modular multiply-add through the 64-bit Barrett step; out = x
                                   (the modular inner loop of the microbenchmarks of Sec. 12.2) */
    GB_MODP_CHAIN_MONT = 11     /* the same chain with the product in Montgomery form (b[i] converted
                                   once, redc per step, Sec. 8.4); out = x, the same residue */
} gb_modp_op;

/* Device pointers on the current device: a, b, c [n] (b and c only where the operation reads
   them; for the two window operations a and b hold n * window values; the chains read a, b and c
   [n] and run `window` >= 1 steps), out [n].  stream: a
   cudaStream_t (NULL: the legacy default stream); the call only enqueues the work.
   GB_EINVAL: p not an odd prime below 2^31, an unknown operation, a 16-bit-only operation with a
   larger p, a window out of range, a null pointer the operation needs. */
gb_status gb_modp_apply(gb_modp_op op, uint32_t p, uint64_t n, uint32_t window, const uint32_t *a,
                        const uint32_t *b, const uint32_t *c, uint32_t *out, void *stream);

/* Host only, no device or context: the critical-pair bookkeeping of the F4 loop replayed on a
   sequence of leading monomials, to check it against a textbook model.  The pairs are those of
   UPDATE (Becker-Weispfenning; the Gebauer-Moeller criteria, Sec. 2.1's S-pairs pruned) with the
   selection of the pipeline (Sec. 4.2: every pair of the least lcm degree).
   lms[nelem * n]: the leading monomials (n exponent bytes each) in insertion order, inserted in
   ngroups groups of group_sizes[g] elements; the elements of one group are inserted together, as
   the new elements of one F4 step are (the result is that of inserting them one at a time in
   order).  select_before[g] (NULL: never): before group g, remove the pairs whose lcm has the
   least degree.  Output: npairs pairs (i, j), i < j, at pairs[2 q], pairs[2 q + 1] (cap pairs at
   most), and in_basis[nelem]: 0 for an element whose leading monomial a later one divides.
   GB_EINVAL: n outside 1..16, sizes that do not add up, a null pointer, more than cap pairs
   (npairs then holds the count). */
gb_status gb_pair_update_replay(uint32_t n, uint32_t nelem, const uint8_t *lms, uint32_t ngroups,
                                const uint32_t *group_sizes, const uint8_t *select_before, uint32_t cap,
                                uint32_t *pairs, uint32_t *npairs, uint8_t *in_basis);

/* ---- autotuning ----------------------------------------------------------------------------- */

/* The reduction of a Macaulay matrix has interchangeable schedules that give the same D' and
   RREF(D') (Sec. 9.2): the sparse row-by-row reduction or the dense blocked elimination on the
   tensor cores; the panel updates of RREF(D') on CUDA cores or on the tensor cores; the RREF
   rounds launched one by one from the host or as one CUDA graph whose loop runs on the device.
   Without tuning a context chooses by fixed shape rules.

   gb_autotune runs copies of the given systems to completion once per candidate schedule
   (three runs), times every step's reduction and RREF on the device, and keeps, per shape
   bucket, the schedule with the least total time.  A reduction's bucket is the prime's class
   (below 2^16 or not) and floor(log2(x + 1)) of its pivots, non-pivot rows and non-pivot columns;
   an RREF's bucket is the class and the same of D''s rows and columns.  It also times the three
   tiles of the prefix sums of the pipeline (4, 8 or 16 values per thread) on device arrays of
   2^8 .. 2^24 values and keeps the fastest per floor(log2(n + 1)); every later scan of the
   context of that size takes it.  From then on every
   single-system reduction of the context (gb_f4_step, gb_groebner, gb_reduce_macaulay) whose
   bucket the table holds takes the tuned schedule; other buckets, and the matrices of a batch,
   keep the rules.  GB_CTX_REDUCE_SPARSE, GB_CTX_REDUCE_DENSE and GB_CTX_NO_GRAPHS still take
   precedence.  Tuning adds to the context's table; a bucket measured again is replaced.
   The systems must belong to ctx and have run no step; they are not modified.  Do not tune a
   context that a server is using.
   GB_EINVAL: null ctx, a null or foreign system, or a system that has run a step. */
typedef struct {
    uint32_t runs;            /* complete runs of all systems (one per candidate schedule) */
    uint32_t steps;           /* F4 steps timed, over all runs */
    uint32_t buckets_reduce;  /* reduction buckets in the context's table */
    uint32_t buckets_rref;    /* RREF buckets in the context's table */
    uint32_t dense_buckets;   /* reduction buckets where the tensor-core schedule won */
    uint32_t buckets_scan;    /* prefix-sum size buckets (tile of 4, 8 or 16 values per thread) */
    double ms_wall;           /* host wall time of the tuning */
} gb_tune_report;

gb_status gb_autotune(gb_ctx *ctx, uint32_t count, gb_system *const *systems, gb_tune_report *report);
/* Write the context's table to a text file (one bucket per line, with the measured times), or
   add the buckets of such a file to the table.  GB_EINVAL: the file cannot be opened or a line
   is malformed (nothing is added then). */
gb_status gb_tune_save(const gb_ctx *ctx, const char *path);
gb_status gb_tune_load(gb_ctx *ctx, const char *path);

/* ---- diagnostics ---------------------------------------------------------------------------- */

/* Number of CUDA kernels this library has launched in this process so far (all contexts); a
   kernel inside a CUDA graph counts once per execution. */
uint64_t gb_kernel_launches(void);
/* Number of CUDA graphs this library has launched in this process so far (all contexts). */
uint64_t gb_graph_launches(void);

/* ---- errors --------------------------------------------------------------------------------- */

const char *gb_status_str(gb_status s);
const char *gb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GB_H */
