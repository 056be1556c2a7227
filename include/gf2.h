/*
 * gf2.h -- C ABI of the GB300 (sm_103a) GF(2) elimination library.
 *
 * Dense matrices over GF(2) (Albrecht & Pernet, "Efficient Decomposition of
 * Dense Matrices over GF(2)"): PLS decomposition with rank (Proposition "PLS
 * decomposition", Sec. 2; Algorithms MMPF, Sec. 4.1, and PLS, Sec. 5), the
 * reduced row echelon form (Definition "Reduced Row Echelon Form", Sec. 2;
 * computed from PLS as in the "PLS" column of Table 1, Sec. 7), the rank, and
 * the product C = C + A.B used as the trailing update (Algorithm PLS, Sec. 5).
 *
 * MATRIX LAYOUT (all entry points). A matrix is (data, m, n, stride):
 *   data   -- DEVICE pointer, 128-byte aligned, owned by the caller;
 *   m, n   -- rows and columns (bits), 0 <= m, n < 2^31;
 *   stride -- row pitch in 64-bit words, a multiple of 16 (128 bytes) and
 *             >= ceil(n / 64).
 * Row i occupies data[i*stride .. i*stride + stride). Column j of row i is bit
 * (j & 63) of word data[i*stride + (j >> 6)]: least significant bit = leftmost
 * column. Bits at columns >= n ("padding") are ignored on input and zero on
 * output. Words past ceil(n/64) in a row are never read or written.
 *
 * PERMUTATIONS. P (length m) and Q (length n) are DEVICE int64 arrays holding
 * swap vectors, as written by the Gaussian PLS algorithm (appendix): for
 * i = 0 .. r-1, row i was swapped with row P[i] (P[i] >= i) and Q[i] is the
 * column of the i-th pivot (strictly increasing). P[i] = i for i >= r and
 * Q[i] = i for i >= r. A = P.L.S is recovered by applying the transpositions
 * i <-> P[i] for i = r-1 down to 0 to the rows of L.S.
 *
 * ASYNCHRONY. Every call enqueues work on `stream` (a cudaStream_t, NULL = the
 * legacy default stream) and returns without synchronising; results (rank
 * included) are in device memory when the stream reaches that point. Host
 * arguments are validated before anything is enqueued.
 *
 * WORKSPACE. Calls that take (work, work_bytes) need at least
 * gf2_workspace_bytes(op, m, n, opts) bytes of DEVICE memory, 256-byte
 * aligned, owned by the caller and not used by anything else until the stream
 * has finished the call. work == NULL makes the library use a workspace it
 * allocates (cudaMalloc) and keeps per device; calls that share that internal
 * workspace must then be ordered on one stream.
 *
 * ERRORS. Every entry point returns 0 (GF2_OK) or a GF2_E* code and never
 * throws. A non-zero return means nothing was enqueued (except GF2_ECUDA from
 * a failed launch, after which the stream's work is undefined).
 */
#ifndef GF2_H
#define GF2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GF2_OK 0
#define GF2_EINVAL 1   /* null pointer, negative or too large size, stride < ceil(n/64), bad opts */
#define GF2_EALIGN 2   /* data not 128-byte aligned, stride not a multiple of 16, work not 256-byte aligned */
#define GF2_ENOMEM 3   /* internal workspace allocation failed */
#define GF2_ECUDA 4    /* a CUDA runtime call failed (see gf2_last_cuda_error) */
#define GF2_ENOSPACE 5 /* work_bytes smaller than gf2_workspace_bytes() */
#define GF2_EDIM 6     /* mismatched dimensions (gf2_mul) */
#define GF2_ETOOBIG 7  /* matrix too large for the fixed scratch of gf2_rank_noalloc */
#define GF2_ETIMEOUT 8 /* a device-side wait gave up (reported by gf2_sync_status) */

/* op codes for gf2_workspace_bytes */
#define GF2_OP_PLS 1
#define GF2_OP_RREF 2
#define GF2_OP_RANK 3
#define GF2_OP_MUL 4

/* trailing-product form for gf2_mul and the recursive PLS */
#define GF2_PRODUCT_AUTO 0
#define GF2_PRODUCT_XOR 1    /* Gray-code XOR tables (Method of the Four Russians) */
#define GF2_PRODUCT_TENSOR 2 /* 0/1 operands on the tensor cores, exact, low bit kept */
#define GF2_PRODUCT_STRASSEN 3        /* Strassen-Winograd recursion, XOR-table leaves (gf2_mul only) */
#define GF2_PRODUCT_STRASSEN_TENSOR 4 /* Strassen-Winograd recursion, tensor-core leaves (gf2_mul only) */

/*
 * Tuning knobs. None of them changes any result (rank, P, Q, L, S and RREF
 * are unique for the pivot rule, whatever the blocking). Pass NULL for the
 * defaults; a field left 0 means "choose automatically".
 */
typedef struct gf2_opts {
    int k;              /* bits per Gray-code table (Sec. 3.1): 8 (0 = 8; stored as 7-bit halves plus one
                           table of the groups' top bits) or 4 (16 tables of 16 entries: cheaper to build,
                           more lookups; the 16-word PLS-form sweeps only: not with the reduced-form RREF
                           routes, tile_words 4 or 8, or the persistent batch) */
    int tile_words;     /* column tile of a table sweep, in words: 0 (default), 4, 8 or 16 */
    int grid_ctas;      /* CTAs of a table sweep; 0 = one per SM but one (left to the overlapping pivot search) */
    int product;        /* GF2_PRODUCT_*; used by gf2_mul */
    int64_t cutoff_cols;/* recursive PLS: MMPF base case at or below this many columns (Sec. 6); 0 = MMPF only.
                           Strassen products: the smallest dimension recursed on (0 = 8192) */
    int rref_method;    /* gf2_rref: GF2_RREF_* (0 = GF2_RREF_AUTO) */
    int hybrid_permille;/* GF2_RREF_HYBRID: switch to PLS once the remaining rows' density reaches this many
                           per mille (Sec. 6, "M+P 0.15"; 0 = 150) */
    int batch_mode;     /* gf2_pls_batched: GF2_BATCH_* (0 = GF2_BATCH_AUTO) */
    int panels_per_sweep;/* MMPF in PLS form (gf2_pls, gf2_rank, gf2_rref's PLS route): 1 = one table sweep of
                           the trailing block per 64-column panel; 2 = the pivots of two panels first, then one
                           sweep for both (half the trailing block's DRAM traffic); 0 = the library's choice.
                           Same results either way. Ignored by the reduced-form RREF routes and the batch */
    int reserved[4];    /* must be zero */
} gf2_opts;

/* schedules of gf2_pls_batched (same results) */
#define GF2_BATCH_AUTO 0       /* persistent unless a member would need a team of more than 16 CTAs */
#define GF2_BATCH_STEPS 1      /* two launches per panel step over all matrices that have that panel */
#define GF2_BATCH_PERSISTENT 2 /* one persistent launch: teams of CTAs take whole matrices (16-word tiles only) */

/* routes of gf2_rref (all reach the same, unique, reduced row echelon form) */
#define GF2_RREF_AUTO 0   /* the library's choice (currently GF2_RREF_PLS) */
#define GF2_RREF_PLS 1    /* PLS decomposition, then the upper solve (Table 1's "PLS" column) */
#define GF2_RREF_M4RI 2   /* Algorithm M4RI (Sec. 3.1): each panel's tables clear the rows above and below */
#define GF2_RREF_HYBRID 3 /* "M+P" (Sec. 6-7): M4RI panels while the remaining rows are sparse, then PLS panels
                             and the upper solve over the PLS panels' pivots only */

/*
 * Bytes of workspace an operation needs for an m x n matrix. For GF2_OP_MUL
 * pass the inner dimension k as m and the column count n as n: the tensor-core
 * product keeps B transposed there (n x ceil(k/64) words, rounded to whole
 * 128-bit chunks); the XOR-table product needs none; the Strassen forms are
 * sized for a k x k A (use gf2_mul_workspace_bytes for any shape). Returns 0
 * for invalid sizes.
 */
size_t gf2_workspace_bytes(int op, int64_t m, int64_t n, const gf2_opts *opts);

/*
 * Workspace bytes of gf2_mul for A m x k, B k x n under opts->product: 0 for the
 * XOR-table form; B^T for the tensor-core form; for the Strassen forms, the
 * product A.B when accumulating, each level's three block temporaries
 * (m/2 x k/2, k/2 x n/2, m/2 x n/2 at the top, a quarter of that per level
 * down) and the leaf's own. Returns 0 for invalid arguments.
 */
size_t gf2_mul_workspace_bytes(int64_t m, int64_t k, int64_t n, const gf2_opts *opts);

/*
 * PLS decomposition with rank, in place (Proposition "PLS decomposition";
 * computed by block elimination over 64-column panels following MMPF,
 * Sec. 4.1: pivot search, Gray-code tables of the pivot rows, table-driven row
 * additions that write the multipliers of L, and the final compression of L).
 *
 * On return (stream-ordered): A holds L strictly below the diagonal in
 * columns [0, r) (unit diagonal implied) and S in rows [0, r): row i < r is
 * [L_i in cols < i | 1 at col i | 0 up to col Q[i] | S_i right of Q[i] in its
 * original columns]; rows >= r hold only L. *rank = r. P, Q as above.
 * Identical, bit for bit, to the Gaussian PLS algorithm of the appendix.
 * With opts->cutoff_cols > 0 and n above it, the recursive PLS of Sec. 5 runs
 * instead; its trailing products are sized by the rank of each base case, so
 * that route waits for `stream` (host-blocking) once per base case. The
 * default (MMPF panels) never waits.
 *   A      -- device, m x n, stride words per row (layout above), in/out;
 *   P, Q   -- device int64, length m and n, out (may not alias A or work);
 *   rank   -- device int64, out.
 * m == 0 or n == 0 returns GF2_OK with rank 0 and identity P, Q.
 */
int gf2_pls(uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *P, int64_t *Q, int64_t *rank,
            void *work, size_t work_bytes, const gf2_opts *opts, void *stream);

/*
 * Reduced row echelon form, in place (Definition "Reduced Row Echelon Form").
 * opts->rref_method picks the route; all give the same (unique) result:
 *   GF2_RREF_PLS (default): the PLS route of Table 1: PLS decomposition, then
 *     R = (S restricted to its pivot columns)^-1 . S by an upper-triangular
 *     solve over 64-pivot blocks;
 *   GF2_RREF_M4RI: Algorithm M4RI (Sec. 3.1): every 64-column panel's pivot
 *     search, then one table sweep that clears the panel's pivot columns in
 *     every other row, above and below;
 *   GF2_RREF_HYBRID: M4RI sweeps while the density of the remaining rows (the
 *     set bits of their next panel word, counted by each sweep) stays below
 *     opts->hybrid_permille, PLS sweeps from then on, then the upper solve
 *     over the pivots found after the switch (Sec. 6, "M+P").
 * On return rows [0, r) of A hold the RREF and rows [r, m) are zero.
 *   pivots -- device int64, length n, nullable: pivots[i] = column of the
 *             leading 1 of row i for i < r (the column rank profile), i for i >= r;
 *   rank   -- device int64, out.
 */
int gf2_rref(uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank, int64_t *pivots,
             void *work, size_t work_bytes, const gf2_opts *opts, void *stream);

/*
 * Rank only (the return value of the PLS algorithms). A is NOT modified: the
 * elimination runs on a copy inside the workspace.
 */
int gf2_rank(const uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank, void *work,
             size_t work_bytes, const gf2_opts *opts, void *stream);

/*
 * Product over GF(2): C = A.B (accumulate == 0) or C = C + A.B (accumulate
 * != 0), the trailing update A_SE <- A_SE + A_SW.A_NE of Algorithm PLS
 * (Sec. 5). A is m x k, B is k x n, C is m x n, each with its own stride.
 * C must not overlap A or B. opts->product picks the XOR-table form, the
 * tensor-core form, or Strassen-Winograd recursion over either (7 half-size
 * products and 15 block XORs per level, taken while m, k, n >= 2 x leaf size
 * and k, n are multiples of 2048; the leaf size is opts->cutoff_cols, default
 * 8192). All forms are bit-exact. work may be NULL (an internal workspace is
 * used), else it holds at least gf2_mul_workspace_bytes(m, k, n, opts) bytes
 * (GF2_ENOSPACE otherwise).
 */
int gf2_mul(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb,
            int64_t m, int64_t k, int64_t n, int accumulate, void *work, size_t work_bytes,
            const gf2_opts *opts, void *stream);

/*
 * Batched PLS: many independent matrices in one call (the paper decomposes one
 * matrix at a time; the batch runs the same MMPF block elimination, Sec. 4.1,
 * on every matrix). Two schedules (opts->batch_mode): GF2_BATCH_STEPS runs
 * step b -- the pivot search and the table sweep of panel b -- as one launch
 * over all matrices that have a panel b; GF2_BATCH_PERSISTENT runs the whole
 * batch in one cooperative launch with one CTA per SM, where the largest
 * matrices are eliminated by teams of CTAs (barriers between the pivot search
 * and the sweep of each panel, bounded waits reporting GF2_ETIMEOUT) and the
 * others one per CTA, taken from a device work queue.
 * Each matrix's results are bit for bit those of gf2_pls on it alone without
 * the recursive split (opts->cutoff_cols is ignored).
 *   items  -- HOST array of `count` descriptors; the pointers inside are device
 *             pointers (A in/out, P and Q out, as for gf2_pls). Matrices and
 *             their P, Q must not overlap one another;
 *   ranks  -- device int64[count], out: ranks[i] = rank of matrix i;
 *   work   -- device, gf2_pls_batched_workspace_bytes(items, count, opts)
 *             bytes (which reads only the sizes m, n, stride of the items and
 *             returns 0 for invalid ones), or NULL for the library's internal
 *             workspace.
 * Sizes are read on the host (the schedule of launches depends on them).
 * count == 0 returns GF2_OK. Items with m == 0 or n == 0 get rank 0 and
 * identity P, Q.
 */
typedef struct {
    uint64_t *A;    /* device, m x n, stride words per row */
    int64_t m, n, stride;
    int64_t *P;     /* device int64, length m */
    int64_t *Q;     /* device int64, length n */
} gf2_batch_item;

size_t gf2_pls_batched_workspace_bytes(const gf2_batch_item *items, int64_t count, const gf2_opts *opts);
int gf2_pls_batched(const gf2_batch_item *items, int64_t count, int64_t *ranks, void *work, size_t work_bytes,
                    const gf2_opts *opts, void *stream);

/*
 * The persistent schedule's plan, on the host only (no device call): which
 * matrices of a gf2_pls_batched call get a team of CTAs and which go to the
 * device work queue, for a launch of `ctas` CTAs (gf2_pls_batched uses one
 * per SM). The plan reads only m and n of the items. Outputs are host arrays:
 *   team_of     -- int[ctas]: the team of each CTA, or -1 (a queue worker);
 *                  every team is a contiguous range of a power-of-two number
 *                  of CTAs;
 *   team_size   -- int[ctas] (at most ctas / 2 teams are written): CTAs per team;
 *   member_team -- int[count]: the team of each matrix, or -1 for the queue.
 * Returns the number of teams, or -1 for invalid arguments (bad sizes, ctas
 * outside [1, 1024], a NULL output).
 */
int gf2_batch_plan(const gf2_batch_item *items, int64_t count, int ctas, int *team_of, int *team_size,
                   int *member_team);

/*
 * Rank without allocating device memory. The paper has no counterpart. Some
 * callers cannot call cudaMalloc: a plug-in inside a host application that
 * owns the whole device-memory budget is not allowed to; a latency-bound loop
 * cannot take the device-wide synchronisation and the milliseconds cudaMalloc
 * and cudaFree may cost; a process whose device memory is already reserved by
 * another framework's caching allocator may see the allocation fail. This
 * entry point computes exactly what gf2_rank computes (same arguments, A
 * unchanged), but its workspace is one fixed array of
 * GF2_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits. No call allocates or frees
 * device memory, and none is recorded into or replayed from a library-owned
 * CUDA graph: each call enqueues the elimination directly on `stream` (and on
 * a side stream of the library, ordered by events).
 *   Limit: matrices whose rank workspace, gf2_workspace_bytes(GF2_OP_RANK, m,
 *   n, NULL), exceeds GF2_NOALLOC_SCRATCH_BYTES (4 MiB; e.g. 4096 x 4096 fits,
 *   8192 x 8192 does not) are refused with GF2_ETOOBIG before anything is
 *   enqueued. Other argument errors are those of gf2_rank.
 *   First call per device: with that device current, it looks up the array's
 *   device address (cudaGetSymbolAddress) and creates the side stream and
 *   three events it reuses from then on; make that first call before any
 *   stream capture.
 *   Sharing: every call on a device uses that device's one array, which keeps
 *   the last call's contents (each call re-initialises everything it reads).
 *   Calls whose work can overlap on the GPU, e.g. on two streams of the same
 *   device, race on the array; order them on one stream. Concurrent host
 *   threads are serialised while they enqueue.
 */
#define GF2_NOALLOC_SCRATCH_BYTES (4u << 20)
int gf2_rank_noalloc(const uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank, void *stream);

/*
 * Device-side errors. Kernels that wait on the tensor cores or on a flag give
 * up after a bounded time (2 s) instead of spinning forever; they then record
 * GF2_ETIMEOUT in a per-device status word and finish without writing their
 * outputs. gf2_sync_status waits for `stream` (host-blocking), returns the
 * recorded code (GF2_OK if none) and clears it. The word is per device and
 * sticky: an error from any stream stays until it is read.
 */
int gf2_sync_status(void *stream);

/*
 * Diagnostic for the path above (not part of the method): launches one kernel
 * that waits on a device flag nothing ever sets, with the wait limited to
 * limit_ns nanoseconds (capped at the library's 2 s limit). It returns as soon
 * as the launch is enqueued; a following gf2_sync_status reports GF2_ETIMEOUT.
 */
int gf2_diag_wait_timeout(uint64_t limit_ns, void *stream);

/*
 * Autotuner (not part of the method; no knob changes a result). Times the
 * candidate settings of gf2_opts for `op` on a seeded synthetic m x n matrix of
 * Bernoulli(density) bits on the current device, on `stream`, and returns the
 * fastest in *best (and its mean time in *ms_out, nullable). Host-blocking; it
 * allocates and frees its own device buffers. Candidates:
 *   GF2_OP_PLS / RREF / RANK: tile_words 4, 8 and 16; for PLS with n > 8192 also
 *     the recursive split at 4096 columns with the XOR-table and the
 *     tensor-core product; for RREF also the M4RI route and the hybrid at
 *     150 and 200 per mille;
 *   GF2_OP_MUL (C = A.B with A m x n, B n x n): the XOR-table and the
 *     tensor-core product, and where a level applies (m, n >= 16384, n a
 *     multiple of 2048) Strassen-Winograd over either.
 * The answer is cached per (device, op, ceil(log2 m), ceil(log2 n), density
 * bucket {>= 0.3, >= 0.03, less}); a repeated call returns it without timing.
 * GF2_EINVAL for bad arguments, GF2_ENOMEM if no candidate fits in memory.
 */
int gf2_autotune(int op, int64_t m, int64_t n, double density, gf2_opts *best, double *ms_out, void *stream);

/*
 * Replay of repeated calls (not part of the method; no result changes). One
 * elimination is a few hundred dependent kernel launches on two streams. When
 * gf2_pls (without the recursive split), gf2_rref or gf2_rank is called again
 * with exactly the same arguments (pointers, sizes, options, stream, device),
 * the library captures that call's launches into a CUDA graph and launches the
 * graph on `stream` from then on; the graph reads the buffers' current
 * contents, so the results are those of a direct call. The first occurrence of
 * an argument list runs directly; at most 32 graphs are kept (least recently
 * used dropped). Calls are never captured while launch timing (gf2_prof_enable
 * flag 2) is on, while `stream` is itself being captured by the caller (the
 * launches then go into the caller's graph), or when capture fails.
 * Freeing a buffer and allocating another at the same address keeps replays
 * valid. gf2_replay_enable(0) switches replay off (process-wide; default on);
 * gf2_replay_stats reports how many graphs were captured and how many calls
 * were replayed since the process started (either pointer may be NULL).
 */
void gf2_replay_enable(int on);
void gf2_replay_stats(long long *captured, long long *replayed);

/* Human-readable text for a GF2_* code (static storage). */
const char *gf2_strerror(int code);

/* cudaError_t value of the last CUDA failure seen by this thread (0 if none). */
int gf2_last_cuda_error(void);

/* Library version: major*10000 + minor*100 + patch. */
int gf2_version(void);

/*
 * Diagnostics (not part of the method). flags: 1 = count every kernel launch
 * of the library; 2 = also bracket each launch of the timed kernel classes
 * with a pair of CUDA events on the launching stream. gf2_prof_collect() waits
 * for the recorded events (host-blocking), adds their elapsed times to the
 * class totals and returns the totals of class `cls` since gf2_prof_reset().
 * Profiling state is process-wide; not for concurrent use from several threads.
 */
#define GF2_PROF_SWEEP 0 /* table sweep of a panel (MakeTable1 + AddRowsFromTable) */
#define GF2_PROF_PIVOT 1 /* pivot search of a panel (PlsSubmatrix) */
#define GF2_PROF_RREF 2  /* one 64-pivot block of the RREF back substitution */
#define GF2_PROF_MUL 3   /* product kernels */
#define GF2_PROF_COORDS 4 /* coordinates and multipliers of the rows of a two-panel sweep step */
#define GF2_PROF_CLASSES 5
void gf2_prof_enable(int flags);
void gf2_prof_reset(void);
long long gf2_prof_launches(void);
int gf2_prof_collect(int cls, double *ms_total, long long *launches);

#ifdef __cplusplus
}
#endif
#endif /* GF2_H */
