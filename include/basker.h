/*
 * basker.h -- C ABI of the GB300 sparse LU library (libbasker_gb300.so).
 *
 * The library factors A (n x n, CSC) as the paper "Basker: A Threaded Sparse LU
 * Factorization Utilizing Hierarchical Parallelism and Data Layouts" (Booth,
 * Rajamanickam, Thornquist, arXiv 1601.05725) describes: A is permuted by fixed
 * row/column permutations P, Q into block triangular form (BTF, Sec. II and
 * III-A), only the diagonal blocks are factored (Sec. II), one diagonal block may
 * carry a nested-dissection (ND) tree (Sec. III-C), and every block is factored
 * with the left-looking Gilbert-Peierls method (Algorithm 1) with threshold
 * partial pivoting confined to the block, or to the ND node (the diagonal blocks
 * A_ii / A_jj of Fig. 3a).  Refactorization reuses the pattern for a sequence of
 * matrices (Sec. V, the circuit-simulation sequence), and the solve is the BTF
 * back-substitution with the off-diagonal blocks kept as values of A (Sec. III-B).
 *
 * Conventions for every entry point:
 *   - Indices are 0-based int32.  CSC: colptr[n+1], rowind[nnz], rows strictly
 *     increasing inside a column.
 *   - "new -> old" permutations: B = A(P,Q) means B(i,j) = A(P[i], Q[j]).
 *   - Pointers named *_dev are device pointers (CUDA global memory) read or
 *     written in stream order on the stream passed in; *_host are host pointers.
 *   - Streams are passed as void* holding a cudaStream_t (NULL = legacy default).
 *   - The caller owns every array it passes; the library copies what it keeps.
 *     The handle owns all device memory the library allocates.
 *   - Return value: a basker_status (0 = success).  A handle is not thread-safe:
 *     use one handle from one host thread and one stream at a time.
 *   - No entry point falls back to the CPU: device work runs only in this
 *     library's CUDA kernels.
 */
#ifndef BASKER_GB300_H
#define BASKER_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct basker_s *basker_t;

typedef enum {
    BASKER_OK = 0,
    BASKER_ERR_INVALID_ARG = 1,   /* bad size, pointer, permutation or CSC pattern */
    BASKER_ERR_NOT_BTF = 2,       /* an entry of B lies below the diagonal blocks (Sec. II) */
    BASKER_ERR_BAD_ND = 3,        /* an entry joins two ND nodes on different branches (Sec. III-C) */
    BASKER_ERR_SINGULAR = 4,      /* no nonzero pivot candidate; basker_info gives the column */
    BASKER_ERR_NAN = 5,           /* a non-finite value in a factored column; column in basker_info */
    BASKER_ERR_OOM = 6,           /* device or host allocation failed */
    BASKER_ERR_TIMEOUT = 7,       /* an in-kernel wait exceeded options.wait_budget_cycles */
    BASKER_ERR_CUDA = 8,          /* a CUDA runtime call failed */
    BASKER_ERR_NOT_FACTORED = 9   /* refactor/solve/export before a successful factor */
} basker_status;

typedef struct {
    double tau;                   /* pivot threshold in (0,1]; default 1e-3 */
    double slack;                 /* extra L/U capacity over the symbolic count; default 1.0 */
    long long wait_budget_cycles; /* clock64 cycles any in-kernel wait may spin; default 2e10 */
    int factor_mode;              /* 0 (default): the in-node phase of an ND separator whose
                                     column state fits in shared memory runs as one dense
                                     right-looking elimination by a block of threads; 1: every
                                     in-node phase column by column in one warp.  The
                                     factors are the same (other values: INVALID_ARG) */
    int timing;                   /* nonzero: record CUDA events around every kernel launch
                                     on the caller's stream; totals in basker_info */
    int precision;                /* 0 (default): FP64 factorization and solve.
                                     1: FP32 factorization and FP32 triangular solves,
                                     refined in FP64 (residual b - A x, update and backward
                                     error in FP64) until the backward error reaches ir_tol;
                                     a factorization whose pivot growth exceeds growth_limit,
                                     that fails in FP32, or whose refinement stalls is redone
                                     in FP64 (BASKER_OK; basker_info counts it).
                                     2: FP64 factorization; every solve refined in FP64
                                     the same way until its backward error reaches ir_tol
                                     (at most ir_max_iter solves; no FP64 redo needed) */
    int ir_max_iter;              /* precision 1, 2: refinement steps at most; default 10 */
    double ir_tol;                /* precision 1, 2: backward error to reach; default 1e-13 */
    double growth_limit;          /* precision 1: max over BTF blocks of max|U_d| / max|B_d|
                                     above which the FP32 factors are not used; default 1e4 */
    int refactor_switch;          /* the pivots a refactorization's stored-pattern pass
                                     rejected are resolved, 0 (default): by rounds of
                                     column recomputation until they have taken as long
                                     as the handle's last complete factorization, the rest
                                     then one complete Algorithm 1 pass with the previous
                                     pivots preferred (that pass at once when more than
                                     max(16, n/200) pivots were rejected); 1: rounds
                                     only; 2: the complete
                                     pass at once; 3: when every ND separator fits the
                                     dense elimination, the repair pass (one block of
                                     threads per ND leaf or BTF block walks its columns
                                     from the first rejection on, in column order, on the
                                     device, with no host round trip), else as 0.  The
                                     factors are the same in every mode (other values:
                                     INVALID_ARG). */
    int graphs;                   /* nonzero (default): the launches that follow every
                                     factorization are replayed from a CUDA graph captured
                                     once per L/U arena; 0: launched one by one */
    int symbolic_mode;            /* 0 (default): basker_symbolic sizes L and U by a structural
                                     Gilbert-Peierls pass under the natural pivots (exact
                                     counts, and the pattern and schedule that let
                                     basker_factor take the refactorization's path);
                                     1: by Algorithm 3's elimination-tree counts of the
                                     symmetric structure (upper bounds, no pattern stored,
                                     cheaper; every basker_factor runs the complete pass);
                                     2: by Algorithm 3 with its interval estimates (Sec.
                                     III-C): the leaves and BTF blocks counted as in 1,
                                     every separator column taken dense between the lowest
                                     and highest row its descendants' lest ranges give
                                     (looser upper bounds of 1's, column by column; no
                                     pattern stored); other values: INVALID_ARG */
    int reserved[1];
} basker_options;

typedef struct {
    int32_t n;
    int32_t nblocks;              /* BTF blocks */
    int32_t nd_block;             /* ND block index or -1 */
    int32_t nd_leaves;
    int64_t nnz_a;                /* entries of A */
    int64_t nnz_l;                /* stored strictly-lower entries of L (unit diagonal implied) */
    int64_t nnz_u;                /* stored entries of U, diagonal included */
    int64_t nnz_l_sym, nnz_u_sym; /* symbolic counts under the preferred (diagonal) pivots */
    double flops;                 /* sum_j l_j (2 u_j + 1) of the current factors */
    int32_t failed_column;        /* column named by SINGULAR / NAN, else -1 */
    int32_t last_repivot_columns; /* columns recomputed by the reach in the last refactor */
    int32_t off_diagonal_pivots;  /* columns whose pivot is not the natural row */
    int32_t capacity_regrows;     /* times the L/U arena was regrown */
    int64_t device_bytes;         /* device memory held by the handle */
    int32_t gp_launches;          /* kernel launches of the last factor/refactor */
    int32_t static_launches;
    int64_t kernel_launches;      /* all kernel launches since basker_symbolic */
    double kernel_ms[10];         /* with options.timing: device time per kernel kind since
                                     the last basker_info call: [0] value gather,
                                     [1] stored-pattern refactor, [2] DAG levels,
                                     [3] in-node Algorithm 1, [4] separator descendant
                                     phase, [5] solve, [6] separators' in-node phase as
                                     dense eliminations,
                                     [7] refactorization rounds after the stored-pattern
                                     pass, [8] factors transposed into rows for the
                                     solve, [9] FP64 refinement (precision 1) */
    int32_t internal_site;        /* nonzero: code of the internal consistency check that
                                     failed (reported as INVALID_ARG), for diagnosis */
    int32_t internal_col;         /* column of that check */
    int32_t last_rounds;          /* redo rounds of the last refactor (0: no pivot rejected) */
    int32_t ir_iterations;        /* precision 1: refinement steps of the last solve */
    int32_t ir_fallbacks;         /* precision 1: factorizations redone in FP64 so far */
    int32_t precision_used;       /* arithmetic of the factors the last solve used: 0 FP64, 1 FP32 */
    int32_t tuned_static_blocks;  /* basker_autotune's choices (0: defaults): persistent blocks */
    int32_t tuned_solve_blocks;   /* of the stored-pattern pass and of the solve */
    double ir_eta;                /* precision 1: backward error after the last solve's refinement */
    double growth;                /* precision 1: pivot growth of the last FP32 factorization */
    int32_t kernel_calls[10];     /* launches per kernel kind (as kernel_ms) since the last
                                     basker_info call, counted with or without timing */
    int32_t cuda_error;           /* after a CUDA status: the runtime's error code of the last
                                     failing call made by this thread, and */
    int32_t cuda_line;            /* the library source line of that call (diagnosis) */
    int64_t rounds_columns;       /* columns processed by refactorization rounds since the
                                     last basker_info call */
    int32_t full_refactors;       /* refactorizations finished by a complete Algorithm 1
                                     pass instead of rounds (options.refactor_switch) */
    int32_t graph_launches;       /* CUDA graph replays so far (options.graphs) */
    int32_t static_factors;       /* basker_factor calls served by the stored-pattern path
                                     (natural pivots preferred) instead of a complete pass */
    int32_t pad1;
} basker_info_t;

/* Defaults listed in basker_options. */
void basker_default_options(basker_options *opt);

/* The symbolic counts alone, on the host (no device, no handle): the same
 * arguments as basker_symbolic, then mode (0: the structural pass under the
 * natural pivots, exact for those pivots; 1: Algorithm 3's elimination-tree
 * counts of the symmetric structure, Sec. III-C, an upper bound of mode 0's; 2:
 * Algorithm 3 with the interval (lest) estimates for the separators, an upper
 * bound of mode 1's) and
 * two host arrays of n ints (either may be NULL) receiving each column's L count
 * (strictly lower entries) and U count (diagonal included).  Errors: INVALID_ARG,
 * NOT_BTF, BAD_ND; the arrays are untouched on error. */
int basker_symbolic_counts(int32_t n, const int32_t *colptr, const int32_t *rowind,
                           const int32_t *P, const int32_t *Q,
                           int32_t nblocks, const int32_t *block_ptr,
                           int32_t nd_block, int32_t nd_leaves, const int32_t *nd_node_ptr,
                           int mode, int32_t *l_count, int32_t *u_count);

/* Analyse a pattern (host arrays; Sec. III-A/III-C orderings are inputs).
 *   n, colptr, rowind: pattern of A (host).
 *   P, Q: host, new -> old permutations putting A in BTF order.
 *   nblocks, block_ptr[nblocks+1]: BTF block boundaries in B's numbering
 *     (0 = b_0 < b_1 < ... < b_nblocks = n).
 *   nd_block: index of the block carrying the ND tree, or -1.
 *   nd_leaves: power of two; nd_node_ptr[2*nd_leaves]: row/column boundaries of
 *     the ND nodes in postorder (left subtree, right subtree, separator), from
 *     block_ptr[nd_block] to block_ptr[nd_block+1]; nodes may be empty.
 *   opt: options (NULL = defaults).  out: receives the handle.
 * Checks the BTF and ND invariants, runs the structural pass or Algorithm 3's
 * counts (options.symbolic_mode: capacities, the level schedule of Algorithm 4's
 * dependency tree), allocates the device arena and uploads the plan.  Errors: INVALID_ARG, NOT_BTF, BAD_ND, OOM, CUDA;
 * *out is NULL on error. */
int basker_symbolic(int32_t n, const int32_t *colptr, const int32_t *rowind,
                    const int32_t *P, const int32_t *Q,
                    int32_t nblocks, const int32_t *block_ptr,
                    int32_t nd_block, int32_t nd_leaves, const int32_t *nd_node_ptr,
                    const basker_options *opt, basker_t *out);

/* Numeric factorization (Algorithm 1 on every BTF block; Algorithm 4's levels on
 * the ND block).  values_dev: nnz(A) doubles, device, in A's CSC order.  Pivots
 * prefer the natural row.  Synchronises the stream at the end to read a 16-byte
 * status.  Errors: SINGULAR, NAN (column in basker_info), TIMEOUT, CUDA, OOM. */
int basker_factor(basker_t h, const double *values_dev, void *stream);

/* Refactorization of a new matrix with the same pattern (Sec. V): each column
 * prefers the pivot row of the previous factorization; columns that keep it are
 * computed on the stored pattern (column-level dataflow), and a node whose
 * column rejects its preferred pivot is recomputed from that column on with the
 * reach of Algorithm 1, together with its ancestors.  The result equals a fresh
 * factorization with those preferences.  Errors as basker_factor, and
 * NOT_FACTORED. */
int basker_refactor(basker_t h, const double *values_dev, void *stream);

/* Solve A X = B for nrhs right-hand sides (column-major, leading dimensions ldb,
 * ldx >= n, device pointers; b_dev and x_dev may not overlap).  BTF blocks from
 * last to first: subtract the off-diagonal blocks' products, then the L and U
 * solves of the block.  Asynchronous on the stream.  With options.precision 1
 * the solves run on the FP32 factors and are refined in FP64 (each step
 * synchronises the stream once to test the backward error); a stalled
 * refinement refactors in FP64 and solves with those factors.  Errors:
 * INVALID_ARG, NOT_FACTORED, CUDA, OOM. */
int basker_solve(basker_t h, int32_t nrhs, const double *b_dev, int32_t ldb,
                 double *x_dev, int32_t ldx, void *stream);

/* End-to-end call on host buffers: copies values and b from host memory to the
 * device, refactors (or factors, if refactor != 0 is not possible yet), solves
 * and copies x back, synchronising the stream.  values_host: nnz(A) doubles in
 * A's CSC order; b_host/x_host: n x nrhs column-major (ld = n). */
int basker_refactor_solve_host(basker_t h, const double *values_host, int32_t nrhs,
                               const double *b_host, double *x_host, void *stream);

/* Launch-size tuning (no counterpart in the paper).  The stored-pattern pass,
 * the refactorization rounds and the solve are persistent kernels whose warps
 * claim work; how many blocks they launch changes their speed, not their
 * results.  This runs refactor(values_dev) + solve(b_dev) (one right-hand side,
 * device pointers, n doubles) a few times for each candidate launch size, one
 * kernel at a time, and keeps the fastest on the handle; basker_info reports the
 * choices.  The handle's factors and pivots are those of values_dev afterwards.
 * Blocks the stream.  Errors: those of basker_refactor / basker_solve
 * (the handle then keeps the default sizes). */
int basker_autotune(basker_t h, const double *values_dev, const double *b_dev, void *stream);

/* The latencies that bound one link of a dependency chain of the factorization
 * or the solve (Sec. IV: a thread waits point to point for what it reads), on
 * the current device, for performance models: ns_out[0] = one flag handoff
 * between two blocks through global memory (a release store seen by an acquire
 * load), ns_out[1] = one dependent FP64 fma, ns_out[2] = one dependent FP64
 * division.  ns_out: 3 host doubles.  No handle; synchronous; allocates and
 * frees a few bytes of device memory.  Errors: INVALID_ARG (null), OOM, CUDA,
 * TIMEOUT (a handoff wait ran past 2e9 cycles; nothing is written). */
int basker_probe_latency(double *ns_out);

/* Size, in doubles, of the fixed device array basker_solve_noalloc works in
 * (8 MiB on every GPU that loads the library, held until the process exits). */
#define BASKER_NOALLOC_SCRATCH_DOUBLES (1 << 20)

/* basker_solve for callers that must not allocate device memory.  The paper has
 * no counterpart; this entry point exists for users of the library, such as a
 * simulator's time-step loop whose device memory is all reserved up front by
 * its own pool or caching allocator (a cudaMalloc there can fail while the pool
 * holds the memory, and cudaFree synchronises the whole device), which still
 * need to solve with factors made earlier.
 *   Same arguments and results as basker_solve; the handle must be factored.
 *   The solve's two work vectors (the forward results and the solution by
 *   pivot step, n * nrhs doubles each) live in one array of
 *   BASKER_NOALLOC_SCRATCH_DOUBLES doubles compiled into the library; its other
 *   buffers (per-row flags, the factors by rows) are the handle's, made when it
 *   was factored.  So the call performs no cudaMalloc, cudaFree or other
 *   allocation.  It needs 2 * nrhs * n doubles; larger requests return
 *   BASKER_ERR_INVALID_ARG without launching anything, and so does a handle with
 *   options.precision 1 or 2 (refined solves, whose refinement needs buffers of
 *   its own).  With options.timing the call records no kernel time; it sets
 *   basker_info's precision_used to 0 (FP64 factors).
 *   The first call on a device looks up the array's device address (with that
 *   device current) and caches it; make that first call before any stream
 *   capture begins.
 *   All calls, from every handle, share the one array and the solve leaves its
 *   contents behind; everything the solve reads it writes first in the same
 *   call.  Calls whose work overlaps on the GPU (different streams, or
 *   concurrent host threads) race on the array: serialise them.
 *   Errors: INVALID_ARG, NOT_FACTORED, CUDA. */
int basker_solve_noalloc(basker_t h, int32_t nrhs, const double *b_dev, int32_t ldb,
                         double *x_dev, int32_t ldx, void *stream);

/* Counters of the handle (sizes, flops, failing column, repivots). */
int basker_info(basker_t h, basker_info_t *out);

/* Copy the factors to host memory, in B's coordinates: prow[k] = B row pivoted
 * at step k (n ints); L strictly lower with rows = pivot steps, U upper with the
 * diagonal last, each column sorted by step.  Call with Li == NULL to get the
 * sizes only (*nnz_l, *nnz_u).  Lp/Up are int64[n+1].  Synchronises. */
int basker_export(basker_t h, int32_t *prow, int64_t *Lp, int32_t *Li, double *Lx,
                  int64_t *Up, int32_t *Ui, double *Ux, int64_t *nnz_l, int64_t *nnz_u);

/* Release the handle and all its device memory (NULL is allowed). */
void basker_free(basker_t h);

/* Static string naming a status. */
const char *basker_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* BASKER_GB300_H */
