// basker_internal.h -- plan, task and device-view types of the CUDA library.
//
// Layout in device memory (one arena per handle, all in B = A(P,Q) coordinates):
//   Bp[n+1], Bi[nnzB]        pattern of B, rows sorted; dstart[c] = first entry of
//                            column c inside its diagonal block (entries above it are
//                            the off-diagonal BTF blocks, kept for the solve)
//   bmap[nnzB]               B entry -> index in A's CSC value array (value gather)
//   Bx[nnzB]                 values of B (double)
//   L: Lbeg[n] (int64), Lcnt[n], Li (B rows, ascending), Lx   strictly lower part
//   U: Ubeg[n] (int64), Ucnt[n], Ui (pivot steps, ascending, diagonal last), Ux
//   prow[k] = B row pivoted at step k, pinv = its inverse (-1 = not yet pivoted)
//   Each task (a BTF block, or an ND node) owns one contiguous region of L and of
//   U; its columns are stored one after the other in column order.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/basker.h"

#define BK_MAX_ANC 16          // ND depth limit (65,536 leaves)
#define BK_WARP 32

// One unit of Algorithm 1 work: the columns of a BTF block or of an ND node,
// factored in order by one warp.  Rows of the task's "space" are the only rows a
// column of the task can touch: its subtree [sp_lo, hi) (descendants are already
// pivoted, the node's own rows [lo, hi) are the pivot candidates) followed by the
// rows of its ND ancestors (never pivoted here, they receive the L_kj entries).
struct bk_task {
    int32_t c0, c1;            // columns to factor, c0 >= lo (c0 > lo: a partial redo)
    int32_t lo, hi;            // the node's own rows / columns
    int32_t sp_lo;             // first row of the subtree
    int32_t nanc;              // number of ancestor ranges (ascending rows)
    int32_t anc_lo[BK_MAX_ANC];     // entries past nanc hold INT32_MAX (a sorted table
    int32_t anc_hi[BK_MAX_ANC];     // of 16 for a branch-free search)
    int32_t anc_cum[BK_MAX_ANC];    // rows of the ancestors before range a (INT32_MAX past nanc)
    int32_t anc_sh[BK_MAX_ANC];     // anc_cum[a] - anc_lo[a]: slot = r + (hi - base) + anc_sh[a]
    int32_t space;             // (hi - sp_lo) + sum of ancestor sizes
    int32_t lspace;            // (hi - lo) + sum of ancestor sizes (rows that can be unpivoted)
    int64_t lbeg, lend;        // L region
    int64_t ubeg, uend;        // U region
    int64_t wsoff;             // offset (bytes) of x + bitmaps in the global workspace, -1 = shared
    int64_t ahoff;             // separators: first double of the task's A-hat columns (lspace each)
    int64_t aboff;             // separators: first word of their pattern bitmaps (ceil(lspace/32) each)
    int32_t level;             // height in the ND tree (0: leaves and small BTF blocks)
    int32_t node;              // ND node (postorder) or -1
    int32_t block;             // BTF block
    int32_t dense;             // separators: refactorizations recompute it by the descendant
                               // phase and the dense elimination (the stored-pattern pass skips it)
};

// Status word written by the kernels (device), read back once per call.
struct bk_status {
    unsigned long long first_fail;   // min over failures of (column << 8 | code)
    int32_t capacity;                // nonzero: an L/U region overflowed
    int32_t timeout;                 // nonzero: a wait gave up
    int32_t static_fail;             // columns that rejected their preferred pivot (stored-pattern pass)
    int32_t offdiag;                 // number of columns pivoting off the natural row
    int32_t internal_site;           // first internal-consistency check that fired (0 = none)
    int32_t internal_col;            // and its column
    int32_t repaired;                // columns recomputed by the repair kernel
    int32_t pad;
};

enum { BK_CODE_SINGULAR = 1, BK_CODE_NAN = 2, BK_CODE_INTERNAL = 3 };  // INTERNAL: an index outside its space
enum { BK_DD_RESOLVE = 1, BK_DD_DESC = 2 };    // refactor round flags of a task

// Everything the kernels read, as raw device pointers (passed by value).
struct bk_dev {
    int32_t n;
    int32_t ntasks;
    int32_t prec;                    // arithmetic of the factorization: 0 FP64, 1 FP32 (value
                                     // arrays keep 8-byte slots; FP32 uses them as float arrays)
    const int32_t *Bp, *Bi, *dstart, *bmap, *col_task;
    double *Bx;
    bk_task *tasks;
    int32_t *prow, *pinv;
    const int32_t *pref;             // refactor: the previous pivot rows, preferred
    int64_t *Lbeg, *Ubeg;            // per column: region start
    int64_t *Lend, *Uend;            // per column: region end (capacity)
    int32_t *Lcnt, *Ucnt;
    unsigned long long *pool;        // [0] next free L entry, [1] next free U entry (spill pools)
    int64_t lpool_end, upool_end;    // array sizes: regions of the layout, then the pools
    int32_t *Li, *Ui;
    double *Lx, *Ux;
    bk_status *status;
    int32_t *col_over;               // per column: 1 = its L region overflowed, 2 = its U region
    int32_t *task_stop;              // per task: nonzero once it or a descendant ran out of room
    int32_t *task_fail;              // per task: first column that rejected its preferred pivot
    int32_t *col_fail;               // per column: 1 if it rejected its preferred pivot
    int32_t *dd_start, *dd_flags;    // per task: first column and flags of the current round
    int32_t *touch;                  // per row: epoch of the round that changed its pivot status
    int32_t *dirty_ep;               // per column: epoch of the round that recomputed it
    int32_t *pchg_ep;                // per column: epoch of the round that recomputed it by the reach
    int32_t *touch_ref, *dirty_ref, *pchg_ref;   // the same, numbered by refactorization
    unsigned char *ws;               // global workspace (zero between uses)
    unsigned long long *trace;       // per-item timeline (builds with BK_TRACE only; else null)
    int32_t *done;                   // per column: epoch of its last completion (static kernel)
    int32_t *order;                  // static kernel claim order (topological)
    const int32_t *iorder;           // levels kernel claim order: tasks by level, interleaved
    int32_t *counter;                // claim counters
    int32_t *level;                  // per column level in the static DAG
    double *ahat;                    // separator columns after the descendant phase (dense, L-space)
    uint32_t *abits;                 // their patterns
    int32_t *dcnt;                   // per column: U entries written by the descendant phase
    unsigned char *wsd;              // descendant-phase workspace, one slice per warp
    int64_t wsd_slice;               // bytes per slice
    int32_t wsd_warps;
    int32_t dd_words;                // reach bitmaps per warp in shared memory (0: in the slice)
    double *sx;                      // static kernel: per-warp dense x slices
    int64_t sx_stride;               // doubles per warp slice
    int32_t sx_warps;
    // solve
    int32_t nblocks;
    const int32_t *block_ptr;
    const int32_t *P, *Q;
};

// Value arrays seen in the factorization's arithmetic type V.
template <typename V> __host__ __device__ __forceinline__ V *vals(double *p) { return reinterpret_cast<V *>(p); }

// Host-side plan built by the symbolic pass.
struct bk_plan {
    int32_t n = 0, nblocks = 0, nd_block = -1, nd_leaves = 0, depth = 0;
    int64_t nnz = 0;
    std::vector<int32_t> P, Q, block_ptr, nd_ptr, nd_first, nd_height;
    std::vector<int32_t> Bp, Bi, bmap, dstart;
    std::vector<bk_task> tasks;
    std::vector<int32_t> col_task;
    std::vector<std::vector<int32_t>> level_tasks;   // task ids per GP level
    // pattern under the preferred (natural) pivots, in the task-region layout
    std::vector<int64_t> sLbeg, sUbeg, lcapc, ucapc;  // region starts; per-column capacities
    std::vector<int32_t> sLcnt, sUcnt, sLi, sUi, sprow;
    std::vector<int32_t> slevel, sorder;              // static DAG levels and claim order
    std::vector<int32_t> iorder;                      // tasks by level, each level's tasks taking turns
    int64_t lcap = 0, ucap = 0, nnz_l_sym = 0, nnz_u_sym = 0;
    int64_t lpool = 0, upool = 0;                     // spill pools after the layout's regions
    int64_t ws_bytes = 0;                             // GP global workspace
    int64_t ahat_doubles = 0, ahat_words = 0;         // separator A-hat scratch
    int64_t wsd_slice = 0;                            // column-per-warp slice of level 0 (bytes)
    int32_t wsd_warps = 0;                            // and its slices
    // per ND level: the slice its tasks need (x over the largest space, bitmaps)
    // and the slices that fit the workspace; the workspace holds wsd_bytes
    std::vector<int64_t> level_slice;
    std::vector<int32_t> level_warps;
    int64_t wsd_bytes = 0;
    int32_t dd_words = 0;                             // shared-memory reach bitmaps per warp (words)
    std::vector<int32_t> level_dd_words;              // the same for the tasks of each ND level
    int32_t max_space = 0;
    int32_t symbolic_singular = -1;                   // first column without a structural pivot
    bool counts_only = false;                         // Algorithm 3's counts: no pattern, no schedule
    double slack = 0.5;
};

// symbolic.cpp
void bk_task_ranges(bk_task &T);   // the padded ancestor tables from anc_lo / anc_hi / nanc
int bk_plan_build(int32_t n, const int32_t *colptr, const int32_t *rowind, const int32_t *P,
                  const int32_t *Q, int32_t nblocks, const int32_t *block_ptr, int32_t nd_block,
                  int32_t nd_leaves, const int32_t *nd_node_ptr, double slack, bk_plan &plan,
                  int32_t *bad_col, int mode = 0);
void bk_plan_layout(bk_plan &plan);                      // L/U regions, workspaces
void bk_plan_regrow(bk_plan &plan, const int32_t *over); // after an overflow (per-column flags)
size_t bk_task_smem_bytes(const bk_task &t);
// kernels_dense.cu: the in-node phase of a separator as one dense elimination
#define BK_DENSE_SMEM (200 * 1024)
// refactorization rounds: a waited-for step's L column staged in shared memory,
// up to BK_DD_SCAP entries (rows, values with 16 entries of slack for the
// 16-byte boundaries, and what each row adds), per warp
#define BK_DD_SCAP 512
// per warp: rows, values, what each row adds, the x values under the rows, the
// column's own previous L rows (compared with the new ones), the rows prestaged
// before a wait and the rows' slots
#define BK_DD_STAGE_BYTES ((BK_DD_SCAP + 16) * 12 + BK_DD_SCAP * 12 + (BK_DD_SCAP + 16) * 8 + BK_DD_SCAP * 4)
size_t bk_dense_node_smem(const bk_task &t);
bool bk_dense_node_eligible(const bk_task &t);
// separators of at least BK_DENSE_CLUSTER_MIN columns run on a cluster of
// BK_DENSE_CLUSTER blocks (columns dealt round-robin), smaller ones on one block
#define BK_DENSE_CLUSTER 8
#define BK_DENSE_CLUSTER_MIN 64
int bk_dense_node_cluster(const bk_task &t);
void bk_launch_dense_nodes(const bk_dev &d, const int32_t *task_ids, int32_t ntasks, size_t smem, double tau,
                           int pref_mode, int cluster, void *stream);
bool bk_task_fits_smem(const bk_task &t);

// kernels (launchers), kernels_*.cu
void bk_launch_gather(const bk_dev &d, const double *values, int64_t nnz, void *stream);
void bk_launch_gp_tasks(const bk_dev &d, const int32_t *task_ids, const int32_t *task_c0,
                        int32_t ntasks, size_t smem, double tau, int pref_mode, void *stream);
// ncols_dev (if not null): the number of columns, read on the device (ncols is
// then the largest it can be, for the launch size)
void bk_launch_gp_desc(const bk_dev &d, const int32_t *cols, int32_t ncols, int32_t *counter,
                       void *stream, const int32_t *ncols_dev = nullptr);
// kernels_desc.cu: the descendant phase on the stored patterns, verified; the
// columns that fail are listed in redo[0 .. *nredo) for bk_launch_gp_desc
// sizes of the descendant phase's on-chip layout for one ND level
struct bk_desc_par {
    int32_t hmask;      // slot table entries - 1 (a power of two minus one)
    int32_t xs, xl;     // stored steps and L-space rows of a column kept on chip, at most
    int32_t prs_words;  // words of the bitmap over the largest descendant space
    int32_t cap;        // L entries per staging buffer (512 or 1024)
    size_t smem;        // dynamic shared memory (0: the bitmap does not fit; reach kernel only)
};
bk_desc_par bk_desc_fast_params(const bk_plan &pl, int32_t level);
void bk_launch_desc_fast(const bk_dev &d, const int32_t *cols, int32_t ncols, int32_t *counter, int32_t *redo,
                         int32_t *nredo, const bk_desc_par &par, void *stream);
void bk_launch_dd(const bk_dev &d, const int32_t *cols, int32_t ncols, int32_t *counter, double tau,
                  int32_t epoch, long long budget, int32_t refno, void *stream, int max_warps = 0);
void bk_launch_static(const bk_dev &d, int32_t ncols, double tau, int32_t epoch,
                      long long budget, int blocks, void *stream);
void bk_launch_levels(const bk_dev &d, int32_t epoch, long long budget, int blocks, void *stream,
                      bool check = false);
int bk_static_blocks();
// kernels_repair.cu: the rejected pivots of the ND leaves and BTF blocks resolved
// in column order after the stored-pattern pass (one warp per task)
size_t bk_repair_smem(const bk_task *tasks, const int32_t *ids, int32_t count, size_t limit);
void bk_launch_repair(const bk_dev &d, const int32_t *tasks, int32_t ntasks, int32_t *counter, double tau,
                      size_t smem, int ctas, void *stream);
size_t bk_gp_smem_limit();
