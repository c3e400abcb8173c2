// solve_internal.h -- the BTF solve by rows (kernels_solve.cu, solve_plan.cpp).
#pragma once

#include <cstdint>
#include <vector>

#include "basker_internal.h"

// Factors by rows in pivot-step space, rebuilt after every factorization: row i
// of L holds (k, L(i,k)) for k < i in ascending k; row i of U holds (k, U(i,k))
// for k > i in descending k; Ud[i] = U(i,i).  Row-wise evaluation in these orders
// performs, for every entry of the solution, the same fma sequence as the
// column-wise sweeps of the BTF solve.
struct bk_rows {
    int64_t *Lrp, *Urp;          // n + 1 row starts
    int32_t *Lrk, *Urk;          // column steps
    double *Lrx, *Urx;           // values
    int32_t *Ls;                 // L's row indices as steps, in L's column order
    int32_t *tk;                 // unsorted scatter (steps), capacity max(L, U) entries
    double *tx;                  // unsorted scatter (values)
    double *Ud;                  // n diagonal entries of U
    int32_t *cnt;                // 2 (n + 1) row counts and cursors
    int64_t *part;               // per-block partial sums of the row-start scan
    // rows longer than BK_LONG_ROW are ordered by a column bitmap, one block a row
    int32_t *longs;              // [0] count, then the long rows
    uint32_t *sbits;             // per block: the row's column bitmap
    int32_t *spre;               // per block: popcount prefix of the bitmap words
    int64_t swords;              // words of each block's bitmap (n / 32 + 2)
};

#define BK_LONG_ROW 512
#define BK_LONG_CTAS 64

struct bk_solve_dev {
    int32_t nitems;               // every step forward and backward, and every ND separator twice
    int32_t *items;               // k < n: forward row k; n + t: forward sweep of separator task t;
                                  // ~k, ~(n + t): the same backward
    // ND leaves: their rows' places in items are filled after every factorization,
    // all leaves together, in order of the factorization's column levels
    // (increasing forward, decreasing backward; see kernels_solve.cu)
    int32_t nleaves;
    const int32_t *leaf_tasks;
    int32_t leaf_rows, leaf_f0, leaf_b0, leaf_maxrows;
    int32_t *leaf_bad;            // per leaf: the levels do not order its forward rows
    int32_t *lcnt;                // 2 (leaf_maxrows + 1): per-key counts, then starts
    const int32_t *cutlo, *cuthi; // per step: its separator's own rows [lo, hi), or lo = hi = -1
    const int32_t *offp, *offj, *offpos;  // coupling of B by row: columns of later blocks
    int32_t *fdone, *bdone;       // per-step flags of the forward and the backward pass
    double *w;                    // n x nrhs, forward results by step
    double *z;                    // n x nrhs, the solution by step
    bk_rows r;
    // the separators' own triangles: the sweep items of items (n + t forward,
    // ~(n + t) backward) in claim order; sweeper block b of nsb takes the sweeps
    // b, b + nsb, ... (a whole block a sweep; the row warps skip them)
    int32_t nsweeps;
    const int32_t *sweeps;
    int32_t sw_win;               // entries of a column copied ahead per pipeline stage
    int32_t sw_zrows;             // a node of up to this many rows is swept in shared memory
    size_t sw_smem;               // the kernel's dynamic shared memory (a sweeper's needs)
    int32_t sw_cap[2];            // co-resident blocks with it (FP64, FP32 kernel)
};

struct bk_solve_plan {
    std::vector<int32_t> items, offp, offj, offpos, cutlo, cuthi, leaf_tasks, sweeps;
    int32_t leaf_rows = 0, leaf_f0 = -1, leaf_b0 = -1, leaf_maxrows = 0;
    int32_t sw_maxm = 0;          // rows of the largest separator
};

void bk_solve_plan_build(const bk_plan &pl, bk_solve_plan &sp);
void bk_launch_rows(const bk_dev &d, const bk_rows &r, void *stream);
void bk_launch_leaf_order(const bk_dev &d, const bk_solve_dev &s, void *stream);
// permute: b is indexed by A's rows and x by A's columns (b(P), x(Q)); otherwise
// both are in B's row / column space (the refinement's corrections).
void bk_launch_solve(const bk_dev &d, const bk_solve_dev &s, int32_t nrhs, const double *b, int32_t ldb,
                     double *x, int32_t ldx, int32_t epoch, long long budget, void *stream, bool permute = true,
                     int max_ctas = 0);
int bk_solve_blocks();   // persistent blocks of the solve kernel at full occupancy (4 warps each)
// The sweep geometry of a plan (sw_win, sw_zrows) and the kernel's dynamic
// shared memory for it.
void bk_solve_sweep_setup(bk_solve_dev &s, int32_t sw_maxm);
