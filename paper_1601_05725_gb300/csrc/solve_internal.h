// solve_internal.h -- work items of the BTF / ND solve (kernels_solve.cu).
#pragma once

#include <cstdint>
#include <vector>

#include "basker_internal.h"

enum { BK_ITEM_BLOCK = 0, BK_ITEM_FWD = 1, BK_ITEM_BWD = 2 };

struct bk_sitem {
    int32_t type;
    int32_t task;
    int32_t dep_beg, dep_end;     // items to wait for (indices into deps)
    int32_t desc_beg, desc_end;   // FWD: descendant tasks whose buffers hold this node's terms
};

struct bk_solve_dev {
    int32_t nitems;
    const bk_sitem *items;
    const int32_t *deps;
    const int32_t *desc;
    int32_t *item_done;
    const int32_t *offp, *offj, *offpos;   // coupling entries of B by row: columns of later blocks
    const int64_t *acc_off;                // per task: first slot of its contribution buffer
    int64_t acc_stride;                    // slots per right-hand side
    double *acc;
    double *w;                             // n x nrhs, indexed by pivot step
    const int32_t *Ls;                     // L's row indices as pivot steps
    int64_t smem_bytes;                    // dynamic shared memory of the solve kernel
};

struct bk_solve_plan {
    std::vector<bk_sitem> items;
    std::vector<int32_t> deps, desc, offp, offj, offpos;
    std::vector<int64_t> acc_off;
    int64_t acc_stride = 0;
    int64_t smem_bytes = 0;                // largest item (own rows + ancestor buffer), capped
};

void bk_solve_plan_build(const bk_plan &pl, bk_solve_plan &sp);
void bk_launch_lsteps(const bk_dev &d, int *Ls, void *stream);
void bk_launch_solve(const bk_dev &d, const bk_solve_dev &s, int32_t nrhs, const double *b, int32_t ldb,
                     double *x, int32_t ldx, int32_t epoch, long long budget, void *stream);
