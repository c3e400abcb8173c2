// solve_plan.cpp -- claim order and coupling rows of the BTF solve (host side).
#include <algorithm>

#include "solve_internal.h"

void bk_solve_plan_build(const bk_plan &pl, bk_solve_plan &sp)
{
    const int32_t n = pl.n;
    std::vector<int32_t> blk((size_t)n);
    for (int32_t d = 0; d < pl.nblocks; d++)
        for (int32_t i = pl.block_ptr[(size_t)d]; i < pl.block_ptr[(size_t)d + 1]; i++) blk[(size_t)i] = d;
    // Coupling entries (above the diagonal blocks) grouped by row of B.  The BTF
    // solve runs the blocks from last to first and, after block d, subtracts
    // B(r, j) z_j for its columns j in ascending order from the rows of earlier
    // blocks; each row takes its terms in that order: block descending, then
    // column ascending.
    sp.offp.assign((size_t)n + 1, 0);
    for (int32_t j = 0; j < n; j++)
        for (int32_t e = pl.Bp[(size_t)j]; e < pl.dstart[(size_t)j]; e++) sp.offp[(size_t)pl.Bi[(size_t)e] + 1]++;
    for (int32_t r = 0; r < n; r++) sp.offp[(size_t)r + 1] += sp.offp[(size_t)r];
    sp.offj.assign((size_t)sp.offp[(size_t)n], 0);
    sp.offpos.assign((size_t)sp.offp[(size_t)n], 0);
    {
        std::vector<int32_t> cur(sp.offp.begin(), sp.offp.end() - 1);
        for (int32_t d = pl.nblocks - 1; d >= 0; d--)
            for (int32_t j = pl.block_ptr[(size_t)d]; j < pl.block_ptr[(size_t)d + 1]; j++)
                for (int32_t e = pl.Bp[(size_t)j]; e < pl.dstart[(size_t)j]; e++) {
                    const int32_t r = pl.Bi[(size_t)e];
                    sp.offj[(size_t)cur[(size_t)r]] = j;
                    sp.offpos[(size_t)cur[(size_t)r]++] = e;
                }
    }
    // Claim order: blocks from last to first; in each, the forward rows, then the
    // backward rows.  Every item waits only for items claimed before it.  In a
    // block without ND the forward rows go in ascending step order and the
    // backward rows in descending order.  In the ND block, forward, tree levels
    // from the leaves up; backward, levels from the root down.  The rows of the
    // nodes of a level take turns row by row (ascending in each node forward,
    // descending backward), so that the warps in flight cover the whole level.
    // A leaf's rows are complete row items.  A separator (a node above others)
    // is dense: its row items take only the terms from outside the node
    // (coupling and descendants forward, ancestors backward), and one sweep item
    // per separator, after its rows, solves the node's own triangle in one block.
    sp.items.clear();
    sp.sweeps.clear();
    sp.sw_maxm = 0;
    sp.items.reserve((size_t)2 * (size_t)n + 2 * pl.tasks.size());
    sp.cutlo.assign((size_t)n, -1);
    sp.cuthi.assign((size_t)n, -1);
    int32_t maxh = 0;
    for (const auto &T : pl.tasks) maxh = std::max(maxh, T.level);
    auto is_sep = [&](const bk_task &T) { return T.node >= 0 && T.sp_lo < T.lo; };
    for (const auto &T : pl.tasks)
        if (is_sep(T))
            for (int32_t i = T.lo; i < T.hi; i++) {
                sp.cutlo[(size_t)i] = T.lo;
                sp.cuthi[(size_t)i] = T.hi;
            }
    auto interleave = [&](const std::vector<int32_t> &tasks, bool fwd) {
        int32_t longest = 0;
        for (int32_t t : tasks) longest = std::max(longest, pl.tasks[(size_t)t].hi - pl.tasks[(size_t)t].lo);
        for (int32_t q = 0; q < longest; q++)
            for (int32_t t : tasks) {
                const bk_task &T = pl.tasks[(size_t)t];
                if (q >= T.hi - T.lo) continue;
                sp.items.push_back(fwd ? T.lo + q : ~(T.hi - 1 - q));
            }
        for (int32_t t : tasks)
            if (is_sep(pl.tasks[(size_t)t])) {
                sp.items.push_back(fwd ? n + t : ~(n + t));
                sp.sweeps.push_back(fwd ? n + t : ~(n + t));
                sp.sw_maxm = std::max(sp.sw_maxm, pl.tasks[(size_t)t].hi - pl.tasks[(size_t)t].lo);
            }
    };
    // Height-0 tasks (ND leaves, and BTF blocks when no coupling entry ties
    // the blocks together) get their order after each factorization (leaf_*).
    auto note_leaves = [&](const std::vector<int32_t> &tasks) {
        sp.leaf_tasks = tasks;
        sp.leaf_rows = 0;
        for (int32_t t : tasks) {
            sp.leaf_rows += pl.tasks[(size_t)t].hi - pl.tasks[(size_t)t].lo;
            sp.leaf_maxrows = std::max(sp.leaf_maxrows, pl.tasks[(size_t)t].hi - pl.tasks[(size_t)t].lo);
        }
    };
    if (sp.offp[(size_t)n] == 0) {
        // no coupling: every block is independent; all tasks by height together
        std::vector<std::vector<int32_t>> by_height((size_t)maxh + 1);
        for (size_t t = 0; t < pl.tasks.size(); t++) by_height[(size_t)pl.tasks[t].level].push_back((int32_t)t);
        note_leaves(by_height[0]);
        sp.leaf_f0 = (int32_t)sp.items.size();
        for (int32_t h = 0; h <= maxh; h++) interleave(by_height[(size_t)h], true);
        for (int32_t h = maxh; h >= 1; h--) interleave(by_height[(size_t)h], false);
        sp.leaf_b0 = (int32_t)sp.items.size();
        interleave(by_height[0], false);
        return;
    }
    for (int32_t d = pl.nblocks - 1; d >= 0; d--) {
        const int32_t k0 = pl.block_ptr[(size_t)d], k1 = pl.block_ptr[(size_t)d + 1];
        if (d != pl.nd_block) {
            for (int32_t k = k0; k < k1; k++) sp.items.push_back(k);
            for (int32_t k = k1 - 1; k >= k0; k--) sp.items.push_back(~k);
            continue;
        }
        std::vector<std::vector<int32_t>> by_height((size_t)maxh + 1);
        for (size_t t = 0; t < pl.tasks.size(); t++)
            if (pl.tasks[t].block == d) by_height[(size_t)pl.tasks[t].level].push_back((int32_t)t);
        // the leaves (height 0) get their order after each factorization; their
        // places here hold a valid order until then
        note_leaves(by_height[0]);
        sp.leaf_f0 = (int32_t)sp.items.size();
        for (int32_t h = 0; h <= maxh; h++) interleave(by_height[(size_t)h], true);
        for (int32_t h = maxh; h >= 1; h--) interleave(by_height[(size_t)h], false);
        sp.leaf_b0 = (int32_t)sp.items.size();
        interleave(by_height[0], false);
    }
}
