// solve_plan.cpp -- items and dependencies of the BTF / ND solve (host side).
#include <algorithm>

#include "solve_internal.h"

void bk_solve_plan_build(const bk_plan &pl, bk_solve_plan &sp)
{
    const int32_t n = pl.n;
    // coupling entries (above the diagonal blocks), grouped by row of B
    std::vector<int32_t> blk((size_t)n);
    for (int32_t d = 0; d < pl.nblocks; d++)
        for (int32_t i = pl.block_ptr[(size_t)d]; i < pl.block_ptr[(size_t)d + 1]; i++) blk[(size_t)i] = d;
    sp.offp.assign((size_t)n + 1, 0);
    for (int32_t j = 0; j < n; j++)
        for (int32_t e = pl.Bp[(size_t)j]; e < pl.dstart[(size_t)j]; e++) sp.offp[(size_t)pl.Bi[(size_t)e] + 1]++;
    for (int32_t r = 0; r < n; r++) sp.offp[(size_t)r + 1] += sp.offp[(size_t)r];
    sp.offj.assign((size_t)sp.offp[(size_t)n], 0);
    sp.offpos.assign((size_t)sp.offp[(size_t)n], 0);
    {
        std::vector<int32_t> cur(sp.offp.begin(), sp.offp.end() - 1);
        for (int32_t j = 0; j < n; j++)
            for (int32_t e = pl.Bp[(size_t)j]; e < pl.dstart[(size_t)j]; e++) {
                const int32_t r = pl.Bi[(size_t)e];
                sp.offj[(size_t)cur[(size_t)r]] = j;
                sp.offpos[(size_t)cur[(size_t)r]++] = e;
            }
    }
    // items: blocks from last to first; the ND block as forward items in
    // postorder followed by backward items in reverse postorder
    const size_t nt = pl.tasks.size();
    std::vector<int32_t> fwd_item(nt, -1), bwd_item(nt, -1), node_task;
    if (pl.nd_block >= 0) {
        node_task.assign((size_t)(2 * pl.nd_leaves - 1), -1);
        for (size_t t = 0; t < nt; t++)
            if (pl.tasks[t].node >= 0) node_task[(size_t)pl.tasks[t].node] = (int32_t)t;
    }
    sp.items.clear();
    std::vector<int32_t> block_tasks;
    for (int32_t d = pl.nblocks - 1; d >= 0; d--) {
        block_tasks.clear();
        for (size_t t = 0; t < nt; t++)
            if (pl.tasks[t].block == d) block_tasks.push_back((int32_t)t);
        if (d != pl.nd_block) {
            for (int32_t t : block_tasks) {
                fwd_item[(size_t)t] = bwd_item[(size_t)t] = (int32_t)sp.items.size();
                sp.items.push_back({BK_ITEM_BLOCK, t, 0, 0, 0, 0});
            }
        } else {
            std::sort(block_tasks.begin(), block_tasks.end(),
                      [&](int32_t a, int32_t b) { return pl.tasks[(size_t)a].node < pl.tasks[(size_t)b].node; });
            for (int32_t t : block_tasks) {
                fwd_item[(size_t)t] = (int32_t)sp.items.size();
                sp.items.push_back({BK_ITEM_FWD, t, 0, 0, 0, 0});
            }
            for (auto it = block_tasks.rbegin(); it != block_tasks.rend(); ++it) {
                bwd_item[(size_t)*it] = (int32_t)sp.items.size();
                sp.items.push_back({BK_ITEM_BWD, *it, 0, 0, 0, 0});
            }
        }
    }
    // the item after which z_j is final
    std::vector<int32_t> zitem((size_t)n);
    for (int32_t j = 0; j < n; j++) zitem[(size_t)j] = bwd_item[(size_t)pl.col_task[(size_t)j]];
    // dependencies and descendant lists
    sp.deps.clear();
    sp.desc.clear();
    std::vector<int32_t> tmp;
    for (auto &it : sp.items) {
        const bk_task &T = pl.tasks[(size_t)it.task];
        tmp.clear();
        it.desc_beg = it.desc_end = (int32_t)sp.desc.size();
        if (it.type != BK_ITEM_BWD) {
            for (int32_t k = T.lo; k < T.hi; k++)          // coupling rows of this block / node
                for (int32_t e = sp.offp[(size_t)k]; e < sp.offp[(size_t)k + 1]; e++)
                    tmp.push_back(zitem[(size_t)sp.offj[(size_t)e]]);
        }
        if (it.type == BK_ITEM_FWD) {
            for (int32_t u = pl.nd_first[(size_t)T.node]; u < T.node; u++) {
                const int32_t ut = node_task[(size_t)u];
                if (ut < 0) continue;
                tmp.push_back(fwd_item[(size_t)ut]);
                sp.desc.push_back(ut);
            }
            it.desc_end = (int32_t)sp.desc.size();
        }
        if (it.type == BK_ITEM_BWD) {
            tmp.push_back(fwd_item[(size_t)it.task]);
            for (int32_t a = 0; a < T.nanc; a++) {
                // ancestors are identified by their row ranges
                for (size_t u = 0; u < nt; u++)
                    if (pl.tasks[u].node >= 0 && pl.tasks[u].lo == T.anc_lo[a] && pl.tasks[u].hi == T.anc_hi[a])
                        tmp.push_back(bwd_item[u]);
            }
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        it.dep_beg = (int32_t)sp.deps.size();
        for (int32_t v : tmp) sp.deps.push_back(v);
        it.dep_end = (int32_t)sp.deps.size();
    }
    // contribution buffers of ND nodes: one slot per ancestor row
    sp.acc_off.assign(nt, 0);
    int64_t off = 0;
    for (size_t t = 0; t < nt; t++) {
        sp.acc_off[t] = off;
        if (pl.tasks[t].node >= 0) off += pl.tasks[t].lspace - (pl.tasks[t].hi - pl.tasks[t].lo);
    }
    sp.acc_stride = std::max<int64_t>(off, 1);
    // shared memory of one solve item: its own rows and its ancestor buffer
    int64_t need = 0;
    const int64_t cap = 200 * 1024;
    for (const auto &it : sp.items) {
        const bk_task &T = pl.tasks[(size_t)it.task];
        const int64_t own = T.hi - T.lo, anc = it.type == BK_ITEM_BLOCK ? 0 : T.lspace - own;
        const int64_t b = 8 * (own + anc);
        if (b <= cap) need = std::max(need, b);
    }
    sp.smem_bytes = (need + 15) & ~(int64_t)15;
}
