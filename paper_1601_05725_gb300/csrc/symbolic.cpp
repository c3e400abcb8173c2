// symbolic.cpp -- host planner of the CUDA library (basker_symbolic).
//
// Validates the input, forms the pattern of B = A(P,Q) (the BTF form of Sec. II /
// III-A), checks that B is block upper triangular and that, inside the ND block,
// every entry joins two nodes on one root path (the separators of Sec. III-C
// disconnect their halves), builds the tasks of the level schedule (Algorithm 4's
// dependency tree: leaves and small BTF blocks first, then separators by height),
// and sizes every column's L and U storage: by default with a structural
// Gilbert-Peierls pass under the preferred (natural) pivots (exact counts for
// those pivots, plus the pattern and a static schedule for the first
// factorization; symmetric pruning of the reach graph, Eisenstat and Liu, keeps
// its cost near |L+U|), or with Algorithm 3's counts, which store no pattern:
// exact elimination-tree counts everywhere (options.symbolic_mode 1), or exact at
// the leaves and the paper's interval estimates for the separators
// (options.symbolic_mode 2).  Slack covers pivoting.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "basker_internal.h"

namespace {

bool is_permutation(int32_t n, const int32_t *p)
{
    std::vector<char> seen((size_t)n, 0);
    for (int32_t i = 0; i < n; i++) {
        if (p[i] < 0 || p[i] >= n || seen[(size_t)p[i]]) return false;
        seen[(size_t)p[i]] = 1;
    }
    return true;
}

// Complete binary ND tree in postorder: children before the separator above them.
int32_t number_tree(int32_t height, int32_t &next, std::vector<int32_t> &first,
                    std::vector<int32_t> &h, std::vector<int32_t> &parent)
{
    int32_t start = next, a = -1, b = -1;
    if (height > 0) {
        a = number_tree(height - 1, next, first, h, parent);
        b = number_tree(height - 1, next, first, h, parent);
    }
    int32_t t = next++;
    first[(size_t)t] = start;
    h[(size_t)t] = height;
    if (a >= 0) { parent[(size_t)a] = t; parent[(size_t)b] = t; }
    return t;
}

// Sort distinct non-negative ints: a comparison sort for short lists, a bitmap
// over the value range for long ones (linear in the count and the range / 64; the
// reach of a column tied to much of its block lists that many steps).  bits has a
// word per 64 values and is left zero.
void sort_ints(std::vector<int32_t> &v, std::vector<uint64_t> &bits)
{
    if (v.size() < 512) {
        std::sort(v.begin(), v.end());
        return;
    }
    int32_t lo = v[0], hi = v[0];
    for (int32_t x : v) {
        lo = std::min(lo, x);
        hi = std::max(hi, x);
        bits[(size_t)x >> 6] |= 1ull << (x & 63);
    }
    size_t k = 0;
    for (size_t w = (size_t)lo >> 6; w <= ((size_t)hi >> 6); w++) {
        uint64_t b = bits[w];
        bits[w] = 0;
        while (b) {
            const int t = __builtin_ctzll(b);
            b &= b - 1;
            v[k++] = (int32_t)(w * 64 + (size_t)t);
        }
    }
}

}  // namespace

// Column state of the in-node kernel: x over the L-space, a bitmap of own steps,
// a bitmap of L-space rows, a bitmap of own rows touched by a redo, and caches of
// the node's own pivots and L offsets.
size_t bk_task_smem_bytes(const bk_task &t)
{
    size_t own = (size_t)(t.hi - t.lo);
    // x, cached L offsets, step / row / touched bitmaps, cached pinv, prow, Lcnt
    return (size_t)t.lspace * 8 + own * 8 + 2 * ((own + 31) / 32) * 4 + (((size_t)t.lspace + 31) / 32) * 4 +
           3 * own * 4 + 16;
}

bool bk_task_fits_smem(const bk_task &t) { return bk_task_smem_bytes(t) <= bk_gp_smem_limit(); }

// The lower adjacency of the symmetric structure inside each diagonal block (for
// each column c the rows i < c with B(i,c) != 0 or B(c,i) != 0) and its
// elimination tree (Liu's algorithm with path compression).
struct SymTree {
    std::vector<int64_t> ap;
    std::vector<int32_t> ai, parent;
};

static void sym_tree(const bk_plan &pl, SymTree &st)
{
    const int32_t n = pl.n;
    std::vector<int32_t> blk((size_t)n);
    for (int32_t d = 0; d < pl.nblocks; d++)
        for (int32_t i = pl.block_ptr[(size_t)d]; i < pl.block_ptr[(size_t)d + 1]; i++) blk[(size_t)i] = d;
    st.ap.assign((size_t)n + 1, 0);
    for (int32_t c = 0; c < n; c++)
        for (int32_t e = pl.dstart[(size_t)c]; e < pl.Bp[(size_t)c + 1]; e++) {
            const int32_t r = pl.Bi[(size_t)e];
            if (r == c || blk[(size_t)r] != blk[(size_t)c]) continue;
            st.ap[(size_t)std::max(r, c) + 1]++;
        }
    for (int32_t c = 0; c < n; c++) st.ap[(size_t)c + 1] += st.ap[(size_t)c];
    st.ai.assign((size_t)st.ap[(size_t)n], 0);
    std::vector<int64_t> fill(st.ap.begin(), st.ap.end() - 1);
    for (int32_t c = 0; c < n; c++)
        for (int32_t e = pl.dstart[(size_t)c]; e < pl.Bp[(size_t)c + 1]; e++) {
            const int32_t r = pl.Bi[(size_t)e];
            if (r == c || blk[(size_t)r] != blk[(size_t)c]) continue;
            st.ai[(size_t)fill[(size_t)std::max(r, c)]++] = std::min(r, c);
        }
    st.parent.assign((size_t)n, -1);
    std::vector<int32_t> anc((size_t)n, -1);
    for (int32_t c = 0; c < n; c++)
        for (int64_t e = st.ap[(size_t)c]; e < st.ap[(size_t)c + 1]; e++) {
            int32_t r = st.ai[(size_t)e];
            while (anc[(size_t)r] != -1 && anc[(size_t)r] != c) {
                const int32_t t = anc[(size_t)r];
                anc[(size_t)r] = c;
                r = t;
            }
            if (anc[(size_t)r] == -1) {
                anc[(size_t)r] = c;
                st.parent[(size_t)r] = c;
            }
        }
}

static void finish_counts(bk_plan &pl)
{
    int64_t nl = 0, nu = 0;
    for (int32_t c = 0; c < pl.n; c++) {
        nl += pl.sLcnt[(size_t)c];
        nu += pl.sUcnt[(size_t)c];
    }
    pl.nnz_l_sym = nl;
    pl.nnz_u_sym = nu;
    pl.sLi.clear();
    pl.sUi.clear();
    pl.sprow.clear();
    pl.slevel.clear();
    pl.sorder.clear();
}

// Algorithm 3's counts (Sec. III-C, parallel symbolic factorization), per BTF
// diagonal block: the elimination tree of the symmetric structure B_dd + B_dd^T
// (one tree for the whole ND block: its separators are the ancestors of their
// subtrees, so the tree holds the leaves' trees, the L_ki rows and the U_ij
// columns), then for every column c the row subtree of c (the nodes met walking
// up from each i < c adjacent to c, stopping at a node already met for c).  Its
// size + 1 is U(:,c)'s count; the number of later row subtrees that contain a
// node j is L(:,j)'s count.  These are the counts of the Cholesky factor of the
// symmetric structure, which contains the LU pattern of the natural pivots, so
// they never fall below the structural pass's counts (equal for a symmetric
// pattern); they cost O(|L + U|) node visits.  No pattern is stored
// (options.symbolic_mode 1).
static void etree_counts(bk_plan &pl)
{
    const int32_t n = pl.n;
    pl.sLcnt.assign((size_t)n, 0);
    pl.sUcnt.assign((size_t)n, 0);
    SymTree st;
    sym_tree(pl, st);
    // row subtrees
    std::vector<int32_t> mark((size_t)n, -1);
    for (int32_t c = 0; c < n; c++) {
        int32_t uc = 1;
        mark[(size_t)c] = c;
        for (int64_t e = st.ap[(size_t)c]; e < st.ap[(size_t)c + 1]; e++)
            for (int32_t r = st.ai[(size_t)e]; r >= 0 && mark[(size_t)r] != c; r = st.parent[(size_t)r]) {
                mark[(size_t)r] = c;
                uc++;
                pl.sLcnt[(size_t)r]++;
            }
        pl.sUcnt[(size_t)c] = uc;
    }
    finish_counts(pl);
}

// Algorithm 3's reading of the upper tree levels (options.symbolic_mode 2).  The
// ND leaves and the BTF blocks (tree levels -1 and 0) are counted exactly, by the
// row subtrees above; for each of their columns t the rows of L(:,t) in every
// ancestor node are kept as a range (lest: the lowest and the highest row).  The
// separators are then estimated level by level up the tree: a row t below
// separator column c is taken to reach c (an entry U(t,c)) when c lies in t's
// range for c's node (for the symmetric structure the columns of U's row t are
// the rows of L's column t, so lest also serves as uest), and column c's rows in
// each node (its own, each ancestor) are taken dense between the lowest and the
// highest row of the ranges of those t, of the column's own entries, and of the
// earlier columns of its node that reach it.  Each range holds the exact rows,
// so the estimates bound the tree counts (mode 1) from above, column by column.
static void interval_counts(bk_plan &pl)
{
    const int32_t n = pl.n;
    pl.sLcnt.assign((size_t)n, 0);
    pl.sUcnt.assign((size_t)n, 0);
    SymTree st;
    sym_tree(pl, st);
    auto task_of = [&](int32_t c) -> const bk_task & { return pl.tasks[(size_t)pl.col_task[(size_t)c]]; };
    auto exact = [&](int32_t c) { return task_of(c).level == 0; };
    // lest: per column, one range per ancestor node and one for its own node
    std::vector<int64_t> off((size_t)n + 1, 0);
    for (int32_t c = 0; c < n; c++) off[(size_t)c + 1] = off[(size_t)c] + task_of(c).nanc + 1;
    std::vector<int32_t> lmin((size_t)off[(size_t)n], INT32_MAX), lmax((size_t)off[(size_t)n], -1);
    auto anc_slot = [](const bk_task &K, int32_t r) {
        for (int32_t a = 0; a < K.nanc; a++)
            if (r >= K.anc_lo[a] && r < K.anc_hi[a]) return a;
        return -1;
    };
    // exact levels: row subtrees, which stop at the first separator column
    std::vector<int32_t> mark((size_t)n, -1);
    for (int32_t c = 0; c < n; c++) {
        const bool crow = exact(c);
        int32_t uc = 1;
        mark[(size_t)c] = c;
        for (int64_t e = st.ap[(size_t)c]; e < st.ap[(size_t)c + 1]; e++)
            for (int32_t r = st.ai[(size_t)e]; r >= 0 && mark[(size_t)r] != c; r = st.parent[(size_t)r]) {
                if (!exact(r)) break;                // a separator column: estimated below
                mark[(size_t)r] = c;
                uc++;
                pl.sLcnt[(size_t)r]++;
                if (!crow) {                         // row c of an ancestor node in L(:,r)
                    const int32_t a = anc_slot(task_of(r), c);
                    if (a >= 0) {
                        const int64_t k = off[(size_t)r] + a;
                        lmin[(size_t)k] = std::min(lmin[(size_t)k], c);
                        lmax[(size_t)k] = std::max(lmax[(size_t)k], c);
                    }
                }
            }
        if (crow) pl.sUcnt[(size_t)c] = uc;
    }
    // the upper adjacency (rows r > c of each column's symmetric structure)
    std::vector<int64_t> up((size_t)n + 1, 0);
    for (int32_t r = 0; r < n; r++)
        for (int64_t e = st.ap[(size_t)r]; e < st.ap[(size_t)r + 1]; e++) up[(size_t)st.ai[(size_t)e] + 1]++;
    for (int32_t c = 0; c < n; c++) up[(size_t)c + 1] += up[(size_t)c];
    std::vector<int32_t> ui((size_t)up[(size_t)n]);
    {
        std::vector<int64_t> fill(up.begin(), up.end() - 1);
        for (int32_t r = 0; r < n; r++)
            for (int64_t e = st.ap[(size_t)r]; e < st.ap[(size_t)r + 1]; e++)
                ui[(size_t)fill[(size_t)st.ai[(size_t)e]]++] = r;
    }
    // separators, children before parents (the tasks are in postorder)
    for (const bk_task &J : pl.tasks) {
        if (J.level == 0 || J.node < 0) continue;
        const int32_t m = J.hi - J.lo, ns = J.nanc, w = ns + 1;     // ranges: ancestors, then own
        std::vector<int32_t> cnt((size_t)m, 0), rmin((size_t)m * w, INT32_MAX), rmax((size_t)m * w, -1);
        auto hull = [&](int32_t c, int32_t q, int32_t lo, int32_t hi) {
            if (hi < lo) return;
            const size_t k = (size_t)(c - J.lo) * w + q;
            rmin[k] = std::min(rmin[k], lo);
            rmax[k] = std::max(rmax[k], hi);
        };
        // rows below the separator: a range covering column c reaches it
        for (int32_t t = J.sp_lo; t < J.lo; t++) {
            const bk_task &K = task_of(t);
            const int32_t a = anc_slot(K, J.lo);
            if (a < 0) continue;
            const int64_t k0 = off[(size_t)t];
            const int32_t mn = lmin[(size_t)k0 + a], mx = lmax[(size_t)k0 + a];
            for (int32_t c = std::max(mn, J.lo); c <= std::min(mx, J.hi - 1); c++) {
                cnt[(size_t)(c - J.lo)]++;
                for (int32_t q = 0; q < ns; q++)
                    hull(c, q, lmin[(size_t)k0 + a + 1 + q], lmax[(size_t)k0 + a + 1 + q]);
                hull(c, ns, std::max(mn, c + 1), mx);
            }
        }
        for (int32_t c = J.lo; c < J.hi; c++) {
            // the column's own entries
            for (int64_t e = up[(size_t)c]; e < up[(size_t)c + 1]; e++) {
                const int32_t r = ui[(size_t)e];
                if (r < J.hi) {
                    hull(c, ns, r, r);
                } else {
                    const int32_t q = anc_slot(J, r);
                    if (q >= 0) hull(c, q, r, r);
                }
            }
            const size_t k = (size_t)(c - J.lo) * w;
            int64_t lc = 0;
            for (int32_t q = 0; q <= ns; q++)
                if (rmax[k + q] >= rmin[k + q]) lc += rmax[k + q] - rmin[k + q] + 1;
            pl.sLcnt[(size_t)c] = (int32_t)lc;
            pl.sUcnt[(size_t)c] = cnt[(size_t)(c - J.lo)] + 1;
            for (int32_t q = 0; q <= ns; q++) {
                lmin[(size_t)off[(size_t)c] + q] = rmin[k + q];
                lmax[(size_t)off[(size_t)c] + q] = rmax[k + q];
            }
            // the later columns of the node that this column's own range reaches
            const int32_t mn = rmin[k + ns], mx = rmax[k + ns];
            for (int32_t c2 = std::max(mn, c + 1); c2 <= mx && c2 < J.hi; c2++) {
                cnt[(size_t)(c2 - J.lo)]++;
                for (int32_t q = 0; q < ns; q++) hull(c2, q, rmin[k + q], rmax[k + q]);
                hull(c2, ns, std::max(mn, c2 + 1), mx);
            }
        }
    }
    finish_counts(pl);
}

// The ancestor ranges as sorted tables of BK_MAX_ANC entries (unused ones
// INT32_MAX) with each range's first slot, so that a row's slot is found by a
// fixed four-step binary search (slot_of in device_util.cuh).
void bk_task_ranges(bk_task &T)
{
    int32_t cum = 0;
    for (int32_t a = 0; a < BK_MAX_ANC; a++) {
        if (a < T.nanc) {
            T.anc_cum[a] = cum;
            T.anc_sh[a] = cum - T.anc_lo[a];
            cum += T.anc_hi[a] - T.anc_lo[a];
        } else {
            T.anc_lo[a] = T.anc_hi[a] = T.anc_cum[a] = INT32_MAX;
            T.anc_sh[a] = 0;
        }
    }
}

int bk_plan_build(int32_t n, const int32_t *colptr, const int32_t *rowind, const int32_t *P,
                  const int32_t *Q, int32_t nblocks, const int32_t *block_ptr, int32_t nd_block,
                  int32_t nd_leaves, const int32_t *nd_node_ptr, double slack, bk_plan &pl,
                  int32_t *bad_col, int mode)
{
    *bad_col = -1;
    if (n < 0 || nblocks < 0 || (n > 0 && nblocks < 1) || !colptr || (n > 0 && (!P || !Q || !block_ptr)))
        return BASKER_ERR_INVALID_ARG;
    if (colptr[0] != 0) return BASKER_ERR_INVALID_ARG;
    for (int32_t j = 0; j < n; j++) {
        if (colptr[j + 1] < colptr[j]) return BASKER_ERR_INVALID_ARG;
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++)
            if (rowind[p] < 0 || rowind[p] >= n || (p > colptr[j] && rowind[p] <= rowind[p - 1]))
                return BASKER_ERR_INVALID_ARG;
    }
    if (n > 0 && (!is_permutation(n, P) || !is_permutation(n, Q))) return BASKER_ERR_INVALID_ARG;
    if (block_ptr[0] != 0 || block_ptr[nblocks] != n) return BASKER_ERR_INVALID_ARG;
    for (int32_t d = 0; d < nblocks; d++)
        if (block_ptr[d + 1] <= block_ptr[d]) return BASKER_ERR_INVALID_ARG;

    pl.n = n;
    pl.nblocks = nblocks;
    pl.slack = slack;
    pl.P.assign(P, P + n);
    pl.Q.assign(Q, Q + n);
    pl.block_ptr.assign(block_ptr, block_ptr + nblocks + 1);
    std::vector<int32_t> blk((size_t)n);
    for (int32_t d = 0; d < nblocks; d++)
        for (int32_t i = block_ptr[d]; i < block_ptr[d + 1]; i++) blk[(size_t)i] = d;

    // ---- ND tree of one block
    std::vector<int32_t> node_of;
    std::vector<int32_t> parent;
    pl.nd_block = -1;
    if (nd_block >= 0) {
        int32_t depth = 0;
        while ((1 << depth) < nd_leaves && depth < 30) depth++;
        if (nd_block >= nblocks || nd_leaves < 1 || (1 << depth) != nd_leaves || depth > BK_MAX_ANC || !nd_node_ptr)
            return BASKER_ERR_INVALID_ARG;
        int32_t nodes = 2 * nd_leaves - 1;
        if (nd_node_ptr[0] != block_ptr[nd_block] || nd_node_ptr[nodes] != block_ptr[nd_block + 1])
            return BASKER_ERR_INVALID_ARG;
        for (int32_t t = 0; t < nodes; t++)
            if (nd_node_ptr[t + 1] < nd_node_ptr[t]) return BASKER_ERR_INVALID_ARG;
        pl.nd_block = nd_block;
        pl.nd_leaves = nd_leaves;
        pl.depth = depth;
        pl.nd_ptr.assign(nd_node_ptr, nd_node_ptr + nodes + 1);
        pl.nd_first.assign((size_t)nodes, 0);
        pl.nd_height.assign((size_t)nodes, 0);
        parent.assign((size_t)nodes, -1);
        int32_t next = 0;
        number_tree(depth, next, pl.nd_first, pl.nd_height, parent);
        node_of.assign((size_t)n, -1);
        for (int32_t t = 0; t < nodes; t++)
            for (int32_t i = nd_node_ptr[t]; i < nd_node_ptr[t + 1]; i++) node_of[(size_t)i] = t;
    }

    // ---- B = A(P,Q), rows sorted, with the map back to A's entries
    int64_t nnz = colptr[n];
    if (nnz >= (int64_t)1 << 31) return BASKER_ERR_INVALID_ARG;
    pl.nnz = nnz;
    std::vector<int32_t> Pinv((size_t)n);
    for (int32_t i = 0; i < n; i++) Pinv[(size_t)P[i]] = i;
    pl.Bp.assign((size_t)n + 1, 0);
    for (int32_t j = 0; j < n; j++) pl.Bp[(size_t)j + 1] = pl.Bp[(size_t)j] + (colptr[Q[j] + 1] - colptr[Q[j]]);
    pl.Bi.resize((size_t)nnz);
    pl.bmap.resize((size_t)nnz);
    pl.dstart.resize((size_t)n);
    std::vector<std::pair<int32_t, int32_t>> tmp;
    for (int32_t j = 0; j < n; j++) {
        int32_t q = Q[j];
        tmp.clear();
        for (int32_t p = colptr[q]; p < colptr[q + 1]; p++) tmp.emplace_back(Pinv[(size_t)rowind[p]], p);
        std::sort(tmp.begin(), tmp.end());
        int32_t o = pl.Bp[(size_t)j];
        int32_t k0 = block_ptr[blk[(size_t)j]];
        int32_t ds = -1;
        for (size_t k = 0; k < tmp.size(); k++) {
            int32_t r = tmp[k].first;
            pl.Bi[(size_t)o + k] = r;
            pl.bmap[(size_t)o + k] = tmp[k].second;
            if (blk[(size_t)r] > blk[(size_t)j]) { *bad_col = j; return BASKER_ERR_NOT_BTF; }
            if (ds < 0 && r >= k0) ds = o + (int32_t)k;
            if (node_of.size() && blk[(size_t)j] == pl.nd_block && r >= k0) {
                int32_t a = node_of[(size_t)r], b = node_of[(size_t)j];
                bool rel = (pl.nd_first[(size_t)a] <= b && b <= a) || (pl.nd_first[(size_t)b] <= a && a <= b);
                if (!rel) { *bad_col = j; return BASKER_ERR_BAD_ND; }
            }
        }
        pl.dstart[(size_t)j] = ds < 0 ? pl.Bp[(size_t)j + 1] : ds;
    }

    // ---- tasks: BTF blocks, ND nodes (postorder), each with its row space
    pl.tasks.clear();
    pl.col_task.assign((size_t)n, -1);
    int32_t maxlevel = 0;
    for (int32_t d = 0; d < nblocks; d++) {
        if (d == pl.nd_block) {
            int32_t nodes = 2 * nd_leaves - 1;
            for (int32_t t = 0; t < nodes; t++) {
                if (pl.nd_ptr[(size_t)t + 1] == pl.nd_ptr[(size_t)t]) continue;
                bk_task T;
                std::memset(&T, 0, sizeof T);
                T.lo = T.c0 = pl.nd_ptr[(size_t)t];
                T.hi = T.c1 = pl.nd_ptr[(size_t)t + 1];
                T.sp_lo = pl.nd_ptr[(size_t)pl.nd_first[(size_t)t]];
                T.nanc = 0;
                int32_t lsp = T.hi - T.lo;
                for (int32_t a = parent[(size_t)t]; a >= 0; a = parent[(size_t)a]) {
                    if (pl.nd_ptr[(size_t)a + 1] == pl.nd_ptr[(size_t)a]) continue;
                    T.anc_lo[T.nanc] = pl.nd_ptr[(size_t)a];
                    T.anc_hi[T.nanc] = pl.nd_ptr[(size_t)a + 1];
                    lsp += T.anc_hi[T.nanc] - T.anc_lo[T.nanc];
                    T.nanc++;
                }
                T.space = (T.hi - T.sp_lo) + (lsp - (T.hi - T.lo));
                T.lspace = lsp;
                bk_task_ranges(T);
                T.level = pl.nd_height[(size_t)t];
                T.node = t;
                T.block = d;
                maxlevel = std::max(maxlevel, T.level);
                for (int32_t c = T.lo; c < T.hi; c++) pl.col_task[(size_t)c] = (int32_t)pl.tasks.size();
                pl.tasks.push_back(T);
            }
        } else {
            bk_task T;
            std::memset(&T, 0, sizeof T);
            T.lo = T.c0 = T.sp_lo = block_ptr[d];
            T.hi = T.c1 = block_ptr[d + 1];
            T.space = T.lspace = T.hi - T.lo;
            bk_task_ranges(T);
            T.level = 0;
            T.node = -1;
            T.block = d;
            for (int32_t c = T.lo; c < T.hi; c++) pl.col_task[(size_t)c] = (int32_t)pl.tasks.size();
            pl.tasks.push_back(T);
        }
    }
    pl.level_tasks.assign((size_t)maxlevel + 1, {});
    for (size_t i = 0; i < pl.tasks.size(); i++) pl.level_tasks[(size_t)pl.tasks[i].level].push_back((int32_t)i);
    // a topological order of the columns with breadth: the tasks of a level take
    // turns column by column (a column depends on earlier columns of its task and
    // on the tasks below it)
    pl.iorder.clear();
    pl.iorder.reserve((size_t)n);
    for (const auto &lt : pl.level_tasks) {
        auto len = [&](int32_t t) { return pl.tasks[(size_t)t].c1 - pl.tasks[(size_t)t].c0; };
        int32_t longest = 0;
        for (int32_t t : lt) longest = std::max(longest, len(t));
        // rounds q = 0 .. longest - 1: the tasks longer than q in the level's order;
        // the list of active tasks shrinks as they end, so the work is O(columns)
        std::vector<int32_t> active(lt.begin(), lt.end());
        for (int32_t q = 0; q < longest; q++) {
            size_t w = 0;
            for (size_t i = 0; i < active.size(); i++) {
                const int32_t t = active[i];
                if (q < len(t)) {
                    pl.iorder.push_back(pl.tasks[(size_t)t].c0 + q);
                    active[w++] = t;
                }
            }
            active.resize(w);
        }
    }
    pl.max_space = 0;
    for (auto &T : pl.tasks) pl.max_space = std::max(pl.max_space, T.space);

    pl.counts_only = mode == 1 || mode == 2;
    if (pl.counts_only) {
        if (mode == 1) etree_counts(pl);
        else interval_counts(pl);
        pl.symbolic_singular = -1;
        bk_plan_layout(pl);
        return BASKER_OK;
    }

    // ---- structural Gilbert-Peierls pass under the preferred pivots
    std::vector<int32_t> pinv((size_t)n, -1), mark((size_t)n, -1);
    pl.sprow.assign((size_t)n, -1);
    std::vector<int64_t> Lst((size_t)n + 1, 0), Ust((size_t)n + 1, 0);
    std::vector<int32_t> Lrows, Usteps;            // flat, column order
    std::vector<int32_t> g;                        // reach graph: copy of L rows, prunable
    std::vector<int64_t> gbeg((size_t)n, 0);
    std::vector<int32_t> gend((size_t)n, 0), glen((size_t)n, 0);
    std::vector<char> pruned((size_t)n, 0);
    std::vector<int32_t> stack, spos, lrow, ustep;
    std::vector<uint64_t> sortbits(((size_t)n + 63) / 64 + 1, 0);
    pl.symbolic_singular = -1;
    for (int32_t c = 0; c < n; c++) {
        const bk_task &T = pl.tasks[(size_t)pl.col_task[(size_t)c]];
        lrow.clear();
        ustep.clear();
        for (int32_t p = pl.dstart[(size_t)c]; p < pl.Bp[(size_t)c + 1]; p++) {
            int32_t r0 = pl.Bi[(size_t)p];
            if (mark[(size_t)r0] == c) continue;
            mark[(size_t)r0] = c;
            stack.assign(1, r0);
            spos.assign(1, 0);
            while (!stack.empty()) {
                int32_t r = stack.back();
                int32_t j = pinv[(size_t)r];
                bool pushed = false;
                if (j >= 0) {
                    int32_t &k = spos.back();
                    while (k < gend[(size_t)j]) {
                        int32_t r2 = g[(size_t)(gbeg[(size_t)j] + k)];
                        k++;
                        if (mark[(size_t)r2] != c) {
                            mark[(size_t)r2] = c;
                            stack.push_back(r2);
                            spos.push_back(0);
                            pushed = true;
                            break;
                        }
                    }
                }
                if (!pushed) {
                    if (j >= 0) ustep.push_back(j); else lrow.push_back(r);
                    stack.pop_back();
                    spos.pop_back();
                }
            }
        }
        sort_ints(ustep, sortbits);
        sort_ints(lrow, sortbits);
        int32_t piv = -1;
        if (mark[(size_t)c] == c && pinv[(size_t)c] < 0) piv = c;
        else
            for (int32_t r : lrow)
                if (r >= T.lo && r < T.hi) { piv = r; break; }
        if (piv < 0 && pl.symbolic_singular < 0) pl.symbolic_singular = c;
        for (int32_t j : ustep) Usteps.push_back(j);
        Usteps.push_back(c);
        gbeg[(size_t)c] = (int64_t)g.size();
        for (int32_t r : lrow)
            if (r != piv) { Lrows.push_back(r); g.push_back(r); }
        glen[(size_t)c] = gend[(size_t)c] = (int32_t)((int64_t)g.size() - gbeg[(size_t)c]);
        Lst[(size_t)c + 1] = (int64_t)Lrows.size();
        Ust[(size_t)c + 1] = (int64_t)Usteps.size();
        if (piv >= 0) { pinv[(size_t)piv] = c; pl.sprow[(size_t)c] = piv; }
        // symmetric pruning: a column j of the reach whose L holds the new pivot row
        // keeps only its already pivoted rows for later reaches
        if (piv >= 0)
            for (int32_t j : ustep) {
                if (pruned[(size_t)j]) continue;
                int32_t *gj = g.data() + gbeg[(size_t)j];
                int32_t len = glen[(size_t)j];
                bool has = false;
                for (int32_t k = 0; k < len; k++) if (gj[k] == piv) { has = true; break; }
                if (!has) continue;
                int32_t head = 0, tail = len;
                while (head < tail) {
                    if (pinv[(size_t)gj[head]] >= 0) head++;
                    else std::swap(gj[head], gj[--tail]);
                }
                gend[(size_t)j] = tail;
                pruned[(size_t)j] = 1;
            }
    }
    pl.nnz_l_sym = (int64_t)Lrows.size();
    pl.nnz_u_sym = (int64_t)Usteps.size();

    // ---- static DAG levels (column c waits for the steps of U(:,c)) and claim order
    pl.slevel.assign((size_t)n, 0);
    int32_t nlev = 0;
    for (int32_t c = 0; c < n; c++) {
        int32_t lv = 0;
        for (int64_t k = Ust[(size_t)c]; k < Ust[(size_t)c + 1] - 1; k++)
            lv = std::max(lv, pl.slevel[(size_t)Usteps[(size_t)k]] + 1);
        pl.slevel[(size_t)c] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    std::vector<int64_t> cnt((size_t)nlev + 1, 0);
    for (int32_t c = 0; c < n; c++) cnt[(size_t)pl.slevel[(size_t)c] + 1]++;
    for (int32_t l = 0; l < nlev; l++) cnt[(size_t)l + 1] += cnt[(size_t)l];
    pl.sorder.assign((size_t)n, 0);
    for (int32_t c = 0; c < n; c++) pl.sorder[(size_t)cnt[(size_t)pl.slevel[(size_t)c]]++] = c;

    // ---- keep the symbolic pattern column by column (laid out by bk_plan_layout)
    pl.sLcnt.assign((size_t)n, 0);
    pl.sUcnt.assign((size_t)n, 0);
    for (int32_t c = 0; c < n; c++) {
        pl.sLcnt[(size_t)c] = (int32_t)(Lst[(size_t)c + 1] - Lst[(size_t)c]);
        pl.sUcnt[(size_t)c] = (int32_t)(Ust[(size_t)c + 1] - Ust[(size_t)c]);
    }
    pl.sLi.swap(Lrows);
    pl.sUi.swap(Usteps);
    bk_plan_layout(pl);
    return BASKER_OK;
}

// Largest possible L and U counts of column c: the unpivoted rows of its node
// other than the pivot plus its ancestors' rows; the earlier steps of its subtree
// plus the diagonal.
static int64_t l_bound(const bk_task &T, int32_t c) { return (int64_t)(T.hi - c - 1) + (T.lspace - (T.hi - T.lo)); }
static int64_t u_bound(const bk_task &T, int32_t c) { return (int64_t)(c - T.sp_lo) + 1; }

static void prefix_layout(bk_plan &pl)
{
    const int32_t n = pl.n;
    pl.sLbeg.assign((size_t)n + 1, 0);
    pl.sUbeg.assign((size_t)n + 1, 0);
    for (int32_t c = 0; c < n; c++) {
        pl.sLbeg[(size_t)c + 1] = pl.sLbeg[(size_t)c] + pl.lcapc[(size_t)c];
        pl.sUbeg[(size_t)c + 1] = pl.sUbeg[(size_t)c] + pl.ucapc[(size_t)c];
    }
    pl.lcap = pl.sLbeg[(size_t)n];
    pl.ucap = pl.sUbeg[(size_t)n];
    // a column that outgrows its region moves to a region of the spill pool
    pl.lpool = pl.lcap / 2 + (1 << 20);
    pl.upool = pl.ucap / 2 + (1 << 20);
}

// After an overflow (a spill pool ran out): a column that overflowed gets four
// times its room, the later columns of the same task twice theirs (pivoting moved
// fill there), each at most its upper bound; the pools grow with the regions.
// Growing geometrically rather than to the bounds keeps the arena proportional to
// the fill: the bounds of a large ND block sum to many times |L + U|.
void bk_plan_regrow(bk_plan &pl, const int32_t *over)
{
    for (const bk_task &T : pl.tasks) {
        bool al = false, au = false;
        for (int32_t c = T.lo; c < T.hi; c++) {
            const size_t k = (size_t)c;
            if (over[k] & 1) { pl.lcapc[k] = std::min<int64_t>(4 * pl.lcapc[k] + 64, l_bound(T, c)); al = true; }
            else if (al) pl.lcapc[k] = std::min<int64_t>(2 * pl.lcapc[k] + 8, l_bound(T, c));
            if (over[k] & 2) { pl.ucapc[k] = std::min<int64_t>(4 * pl.ucapc[k] + 64, u_bound(T, c)); au = true; }
            else if (au) pl.ucapc[k] = std::min<int64_t>(2 * pl.ucapc[k] + 8, u_bound(T, c));
        }
    }
    prefix_layout(pl);
}

// Per-column L and U regions: count x (1 + slack) + a margin, at most the
// column's upper bound.  Columns are stored one after the other, so Lbeg[c] is a
// prefix sum of the capacities.
void bk_plan_layout(bk_plan &pl)
{
    int32_t n = pl.n;
    pl.lcapc.assign((size_t)n, 0);
    pl.ucapc.assign((size_t)n, 0);
    for (int32_t c = 0; c < n; c++) {
        const bk_task &T = pl.tasks[(size_t)pl.col_task[(size_t)c]];
        const double f = 1.0 + pl.slack;
        pl.lcapc[(size_t)c] = std::min<int64_t>((int64_t)(pl.sLcnt[(size_t)c] * f) + 8, l_bound(T, c));
        pl.ucapc[(size_t)c] = std::min<int64_t>((int64_t)(pl.sUcnt[(size_t)c] * f) + 8, u_bound(T, c));
    }
    prefix_layout(pl);
    // global workspace of the in-node tasks whose column state does not fit in
    // shared memory, 256-byte aligned
    int64_t off = 0;
    for (auto &T : pl.tasks) {
        if (bk_task_fits_smem(T)) { T.wsoff = -1; continue; }
        T.wsoff = off;
        off += ((int64_t)bk_task_smem_bytes(T) + 255) & ~(int64_t)255;
    }
    // separators: A-hat scratch (dense over the L-space per column) and the
    // descendant-phase slice (x over the whole space plus two bitmaps)
    // column-per-warp kernels (separator descendant phase, refactor rounds): one
    // slice per warp holding x over a task's whole space and its step / row bitmaps
    int64_t ah = 0, ab = 0;
    std::vector<int64_t> level_cols(pl.level_tasks.size(), 0), level_slice(pl.level_tasks.size(), 256);
    for (auto &T : pl.tasks) {
        T.ahoff = T.aboff = 0;
        const int64_t own = T.hi - T.lo, words = (T.lspace + 31) / 32;
        // x over the space, then the reach's step and row bitmaps, or (the
        // descendant phase on stored patterns) a mark byte per slot
        int64_t sl = (int64_t)T.space * 8 +
                     std::max<int64_t>(((int64_t)(T.hi - T.sp_lo) + 31) / 32 * 4 + words * 4, (int64_t)T.space);
        level_slice[(size_t)T.level] = std::max(level_slice[(size_t)T.level], (sl + 255) & ~(int64_t)255);
        level_cols[(size_t)T.level] += own;
        if (T.sp_lo >= T.lo) continue;
        T.ahoff = ah;
        T.aboff = ab;
        ah += own * T.lspace;
        ab += own * words;
    }
    pl.ahat_doubles = std::max<int64_t>(ah, 1);
    pl.ahat_words = std::max<int64_t>(ab, 1);
    // the reach's step and row bitmaps fit in shared memory for four warps a block
    // (beside the rounds' staging areas), per ND level: the rounds of a level
    // launch with its own tasks' bitmaps
    auto fits = [](int64_t w) { return 4 * w * 4 + 4 * BK_DD_STAGE_BYTES <= 160 * 1024; };
    int64_t bw = 0;
    pl.level_dd_words.assign(pl.level_tasks.size(), 0);
    for (auto &T : pl.tasks) {
        const int64_t w = (((int64_t)(T.hi - T.sp_lo) + 31) / 32 + (T.lspace + 31) / 32 + 3) & ~(int64_t)3;
        bw = std::max(bw, w);
        int32_t &lw = pl.level_dd_words[(size_t)T.level];
        lw = (int32_t)std::max<int64_t>(lw, w);
    }
    pl.dd_words = fits(bw) ? (int32_t)bw : 0;
    for (auto &lw : pl.level_dd_words)
        if (!fits(lw)) lw = 0;
    // One workspace serves every level in turn, each with slices of its own size:
    // a level wants one slice per column it processes at once (at most 152 SMs x
    // 16 warps); the workspace holds what level 0 (the leaves and BTF blocks) wants
    // and, for the levels above, up to 1 GiB (a root separator whose space is the
    // whole ND block takes fewer warps rather than gigabytes)
    const size_t nl = level_cols.size();
    int64_t need0 = 0, need = 0, most = 256;
    for (size_t l = 0; l < nl; l++) {
        const int64_t want = std::min<int64_t>(std::max<int64_t>(level_cols[l], 1), 152 * 16) * level_slice[l];
        if (l == 0) need0 = want;
        need = std::max(need, want);
        most = std::max(most, level_slice[l]);
    }
    pl.wsd_bytes = std::max(std::min(need, std::max(need0, (int64_t)1 << 30)), most);
    pl.level_slice = level_slice;
    pl.level_warps.assign(nl, 1);
    for (size_t l = 0; l < nl; l++)
        pl.level_warps[l] = (int32_t)std::max<int64_t>(
            1, std::min<int64_t>(std::min<int64_t>(std::max<int64_t>(level_cols[l], 1), 152 * 16),
                                 pl.wsd_bytes / level_slice[l]));
    pl.wsd_slice = nl ? level_slice[0] : 256;
    pl.wsd_warps = nl ? pl.level_warps[0] : 1;
    pl.ws_bytes = off;
}
