/*
 * basker_oracle.c -- the oracle: a plain, serial, FP64 CPU implementation of the
 * numeric sparse LU that the CUDA library computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file.  It shares no code, header, table or helper
 * with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (Booth, Rajamanickam, Thornquist, "Basker", arXiv 1601.05725):
 *
 *   B = A(P,Q) is block upper triangular (Sec. II, the BTF display; Sec. III-A).
 *   Only the diagonal blocks B_dd are factored (Sec. II: the off-diagonal blocks
 *   enter only the solve).  Each is factored column by column with the
 *   left-looking Gilbert-Peierls method (Algorithm 1):
 *     1. pattern of column c = the set of rows reachable, in the graph of the L
 *        computed so far, from the rows of B_dd(:,c); found by depth-first search;
 *     2. for every pivoted row in the pattern (pivot step j), in a topological
 *        order: x(rows of L(:,j)) -= L(:,j) * x(pivot row of j);
 *     3. select a pivot among the pattern's rows that are not yet pivoted;
 *     4. split x into U(:,c) (rows already pivoted, plus the pivot) and
 *        L(:,c) = x / pivot (the other rows).
 *   In the block that carries nested dissection (Sec. III-C), a pivot for a column
 *   of ND node t may only come from node t's own rows: the leaves of the ND tree
 *   and the separators are the diagonal blocks A_ii / A_jj of the 2D layout
 *   (Fig. 3a; Algorithm 4 pivots inside each leaf block LU_ii and separator block
 *   LU_jj).  Algorithm 4 computes exactly these factors in a parallel schedule;
 *   this file computes them by the plain definition, one column after the other.
 *
 * Readings of points the paper leaves open (each is a documented choice):
 *   - Pivot rule (Algorithm 1 leaves the rule open): threshold partial
 *     pivoting.  m = max |x_r| over the candidates; the preferred row (the row
 *     pivoted at this column by a previous factorization, else the natural row c)
 *     is kept when it is a candidate and |x_pref| >= tau * m; otherwise the
 *     lowest-numbered candidate row with |x_r| == m is taken.
 *   - Topological order (Algorithm 1 leaves it open): ascending pivot step by
 *     default (a valid topological order, because L(:,j) only reaches steps after
 *     j); ORACLE_ORDER_DFS keeps the DFS reverse postorder instead.
 *   - Every update is one fma(-l, m, x); L is scaled by IEEE division; entries
 *     that cancel to zero stay in the pattern.
 *   - A non-finite value anywhere in the column is reported as ORACLE_NAN, no
 *     candidate or a zero maximum as ORACLE_SINGULAR, with the column.
 *
 * Build: plain C99, -O2 -ffp-contract=off (no contraction other than the
 * explicit fma calls, so x86 and Arm hosts give the same bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    ORACLE_OK = 0,
    ORACLE_INVALID = 1,
    ORACLE_NOT_BTF = 2,
    ORACLE_BAD_ND = 3,
    ORACLE_SINGULAR = 4,
    ORACLE_NAN = 5,
    ORACLE_NOMEM = 6,
};

enum { ORACLE_ORDER_ASCENDING = 0, ORACLE_ORDER_DFS = 1 };

typedef struct {
    int n;
    /* B = A(P,Q) in CSC with sorted rows; bmap[e] = index of B's entry e in A */
    int64_t *Bp;
    int *Bi;
    int64_t *bmap;
    double *Bx;
    int *P, *Q;
    int nblocks;
    int *block_ptr;
    int *blk;            /* blk[i] = BTF block of row/column i */
    int nd_block, nd_leaves;
    int *nd_ptr;         /* 2*leaves entries: node t spans [nd_ptr[t], nd_ptr[t+1]) */
    int *nd_first;       /* first node of t's subtree (postorder: subtree = [first, t]) */
    int status, info_col;
    /* factors (after oracle_factor): B row prow[k] is pivoted at step k */
    int *prow, *pinv;
    int64_t *Lp, *Up;    /* n+1 */
    int *Li, *Ui;        /* L rows are B rows during the factorization, steps after it */
    double *Lx, *Ux;
    int64_t lcap, ucap;
    int factored;
} oracle_lu;

/* ------------------------------------------------------------------------- */
/* structure checks                                                           */

static int is_permutation(int n, const int *p, int *scratch)
{
    memset(scratch, 0, sizeof(int) * (size_t)n);
    for (int i = 0; i < n; i++) {
        if (p[i] < 0 || p[i] >= n || scratch[p[i]]) return 0;
        scratch[p[i]] = 1;
    }
    return 1;
}

/* Number the complete binary ND tree in postorder (Fig. 3: leaves 1,2,4,5,
 * separators 3,6, root 7 for four leaves, here 0-based) and record, for each
 * node, the first node of its subtree. */
static int nd_number(int depth, int *counter, int *first)
{
    int start = *counter;
    if (depth > 0) {
        nd_number(depth - 1, counter, first);
        nd_number(depth - 1, counter, first);
    }
    int t = (*counter)++;
    first[t] = start;
    return t;
}

static int nd_node_of(const oracle_lu *h, int r)
{
    /* last node t with nd_ptr[t] <= r; empty nodes are skipped naturally */
    int lo = 0, hi = 2 * h->nd_leaves - 1; /* nodes 0 .. 2L-2 */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (h->nd_ptr[mid] <= r) lo = mid; else hi = mid;
    }
    return lo;
}

static int nd_related(const oracle_lu *h, int a, int b)
{
    /* a is an ancestor-or-self of b, or the other way round */
    return (h->nd_first[a] <= b && b <= a) || (h->nd_first[b] <= a && a <= b);
}

void oracle_free(oracle_lu *h)
{
    if (!h) return;
    free(h->Bp); free(h->Bi); free(h->bmap); free(h->Bx); free(h->P); free(h->Q);
    free(h->block_ptr); free(h->blk); free(h->nd_ptr); free(h->nd_first);
    free(h->prow); free(h->pinv); free(h->Lp); free(h->Up); free(h->Li); free(h->Ui);
    free(h->Lx); free(h->Ux);
    free(h);
}

int oracle_status(const oracle_lu *h, int *info_col)
{
    if (info_col) *info_col = h->info_col;
    return h->status;
}

/* Validate the input and form the pattern of B = A(P,Q) (Sec. II: PAQ in BTF).
 * The returned handle carries a status; it is NULL only if memory runs out. */
oracle_lu *oracle_analyze(int n, const int *Ap, const int *Ai, const int *P, const int *Q,
                          int nblocks, const int *block_ptr, int nd_block, int nd_leaves,
                          const int *nd_node_ptr)
{
    oracle_lu *h = (oracle_lu *)calloc(1, sizeof(oracle_lu));
    if (!h) return NULL;
    h->n = n;
    h->nd_block = -1;
    h->info_col = -1;
    if (n < 0 || nblocks < 0 || (n > 0 && nblocks < 1)) { h->status = ORACLE_INVALID; return h; }
    size_t nn = (size_t)(n > 0 ? n : 1);
    int *scratch = (int *)calloc(nn, sizeof(int));
    h->P = (int *)malloc(sizeof(int) * nn);
    h->Q = (int *)malloc(sizeof(int) * nn);
    h->blk = (int *)malloc(sizeof(int) * nn);
    h->block_ptr = (int *)malloc(sizeof(int) * (size_t)(nblocks + 1));
    h->Bp = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    if (!scratch || !h->P || !h->Q || !h->blk || !h->block_ptr || !h->Bp) {
        free(scratch); h->status = ORACLE_NOMEM; return h;
    }
    /* the CSC pattern of A: monotone column pointers, rows in range, strictly increasing */
    if (Ap[0] != 0) { free(scratch); h->status = ORACLE_INVALID; return h; }
    for (int j = 0; j < n; j++) {
        if (Ap[j + 1] < Ap[j]) { free(scratch); h->status = ORACLE_INVALID; return h; }
        for (int p = Ap[j]; p < Ap[j + 1]; p++) {
            if (Ai[p] < 0 || Ai[p] >= n || (p > Ap[j] && Ai[p] <= Ai[p - 1])) {
                free(scratch); h->status = ORACLE_INVALID; return h;
            }
        }
    }
    if (!is_permutation(n, P, scratch) || !is_permutation(n, Q, scratch)) {
        free(scratch); h->status = ORACLE_INVALID; return h;
    }
    memcpy(h->P, P, sizeof(int) * (size_t)n);
    memcpy(h->Q, Q, sizeof(int) * (size_t)n);
    /* BTF block boundaries: 0 = b_0 < b_1 < ... < b_nblocks = n */
    h->nblocks = nblocks;
    if (block_ptr[0] != 0 || block_ptr[nblocks] != n) { free(scratch); h->status = ORACLE_INVALID; return h; }
    for (int d = 0; d < nblocks; d++) {
        if (block_ptr[d + 1] <= block_ptr[d]) { free(scratch); h->status = ORACLE_INVALID; return h; }
        for (int i = block_ptr[d]; i < block_ptr[d + 1]; i++) h->blk[i] = d;
    }
    memcpy(h->block_ptr, block_ptr, sizeof(int) * (size_t)(nblocks + 1));
    /* the ND tree of one BTF block (Sec. III-C): 2^depth leaves, postorder nodes */
    if (nd_block >= 0) {
        int depth = 0;
        while ((1 << depth) < nd_leaves) depth++;
        if (nd_block >= nblocks || nd_leaves < 1 || (1 << depth) != nd_leaves) {
            free(scratch); h->status = ORACLE_INVALID; return h;
        }
        int nodes = 2 * nd_leaves - 1;
        h->nd_block = nd_block;
        h->nd_leaves = nd_leaves;
        h->nd_ptr = (int *)malloc(sizeof(int) * (size_t)(nodes + 1));
        h->nd_first = (int *)malloc(sizeof(int) * (size_t)nodes);
        if (!h->nd_ptr || !h->nd_first) { free(scratch); h->status = ORACLE_NOMEM; return h; }
        memcpy(h->nd_ptr, nd_node_ptr, sizeof(int) * (size_t)(nodes + 1));
        if (h->nd_ptr[0] != block_ptr[nd_block] || h->nd_ptr[nodes] != block_ptr[nd_block + 1]) {
            free(scratch); h->status = ORACLE_INVALID; return h;
        }
        for (int t = 0; t < nodes; t++)
            if (h->nd_ptr[t + 1] < h->nd_ptr[t]) { free(scratch); h->status = ORACLE_INVALID; return h; }
        int counter = 0;
        nd_number(depth, &counter, h->nd_first);
    }
    /* B = A(P,Q): B(i,j) = A(P[i], Q[j]); rows sorted by counting placement */
    int *Pinv = scratch;
    for (int i = 0; i < n; i++) Pinv[P[i]] = i;
    int64_t nnz = Ap[n];
    for (int j = 0; j < n; j++) h->Bp[j + 1] = h->Bp[j] + (Ap[Q[j] + 1] - Ap[Q[j]]);
    h->Bi = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    h->bmap = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    h->Bx = (double *)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    if (!h->Bi || !h->bmap || !h->Bx) { free(scratch); h->status = ORACLE_NOMEM; return h; }
    for (int j = 0; j < n; j++) {
        int64_t q = h->Bp[j];
        for (int p = Ap[Q[j]]; p < Ap[Q[j] + 1]; p++, q++) {
            h->Bi[q] = Pinv[Ai[p]];
            h->bmap[q] = p;
        }
        /* insertion sort of the column by row (columns are short) */
        for (int64_t a = h->Bp[j] + 1; a < h->Bp[j + 1]; a++) {
            int r = h->Bi[a];
            int64_t m = h->bmap[a];
            int64_t b = a - 1;
            while (b >= h->Bp[j] && h->Bi[b] > r) { h->Bi[b + 1] = h->Bi[b]; h->bmap[b + 1] = h->bmap[b]; b--; }
            h->Bi[b + 1] = r;
            h->bmap[b + 1] = m;
        }
    }
    free(scratch);
    /* BTF invariant: no entry below the diagonal blocks */
    for (int j = 0; j < n; j++)
        for (int64_t p = h->Bp[j]; p < h->Bp[j + 1]; p++)
            if (h->blk[h->Bi[p]] > h->blk[j]) { h->status = ORACLE_NOT_BTF; h->info_col = j; return h; }
    /* ND invariant: inside the ND block an entry joins two nodes on one root path,
     * i.e. separators disconnect their two halves */
    if (h->nd_block >= 0) {
        int k0 = block_ptr[h->nd_block], k1 = block_ptr[h->nd_block + 1];
        for (int j = k0; j < k1; j++) {
            int tj = nd_node_of(h, j);
            for (int64_t p = h->Bp[j]; p < h->Bp[j + 1]; p++) {
                int i = h->Bi[p];
                if (i < k0) continue;
                if (!nd_related(h, nd_node_of(h, i), tj)) { h->status = ORACLE_BAD_ND; h->info_col = j; return h; }
            }
        }
    }
    h->status = ORACLE_OK;
    return h;
}

/* ------------------------------------------------------------------------- */
/* numeric factorization                                                      */

static int grow(void **a, void **b, int64_t *cap, int64_t need, size_t sa, size_t sb)
{
    if (need <= *cap) return 1;
    int64_t nc = *cap ? *cap : 1024;
    while (nc < need) nc *= 2;
    void *na = realloc(*a, sa * (size_t)nc);
    if (!na) return 0;
    *a = na;
    void *nb = realloc(*b, sb * (size_t)nc);
    if (!nb) return 0;
    *b = nb;
    *cap = nc;
    return 1;
}

static int cmp_by_key(const void *a, const void *b)
{
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Factor every diagonal block of B with the values Ax (A's CSC order).
 * pref: NULL (natural rows) or, per column, the B row preferred as its pivot.
 * Returns the status; on failure info_col names the column. */
int oracle_factor(oracle_lu *h, const double *Ax, double tau, const int *pref, int order)
{
    if (h->status != ORACLE_OK && h->status != ORACLE_SINGULAR && h->status != ORACLE_NAN)
        return h->status;
    h->status = ORACLE_OK;
    h->info_col = -1;
    h->factored = 0;
    int n = h->n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    for (int64_t e = 0; e < h->Bp[n]; e++) h->Bx[e] = Ax[h->bmap[e]];
    free(h->prow); free(h->pinv); free(h->Lp); free(h->Up);
    h->prow = (int *)malloc(sizeof(int) * nn);
    h->pinv = (int *)malloc(sizeof(int) * nn);
    h->Lp = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    h->Up = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    double *x = (double *)calloc(nn, sizeof(double));
    int *mark = (int *)malloc(sizeof(int) * nn);      /* column stamp: row is in the pattern */
    int *pattern = (int *)malloc(sizeof(int) * nn);   /* rows of the pattern */
    int *topo = (int *)malloc(sizeof(int) * nn);      /* pivoted rows, DFS finish order */
    int *stack = (int *)malloc(sizeof(int) * nn);
    int64_t *spos = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *keyed = (int64_t *)malloc(sizeof(int64_t) * nn);
    if (!h->prow || !h->pinv || !h->Lp || !h->Up || !x || !mark || !pattern || !topo || !stack || !spos || !keyed) {
        h->status = ORACLE_NOMEM;
        goto done;
    }
    for (int i = 0; i < n; i++) { h->pinv[i] = -1; h->prow[i] = -1; mark[i] = -1; }

    for (int d = 0; d < h->nblocks && h->status == ORACLE_OK; d++) {
        int k0 = h->block_ptr[d], k1 = h->block_ptr[d + 1];
        for (int c = k0; c < k1; c++) {
            /* candidate rows of column c: its BTF block, or its ND node */
            int lo = k0, hi = k1;
            if (d == h->nd_block) {
                int t = nd_node_of(h, c);
                lo = h->nd_ptr[t];
                hi = h->nd_ptr[t + 1];
            }
            /* 1. reach by depth-first search in the graph of L (Algorithm 1's first step):
             *    a row pivoted at step s has an edge to every row of L(:,s) */
            int np = 0, nt = 0;
            for (int64_t p = h->Bp[c]; p < h->Bp[c + 1]; p++) {
                int r0 = h->Bi[p];
                if (r0 < k0 || mark[r0] == c) continue;   /* rows above the block: off-diagonal part */
                int top = 0;
                stack[0] = r0;
                mark[r0] = c;
                pattern[np++] = r0;
                spos[0] = h->pinv[r0] >= 0 ? h->Lp[h->pinv[r0]] : -1;
                while (top >= 0) {
                    int r = stack[top];
                    int s = h->pinv[r];
                    int descended = 0;
                    if (s >= 0) {
                        int64_t end = h->Lp[s + 1];
                        while (spos[top] < end) {
                            int r2 = h->Li[spos[top]++];
                            if (mark[r2] != c) {
                                mark[r2] = c;
                                pattern[np++] = r2;
                                stack[++top] = r2;
                                spos[top] = h->pinv[r2] >= 0 ? h->Lp[h->pinv[r2]] : -1;
                                descended = 1;
                                break;
                            }
                        }
                    }
                    if (!descended) {
                        if (s >= 0) topo[nt++] = r;      /* finished: postorder */
                        top--;
                    }
                }
            }
            /* 2. the order of the updates */
            int nu = nt;
            if (order == ORACLE_ORDER_ASCENDING) {
                for (int k = 0; k < nu; k++) keyed[k] = ((int64_t)h->pinv[topo[k]] << 32) | (uint32_t)topo[k];
                qsort(keyed, (size_t)nu, sizeof(int64_t), cmp_by_key);
                for (int k = 0; k < nu; k++) topo[k] = (int)(keyed[k] & 0xffffffff);
            } else {
                for (int a = 0, b = nu - 1; a < b; a++, b--) { int t = topo[a]; topo[a] = topo[b]; topo[b] = t; }
            }
            /* 3. x = B_dd(:,c), then the sparse triangular solve (Algorithm 1's update loop) */
            for (int64_t p = h->Bp[c]; p < h->Bp[c + 1]; p++)
                if (h->Bi[p] >= k0) x[h->Bi[p]] = h->Bx[p];
            for (int k = 0; k < nu; k++) {
                int r = topo[k];
                int s = h->pinv[r];
                double m = x[r];
                for (int64_t p = h->Lp[s]; p < h->Lp[s + 1]; p++)
                    x[h->Li[p]] = fma(-h->Lx[p], m, x[h->Li[p]]);
            }
            /* 4. pivot (Algorithm 1's pivot selection) among unpivoted pattern rows of [lo, hi) */
            double amax = 0.0;
            int ncand = 0, bad = 0;
            for (int k = 0; k < np; k++) {
                int r = pattern[k];
                double v = x[r];
                if (!isfinite(v)) bad = 1;
                if (h->pinv[r] < 0 && r >= lo && r < hi) {
                    ncand++;
                    if (fabs(v) > amax) amax = fabs(v);
                }
            }
            int piv = -1;
            if (bad) {
                h->status = ORACLE_NAN;
            } else if (ncand == 0 || amax == 0.0) {
                h->status = ORACLE_SINGULAR;
            } else {
                int pr = pref ? pref[c] : c;
                if (pr >= lo && pr < hi && pr < n && mark[pr] == c && h->pinv[pr] < 0 &&
                    fabs(x[pr]) >= tau * amax) {
                    piv = pr;
                } else {
                    for (int k = 0; k < np; k++) {
                        int r = pattern[k];
                        if (h->pinv[r] < 0 && r >= lo && r < hi && fabs(x[r]) == amax && (piv < 0 || r < piv))
                            piv = r;
                    }
                }
            }
            if (piv < 0) {
                h->info_col = c;
                for (int k = 0; k < np; k++) x[pattern[k]] = 0.0;
                break;
            }
            /* 5. copy x into U(:,c) and L(:,c) (Algorithm 1's final copy) */
            int64_t lnz = h->Lp[c], unz = h->Up[c];
            if (!grow((void **)&h->Ui, (void **)&h->Ux, &h->ucap, unz + nu + 1, sizeof(int), sizeof(double)) ||
                !grow((void **)&h->Li, (void **)&h->Lx, &h->lcap, lnz + np, sizeof(int), sizeof(double))) {
                h->status = ORACLE_NOMEM;
                break;
            }
            /* U entries in ascending step order, the diagonal last */
            for (int k = 0; k < nu; k++) keyed[k] = ((int64_t)h->pinv[topo[k]] << 32) | (uint32_t)topo[k];
            qsort(keyed, (size_t)nu, sizeof(int64_t), cmp_by_key);
            for (int k = 0; k < nu; k++) {
                int r = (int)(keyed[k] & 0xffffffff);
                h->Ui[unz] = h->pinv[r];
                h->Ux[unz++] = x[r];
            }
            double pv = x[piv];
            h->Ui[unz] = c;
            h->Ux[unz++] = pv;
            for (int k = 0; k < np; k++) {
                int r = pattern[k];
                if (h->pinv[r] < 0 && r != piv) {
                    h->Li[lnz] = r;
                    h->Lx[lnz++] = x[r] / pv;
                }
            }
            h->Lp[c + 1] = lnz;
            h->Up[c + 1] = unz;
            h->pinv[piv] = c;
            h->prow[c] = piv;
            for (int k = 0; k < np; k++) x[pattern[k]] = 0.0;
        }
    }
    if (h->status == ORACLE_OK) {
        /* L rows: B rows -> pivot steps, then each column sorted by step */
        for (int c = 0; c < n; c++) {
            int64_t s = h->Lp[c], e = h->Lp[c + 1];
            for (int64_t p = s; p < e; p++) h->Li[p] = h->pinv[h->Li[p]];
            for (int64_t a = s + 1; a < e; a++) {
                int r = h->Li[a];
                double v = h->Lx[a];
                int64_t b = a - 1;
                while (b >= s && h->Li[b] > r) { h->Li[b + 1] = h->Li[b]; h->Lx[b + 1] = h->Lx[b]; b--; }
                h->Li[b + 1] = r;
                h->Lx[b + 1] = v;
            }
        }
        h->factored = 1;
    }
done:
    free(x); free(mark); free(pattern); free(topo); free(stack); free(spos); free(keyed);
    return h->status;
}

void oracle_sizes(const oracle_lu *h, int64_t *lnz, int64_t *unz)
{
    *lnz = h->factored ? h->Lp[h->n] : 0;
    *unz = h->factored ? h->Up[h->n] : 0;
}

/* Factors in B's coordinates: prow[k] = B row pivoted at step k; L strictly lower
 * (unit diagonal implied) and U upper with the diagonal last, rows = pivot steps,
 * each column in ascending order. */
int oracle_export(const oracle_lu *h, int *prow, int64_t *Lp, int *Li, double *Lx,
                  int64_t *Up, int *Ui, double *Ux)
{
    if (!h->factored) return ORACLE_INVALID;
    int n = h->n;
    memcpy(prow, h->prow, sizeof(int) * (size_t)n);
    memcpy(Lp, h->Lp, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(Up, h->Up, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(Li, h->Li, sizeof(int) * (size_t)h->Lp[n]);
    memcpy(Lx, h->Lx, sizeof(double) * (size_t)h->Lp[n]);
    memcpy(Ui, h->Ui, sizeof(int) * (size_t)h->Up[n]);
    memcpy(Ux, h->Ux, sizeof(double) * (size_t)h->Up[n]);
    return ORACLE_OK;
}

/* Solve A x = b for nrhs right-hand sides (column-major, leading dims ldb, ldx).
 * BTF back-substitution (Sec. III-B: the off-diagonal blocks keep the values of B
 * and enter through a matrix-vector product): blocks from last to first, each one
 * L (unit) forward and U backward solve on the pivoted right-hand side. */
int oracle_solve(const oracle_lu *h, int nrhs, const double *b, int ldb, double *x, int ldx)
{
    if (!h->factored) return ORACLE_INVALID;
    int n = h->n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *c = (double *)malloc(sizeof(double) * nn);
    double *z = (double *)malloc(sizeof(double) * nn);
    if (!c || !z) { free(c); free(z); return ORACLE_NOMEM; }
    for (int q = 0; q < nrhs; q++) {
        const double *bq = b + (size_t)q * (size_t)ldb;
        for (int i = 0; i < n; i++) c[i] = bq[h->P[i]];
        for (int d = h->nblocks - 1; d >= 0; d--) {
            int k0 = h->block_ptr[d], k1 = h->block_ptr[d + 1];
            for (int k = k0; k < k1; k++) z[k] = c[h->prow[k]];
            for (int k = k0; k < k1; k++)                        /* L w = P c */
                for (int64_t p = h->Lp[k]; p < h->Lp[k + 1]; p++)
                    z[h->Li[p]] = fma(-h->Lx[p], z[k], z[h->Li[p]]);
            for (int k = k1 - 1; k >= k0; k--) {                 /* U z = w */
                int64_t dg = h->Up[k + 1] - 1;                   /* diagonal is last */
                z[k] = z[k] / h->Ux[dg];
                for (int64_t p = h->Up[k]; p < dg; p++)
                    z[h->Ui[p]] = fma(-h->Ux[p], z[k], z[h->Ui[p]]);
            }
            for (int j = k0; j < k1; j++)                        /* c_e -= B_ed z_d, e < d */
                for (int64_t p = h->Bp[j]; p < h->Bp[j + 1] && h->Bi[p] < k0; p++)
                    c[h->Bi[p]] = fma(-h->Bx[p], z[j], c[h->Bi[p]]);
        }
        double *xq = x + (size_t)q * (size_t)ldx;
        for (int j = 0; j < n; j++) xq[h->Q[j]] = z[j];
    }
    free(c);
    free(z);
    return ORACLE_OK;
}

/* B's pattern and values (after oracle_factor), for the tests' checks. */
void oracle_bsizes(const oracle_lu *h, int64_t *nnz) { *nnz = h->Bp[h->n]; }

void oracle_bexport(const oracle_lu *h, int64_t *Bp, int *Bi, double *Bx)
{
    memcpy(Bp, h->Bp, sizeof(int64_t) * (size_t)(h->n + 1));
    memcpy(Bi, h->Bi, sizeof(int) * (size_t)h->Bp[h->n]);
    memcpy(Bx, h->Bx, sizeof(double) * (size_t)h->Bp[h->n]);
}
