// kernels_dense.cu -- the in-node phase of an ND separator as a dense
// right-looking elimination, one block of threads per separator.
//
// After the descendant phase (Algorithm 4's solves with the descendants' L and
// the reductions into A-hat) every column of separator j is a dense vector over
// its L-space (own rows, then the ancestors' rows) with a pattern bitmap: the
// block A-hat_jj stacked on the rows of the L_kj below it.  Algorithm 1 on these
// columns, one after the other, is the same computation as a right-looking
// elimination of the stacked block: at step k the pivot of column k is chosen
// (threshold partial pivoting among the separator's unpivoted rows, the
// preferred row first), L(:,k) is the column over the pivot, and every later
// column whose pattern holds the pivot row receives that entry as U(k, c) and the
// update x -= L(:,k) U(k,c), one fma per entry, which also extends its pattern.
// Each entry so receives its updates in ascending step order, the order of the
// column-by-column form, so the factors are identical bit for bit; the steps a
// column receives are exactly those whose pivot row lies in its pattern at that
// time, as in the column's reach.
//
// Step k in two phases.  First, warp 0 copies column k into shared memory,
// applies step k - 1 to it there, chooses its pivot, ranks the L entries (a
// prefix sum over the pattern words) and divides, while warps 1..31 apply step
// k - 1 to the columns after k (one warp a column, one L entry per lane, eight
// independent loads in flight per lane).  Second, one thread per later column
// takes its U(k, c) (moving the column's U region if full).  The L column of a
// step is double-buffered in shared memory, so that step k - 1's is still being
// applied while step k's is built.  The dense block lives in the A-hat scratch
// (L2-resident).
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include <cooperative_groups.h>

#include "basker_internal.h"
#include "device_util.cuh"
#include "trace.cuh"

using namespace bk;
namespace cg = cooperative_groups;

namespace {

constexpr int DN_THREADS = 1024;
constexpr int DN_WARPS = DN_THREADS / 32;

struct DnShared {
    bk_task T;
    // nonzero: leave (failure, overflow, or an earlier failure elsewhere).  Read
    // right after the cluster barrier of step k from stop[k & 1], which is written
    // only before that barrier: by step k's first phase or step k - 1's second
    // phase.  Every block thus leaves after the same step.
    int stop[2];
    int pslot[2];        // pivot slot of the step (by step parity), in the step owner's copy
    int cnt[2];          // L count of the step (by step parity), in the step owner's copy
};

// Every block of the cluster sees stop[parity]: written into each block's copy.
__device__ __forceinline__ void cluster_stop(cg::cluster_group &cl, DnShared &S, int parity)
{
    for (unsigned r = 0; r < cl.num_blocks(); r++) *cl.map_shared_rank(&S.stop[parity], r) = 1;
}

template <typename V>
__global__ void __launch_bounds__(DN_THREADS) bk_dense_node_kernel(bk_dev d, const int32_t *__restrict__ task_ids,
                                                                   double tau, int pref_mode)
{
    V *const Lx = vals<V>(d.Lx);
    V *const Ux = vals<V>(d.Ux);
    V *const Ahat = vals<V>(d.ahat);
    cg::cluster_group cl = cg::this_cluster();
    const int CN = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    __shared__ DnShared S;
    extern __shared__ __align__(16) unsigned char dsm[];
    const int tid_x = threadIdx.x, lane = tid_x & 31, wid = tid_x >> 5;
    const int tid = task_ids[blockIdx.x / CN];
    BK_TSTART(t0);
    if (wid == 0) load_task(S.T, d.tasks + tid, lane);
    if (tid_x == 0) S.stop[0] = S.stop[1] = 0;
    __syncthreads();
    const bk_task &T = S.T;
    const int nown = T.hi - T.lo, lsp = T.lspace, nrw = (lsp + 31) >> 5;
    // shared layout (8-byte slots first): ub[nown] ue[nown] (int64) | lval[2][lsp] colv[lsp]
    // mval[nown] (V in 8-byte slots) | nu[nown] spiv[nown] lsl[2][lsp] wpre[nrw] lbits[2][nrw]
    // colb[nrw] (32-bit) | cbad[nown] chit[nown] (bytes).  Per-column state is kept by
    // the block that owns the column (column k: block k mod CN); spiv by every block.
    int64_t *ubs = reinterpret_cast<int64_t *>(dsm);
    int64_t *ues = ubs + nown;
    double *slots = reinterpret_cast<double *>(ues + nown);
    V *lval0 = reinterpret_cast<V *>(slots);
    V *lval1 = reinterpret_cast<V *>(slots + lsp);
    V *colv = reinterpret_cast<V *>(slots + 2 * lsp);
    V *mval = reinterpret_cast<V *>(slots + 3 * lsp);
    int32_t *nus = reinterpret_cast<int32_t *>(slots + 3 * lsp + nown);
    int32_t *spiv = nus + nown;
    int32_t *lsl0 = spiv + nown;
    int32_t *lsl1 = lsl0 + lsp;
    int32_t *wpre = lsl1 + lsp;
    uint32_t *lbits0 = reinterpret_cast<uint32_t *>(wpre + nrw);
    uint32_t *lbits1 = lbits0 + nrw;
    uint32_t *colb = lbits1 + nrw;
    unsigned char *cbad = reinterpret_cast<unsigned char *>(colb + nrw);
    unsigned char *chit = cbad + nown;

    V *const A = Ahat + T.ahoff;                       // column k at A + k * lsp
    uint32_t *const AB = d.abits + T.aboff;            // column k at AB + k * nrw
    for (int k = tid_x; k < nown; k += DN_THREADS) {
        const int c = T.lo + k;
        if (k % CN == rank) {
            ubs[k] = d.Ubeg[c];
            ues[k] = d.Uend[c];
            nus[k] = d.dcnt[c];
        }
        spiv[k] = -1;
        cbad[k] = 0;
        chit[k] = 0;
    }
    // entries outside the patterns hold stale values: zero them (own columns)
    for (int64_t e = tid_x; e < (int64_t)nown * lsp; e += DN_THREADS) {
        const int k = (int)(e / lsp), s = (int)(e % lsp);
        if (k % CN != rank) continue;
        if (!((AB[(int64_t)k * nrw + (s >> 5)] >> (s & 31)) & 1u)) A[e] = V(0);
    }
    cl.sync();

    for (int k = 0; k < nown; ++k) {
        const int c = T.lo + k;
        const int b = k & 1;
        const int owner = k % CN;
        V *const lval = b ? lval1 : lval0;
        int32_t *const lsl = b ? lsl1 : lsl0;
        uint32_t *const lbits = b ? lbits1 : lbits0;
        const V *const lval_p = b ? lval0 : lval1;     // step k - 1
        const int32_t *const lsl_p = b ? lsl0 : lsl1;
        const uint32_t *const lbits_p = b ? lbits0 : lbits1;
        const int cnt_p = k > 0 ? S.cnt[b ^ 1] : 0;
        if (rank != owner || wid > 0) {
            // ---- step k - 1 on this block's columns after k (one warp a column)
            const int nw = rank == owner ? DN_WARPS - 1 : DN_WARPS;
            const int w0 = rank == owner ? wid - 1 : wid;
            int first = k + 1 + ((rank - (k + 1) % CN) + CN) % CN;   // first own column after k
            for (int k2 = first + w0 * CN; k2 < nown && k > 0; k2 += nw * CN) {
                if (!chit[k2]) continue;
                uint32_t *const b2 = AB + (int64_t)k2 * nrw;
                for (int w = lane; w < nrw; w += 32) b2[w] |= lbits_p[w];
                V *const a2 = A + (int64_t)k2 * lsp;
                const V m = mval[k2];
                int q = lane;
                for (; q + 7 * 32 < cnt_p; q += 8 * 32) {
                    int sl[8];
                    V xv[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) sl[u] = lsl_p[q + 32 * u];
#pragma unroll
                    for (int u = 0; u < 8; u++) xv[u] = a2[sl[u]];
#pragma unroll
                    for (int u = 0; u < 8; u++) a2[sl[u]] = fma(-lval_p[q + 32 * u], m, xv[u]);
                }
                for (; q < cnt_p; q += 32) {
                    const int s0 = lsl_p[q];
                    a2[s0] = fma(-lval_p[q], m, a2[s0]);
                }
            }
        } else {
            // ---- the owner's warp 0: column k into shared memory, step k - 1
            // applied to it, then its pivot and L(:,k)
            const int pref = pref_mode ? d.pref[c] : c;
            int64_t lb = d.Lbeg[c], le = d.Lend[c];
            bool stop = false;
            if ((k & 15) == 0) stop = __shfl_sync(BK_FULL, (int)should_stop(d, tid, c), 0) != 0;
            const V *const ac = A + (int64_t)k * lsp;
            const uint32_t *const bc = AB + (int64_t)k * nrw;
            for (int w = lane; w < nrw; w += 32) colb[w] = bc[w];
#pragma unroll 8
            for (int s = lane; s < lsp; s += 32) colv[s] = ac[s];
            __syncwarp();
            if (k > 0 && chit[k]) {
                const V m = mval[k];
                for (int w = lane; w < nrw; w += 32) colb[w] |= lbits_p[w];
                for (int q = lane; q < cnt_p; q += 32) {
                    const int s0 = lsl_p[q];
                    colv[s0] = fma(-lval_p[q], m, colv[s0]);
                }
                __syncwarp();
            }
            V amax = V(0);
            int ncand = 0;
            bool bad = cbad[k] != 0;
            for (int s = lane; s < lsp; s += 32) {
                if (!((colb[s >> 5] >> (s & 31)) & 1u)) continue;
                const V v = colv[s];
                if (!isfinite(v)) bad = true;
                if (s < nown) {
                    ncand++;
                    amax = fmax(amax, fabs(v));
                }
            }
            amax = warp_max(amax);
            ncand = warp_sum(ncand);
            bad = __any_sync(BK_FULL, bad);
            int ps = -1;
            if (!stop && !bad && ncand > 0 && amax > V(0)) {
                const int pr = pref - T.lo;
                if (pr >= 0 && pr < nown && spiv[pr] < 0 && ((colb[pr >> 5] >> (pr & 31)) & 1u) &&
                    (double)fabs(colv[pr]) >= tau * (double)amax) {
                    ps = pr;
                } else {
                    // the lowest candidate row holding the maximum
                    int best = INT_MAX;
                    for (int s = lane; s < nown; s += 32)
                        if (((colb[s >> 5] >> (s & 31)) & 1u) && fabs(colv[s]) == amax) { best = s; break; }
                    ps = warp_min(best);
                    if (ps == INT_MAX) {             // cannot happen: amax is one of the values
                        if (lane == 0) report_internal(d.status, c, 40);
                        ps = -1;
                    }
                }
            } else if (!stop && lane == 0) {
                report_fail(d.status, c, bad ? BK_CODE_NAN : BK_CODE_SINGULAR);
            }
            if (ps >= 0) {
                // ranks of the L entries (the pattern without the pivot, ascending
                // slots) and the pattern words they add to the columns they update
                int carry = 0;
                for (int w0 = 0; w0 < nrw; w0 += 32) {
                    const int w = w0 + lane;
                    uint32_t bits = w < nrw ? colb[w] : 0u;
                    if (w == (ps >> 5)) bits &= ~(1u << (ps & 31));
                    const int cnt = __popc(bits);
                    const int pre = warp_exscan(cnt, lane);
                    if (w < nrw) {
                        wpre[w] = carry + pre;
                        lbits[w] = bits;
                    }
                    carry += __shfl_sync(BK_FULL, pre + cnt, 31);
                }
                // L region (a larger pool region when the count outgrows it)
                bool fail = false;
                if (lb + carry > le) {
                    const int64_t cap = min((long long)(2 * (int64_t)carry + 16),
                                            (long long)((T.hi - c - 1) + (lsp - nown)));
                    int64_t nb = 0;
                    if (lane == 0) nb = pool_alloc(d.pool, d.lpool_end, cap);
                    nb = __shfl_sync(BK_FULL, nb, 0);
                    if (nb < 0) {
                        fail = true;
                        if (lane == 0) report_overflow(d, T, tid, c, 1);
                    } else {
                        lb = nb;
                        if (lane == 0) {
                            d.Lbeg[c] = lb;
                            d.Lend[c] = nb + cap;
                        }
                    }
                }
                __syncwarp();
                if (fail) {
                    if (lane == 0) cluster_stop(cl, S, b);
                } else {
                    const V xp = colv[ps];
                    // L(:,c) = x / pivot over the pattern
                    for (int s = lane; s < lsp; s += 32) {
                        const int w = s >> 5, bt = s & 31;
                        const uint32_t bits = lbits[w];
                        if (!((bits >> bt) & 1u)) continue;
                        const int pos = wpre[w] + __popc(bits & ((1u << bt) - 1u));
                        const V q = colv[s] / xp;
                        d.Li[lb + pos] = row_of_lslot(T, s);
                        Lx[lb + pos] = q;
                        lsl[pos] = s;
                        lval[pos] = q;
                    }
                    if (lane == 0) {
                        const int piv = T.lo + ps;
                        const int64_t u = ubs[k] + nus[k];
                        d.Ui[u] = c;
                        Ux[u] = xp;
                        d.Ucnt[c] = nus[k] + 1;
                        d.Lcnt[c] = carry;
                        d.pinv[piv] = c;
                        d.prow[c] = piv;
                        if (piv != c) atomicAdd(&d.status->offdiag, 1);
                        S.pslot[b] = ps;
                        S.cnt[b] = carry;
                    }
                }
            } else if (lane == 0) {
                cluster_stop(cl, S, b);
            }
        }
        cl.sync();
        if (S.stop[b]) break;
        // ---- the step's pivot and L(:,k) from its owner's shared memory
        DnShared *const So = cl.map_shared_rank(&S, owner);
        const int ps = So->pslot[b], cnt = So->cnt[b];
        if (rank != owner) {
            const V *const rv = cl.map_shared_rank(lval, owner);
            const int32_t *const rs = cl.map_shared_rank(lsl, owner);
            const uint32_t *const rb = cl.map_shared_rank(lbits, owner);
            for (int q = tid_x; q < cnt; q += DN_THREADS) {
                lsl[q] = rs[q];
                lval[q] = rv[q];
            }
            for (int w = tid_x; w < nrw; w += DN_THREADS) lbits[w] = rb[w];
            if (tid_x == 0) {
                S.pslot[b] = ps;
                S.cnt[b] = cnt;
            }
        }
        if (tid_x == 0) spiv[ps] = k;
        // ---- this block's later columns whose pattern holds the pivot row (one
        // thread a column): U(c, c2) = that entry, which leaves the column
        const int first = k + 1 + ((rank - (k + 1) % CN) + CN) % CN;
        for (int k2 = first + tid_x * CN; k2 < nown; k2 += DN_THREADS * CN) {
            uint32_t *const b2 = AB + (int64_t)k2 * nrw;
            const uint32_t w = b2[ps >> 5];
            const bool hit = (w >> (ps & 31)) & 1u;
            chit[k2] = hit;
            if (!hit) continue;
            V *const a2 = A + (int64_t)k2 * lsp;
            const V m = a2[ps];
            mval[k2] = m;
            int64_t ub = ubs[k2], ue = ues[k2];
            const int nu = nus[k2];
            if (ub + nu + 2 > ue) {
                const int c2 = T.lo + k2;
                const int64_t cap = grown_ucap(nu, (int64_t)(c2 - T.sp_lo) + 1);
                const int64_t nb = pool_alloc(d.pool + 1, d.upool_end, cap);
                if (nb < 0) {
                    report_overflow(d, T, tid, c2, 2);
                    cluster_stop(cl, S, b ^ 1);
                    chit[k2] = 0;
                    continue;
                }
                for (int q = 0; q < nu; q++) {
                    d.Ui[nb + q] = d.Ui[ub + q];
                    Ux[nb + q] = Ux[ub + q];
                }
                ub = nb;
                ue = nb + cap;
                d.Ubeg[c2] = ub;
                d.Uend[c2] = ue;
                ubs[k2] = ub;
                ues[k2] = ue;
            }
            d.Ui[ub + nu] = c;
            Ux[ub + nu] = m;
            nus[k2] = nu + 1;
            if (!isfinite(m)) cbad[k2] = 1;
            a2[ps] = V(0);
            b2[ps >> 5] = w & ~(1u << (ps & 31));
        }
        __syncthreads();
    }
    // no block leaves while another may still read its shared memory
    cl.sync();
    if (rank == 0 && tid_x == 0) BK_TREC(d.trace, BK_TR_DENSE, 0, tid, t0);
}

}  // namespace

size_t bk_dense_node_smem(const bk_task &T)
{
    const size_t own = (size_t)(T.hi - T.lo), lsp = (size_t)T.lspace, nrw = (lsp + 31) / 32;
    return own * 16 + 3 * lsp * 8 + own * 8 + own * 8 + 2 * lsp * 4 + 4 * nrw * 4 + 2 * own + 16;
}

bool bk_dense_node_eligible(const bk_task &T)
{
    return T.sp_lo < T.lo && T.hi > T.lo && bk_dense_node_smem(T) <= BK_DENSE_SMEM;
}

void bk_launch_dense_nodes(const bk_dev &d, const int32_t *task_ids, int32_t ntasks, size_t smem, double tau,
                           int pref_mode, int cluster, void *stream)
{
    if (ntasks <= 0) return;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(bk_dense_node_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, BK_DENSE_SMEM);
        cudaFuncSetAttribute(bk_dense_node_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, BK_DENSE_SMEM);
    });
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntasks * cluster));
    cfg.blockDim = dim3(DN_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (d.prec)
        cudaLaunchKernelEx(&cfg, bk_dense_node_kernel<float>, d, task_ids, tau, pref_mode);
    else
        cudaLaunchKernelEx(&cfg, bk_dense_node_kernel<double>, d, task_ids, tau, pref_mode);
}

int bk_dense_node_cluster(const bk_task &T)
{
    return T.hi - T.lo >= BK_DENSE_CLUSTER_MIN ? BK_DENSE_CLUSTER : 1;
}
