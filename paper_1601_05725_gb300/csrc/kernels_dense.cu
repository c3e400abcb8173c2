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
constexpr int DN_CG = 4;             // warps of the owner block that build a step's column

// the column group's barrier (named barrier 1, DN_CG warps)
__device__ __forceinline__ void cg_bar() { asm volatile("bar.sync 1, %0;" ::"n"(DN_CG * 32) : "memory"); }

struct DnShared {
    bk_task T;
    // nonzero: leave (failure, overflow, or an earlier failure elsewhere).  Read
    // right after the first cluster barrier of step k from stop[k & 1], which is
    // written only before that barrier: by step k's first phase or step k - 1's
    // second phase.  Every block thus leaves after the same step.
    int stop[2];
    int pslot[2];        // pivot slot of the step (by step parity), in the step owner's copy
    int cnt[2];          // L count of the step (by step parity), in the step owner's copy
    double xp[2];        // the pivot's value (the step owner's copy)
    long long lb[2];     // start of L(:,c) (the step owner's copy)
    int cstop;           // the column group's stop decision
    unsigned long long redk[DN_CG];  // the column group's reductions
    int redc[DN_CG], redb[DN_CG], redi[DN_CG];
};

// Every block of the cluster sees stop[parity]: written into each block's copy.
__device__ __forceinline__ void cluster_stop(cg::cluster_group &cl, DnShared &S, int parity)
{
    for (unsigned r = 0; r < cl.num_blocks(); r++) *cl.map_shared_rank(&S.stop[parity], r) = 1;
}

// Shared memory of a block, in bytes: the base layout, and the block's own
// columns of the dense block with their pattern words (columns k with
// k mod cluster == rank), kept on chip when they fit.
__host__ __device__ inline size_t dn_base_bytes(int own, int lsp)
{
    const size_t nrw = ((size_t)lsp + 31) / 32;
    return (size_t)own * 16 + 3 * (size_t)lsp * 8 + (size_t)own * 8 + (size_t)own * 8 + 2 * (size_t)lsp * 4 +
           (4 * nrw + 1) * 4 + 2 * (size_t)own + 16;
}

__host__ __device__ inline size_t dn_local_bytes(int own, int lsp, int cluster)
{
    const size_t nloc = ((size_t)own + cluster - 1) / cluster, nrw = ((size_t)lsp + 31) / 32;
    return nloc * (size_t)lsp * 8 + nloc * nrw * 4;
}

template <typename V>
__global__ void __launch_bounds__(DN_THREADS) bk_dense_node_kernel(bk_dev d, const int32_t *__restrict__ task_ids,
                                                                   double tau, int pref_mode, size_t smem_bytes)
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
    // the block's columns on chip when they fit in the shared memory given
    const bool onchip = dn_base_bytes(nown, lsp) + dn_local_bytes(nown, lsp, CN) <= smem_bytes;
    const int nloc = onchip ? (nown + CN - 1) / CN : 0;
    // shared layout (8-byte slots first): ub[nown] ue[nown] (int64) | lval[2][lsp] colv[lsp]
    // mval[nown] loc[nloc][lsp] (V in 8-byte slots) | nus[nown] spiv[nown] lsl[2][lsp] wpre[nrw + 1]
    // lbits[2][nrw] colb[nrw] locb[nloc][nrw] (32-bit) | cbad[nown] chit[nown] (bytes).
    // Per-column state is kept by the block that owns the column (column k: block
    // k mod CN, local index k / CN); spiv by every block.
    int64_t *ubs = reinterpret_cast<int64_t *>(dsm);
    int64_t *ues = ubs + nown;
    double *slots = reinterpret_cast<double *>(ues + nown);
    V *lval0 = reinterpret_cast<V *>(slots);
    V *lval1 = reinterpret_cast<V *>(slots + lsp);
    V *colv = reinterpret_cast<V *>(slots + 2 * lsp);
    V *mval = reinterpret_cast<V *>(slots + 3 * lsp);
    double *locslots = slots + 3 * lsp + nown;
    int32_t *nus = reinterpret_cast<int32_t *>(locslots + (int64_t)nloc * lsp);
    int32_t *spiv = nus + nown;
    int32_t *lsl0 = spiv + nown;
    int32_t *lsl1 = lsl0 + lsp;
    int32_t *wpre = lsl1 + lsp;
    uint32_t *lbits0 = reinterpret_cast<uint32_t *>(wpre + nrw + 1);
    uint32_t *lbits1 = lbits0 + nrw;
    uint32_t *colb = lbits1 + nrw;
    uint32_t *locb = colb + nrw;
    unsigned char *cbad = reinterpret_cast<unsigned char *>(locb + (int64_t)nloc * nrw);
    unsigned char *chit = cbad + nown;

    V *const A = Ahat + T.ahoff;                       // column k at A + k * lsp
    uint32_t *const AB = d.abits + T.aboff;            // column k at AB + k * nrw
    // column k of this block (values, pattern words): on chip or in the scratch
    auto colA = [&](int k) -> V * {
        return onchip ? reinterpret_cast<V *>(locslots + (int64_t)(k / CN) * lsp) : A + (int64_t)k * lsp;
    };
    auto colB = [&](int k) -> uint32_t * { return onchip ? locb + (int64_t)(k / CN) * nrw : AB + (int64_t)k * nrw; };
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
    // the block's columns (entries outside the patterns hold stale values: zero)
    for (int64_t e = tid_x; e < (int64_t)nown * lsp; e += DN_THREADS) {
        const int k = (int)(e / lsp), sl = (int)(e % lsp);
        if (k % CN != rank) continue;
        const bool in = (AB[(int64_t)k * nrw + (sl >> 5)] >> (sl & 31)) & 1u;
        if (onchip) colA(k)[sl] = in ? A[e] : V(0);
        else if (!in) A[e] = V(0);
    }
    if (onchip)
        for (int64_t e = tid_x; e < (int64_t)nown * nrw; e += DN_THREADS) {
            const int k = (int)(e / nrw);
            if (k % CN == rank) colB(k)[e % nrw] = AB[e];
        }
    cl.sync();

#ifdef BK_TRACE
    // trace builds: per-phase cycles of thread 0 (owner steps, other steps)
    long long cyc[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
    long long lap_t = clock64();
#define DN_LAP(i)                                                        \
    do {                                                                 \
        const long long t_ = clock64();                                  \
        cyc[rank == owner ? 0 : 1][i] += t_ - lap_t;                     \
        lap_t = t_;                                                      \
    } while (0)
#else
#define DN_LAP(i)
#endif
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
        if (rank != owner || wid >= DN_CG) {
            // ---- step k - 1 on this block's columns after k (one warp a column)
            const int nw = rank == owner ? DN_WARPS - DN_CG : DN_WARPS;
            const int w0 = rank == owner ? wid - DN_CG : wid;
            int first = k + 1 + ((rank - (k + 1) % CN) + CN) % CN;   // first own column after k
            for (int k2 = first + w0 * CN; k2 < nown && k > 0; k2 += nw * CN) {
                if (!chit[k2]) continue;
                uint32_t *const b2 = colB(k2);
                for (int w = lane; w < nrw; w += 32) b2[w] |= lbits_p[w];
                V *const a2 = colA(k2);
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
            // ---- the owner's column group (DN_CG warps): column k, step k - 1
            // applied to it, its pivot; then warp 0 ranks its L entries and takes
            // its L region (the division follows after the cluster barrier, spread
            // over the cluster)
            constexpr int CT = DN_CG * 32;
            const int ct = tid_x;
            const int pref = pref_mode ? d.pref[c] : c;
            int64_t lb = d.Lbeg[c], le = d.Lend[c];      // read early: used after the pivot
            const V *const ac = colA(k);
            const uint32_t *const bc = colB(k);
            const bool upd = k > 0 && chit[k];
            for (int w = ct; w < nrw; w += CT) colb[w] = bc[w] | (upd ? lbits_p[w] : 0u);
            for (int sl = ct; sl < lsp; sl += CT) colv[sl] = ac[sl];
            if (ct == 0) S.cstop = (k & 15) == 0 ? (int)should_stop(d, tid, c) : 0;
            cg_bar();
            if (upd) {
                const V m = mval[k];
                for (int q = ct; q < cnt_p; q += CT) {
                    const int s0 = lsl_p[q];
                    colv[s0] = fma(-lval_p[q], m, colv[s0]);
                }
            }
            cg_bar();
            // magnitudes compared as integers: for finite values the order of |v|
            // is that of the bits with the sign cleared (the non-finite ones are
            // caught by bad first), so the maximum and the rows holding it need no
            // floating-point instruction
            unsigned long long kmax = 0;
            int ncand = 0;
            bool bad = cbad[k] != 0;
            for (int sl = ct; sl < lsp; sl += CT) {
                if (!((colb[sl >> 5] >> (sl & 31)) & 1u)) continue;
                const unsigned long long key = mag_key(colv[sl]);
                if (key >= key_inf<V>()) bad = true;
                if (sl < nown) {
                    ncand++;
                    kmax = key > kmax ? key : kmax;
                }
            }
            kmax = warp_max_key(kmax);
            ncand = warp_sum(ncand);
            bad = __any_sync(BK_FULL, bad);
            if (lane == 0) {
                S.redk[wid] = kmax;
                S.redc[wid] = ncand;
                S.redb[wid] = bad ? 1 : 0;
            }
            cg_bar();
            kmax = 0;
            ncand = 0;
            bad = false;
#pragma unroll
            for (int g = 0; g < DN_CG; g++) {
                kmax = S.redk[g] > kmax ? S.redk[g] : kmax;
                ncand += S.redc[g];
                bad = bad || S.redb[g] != 0;
            }
            const V amax = key_value<V>(kmax);
            const bool stop = S.cstop != 0;
            int ps = -1;
            const bool ok = !stop && !bad && ncand > 0 && kmax > 0;
            const int pr = pref - T.lo;
            const bool take_pref = ok && pr >= 0 && pr < nown && spiv[pr] < 0 && ((colb[pr >> 5] >> (pr & 31)) & 1u) &&
                                   (double)fabs(colv[pr]) >= tau * (double)amax;
            if (ok && !take_pref) {
                // the lowest candidate row holding the maximum
                int best = INT_MAX;
                for (int sl = ct; sl < nown; sl += CT)
                    if (((colb[sl >> 5] >> (sl & 31)) & 1u) && mag_key(colv[sl]) == kmax) { best = sl; break; }
                best = warp_min(best);
                if (lane == 0) S.redi[wid] = best;
            }
            cg_bar();
            if (take_pref) {
                ps = pr;
            } else if (ok) {
                int best = INT_MAX;
#pragma unroll
                for (int g = 0; g < DN_CG; g++) best = min(best, S.redi[g]);
                ps = best;
                if (ps == INT_MAX) {                 // cannot happen: amax is one of the values
                    if (ct == 0) report_internal(d.status, c, 40);
                    ps = -1;
                }
            } else if (!stop && ct == 0) {
                report_fail(d.status, c, bad ? BK_CODE_NAN : BK_CODE_SINGULAR);
            }
            if (wid == 0) {
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
                    if (lane == 0) wpre[nrw] = carry;
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
                    } else if (lane == 0) {
                        const V xp = colv[ps];
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
                        S.xp[b] = (double)xp;
                        S.lb[b] = lb;
                    }
                } else if (lane == 0) {
                    cluster_stop(cl, S, b);
                }
            }
        }
        DN_LAP(0);
        cl.sync();
        DN_LAP(1);
        if (S.stop[b]) break;
        DnShared *const So = cl.map_shared_rank(&S, owner);
        const int ps = So->pslot[b], cnt = So->cnt[b];
        if (tid_x == 0) spiv[ps] = k;
        {
            // ---- L(:,c) = x / pivot over the pattern, one entry a thread, computed
            // by every block from the owner's column (its own copy for its updates;
            // the owner stores it): no second barrier and no gather
            const uint32_t *const rb = cl.map_shared_rank(lbits, owner);
            const int32_t *const rw = cl.map_shared_rank(wpre, owner);
            const V *const rc = cl.map_shared_rank(colv, owner);
            const V xp = (V)So->xp[b];
            const int64_t lb = So->lb[b];
            for (int sl = tid_x; sl < lsp; sl += DN_THREADS) {
                const int w = sl >> 5, bt = sl & 31;
                const uint32_t bits = rb[w];
                if (!((bits >> bt) & 1u)) continue;
                const int pos = rw[w] + __popc(bits & ((1u << bt) - 1u));
                const V q = rc[sl] / xp;
                if (rank == owner) {
                    d.Li[lb + pos] = row_of_lslot(T, sl);
                    Lx[lb + pos] = q;
                }
                lsl[pos] = sl;
                lval[pos] = q;
            }
            if (rank != owner)
                for (int w = tid_x; w < nrw; w += DN_THREADS) lbits[w] = rb[w];
        }
        // ---- this block's later columns whose pattern holds the pivot row (one
        // thread a column): U(c, c2) = that entry, which leaves the column
        const int first = k + 1 + ((rank - (k + 1) % CN) + CN) % CN;
        for (int k2 = first + tid_x * CN; k2 < nown; k2 += DN_THREADS * CN) {
            uint32_t *const b2 = colB(k2);
            const uint32_t w = b2[ps >> 5];
            const bool hit = (w >> (ps & 31)) & 1u;
            chit[k2] = hit;
            if (!hit) continue;
            V *const a2 = colA(k2);
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
        DN_LAP(2);
        if (rank != owner && tid_x == 0) {
            S.pslot[b] = ps;
            S.cnt[b] = cnt;
        }
        __syncthreads();
        DN_LAP(4);
    }
#undef DN_LAP
#ifdef BK_TRACE
    if (tid_x == 0)
        for (int i = 0; i < 5; i++)
            bk_trace_raw(d.trace, BK_TR_PHASE, 40 + i, tid * 16 + rank, (unsigned long long)cyc[0][i],
                         (unsigned long long)cyc[1][i]);
#endif
    // no block leaves while another may still read its shared memory
    cl.sync();
    if (rank == 0 && tid_x == 0) BK_TREC(d.trace, BK_TR_DENSE, 0, tid, t0);
}

}  // namespace

size_t bk_dense_node_smem(const bk_task &T)
{
    const int own = T.hi - T.lo;
    const size_t base = dn_base_bytes(own, T.lspace);
    const size_t full = base + dn_local_bytes(own, T.lspace, bk_dense_node_cluster(T));
    return full <= BK_DENSE_SMEM ? full : base;
}

bool bk_dense_node_eligible(const bk_task &T)
{
    return T.sp_lo < T.lo && T.hi > T.lo && dn_base_bytes(T.hi - T.lo, T.lspace) <= BK_DENSE_SMEM;
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
        cudaLaunchKernelEx(&cfg, bk_dense_node_kernel<float>, d, task_ids, tau, pref_mode, smem);
    else
        cudaLaunchKernelEx(&cfg, bk_dense_node_kernel<double>, d, task_ids, tau, pref_mode, smem);
}

int bk_dense_node_cluster(const bk_task &T)
{
    return T.hi - T.lo >= BK_DENSE_CLUSTER_MIN ? BK_DENSE_CLUSTER : 1;
}
