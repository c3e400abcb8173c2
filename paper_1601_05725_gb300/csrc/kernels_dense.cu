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
// Per step: one warp chooses the pivot and ranks the L entries (a prefix sum over
// the pattern words); all threads divide and store L(:,k), while one thread per
// later column takes its U(k, c) (and moves the column's U region if full); then
// one warp per later column adds L(:,k)'s pattern words and applies the update,
// one L entry per lane, eight independent loads in flight per lane.  The dense
// block lives in the A-hat scratch (L2-resident); the step's L column, the
// multipliers and the per-column U cursors are in shared memory.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "basker_internal.h"
#include "device_util.cuh"

using namespace bk;

namespace {

constexpr int DN_THREADS = 1024;
constexpr int DN_WARPS = DN_THREADS / 32;

struct DnShared {
    bk_task T;
    int stop;            // nonzero: leave (failure, overflow, or an earlier failure elsewhere)
    int pslot;           // this step's pivot slot
    int cnt;             // this step's L count
    int64_t lb;          // this step's L region start
    double xp;           // this step's pivot value (in V)
};

template <typename V>
__global__ void __launch_bounds__(DN_THREADS) bk_dense_node_kernel(bk_dev d, const int32_t *__restrict__ task_ids,
                                                                   double tau, int pref_mode)
{
    V *const Lx = vals<V>(d.Lx);
    V *const Ux = vals<V>(d.Ux);
    V *const Ahat = vals<V>(d.ahat);
    __shared__ DnShared S;
    extern __shared__ __align__(16) unsigned char dsm[];
    const int tid_x = threadIdx.x, lane = tid_x & 31, wid = tid_x >> 5;
    const int tid = task_ids[blockIdx.x];
    if (wid == 0) load_task(S.T, d.tasks + tid, lane);
    if (tid_x == 0) S.stop = 0;
    __syncthreads();
    const bk_task &T = S.T;
    const int nown = T.hi - T.lo, lsp = T.lspace, nrw = (lsp + 31) >> 5;
    // shared layout: ub[nown] ue[nown] (int64) | lval[lsp] mval[nown] (V, 8-byte slots) |
    //                nu[nown] spiv[nown] lsl[lsp] wpre[nrw] lbits[nrw] (32-bit) | cbad[nown] chit[nown] (bytes)
    int64_t *ubs = reinterpret_cast<int64_t *>(dsm);
    int64_t *ues = ubs + nown;
    V *lval = reinterpret_cast<V *>(ues + nown);
    V *mval = reinterpret_cast<V *>(reinterpret_cast<double *>(ues + nown) + lsp);
    int32_t *nus = reinterpret_cast<int32_t *>(reinterpret_cast<double *>(ues + nown) + lsp + nown);
    int32_t *spiv = nus + nown;
    int32_t *lsl = spiv + nown;
    int32_t *wpre = lsl + lsp;
    uint32_t *lbits = reinterpret_cast<uint32_t *>(wpre + nrw);
    unsigned char *cbad = reinterpret_cast<unsigned char *>(lbits + nrw);
    unsigned char *chit = cbad + nown;

    V *const A = Ahat + T.ahoff;                       // column k at A + k * lsp
    uint32_t *const AB = d.abits + T.aboff;            // column k at AB + k * nrw
    for (int k = tid_x; k < nown; k += DN_THREADS) {
        const int c = T.lo + k;
        ubs[k] = d.Ubeg[c];
        ues[k] = d.Uend[c];
        nus[k] = d.dcnt[c];
        spiv[k] = -1;
        cbad[k] = 0;
    }
    // entries outside the patterns hold stale values: zero them
    for (int64_t e = tid_x; e < (int64_t)nown * lsp; e += DN_THREADS) {
        const int k = (int)(e / lsp), s = (int)(e % lsp);
        if (!((AB[(int64_t)k * nrw + (s >> 5)] >> (s & 31)) & 1u)) A[e] = V(0);
    }
    __syncthreads();

    for (int k = 0; k < nown; ++k) {
        const int c = T.lo + k;
        V *const ac = A + (int64_t)k * lsp;
        const uint32_t *const bc = AB + (int64_t)k * nrw;
        // ---- pivot of column c and the ranks of its L entries (warp 0)
        if (wid == 0) {
            bool stop = false;
            if ((k & 15) == 0) stop = __shfl_sync(BK_FULL, (int)should_stop(d, tid, c), 0) != 0;
            V amax = V(0);
            int ncand = 0;
            bool bad = cbad[k] != 0;
#pragma unroll 4
            for (int s = lane; s < lsp; s += 32) {
                if (!((bc[s >> 5] >> (s & 31)) & 1u)) continue;
                const V v = ac[s];
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
                const int pref = pref_mode ? d.pref[c] : c;
                const int pr = pref - T.lo;
                if (pr >= 0 && pr < nown && spiv[pr] < 0 && ((bc[pr >> 5] >> (pr & 31)) & 1u) &&
                    (double)fabs(ac[pr]) >= tau * (double)amax) {
                    ps = pr;
                } else {
                    // the lowest candidate row holding the maximum
                    int best = INT_MAX;
                    for (int s = lane; s < nown; s += 32)
                        if (((bc[s >> 5] >> (s & 31)) & 1u) && fabs(ac[s]) == amax) { best = s; break; }
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
                // slots) and the pattern words they add to a column they update
                int carry = 0;
                for (int w0 = 0; w0 < nrw; w0 += 32) {
                    const int w = w0 + lane;
                    uint32_t bits = w < nrw ? bc[w] : 0u;
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
                int64_t lb = d.Lbeg[c], le = d.Lend[c];
                int fail = 0;
                if (lb + carry > le) {
                    const int64_t cap = min((long long)(2 * (int64_t)carry + 16),
                                            (long long)((T.hi - c - 1) + (lsp - nown)));
                    int64_t nb = 0;
                    if (lane == 0) nb = pool_alloc(d.pool, d.lpool_end, cap);
                    nb = __shfl_sync(BK_FULL, nb, 0);
                    if (nb < 0) {
                        fail = 1;
                        if (lane == 0) report_overflow(d, T, tid, c, 1);
                    } else {
                        lb = nb;
                        le = nb + cap;
                        if (lane == 0) {
                            d.Lbeg[c] = lb;
                            d.Lend[c] = le;
                        }
                    }
                }
                if (lane == 0) {
                    if (fail) {
                        S.stop = 1;
                    } else {
                        const V xp = ac[ps];
                        const int piv = T.lo + ps;
                        const int64_t u = ubs[k] + nus[k];
                        d.Ui[u] = c;
                        Ux[u] = xp;
                        d.Ucnt[c] = nus[k] + 1;
                        d.Lcnt[c] = carry;
                        d.pinv[piv] = c;
                        d.prow[c] = piv;
                        spiv[ps] = c;
                        if (piv != c) atomicAdd(&d.status->offdiag, 1);
                        S.pslot = ps;
                        S.cnt = carry;
                        S.lb = lb;
                        S.xp = (double)xp;
                    }
                }
            } else if (lane == 0) {
                S.stop = 1;
            }
        }
        __syncthreads();
        if (S.stop) return;
        const int ps = S.pslot, cnt = S.cnt;
        const int64_t lb = S.lb;
        const V xp = (V)S.xp;
        // ---- L(:,c) = x / pivot over the pattern (all threads)
        for (int s = tid_x; s < lsp; s += DN_THREADS) {
            const int w = s >> 5, b = s & 31;
            const uint32_t bits = lbits[w];
            if (!((bits >> b) & 1u)) continue;
            const int pos = wpre[w] + __popc(bits & ((1u << b) - 1u));
            const V q = ac[s] / xp;
            d.Li[lb + pos] = row_of_lslot(T, s);
            Lx[lb + pos] = q;
            lsl[pos] = s;
            lval[pos] = q;
        }
        // ---- the later columns whose pattern holds the pivot row (one thread a
        // column): U(c, c2) = that entry, which leaves the column
        for (int k2 = k + 1 + tid_x; k2 < nown; k2 += DN_THREADS) {
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
                    S.stop = 1;
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
        if (S.stop) return;
        // ---- x -= L(:,c) U(c, c2) and the pattern of L(:,c) added (one warp a column)
        for (int k2 = k + 1 + wid; k2 < nown; k2 += DN_WARPS) {
            if (!chit[k2]) continue;
            uint32_t *const b2 = AB + (int64_t)k2 * nrw;
            for (int w = lane; w < nrw; w += 32) b2[w] |= lbits[w];
            V *const a2 = A + (int64_t)k2 * lsp;
            const V m = mval[k2];
            int q = lane;
            for (; q + 7 * 32 < cnt; q += 8 * 32) {
                int sl[8];
                V xv[8];
#pragma unroll
                for (int u = 0; u < 8; u++) sl[u] = lsl[q + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; u++) xv[u] = a2[sl[u]];
#pragma unroll
                for (int u = 0; u < 8; u++) a2[sl[u]] = fma(-lval[q + 32 * u], m, xv[u]);
            }
            for (; q < cnt; q += 32) {
                const int s0 = lsl[q];
                a2[s0] = fma(-lval[q], m, a2[s0]);
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t bk_dense_node_smem(const bk_task &T)
{
    const size_t own = (size_t)(T.hi - T.lo), lsp = (size_t)T.lspace, nrw = (lsp + 31) / 32;
    return own * 16 + lsp * 8 + own * 8 + own * 8 + lsp * 4 + nrw * 8 + 2 * own + 16;
}

bool bk_dense_node_eligible(const bk_task &T)
{
    return T.sp_lo < T.lo && T.hi > T.lo && bk_dense_node_smem(T) <= BK_DENSE_SMEM;
}

void bk_launch_dense_nodes(const bk_dev &d, const int32_t *task_ids, int32_t ntasks, size_t smem, double tau,
                           int pref_mode, void *stream)
{
    if (ntasks <= 0) return;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(bk_dense_node_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, BK_DENSE_SMEM);
        cudaFuncSetAttribute(bk_dense_node_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, BK_DENSE_SMEM);
    });
    if (d.prec)
        bk_dense_node_kernel<float><<<ntasks, DN_THREADS, smem, (cudaStream_t)stream>>>(d, task_ids, tau, pref_mode);
    else
        bk_dense_node_kernel<double><<<ntasks, DN_THREADS, smem, (cudaStream_t)stream>>>(d, task_ids, tau, pref_mode);
}
