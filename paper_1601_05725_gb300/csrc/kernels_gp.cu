// kernels_gp.cu -- numeric Gilbert-Peierls factorization on the GPU.
//
//   bk_gather_kernel   values of A -> B's entries (the fixed permutation P, Q).
//   bk_gp_task_kernel  Algorithm 1, one warp per task (a small BTF block, an ND
//                      leaf, or the in-node phase of an ND separator), columns in
//                      order.  Per column: Algorithm 1's reach and its update loop
//                      are one sweep over a bitmap of pivot
//                      steps, lowest step first (an ascending step order is a
//                      topological order of the reach); then threshold pivoting
//                      among the node's own unpivoted rows (warp max / warp min
//                      by shuffle) and the split of x into L and U.
//   bk_gp_desc_kernel  Algorithm 4's upper off-diagonal solves and reductions for ND separators: one warp per
//                      separator column solves that column against every
//                      descendant's L (the U_ij blocks) and applies the products
//                      to the separator's and ancestors' rows (the reductions into
//                      A-hat_lj and A-hat_jj), lowest step first.  None of this
//                      depends on the separator's own pivots, so all its columns
//                      run at once; the in-node phase then continues each column
//                      with the separator's own steps and picks the pivot.
//
// Within a column every entry receives its updates one fma at a time in
// ascending pivot-step order (descendant steps, then own steps), and L is
// scaled with an IEEE division, the order the reference definition uses.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <climits>

#include "basker_internal.h"
#include "device_util.cuh"
#include "trace.cuh"

using namespace bk;

namespace {

constexpr int DESC_PF = 8;     // L entries per lane in flight in the descendant phase

// B's values in the factorization's type (FP32: rounded to nearest from FP64).
template <typename V>
__global__ void bk_gather_kernel(V *__restrict__ Bx, const double *__restrict__ vals,
                                 const int32_t *__restrict__ bmap, int64_t nnz)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        Bx[e] = (V)__ldg(vals + bmap[e]);
}

__device__ __forceinline__ void set_bit(volatile uint32_t *bm, int i)
{
    atomicOr(const_cast<uint32_t *>(bm) + (i >> 5), 1u << (i & 31));
}

// Lowest set bit at or after word w0 of a bitmap of nw words; -1 if none.
// The bitmap is re-read every call (other lanes set bits between calls).
__device__ __forceinline__ int next_step_bit(const volatile uint32_t *bm, int nw, int &w0, int lane)
{
    while (w0 < nw) {
        const uint32_t v = (w0 + lane < nw) ? bm[w0 + lane] : 0u;
        const uint32_t ball = __ballot_sync(BK_FULL, v != 0u);
        if (ball) {
            const int l = __ffs(ball) - 1;
            const uint32_t bits = __shfl_sync(BK_FULL, v, l);
            w0 += l;
            return (w0 << 5) + (__ffs(bits) - 1);
        }
        w0 += 32;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Algorithm 1 per task.  The column state lives in the task's L-space (own rows,
// then ancestors' rows; base = lo):
//   x   dense values, zero outside the current column's pattern
//   sb  bitmap of own pivot steps still to apply to the column
//   rb  bitmap of L-space rows in the pattern that are not pivoted
//   tb  (mode 2) own rows whose pivot status a recomputed column changed
// A row counts as pivoted at column c when 0 <= pinv[row] < c, so that pinv may
// still hold later columns' previous pivots during a redo.
// pref_mode: 0 prefer the natural row; 1 prefer pref[c]; 2 a redo from task_c0
// that recomputes only the columns whose stored pattern meets a touched row
// (or that rejected their preferred pivot) and keeps the others.
template <typename V>
__global__ void __launch_bounds__(32) bk_gp_task_kernel(bk_dev d, const int32_t *__restrict__ task_ids,
                                                        const int32_t *__restrict__ task_c0, double tau,
                                                        int pref_mode)
{
    const V *const Bx = vals<V>(d.Bx);
    V *const Lx = vals<V>(d.Lx);
    V *const Ux = vals<V>(d.Ux);
    V *const Ahat = vals<V>(d.ahat);
    __shared__ bk_task T;
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x;
    const int tid = task_ids[blockIdx.x];
    load_task(T, d.tasks + tid, lane);
    const int base = T.lo;
    const int nown = T.hi - T.lo;
    const int lsp = T.lspace;
    const int nsw = (nown + 31) >> 5;
    const int nrw = (lsp + 31) >> 5;
    // layout (shared memory, or the task's global workspace slice):
    //   x[lsp] | slbeg[nown] | sb[nsw] | rb[nrw] | tb[nsw] | spinv[nown] | sprow[nown] | slcnt[nown]
    // spinv / sprow / slbeg / slcnt cache pinv, prow, Lbeg, Lcnt of the node's own
    // rows and columns (written through to global memory when they change).
    unsigned char *area = T.wsoff < 0 ? dsm : d.ws + T.wsoff;
    V *x = reinterpret_cast<V *>(area);
    int64_t *slbeg = reinterpret_cast<int64_t *>(area + (size_t)lsp * 8);
    uint32_t *s32 = reinterpret_cast<uint32_t *>(slbeg + nown);
    volatile uint32_t *sb = s32;
    volatile uint32_t *rb = s32 + nsw;
    volatile uint32_t *tb = rb + nrw;
    int32_t *spinv = reinterpret_cast<int32_t *>(s32 + 2 * nsw + nrw);
    int32_t *sprow = spinv + nown;
    int32_t *slcnt = sprow + nown;
    if (T.wsoff < 0) {
        for (int i = lane; i < lsp; i += 32) x[i] = 0.0;
        for (int i = lane; i < nsw + nrw; i += 32) s32[i] = 0u;
    }
    for (int i = lane; i < nsw; i += 32) tb[i] = 0u;
    for (int i = lane; i < nown; i += 32) {
        spinv[i] = d.pinv[T.lo + i];
        sprow[i] = d.prow[T.lo + i];
        slbeg[i] = d.Lbeg[T.lo + i];
        slcnt[i] = d.Lcnt[T.lo + i];
    }
    __syncwarp();
    const bool sep = T.sp_lo < T.lo;               // continue a separator column from A-hat
    const int c_begin = task_c0 ? task_c0[blockIdx.x] : T.lo;

    for (int c = c_begin; c < T.hi; ++c) {
        if (((c - c_begin) & 15) == 0 && __shfl_sync(BK_FULL, (int)should_stop(d, tid, c), 0)) return;
        int64_t ub = d.Ubeg[c], ue = d.Uend[c];
        int64_t lb = d.Lbeg[c], le = d.Lend[c];
        if (pref_mode == 2) {
            // keep a column whose stored pattern meets no touched row and that
            // accepted its preferred pivot: its computation is unchanged
            bool hit = c == c_begin || d.col_fail[c] != 0;
            {
                const int r0 = d.pref[c] - base;     // its own previous pivot row
                if ((unsigned)r0 < (unsigned)nown && (tb[r0 >> 5] >> (r0 & 31)) & 1u) hit = true;
            }
            if (!hit) {
                const int uc = d.Ucnt[c];
                for (int k = lane; k < uc - 1 && !hit; k += 32) {
                    const int j = d.Ui[ub + k];
                    if (j >= T.lo) {
                        const int r = d.pref[j] - base;
                        if ((unsigned)r < (unsigned)nown && (tb[r >> 5] >> (r & 31)) & 1u) hit = true;
                    }
                }
                const int lc = d.Lcnt[c];
                for (int k = lane; k < lc && !hit; k += 32) {
                    const int r = d.Li[lb + k] - base;
                    if ((unsigned)r < (unsigned)nown && (tb[r >> 5] >> (r & 31)) & 1u) hit = true;
                }
            }
            if (!__any_sync(BK_FULL, hit)) continue;
            // recompute: the previous pivot row is touched and free again
            if (lane == 0) {
                const int r0 = d.pref[c];
                if (r0 >= T.lo && r0 < T.hi) {
                    atomicOr(const_cast<uint32_t *>(tb) + ((r0 - base) >> 5), 1u << ((r0 - base) & 31));
                    if (spinv[r0 - base] == c) {
                        spinv[r0 - base] = -1;
                        d.pinv[r0] = -1;
                    }
                }
            }
            __syncwarp();
        }
        int nu = 0;
        bool bad = false;
        if (sep) {
            // A-hat(:,c) = the column after all descendant steps (Algorithm 4's solves with L_ii and reductions)
            nu = d.dcnt[c];
            const V *ah = Ahat + T.ahoff + (int64_t)(c - T.lo) * lsp;
            const uint32_t *ab = d.abits + T.aboff + (int64_t)(c - T.lo) * nrw;
            for (int w = lane; w < nrw; w += 32) {
                uint32_t bits = ab[w];
                uint32_t keep = 0u;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int ls = (w << 5) + b;
                    x[ls] = ah[ls];
                    const int p = ls < nown ? spinv[ls] : -1;
                    if (p >= 0 && p < c && p >= base) set_bit(sb, p - base);
                    else keep |= 1u << b;
                }
                if (keep) atomicOr(const_cast<uint32_t *>(rb) + w, keep);
            }
        } else {
            const int e1 = d.Bp[c + 1];
            for (int e = d.dstart[c] + lane; e < e1; e += 32) {
                const int r = d.Bi[e];
                const int s = slot_of(T, base, r);
                if (s < 0) { report_internal(d.status, c, 11); continue; }
                x[s] = Bx[e];
                const int p = s < nown ? spinv[s] : -1;
                if (p >= 0 && p < c) {
                    if (p >= base) set_bit(sb, p - base);
                    else report_internal(d.status, c, 12);
                } else {
                    set_bit(rb, s);
                }
            }
        }
        __syncwarp();

        // Algorithm 1's reach and updates: own pivot steps, lowest first (each at most once)
        int w0 = 0;
        for (int iter = 0;; iter++) {
            const int jb = next_step_bit(sb, nsw, w0, lane);
            if (jb < 0) break;
            const int j = base + jb;
            const int sp = sprow[jb] - base;       // a pivoted own row: slot = row - lo
            if (iter > nown || j >= c || (unsigned)sp >= (unsigned)nown) {
                if (lane == 0) report_internal(d.status, c, 13);
                return;
            }
            const V m = x[sp];
            __syncwarp();
            if (lane == 0) {
                atomicAnd(const_cast<uint32_t *>(sb) + (jb >> 5), ~(1u << (jb & 31)));
                x[sp] = 0.0;
            }
            if (!isfinite(m)) bad = true;
            if (ub + nu + 2 > ue) {
                // move the column to a larger pool region (twice its entries so far)
                const int64_t cap = grown_ucap(nu, (int64_t)(c - T.sp_lo) + 1);
                int64_t nb = 0;
                if (lane == 0) nb = pool_alloc(d.pool + 1, d.upool_end, cap);
                nb = __shfl_sync(BK_FULL, nb, 0);
                if (nb < 0) {
                    if (lane == 0) report_overflow(d, T, tid, c, 2);
                    return;
                }
                for (int k = lane; k < nu; k += 32) {
                    d.Ui[nb + k] = d.Ui[ub + k];
                    Ux[nb + k] = Ux[ub + k];
                }
                __syncwarp();
                ub = nb;
                ue = nb + cap;
                if (lane == 0) {
                    d.Ubeg[c] = ub;
                    d.Uend[c] = ue;
                }
            }
            if (lane == 0) {
                d.Ui[ub + nu] = j;
                Ux[ub + nu] = m;
            }
            nu++;
            const int64_t jl = slbeg[jb];
            const int jc = slcnt[jb];
            for (int k = lane; k < jc; k += 32) {
                const int r = d.Li[jl + k];
                const V l = Lx[jl + k];
                const int s = slot_of(T, base, r);
                if (s < 0) { report_internal(d.status, c, 14); continue; }
                x[s] = fma(-l, m, x[s]);
                const int p = s < nown ? spinv[s] : -1;
                if (p >= 0 && p < c) {
                    if (p > j) set_bit(sb, p - base);
                    else report_internal(d.status, c, 15);
                } else {
                    set_bit(rb, s);
                }
            }
            __syncwarp();
        }

        // Algorithm 1's pivot selection: threshold pivot among the unpivoted own rows
        unsigned long long km = 0;          // largest own magnitude, as a key
        int ncand = 0;
        for (int w = lane; w < nrw; w += 32) {
            uint32_t bits = rb[w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int ls = (w << 5) + b;
                const V v = x[ls];
                if (!isfinite(v)) bad = true;
                if (ls < nown) {
                    ncand++;
                    km = key_max(km, mag_key(v));
                }
            }
        }
        km = warp_max_key(km);
        const V amax = key_value<V>(km);
        ncand = warp_sum(ncand);
        bad = __any_sync(BK_FULL, bad);
        int piv = -1;
        if (!bad && ncand > 0 && amax > 0.0) {
            const int pref = pref_mode ? d.pref[c] : c;
            if (pref >= T.lo && pref < T.hi && (spinv[pref - base] < 0 || spinv[pref - base] >= c) &&
                (double)fabs(x[pref - base]) >= tau * (double)amax) {
                piv = pref;
            } else {
                int best = INT_MAX;
                for (int w = lane; w < nsw; w += 32) {
                    uint32_t bits = rb[w];
                    while (bits) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const int ls = (w << 5) + b;
                        if (ls < nown && mag_key(x[ls]) == km) { best = ls; break; }
                    }
                    if (best != INT_MAX) break;
                }
                best = warp_min(best);
                piv = base + best;
            }
        }
        if (piv < 0) {
            if (lane == 0) report_fail(d.status, c, bad ? BK_CODE_NAN : BK_CODE_SINGULAR);
            return;
        }

        // Algorithm 1's copy to L and U: U(:,c) got the steps above, the pivot closes it, L(:,c) = x / pivot
        const V xp = x[piv - base];
        if (lane == 0) {
            d.Ui[ub + nu] = c;
            Ux[ub + nu] = xp;
        }
        nu++;
        const int pl = piv - base;
        {
            int cnt_all = 0;
            for (int w = lane; w < nrw; w += 32) cnt_all += __popc(rb[w]);
            cnt_all = warp_sum(cnt_all) - 1;          // without the pivot
            if (lb + cnt_all > le) {
                const int64_t cap = min((long long)(2 * (int64_t)cnt_all + 16),
                                        (long long)((T.hi - c - 1) + (lsp - nown)));
                int64_t nb = 0;
                if (lane == 0) nb = pool_alloc(d.pool, d.lpool_end, cap);
                nb = __shfl_sync(BK_FULL, nb, 0);
                if (nb < 0) {
                    if (lane == 0) report_overflow(d, T, tid, c, 1);
                    return;
                }
                lb = nb;
                le = nb + cap;
                if (lane == 0) {
                    d.Lbeg[c] = lb;
                    d.Lend[c] = le;
                    slbeg[c - base] = lb;
                }
            }
        }
        int64_t lpos = lb;
        for (int wbase = 0; wbase < nrw; wbase += 32) {
            const int w = wbase + lane;
            uint32_t bits = w < nrw ? rb[w] : 0u;
            if (w < nrw && bits) rb[w] = 0u;
            if (w == (pl >> 5)) bits &= ~(1u << (pl & 31));
            const int cnt = __popc(bits);
            const int pre = warp_exscan(cnt, lane);
            const int tot = __shfl_sync(BK_FULL, pre + cnt, 31);
            if (lpos + tot > le) {
                if (lane == 0) report_overflow(d, T, tid, c, 1);
                return;
            }
            int64_t q = lpos + pre;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int ls = (w << 5) + b;
                d.Li[q] = row_of_lslot(T, ls);
                Lx[q] = x[ls] / xp;
                x[ls] = 0.0;
                q++;
            }
            lpos += tot;
        }
        __syncwarp();
        if (lane == 0) {
            x[pl] = 0.0;
            d.pinv[piv] = c;
            d.prow[c] = piv;
            spinv[pl] = c;
            sprow[c - base] = piv;
            slcnt[c - base] = (int)(lpos - lb);
            d.Lcnt[c] = (int)(lpos - lb);
            d.Ucnt[c] = nu;
            if (piv != c) atomicAdd(&d.status->offdiag, 1);
            if (pref_mode == 2) atomicOr(const_cast<uint32_t *>(tb) + (pl >> 5), 1u << (pl & 31));
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Descendant phase of separator columns (one warp per column, persistent).
// Column space: subtree rows [sp_lo, hi) then ancestors (base = sp_lo); the step
// bitmap covers descendant steps [sp_lo, lo) only.  The bitmaps sit in shared
// memory when the level's fit (d.dd_words words a warp), else in the slice.
// Every descendant step is final before this kernel, so the step after the
// current one (the lowest set bit once the current one is cleared) has its pivot
// slot, the extent of its L column and its first DSTEP_PF * 32 entries (rows'
// slots, values, the rows' pivot steps) read while the current step is applied;
// a step that the current one adds below that prediction is read when found.
constexpr int DSTEP_PF = 4;
template <typename V>
struct DStep {
    int sp, jc;
    int64_t jl;
    int s[DSTEP_PF], p[DSTEP_PF];
    V l[DSTEP_PF];
};

template <typename V>
__device__ __forceinline__ void read_dstep(const bk_dev &d, const bk_task &T, DStep<V> &st, int j, int ndesc,
                                           int lane)
{
    const int base = T.sp_lo;
    const V *const Lx = vals<V>(d.Lx);
    st.sp = d.prow[j] - base;
    st.jl = d.Lbeg[j];
    st.jc = d.Lcnt[j];
    int r[DSTEP_PF];
#pragma unroll
    for (int u = 0; u < DSTEP_PF; u++) {
        const int q = lane + 32 * u;
        r[u] = q < st.jc ? d.Li[st.jl + q] : -1;
        st.l[u] = q < st.jc ? Lx[st.jl + q] : V(0);
    }
#pragma unroll
    for (int u = 0; u < DSTEP_PF; u++) {
        st.s[u] = r[u] >= 0 ? slot_of(T, base, r[u]) : -2;
        st.p[u] = (st.s[u] >= 0 && st.s[u] < ndesc) ? d.pinv[r[u]] : -1;
    }
}

template <typename V>
__global__ void __launch_bounds__(128) bk_gp_desc_kernel(bk_dev d, const int32_t *__restrict__ cols,
                                                         int32_t ncols, int32_t *counter,
                                                         const int32_t *__restrict__ ncols_dev)
{
    if (ncols_dev) ncols = *ncols_dev;      // a list made on the device (columns left by the fast path)
    const V *const Bx = vals<V>(d.Bx);
    V *const Lx = vals<V>(d.Lx);
    V *const Ux = vals<V>(d.Ux);
    V *const Ahat = vals<V>(d.ahat);
    __shared__ bk_task Ts[4];
    extern __shared__ uint32_t gd_bits[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * 4 + wib;
    if (gw >= d.wsd_warps) return;
    bk_task &T = Ts[wib];
    unsigned char *slice = d.wsd + (int64_t)gw * d.wsd_slice;
    uint32_t *const wbits = gd_bits + (int64_t)wib * d.dd_words;
    for (int i = lane; i < d.dd_words; i += 32) wbits[i] = 0u;
    __syncwarp();
    int cur_task = -1;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(counter, 1);
        k = __shfl_sync(BK_FULL, k, 0);
        if (k >= ncols) break;
        const int c = cols[k];
        BK_TSTART(t0);
        const int tid = d.col_task[c];
        if (__shfl_sync(BK_FULL, (int)should_stop(d, tid, c), 0)) continue;
        if (tid != cur_task) {
            load_task(T, d.tasks + tid, lane);
            cur_task = tid;
        }
        const int base = T.sp_lo;
        const int ndesc = T.lo - T.sp_lo;
        const int lsp = T.lspace;
        const int nsw = (ndesc + 31) >> 5;
        const int nrw = (lsp + 31) >> 5;
        V *x = reinterpret_cast<V *>(slice);
        volatile uint32_t *sb = d.dd_words ? wbits : reinterpret_cast<uint32_t *>(x + T.space);
        volatile uint32_t *rb = sb + nsw;
        int64_t ub = d.Ubeg[c], ue = d.Uend[c];
        bool bad = false;
        int nu = 0;

        const int e1 = d.Bp[c + 1];
        for (int e = d.dstart[c] + lane; e < e1; e += 32) {
            const int r = d.Bi[e];
            const int s = slot_of(T, base, r);
            if (s < 0) { report_internal(d.status, c, 16); continue; }
            x[s] = Bx[e];
            if (s < ndesc) {
                const int p = d.pinv[r];            // descendant rows are all pivoted
                if ((unsigned)(p - base) < (unsigned)ndesc) set_bit(sb, p - base);
                else report_internal(d.status, c, 17);
            } else {
                set_bit(rb, s - ndesc);
            }
        }
        __syncwarp();
        int w0 = 0;
        bool overflow = false, broken = false;
        int jb = next_step_bit(sb, nsw, w0, lane);
        DStep<V> cur, nxt;
        if (jb >= 0) read_dstep(d, T, cur, base + jb, ndesc, lane);
        for (int iter = 0; jb >= 0; iter++) {
            const int j = base + jb;
            const int sp = cur.sp;                 // descendant row: slot = row - sp_lo
            if (iter > ndesc || (unsigned)sp >= (unsigned)ndesc) { broken = true; break; }
            if (lane == 0) atomicAnd(const_cast<uint32_t *>(sb) + (jb >> 5), ~(1u << (jb & 31)));
            __syncwarp();
            int wp = w0;
            const int jbp = next_step_bit(sb, nsw, wp, lane);
            if (jbp >= 0) read_dstep(d, T, nxt, base + jbp, ndesc, lane);
            const V m = x[sp];
            V xv[DSTEP_PF];
#pragma unroll
            for (int u = 0; u < DSTEP_PF; u++) xv[u] = cur.s[u] >= 0 ? x[cur.s[u]] : V(0);
            __syncwarp();
            if (lane == 0) x[sp] = 0.0;
            if (!isfinite(m)) bad = true;
            if (!overflow && ub + nu + 2 > ue) {
                const int64_t cap = grown_ucap(nu, (int64_t)(c - T.sp_lo) + 1);
                int64_t nb = 0;
                if (lane == 0) nb = pool_alloc(d.pool + 1, d.upool_end, cap);
                nb = __shfl_sync(BK_FULL, nb, 0);
                if (nb < 0) {
                    overflow = true;
                } else {
                    for (int k = lane; k < nu; k += 32) {
                        d.Ui[nb + k] = d.Ui[ub + k];
                        Ux[nb + k] = Ux[ub + k];
                    }
                    __syncwarp();
                    ub = nb;
                    ue = nb + cap;
                    if (lane == 0) {
                        d.Ubeg[c] = ub;
                        d.Uend[c] = ue;
                    }
                }
            }
            if (!overflow && lane == 0) {
                d.Ui[ub + nu] = j;
                Ux[ub + nu] = m;
            }
            nu++;
            // the read-ahead entries, then the rest of L(:,j) eight a lane at a time
#pragma unroll
            for (int u = 0; u < DSTEP_PF; u++) {
                const int s = cur.s[u];
                if (s == -2) continue;
                if (s < 0) { report_internal(d.status, c, 18); continue; }
                x[s] = fma(-cur.l[u], m, xv[u]);
                if (s < ndesc) {
                    if (cur.p[u] > j && cur.p[u] < T.lo) set_bit(sb, cur.p[u] - base);
                    else report_internal(d.status, c, 19);
                } else {
                    set_bit(rb, s - ndesc);
                }
            }
            const int64_t jl = cur.jl;
            const int jc = cur.jc;
            for (int q0 = 32 * DSTEP_PF + lane; q0 < jc; q0 += 32 * DESC_PF) {
                int rr[DESC_PF], ss[DESC_PF], pp[DESC_PF];
                V ll[DESC_PF], xw[DESC_PF];
#pragma unroll
                for (int u = 0; u < DESC_PF; u++) {
                    const int q = q0 + 32 * u;
                    rr[u] = q < jc ? d.Li[jl + q] : -1;
                    ll[u] = q < jc ? Lx[jl + q] : V(0);
                }
#pragma unroll
                for (int u = 0; u < DESC_PF; u++) {
                    ss[u] = rr[u] >= 0 ? slot_of(T, base, rr[u]) : -2;
                    xw[u] = ss[u] >= 0 ? x[ss[u]] : V(0);
                    pp[u] = (ss[u] >= 0 && ss[u] < ndesc) ? d.pinv[rr[u]] : -1;
                }
#pragma unroll
                for (int u = 0; u < DESC_PF; u++) {
                    const int s = ss[u];
                    if (s == -2) continue;
                    if (s < 0) { report_internal(d.status, c, 18); continue; }
                    x[s] = fma(-ll[u], m, xw[u]);
                    if (s < ndesc) {
                        if (pp[u] > j && pp[u] < T.lo) set_bit(sb, pp[u] - base);
                        else report_internal(d.status, c, 19);
                    } else {
                        set_bit(rb, s - ndesc);
                    }
                }
            }
            __syncwarp();
            jb = next_step_bit(sb, nsw, w0, lane);
            if (jb >= 0) {
                if (jb == jbp) cur = nxt;
                else read_dstep(d, T, cur, base + jb, ndesc, lane);
            }
        }
        // A-hat(:,c) on the separator's and ancestors' rows, and its pattern
        V *ah = Ahat + T.ahoff + (int64_t)(c - T.lo) * lsp;
        uint32_t *ab = d.abits + T.aboff + (int64_t)(c - T.lo) * nrw;
        for (int w = lane; w < nrw; w += 32) {
            uint32_t bits = rb[w];
            ab[w] = bits;
            if (bits) rb[w] = 0u;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int ls = (w << 5) + b;
                ah[ls] = x[ndesc + ls];
                x[ndesc + ls] = 0.0;
            }
        }
        __syncwarp();
        if (broken) {
            // an impossible step (a bug, never valid input): report it; this warp's
            // workspace slice is no longer clean, the host clears it on error
            if (lane == 0) report_internal(d.status, c, 20);
            return;
        }
        if (lane == 0) {
            d.dcnt[c] = nu;
            if (overflow) report_overflow(d, T, tid, c, 2);
            else if (bad) report_fail(d.status, c, BK_CODE_NAN);
            BK_TREC(d.trace, BK_TR_DESC, 0, c, t0);
        }
        __syncwarp();
    }
}

}  // namespace

size_t bk_gp_smem_limit() { return 220 * 1024; }

void bk_launch_gather(const bk_dev &d, const double *values, int64_t nnz, void *stream)
{
    if (nnz <= 0) return;
    int blocks = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    if (d.prec)
        bk_gather_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(vals<float>(d.Bx), values, d.bmap, nnz);
    else
        bk_gather_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(d.Bx, values, d.bmap, nnz);
}

void bk_launch_gp_tasks(const bk_dev &d, const int32_t *task_ids, const int32_t *task_c0,
                        int32_t ntasks, size_t smem, double tau, int pref_mode, void *stream)
{
    if (ntasks <= 0) return;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(bk_gp_task_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bk_gp_smem_limit());
        cudaFuncSetAttribute(bk_gp_task_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bk_gp_smem_limit());
    });
    if (d.prec)
        bk_gp_task_kernel<float><<<ntasks, 32, smem, (cudaStream_t)stream>>>(d, task_ids, task_c0, tau, pref_mode);
    else
        bk_gp_task_kernel<double><<<ntasks, 32, smem, (cudaStream_t)stream>>>(d, task_ids, task_c0, tau, pref_mode);
}

void bk_launch_gp_desc(const bk_dev &d, const int32_t *cols, int32_t ncols, int32_t *counter,
                       void *stream, const int32_t *ncols_dev)
{
    if (ncols <= 0) return;
    int warps = std::min<int>(ncols, d.wsd_warps);
    // the level's step and row bitmaps, four warps' worth (d.dd_words is set per
    // ND level, 0 when they do not fit)
    const size_t smem = (size_t)4 * d.dd_words * sizeof(uint32_t);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(bk_gp_desc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(bk_gp_desc_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    if (d.prec)
        bk_gp_desc_kernel<float><<<(warps + 3) / 4, 128, smem, (cudaStream_t)stream>>>(d, cols, ncols, counter,
                                                                                      ncols_dev);
    else
        bk_gp_desc_kernel<double><<<(warps + 3) / 4, 128, smem, (cudaStream_t)stream>>>(d, cols, ncols, counter,
                                                                                       ncols_dev);
}

