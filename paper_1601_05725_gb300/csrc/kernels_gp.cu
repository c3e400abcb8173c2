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
//   bk_reset_pivots_kernel  unmark the rows pivoted by columns that are redone.
//
// Within a column every entry receives its updates one fma at a time in
// ascending pivot-step order (descendant steps, then own steps), and L is
// scaled with an IEEE division, the order the reference definition uses.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "basker_internal.h"
#include "device_util.cuh"

using namespace bk;

namespace {

__global__ void bk_gather_kernel(double *__restrict__ Bx, const double *__restrict__ vals,
                                 const int32_t *__restrict__ bmap, int64_t nnz)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        Bx[e] = __ldg(vals + bmap[e]);
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
__global__ void __launch_bounds__(32) bk_gp_task_kernel(bk_dev d, const int32_t *__restrict__ task_ids,
                                                        const int32_t *__restrict__ task_c0, double tau,
                                                        int pref_mode)
{
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
    double *x;
    volatile uint32_t *sb, *rb;
    if (T.wsoff < 0) {
        x = reinterpret_cast<double *>(dsm);
        uint32_t *s = reinterpret_cast<uint32_t *>(x + lsp);
        for (int i = lane; i < lsp; i += 32) x[i] = 0.0;
        for (int i = lane; i < nsw + nrw; i += 32) s[i] = 0u;
        sb = s;
        rb = s + nsw;
        __syncwarp();
    } else {
        x = reinterpret_cast<double *>(d.ws + T.wsoff);
        sb = reinterpret_cast<uint32_t *>(x + lsp);
        rb = sb + nsw;
    }
    const bool sep = T.sp_lo < T.lo;               // continue a separator column from A-hat
    const int c_begin = task_c0 ? task_c0[blockIdx.x] : T.lo;

    for (int c = c_begin; c < T.hi; ++c) {
        if (__shfl_sync(BK_FULL, (int)should_stop(d, tid, c), 0)) return;
        const int64_t ub = d.Ubeg[c], ue = d.Ubeg[c + 1];
        const int64_t lb = d.Lbeg[c], le = d.Lbeg[c + 1];
        int nu = 0;
        bool bad = false;
        if (sep) {
            // A-hat(:,c) = the column after all descendant steps (Algorithm 4's solves with L_ii and reductions)
            nu = d.dcnt[c];
            const double *ah = d.ahat + T.ahoff + (int64_t)(c - T.lo) * lsp;
            const uint32_t *ab = d.abits + T.aboff + (int64_t)(c - T.lo) * nrw;
            for (int w = lane; w < nrw; w += 32) {
                uint32_t bits = ab[w];
                uint32_t keep = 0u;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int ls = (w << 5) + b;
                    x[ls] = ah[ls];
                    const int p = ls < nown ? d.pinv[base + ls] : -1;
                    if (p >= 0 && (unsigned)(p - base) < (unsigned)nown) set_bit(sb, p - base);
                    else keep |= 1u << b;
                }
                if (keep) atomicOr(const_cast<uint32_t *>(rb) + w, keep);
            }
        } else {
            const int e1 = d.Bp[c + 1];
            for (int e = d.dstart[c] + lane; e < e1; e += 32) {
                const int r = d.Bi[e];
                const int s = slot_of(T, base, r);
                if (s < 0) { report_fail(d.status, c, BK_CODE_INTERNAL); continue; }
                x[s] = d.Bx[e];
                const int p = s < nown ? d.pinv[r] : -1;
                if (p >= 0) {
                    if ((unsigned)(p - base) < (unsigned)nown) set_bit(sb, p - base);
                    else report_fail(d.status, c, BK_CODE_INTERNAL);
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
            const int sp = d.prow[j] - base;      // a pivoted own row: slot = row - lo
            if (iter > nown || j >= c || (unsigned)sp >= (unsigned)nown) {
                if (lane == 0) report_fail(d.status, c, BK_CODE_INTERNAL);
                return;
            }
            const double m = x[sp];
            __syncwarp();
            if (lane == 0) {
                atomicAnd(const_cast<uint32_t *>(sb) + (jb >> 5), ~(1u << (jb & 31)));
                x[sp] = 0.0;
            }
            if (!isfinite(m)) bad = true;
            if (ub + nu + 2 > ue) {
                if (lane == 0) report_overflow(d, T, tid, c, 2);
                return;
            }
            if (lane == 0) {
                d.Ui[ub + nu] = j;
                d.Ux[ub + nu] = m;
            }
            nu++;
            const int64_t jl = d.Lbeg[j];
            const int jc = d.Lcnt[j];
            for (int k = lane; k < jc; k += 32) {
                const int r = d.Li[jl + k];
                const double l = d.Lx[jl + k];
                const int s = slot_of(T, base, r);
                if (s < 0) { report_fail(d.status, c, BK_CODE_INTERNAL); continue; }
                x[s] = fma(-l, m, x[s]);
                const int p = s < nown ? d.pinv[r] : -1;
                if (p >= 0) {
                    if (p > j && p < c) set_bit(sb, p - base);
                    else report_fail(d.status, c, BK_CODE_INTERNAL);
                } else {
                    set_bit(rb, s);
                }
            }
            __syncwarp();
        }

        // Algorithm 1's pivot selection: threshold pivot among the unpivoted own rows
        double amax = 0.0;
        int ncand = 0;
        for (int w = lane; w < nrw; w += 32) {
            uint32_t bits = rb[w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int ls = (w << 5) + b;
                const double v = x[ls];
                if (!isfinite(v)) bad = true;
                if (ls < nown) {
                    ncand++;
                    amax = fmax(amax, fabs(v));
                }
            }
        }
        amax = warp_max(amax);
        ncand = warp_sum(ncand);
        bad = __any_sync(BK_FULL, bad);
        int piv = -1;
        if (!bad && ncand > 0 && amax > 0.0) {
            const int pref = pref_mode ? d.pref[c] : c;
            if (pref >= T.lo && pref < T.hi && d.pinv[pref] < 0 && fabs(x[pref - base]) >= tau * amax) {
                piv = pref;
            } else {
                int best = INT_MAX;
                for (int w = lane; w < nsw; w += 32) {
                    uint32_t bits = rb[w];
                    while (bits) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const int ls = (w << 5) + b;
                        if (ls < nown && fabs(x[ls]) == amax) { best = ls; break; }
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
        const double xp = x[piv - base];
        if (lane == 0) {
            d.Ui[ub + nu] = c;
            d.Ux[ub + nu] = xp;
        }
        nu++;
        int64_t lpos = lb;
        const int pl = piv - base;
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
                d.Lx[q] = x[ls] / xp;
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
            d.Lcnt[c] = (int)(lpos - lb);
            d.Ucnt[c] = nu;
            if (piv != c) atomicAdd(&d.status->offdiag, 1);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Descendant phase of separator columns (one warp per column, persistent).
// Column space: subtree rows [sp_lo, hi) then ancestors (base = sp_lo); the step
// bitmap covers descendant steps [sp_lo, lo) only.
__global__ void __launch_bounds__(128) bk_gp_desc_kernel(bk_dev d, const int32_t *__restrict__ cols,
                                                         int32_t ncols, int32_t *counter)
{
    __shared__ bk_task Ts[4];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * 4 + wib;
    if (gw >= d.wsd_warps) return;
    bk_task &T = Ts[wib];
    unsigned char *slice = d.wsd + (int64_t)gw * d.wsd_slice;
    int cur_task = -1;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(counter, 1);
        k = __shfl_sync(BK_FULL, k, 0);
        if (k >= ncols) break;
        const int c = cols[k];
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
        double *x = reinterpret_cast<double *>(slice);
        volatile uint32_t *sb = reinterpret_cast<uint32_t *>(x + T.space);
        volatile uint32_t *rb = sb + nsw;
        const int64_t ub = d.Ubeg[c], ue = d.Ubeg[c + 1];
        bool bad = false;
        int nu = 0;

        const int e1 = d.Bp[c + 1];
        for (int e = d.dstart[c] + lane; e < e1; e += 32) {
            const int r = d.Bi[e];
            const int s = slot_of(T, base, r);
            if (s < 0) { report_fail(d.status, c, BK_CODE_INTERNAL); continue; }
            x[s] = d.Bx[e];
            if (s < ndesc) {
                const int p = d.pinv[r];            // descendant rows are all pivoted
                if ((unsigned)(p - base) < (unsigned)ndesc) set_bit(sb, p - base);
                else report_fail(d.status, c, BK_CODE_INTERNAL);
            } else {
                set_bit(rb, s - ndesc);
            }
        }
        __syncwarp();
        int w0 = 0;
        bool overflow = false, broken = false;
        for (int iter = 0;; iter++) {
            const int jb = next_step_bit(sb, nsw, w0, lane);
            if (jb < 0) break;
            const int j = base + jb;
            const int sp = d.prow[j] - base;       // descendant row: slot = row - sp_lo
            if (iter > ndesc || (unsigned)sp >= (unsigned)ndesc) { broken = true; break; }
            const double m = x[sp];
            __syncwarp();
            if (lane == 0) {
                atomicAnd(const_cast<uint32_t *>(sb) + (jb >> 5), ~(1u << (jb & 31)));
                x[sp] = 0.0;
            }
            if (!isfinite(m)) bad = true;
            if (ub + nu + 2 > ue) overflow = true;
            if (!overflow && lane == 0) {
                d.Ui[ub + nu] = j;
                d.Ux[ub + nu] = m;
            }
            nu++;
            const int64_t jl = d.Lbeg[j];
            const int jc = d.Lcnt[j];
            for (int q = lane; q < jc; q += 32) {
                const int r = d.Li[jl + q];
                const double l = d.Lx[jl + q];
                const int s = slot_of(T, base, r);
                if (s < 0) { report_fail(d.status, c, BK_CODE_INTERNAL); continue; }
                x[s] = fma(-l, m, x[s]);
                if (s < ndesc) {
                    const int p = d.pinv[r];
                    if (p > j && p < T.lo) set_bit(sb, p - base);
                    else report_fail(d.status, c, BK_CODE_INTERNAL);
                } else {
                    set_bit(rb, s - ndesc);
                }
            }
            __syncwarp();
        }
        // A-hat(:,c) on the separator's and ancestors' rows, and its pattern
        double *ah = d.ahat + T.ahoff + (int64_t)(c - T.lo) * lsp;
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
            if (lane == 0) report_fail(d.status, c, BK_CODE_INTERNAL);
            return;
        }
        if (lane == 0) {
            d.dcnt[c] = nu;
            if (overflow) report_overflow(d, T, tid, c, 2);
            else if (bad) report_fail(d.status, c, BK_CODE_NAN);
        }
        __syncwarp();
    }
}

__global__ void bk_reset_pivots_kernel(bk_dev d, const int32_t *__restrict__ task_ids,
                                       const int32_t *__restrict__ task_c0, int32_t ntasks)
{
    for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
        const bk_task &T = d.tasks[task_ids[t]];
        for (int c = task_c0[t] + threadIdx.x; c < T.hi; c += blockDim.x) {
            const int r = d.prow[c];
            if (r >= 0) d.pinv[r] = -1;
        }
    }
}

}  // namespace

size_t bk_gp_smem_limit() { return 160 * 1024; }

void bk_launch_gather(const bk_dev &d, const double *values, int64_t nnz, void *stream)
{
    if (nnz <= 0) return;
    int blocks = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    bk_gather_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(d.Bx, values, d.bmap, nnz);
}

void bk_launch_gp_tasks(const bk_dev &d, const int32_t *task_ids, const int32_t *task_c0,
                        int32_t ntasks, size_t smem, double tau, int pref_mode, void *stream)
{
    if (ntasks <= 0) return;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(bk_gp_task_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bk_gp_smem_limit());
        attr = true;
    }
    bk_gp_task_kernel<<<ntasks, 32, smem, (cudaStream_t)stream>>>(d, task_ids, task_c0, tau, pref_mode);
}

void bk_launch_gp_desc(const bk_dev &d, const int32_t *cols, int32_t ncols, int32_t *counter,
                       void *stream)
{
    if (ncols <= 0) return;
    int warps = std::min<int>(ncols, d.wsd_warps);
    bk_gp_desc_kernel<<<(warps + 3) / 4, 128, 0, (cudaStream_t)stream>>>(d, cols, ncols, counter);
}

void bk_launch_reset_pivots(const bk_dev &d, const int32_t *task_ids, const int32_t *task_c0,
                            int32_t ntasks, void *stream)
{
    if (ntasks <= 0) return;
    bk_reset_pivots_kernel<<<std::min(ntasks, 1024), 128, 0, (cudaStream_t)stream>>>(d, task_ids, task_c0, ntasks);
}
