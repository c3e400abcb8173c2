// kernels_desc.cu -- the descendant phase of ND separator columns on their
// stored patterns (the refactorization of Sec. V; Algorithm 4's solves with the
// descendants' L and the reductions into A-hat).
//
// Column c of separator j receives the updates of its descendant steps:
// x = B(:,c); for each descendant step k of U(:,c), lowest first: U(k,c) =
// x(prow k), x -= L(:,k) U(k,c).  In a refactorization the descendant steps of
// the previous factorization are the reach again unless a descendant changed
// its pattern or its pivots in a way that reaches this column.  One block per
// column applies the stored steps through the block-wide update of
// column_fast.cuh and verifies them against the pivots now in place:
//   * every descendant row an entry (or B(:,c)) touches is the pivot row of a
//     stored step (so no step is missing from the reach), and
//   * the pivot row of every stored step is touched (so no stored step is
//     outside the reach).
// A verified column is exactly the column the reach would give (same steps in
// the same order, one fma per entry), so A-hat(:,c) and U(desc, c) are written
// as the reach kernel would write them.  A column that fails is cleaned up and
// listed for the reach kernel (bk_gp_desc_kernel), which runs next.
//
// Layout.  Compact (a column with at most xs stored steps and an L-space of at
// most xl rows, xs and xl sized per ND level from the symbolic counts of its
// separator columns): x and a mark byte per entry in shared memory, indexed by
// the position of a step in the stored list for the descendant rows (found
// through an open-addressing table from slot to position, built from the stored
// steps' pivot rows; a descendant row not in the table is not the pivot row of a
// stored step) and after them by the L-space slot.  Otherwise x and a mark byte
// per slot in the block's global workspace slice (x over the column's whole
// space does not fit on chip), with a bitmap over the descendant slots holding
// the stored steps' pivot rows in shared memory, in the memory the compact
// layout uses (a block re-initialises it when it switches between the two).
// The level's sizes keep the block's shared memory small enough for all of a
// level's columns to be resident at once (one wave).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "basker_internal.h"
#include "column_fast.cuh"
#include "device_util.cuh"
#include "trace.cuh"

using namespace bk;

namespace {

constexpr int DF_NT = 128;
constexpr int DF_MAXS = 1 << FC_POS_BITS;   // stored steps of a compact column, at most
constexpr int DF_MAXL = 2048;               // L-space rows of a compact column, at most
// L entries per staging buffer: the larger buffers where the level's columns
// still fit on the SMs at once (bk_desc_par::cap picks the kernel)
constexpr int DF_CAP_SMALL = 512, DF_CAP_LARGE = 1024;

template <typename V, int DF_CAP>
__global__ void __launch_bounds__(DF_NT) bk_desc_fast_kernel(bk_dev d, const int32_t *__restrict__ cols,
                                                             int32_t ncols, int32_t *counter, int32_t *redo,
                                                             int32_t *nredo, bk_desc_par par)
{
    const V *const Bx = vals<V>(d.Bx);
    V *const Ux = vals<V>(d.Ux);
    V *const Ahat = vals<V>(d.ahat);
    // compact: the slot table, x, marks; otherwise the prow(S) bitmap (same memory)
    extern __shared__ __align__(16) uint32_t df_smem[];
    __shared__ bk_task T;
    __shared__ FcSmem<V, DF_CAP> fcs;
    __shared__ int red[DF_NT / 32 + 1];
    __shared__ int ctl[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = par.hmask + 1;
    int32_t *const tab = reinterpret_cast<int32_t *>(df_smem);
    V *const xc = reinterpret_cast<V *>(df_smem + H);
    unsigned char *const mc = reinterpret_cast<unsigned char *>(xc + par.xs + par.xl);
    uint32_t *const prs = df_smem;
    for (int i = tid; i < H; i += DF_NT) tab[i] = -1;
    bool table_ready = true;         // the memory holds an empty table (else a zero bitmap)
    int cur_task = -1;
    for (;;) {
        if (tid == 0) ctl[0] = atomicAdd(counter, 1);
        __syncthreads();
        const int k = ctl[0];
        if (k >= ncols) break;
        const int c = cols[k];
        const int task = d.col_task[c];
        if (task != cur_task) {
            if (warp == 0) load_task(T, d.tasks + task, lane);
            cur_task = task;
        }
        __syncthreads();
        BK_TSTART(t0);
        if (__syncthreads_or(tid == 0 && should_stop(d, task, c))) continue;
        const int base = T.sp_lo;
        const int ndesc = T.lo - T.sp_lo;
        const int lsp = T.lspace;
        const int nrw = (lsp + 31) >> 5;
        V *const x = reinterpret_cast<V *>(d.wsd + (int64_t)blockIdx.x * d.wsd_slice);
        unsigned char *const mark = reinterpret_cast<unsigned char *>(x + T.space);
        const int64_t ub = d.Ubeg[c];
        const int ns = d.dcnt[c];
        const int e1 = d.Bp[c + 1];
        if (ns >= 0 && ns <= par.xs && ns <= d.Ucnt[c] - 1 && lsp <= par.xl && ndesc < (1 << (31 - FC_POS_BITS))) {
            // ---- compact: x on chip
            if (!table_ready) {
                __syncthreads();
                for (int i = tid; i < H; i += DF_NT) tab[i] = -1;
                table_ready = true;
                __syncthreads();
            }
            bool ok = true, broken = false;
            for (int q = tid; q < ns; q += DF_NT) {
                const int j = __ldcg(d.Ui + ub + q);
                const int sl = __ldcg(d.prow + j) - base;     // a descendant row's slot
                if (j < base || j >= T.lo || (unsigned)sl >= (unsigned)ndesc) { ok = false; continue; }
                int h = fc_hash(sl, par.hmask);
                for (int probe = 0; probe < H; probe++) {
                    const int old = atomicCAS(tab + h, -1, (sl << FC_POS_BITS) | q);
                    if (old == -1) break;
                    if ((old >> FC_POS_BITS) == sl) {      // two stored steps, one pivot row
                        ok = false;
                        break;
                    }
                    h = (h + 1) & par.hmask;
                }
            }
            for (int i = tid; i < ns + lsp; i += DF_NT) {
                xc[i] = V(0);
                mc[i] = 0;
            }
            ok = __syncthreads_and(ok);
            const FcMap map{tab, par.hmask, ns - ndesc};
            if (ok) {
                for (int e = d.dstart[c] + tid; e < e1; e += DF_NT) {
                    const int sl = slot_of(T, base, d.Bi[e]);
                    if (sl < 0) { broken = true; continue; }
                    const int ix = sl < ndesc ? map.find(sl) : ns + (sl - ndesc);
                    if (ix < 0) { ok = false; continue; }
                    xc[ix] = Bx[e];
                    mc[ix] = 1;
                }
                ok = __syncthreads_and(ok);
            }
            bool bad = false, vfail = false;
            if (ok && !__syncthreads_or(broken)) {
                if (!column_fast_update_cta<V, true, DF_NT, DF_CAP>(d, T, base, d.Ui + ub, ns, Ux + ub, xc, fcs, mc,
                                                                    red, tid, bad, nullptr, ndesc, &vfail, &map))
                    broken = true;
                ok = !__syncthreads_or(vfail);
                if (ok)
                    for (int q = tid; q < ns; q += DF_NT)
                        if (!mc[q]) ok = false;                  // a stored step outside the reach
                ok = __syncthreads_and(ok);
            }
            broken = __syncthreads_or(broken);
            if (ok && !broken) {
                V *const ah = Ahat + T.ahoff + (int64_t)(c - T.lo) * lsp;
                uint32_t *const ab = d.abits + T.aboff + (int64_t)(c - T.lo) * nrw;
                for (int w = tid; w < nrw; w += DF_NT) {
                    uint32_t bits = 0u;
                    for (int b = 0; b < 32; b++) {
                        const int ls = 32 * w + b;
                        if (ls >= lsp) break;
                        if (mc[ns + ls]) {
                            bits |= 1u << b;
                            ah[ls] = xc[ns + ls];
                        }
                    }
                    ab[w] = bits;
                }
                bad = __syncthreads_or(bad);
                if (tid == 0 && bad) report_fail(d.status, c, BK_CODE_NAN);
            } else if (tid == 0) {
                redo[atomicAdd(nredo, 1)] = c;
            }
            // the table back to empty
            __syncthreads();
            for (int i = tid; i < H; i += DF_NT) tab[i] = -1;
            __syncthreads();
            if (tid == 0) BK_TREC(d.trace, BK_TR_DESC, (ok && !broken) ? 3 : 4, c, t0);
            continue;
        }
        if (table_ready) {
            // the bitmap over the descendant slots starts empty
            __syncthreads();
            for (int i = tid; i < par.prs_words; i += DF_NT) prs[i] = 0u;
            table_ready = false;
            __syncthreads();
        }
        bool ok = ns >= 0 && ns <= d.Ucnt[c] - 1;
        // the stored steps must be descendants; their pivot rows form prs
        if (ok)
            for (int q = tid; q < ns; q += DF_NT) {
                const int j = __ldcg(d.Ui + ub + q);
                const int s = __ldcg(d.prow + j) - base;    // a descendant row's slot
                if (j < base || j >= T.lo || (unsigned)s >= (unsigned)ndesc) ok = false;
                else atomicOr(prs + (s >> 5), 1u << (s & 31));
            }
        ok = __syncthreads_and(ok);
        bool broken = false;
        if (ok) {
            for (int e = d.dstart[c] + tid; e < e1; e += DF_NT) {
                const int s = slot_of(T, base, d.Bi[e]);
                if (s < 0) { broken = true; continue; }
                if (s < ndesc && !((prs[s >> 5] >> (s & 31)) & 1u)) ok = false;
                x[s] = Bx[e];
                mark[s] = 1;
            }
            ok = __syncthreads_and(ok);
        }
        bool bad = false, vfail = false;
        if (ok && !__syncthreads_or(broken)) {
            if (!column_fast_update_cta<V, true, DF_NT, DF_CAP>(d, T, base, d.Ui + ub, ns, Ux + ub, x, fcs, mark, red,
                                                                tid, bad, prs, ndesc, &vfail))
                broken = true;
            ok = !__syncthreads_or(vfail);
            // every stored step's pivot row was touched
            if (ok)
                for (int q = tid; q < ns; q += DF_NT) {
                    const int s = __ldcg(d.prow + __ldcg(d.Ui + ub + q)) - base;
                    if (!mark[s]) ok = false;
                }
            ok = __syncthreads_and(ok);
        }
        broken = __syncthreads_or(broken);
        if (ok && !broken) {
            // A-hat(:,c) over the L-space slots and its pattern; the descendant
            // slots (the stored steps' pivot rows) cleared
            V *const ah = Ahat + T.ahoff + (int64_t)(c - T.lo) * lsp;
            uint32_t *const ab = d.abits + T.aboff + (int64_t)(c - T.lo) * nrw;
            for (int w = tid; w < nrw; w += DF_NT) {
                uint32_t bits = 0u;
                for (int b = 0; b < 32; b++) {
                    const int ls = 32 * w + b;
                    if (ls >= lsp) break;
                    if (mark[ndesc + ls]) {
                        bits |= 1u << b;
                        ah[ls] = x[ndesc + ls];
                        x[ndesc + ls] = V(0);
                        mark[ndesc + ls] = 0;
                    }
                }
                ab[w] = bits;
            }
            for (int q = tid; q < ns; q += DF_NT) {
                const int s = __ldcg(d.prow + __ldcg(d.Ui + ub + q)) - base;
                x[s] = V(0);
                mark[s] = 0;
            }
            bad = __syncthreads_or(bad);
            if (tid == 0 && bad) report_fail(d.status, c, BK_CODE_NAN);
        } else {
            // not the reach (or an index outside the space): clean the slice over
            // everything touched, and leave the column to the reach kernel
            for (int e = d.dstart[c] + tid; e < e1; e += DF_NT) {
                const int s = slot_of(T, base, d.Bi[e]);
                if (s >= 0) {
                    x[s] = V(0);
                    mark[s] = 0;
                }
            }
            if (ns > 0 && ns <= d.Ucnt[c] - 1)
                for (int q = warp; q < ns; q += DF_NT / 32) {
                    const int j = __ldcg(d.Ui + ub + q);
                    if ((unsigned)j >= (unsigned)d.n) continue;
                    const int sp = slot_of(T, base, __ldcg(d.prow + j));
                    if (sp >= 0 && lane == 0) {
                        x[sp] = V(0);
                        mark[sp] = 0;
                    }
                    const int64_t jl = __ldcg(d.Lbeg + j);
                    const int jc = __ldcg(d.Lcnt + j);
                    for (int e = lane; e < jc; e += 32) {
                        const int s = slot_of(T, base, __ldcg(d.Li + jl + e));
                        if (s >= 0) {
                            x[s] = V(0);
                            mark[s] = 0;
                        }
                    }
                }
            if (tid == 0) redo[atomicAdd(nredo, 1)] = c;
        }
        // clear the pivot-row bitmap
        if (ns > 0 && ns <= d.Ucnt[c] - 1)
            for (int q = tid; q < ns; q += DF_NT) {
                const int s = __ldcg(d.prow + __ldcg(d.Ui + ub + q)) - base;
                if ((unsigned)s < (unsigned)ndesc) prs[s >> 5] = 0u;
            }
        __syncthreads();
        if (tid == 0) BK_TREC(d.trace, BK_TR_DESC, (ok && !broken) ? 1 : 2, c, t0);
    }
}

}  // namespace

// The compact layout's sizes for the separator columns of ND level `level`: xs
// stored steps (1.5x the largest symbolic U count of the level's columns, as
// pivoting moves patterns), a table of at least 1.5 xs entries, xl the largest
// L-space; the shared memory is the larger of that layout and the bitmap over
// the largest descendant space.  smem 0: the level's descendant phase cannot
// keep the bitmap on chip (every column goes to the reach kernel).
bk_desc_par bk_desc_fast_params(const bk_plan &pl, int32_t level)
{
    bk_desc_par p{};
    int64_t umax = 0, xl = 0, words = 4;
    for (const bk_task &T : pl.tasks) {
        if (T.level != level || T.sp_lo >= T.lo) continue;
        for (int32_t c = T.lo; c < T.hi; c++)
            umax = std::max<int64_t>(umax, c < (int32_t)pl.sUcnt.size() ? pl.sUcnt[(size_t)c] : (int64_t)(c - T.sp_lo + 1));
        xl = std::max<int64_t>(xl, T.lspace);
        words = std::max<int64_t>(words, ((int64_t)(T.lo - T.sp_lo) + 31) / 32);
    }
    int64_t xs = std::min<int64_t>(DF_MAXS, ((umax * 3 / 2) + 63) & ~(int64_t)31);
    if (xl > DF_MAXL) xs = xl = 0;                 // no column of the level fits on chip
    int64_t H = 256;
    while (H < xs + xs / 2) H *= 2;
    const size_t compact = (((size_t)H * 4 + (size_t)(xs + xl) * (sizeof(double) + 1)) + 15) & ~(size_t)15;
    const size_t bitmap = (((size_t)words + 3) & ~(size_t)3) * 4;
    p.hmask = (int32_t)H - 1;
    p.xs = (int32_t)xs;
    p.xl = (int32_t)xl;
    p.prs_words = (int32_t)(((size_t)words + 3) & ~(size_t)3);
    const size_t bytes = std::max(compact, bitmap);
    p.smem = bytes <= 160 * 1024 ? bytes : 0;
    // the larger staging buffers when the blocks the level's columns need on each
    // SM still fit its shared memory with them (static part: the buffers, 24 bytes
    // an entry, plus about 5 KB; 1 KB reserved a block)
    int64_t ncols = 0;
    for (const bk_task &T : pl.tasks)
        if (T.level == level && T.sp_lo < T.lo) ncols += T.hi - T.lo;
    const int64_t per_sm = std::max<int64_t>(1, (ncols + 151) / 152);
    const size_t big = p.smem + (size_t)DF_CAP_LARGE * 24 + 6 * 1024 + 1024;
    p.cap = (size_t)per_sm * big <= 228 * 1024 ? DF_CAP_LARGE : DF_CAP_SMALL;
    return p;
}

void bk_launch_desc_fast(const bk_dev &d, const int32_t *cols, int32_t ncols, int32_t *counter, int32_t *redo,
                         int32_t *nredo, const bk_desc_par &par, void *stream)
{
    if (ncols <= 0) return;
    static std::once_flag once;
    std::call_once(once, [] {
        const int lim = 160 * 1024;
        cudaFuncSetAttribute(bk_desc_fast_kernel<double, DF_CAP_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(bk_desc_fast_kernel<float, DF_CAP_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(bk_desc_fast_kernel<double, DF_CAP_LARGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        cudaFuncSetAttribute(bk_desc_fast_kernel<float, DF_CAP_LARGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    });
    // every column of the level resident at once where the shared memory allows
    const int grid = std::max(1, std::min<int>({ncols, d.wsd_warps, 152 * 8}));
    cudaStream_t s = (cudaStream_t)stream;
    const bool large = par.cap >= DF_CAP_LARGE;
    if (d.prec) {
        if (large)
            bk_desc_fast_kernel<float, DF_CAP_LARGE><<<grid, DF_NT, par.smem, s>>>(d, cols, ncols, counter, redo, nredo, par);
        else
            bk_desc_fast_kernel<float, DF_CAP_SMALL><<<grid, DF_NT, par.smem, s>>>(d, cols, ncols, counter, redo, nredo, par);
    } else {
        if (large)
            bk_desc_fast_kernel<double, DF_CAP_LARGE><<<grid, DF_NT, par.smem, s>>>(d, cols, ncols, counter, redo, nredo, par);
        else
            bk_desc_fast_kernel<double, DF_CAP_SMALL><<<grid, DF_NT, par.smem, s>>>(d, cols, ncols, counter, redo, nredo, par);
    }
}
