// kernels_solve.cu -- x = A^{-1} b with the factors of the BTF diagonal blocks.
//
// BTF back-substitution (Sec. II and III-B: only the diagonal blocks are factored;
// the off-diagonal blocks keep A's values and enter through a product): blocks
// from last to first, c_d -= sum_{e>d} B_de z_e, then L_d w = P_d c_d and
// U_d z_d = w.  The work is a list of items claimed by warps in a topological
// order, each item waiting for the items it needs through flags (point-to-point
// synchronisation, Sec. IV) with a bounded wait:
//   BLOCK d        a BTF block without ND: coupling rows, forward, backward
//   FWD t          ND node t: its rows' coupling terms and the contributions its
//                  descendants left for it, then the forward sweep over its own
//                  columns; contributions to ancestor rows go to the node's own
//                  buffer (read later by the ancestors, in a fixed order)
//   BWD t          ND node t, after its ancestors: backward sweep over its columns,
//                  which updates its own and its descendants' rows
// Values written by other warps are read through L2 (ld.cg).
#include <cuda_runtime.h>

#include <algorithm>

#include "basker_internal.h"
#include "device_util.cuh"
#include "solve_internal.h"

using namespace bk;

namespace {

__device__ __forceinline__ bool wait_items(const bk_dev &d, const bk_solve_dev &s, const bk_sitem &it,
                                           int epoch, long long budget, int lane)
{
    int ok = 1;
    for (int q = it.dep_beg + lane; q < it.dep_end; q += 32) {
        const int *flag = s.item_done + s.deps[q];
        if (ld_acquire(flag) != epoch) {
            const long long t0 = clock64();
            while (ld_acquire(flag) != epoch) {
                if (*reinterpret_cast<const volatile int *>(&d.status->timeout) || clock64() - t0 > budget) {
                    atomicExch(&d.status->timeout, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (!ok) break;
    }
    return !__any_sync(BK_FULL, !ok);
}

// Slot of step i among the ancestor rows of task u (its contribution buffer).
__device__ __forceinline__ int anc_slot(const bk_task &U, int i)
{
    int off = 0;
    for (int a = 0; a < U.nanc; a++) {
        if (i >= U.anc_lo[a] && i < U.anc_hi[a]) return off + (i - U.anc_lo[a]);
        off += U.anc_hi[a] - U.anc_lo[a];
    }
    return -1;
}

// w(k) = b(P(prow k)) - sum of coupling terms of row prow(k) (columns of later blocks)
__device__ __forceinline__ double init_row(const bk_dev &d, const bk_solve_dev &s, int k, int q,
                                           const double *b, int ldb)
{
    const int r = d.prow[k];
    double v = b[(int64_t)q * ldb + d.P[r]];
    for (int e = s.offp[r]; e < s.offp[r + 1]; e++)
        v = fma(-d.Bx[s.offpos[e]], __ldcg(s.w + (int64_t)q * d.n + s.offj[e]), v);
    return v;
}

// Forward sweep over the node's own columns: wl holds the node's own rows (in
// shared memory when they fit), acc its ancestors' rows.  The first 32 entries
// of the next column are loaded while the current one is applied.
__device__ void forward_sweep(const bk_dev &d, const bk_solve_dev &s, const bk_task &T, double *wl,
                              double *acc, int lane)
{
    const int lo = T.lo, hi = T.hi;
    int64_t nb = d.Lbeg[lo];
    int nc = d.Lcnt[lo];
    int ni = lane < nc ? s.Ls[nb + lane] : -1;
    double nv = lane < nc ? d.Lx[nb + lane] : 0.0;
    for (int k = lo; k < hi; k++) {
        const int64_t lb = nb;
        const int lc = nc;
        const int ci = ni;
        const double cv = nv;
        if (k + 1 < hi) {
            nb = d.Lbeg[k + 1];
            nc = d.Lcnt[k + 1];
            ni = lane < nc ? s.Ls[nb + lane] : -1;
            nv = lane < nc ? d.Lx[nb + lane] : 0.0;
        }
        const double wk = wl[k - lo];
        auto apply = [&](int i, double l) {
            if (i > k && i < hi) {
                wl[i - lo] = fma(-l, wk, wl[i - lo]);
            } else {
                const int a = acc ? anc_slot(T, i) : -1;
                if (a >= 0) acc[a] = fma(l, wk, acc[a]);
                else report_internal(d.status, k, 51);
            }
        };
        if (lane < lc) apply(ci, cv);
        for (int t = 32 + lane; t < lc; t += 32) apply(s.Ls[lb + t], d.Lx[lb + t]);
        __syncwarp();
    }
}

// Backward sweep: z_k = w_k / U(k,k), then w -= U(:,k) z_k; own rows in wl, the
// descendants' rows (separators only) in global memory.
__device__ void backward_sweep(const bk_dev &d, const bk_solve_dev &s, const bk_task &T, double *wl,
                               double *wg, int lane)
{
    const int lo = T.lo, hi = T.hi;
    int64_t nb = d.Ubeg[hi - 1];
    int nc = d.Ucnt[hi - 1];
    int ni = lane < nc ? d.Ui[nb + lane] : -1;
    double nv = lane < nc ? d.Ux[nb + lane] : 0.0;
    for (int k = hi - 1; k >= lo; k--) {
        const int64_t ub = nb;
        const int uc = nc;
        const int ci = ni;
        const double cv = nv;
        if (k > lo) {
            nb = d.Ubeg[k - 1];
            nc = d.Ucnt[k - 1];
            ni = lane < nc ? d.Ui[nb + lane] : -1;
            nv = lane < nc ? d.Ux[nb + lane] : 0.0;
        }
        const double zk = wl[k - lo] / d.Ux[ub + uc - 1];
        auto apply = [&](int i, double u) {
            if (i >= lo) wl[i - lo] = fma(-u, zk, wl[i - lo]);
            else wg[i] = fma(-u, zk, __ldcg(wg + i));
        };
        if (lane < uc - 1) apply(ci, cv);
        for (int t = 32 + lane; t < uc - 1; t += 32) apply(d.Ui[ub + t], d.Ux[ub + t]);
        __syncwarp();
        if (lane == 0) wl[k - lo] = zk;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32) bk_solve_kernel(bk_dev d, bk_solve_dev s, int32_t nrhs,
                                                      const double *__restrict__ b, int32_t ldb,
                                                      double *x, int32_t ldx, int32_t epoch,
                                                      long long budget)
{
    extern __shared__ __align__(16) double sw[];
    __shared__ bk_task T;
    __shared__ bk_task U;
    const int lane = threadIdx.x;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(d.counter + 2, 1);
        k = __shfl_sync(BK_FULL, k, 0);
        if (k >= s.nitems) break;
        const bk_sitem it = s.items[k];
        if (!wait_items(d, s, it, epoch, budget, lane)) return;
        load_task(T, d.tasks + it.task, lane);
        const int nown = T.hi - T.lo;
        const int na = it.type == BK_ITEM_BLOCK ? 0 : T.lspace - nown;
        const bool fits = (int64_t)(nown + na) * 8 <= s.smem_bytes;
        for (int q = 0; q < nrhs; q++) {
            double *w = s.w + (int64_t)q * d.n;
            double *wl = fits ? sw : w + T.lo;
            double *accg = s.acc + (int64_t)q * s.acc_stride + s.acc_off[it.task];
            double *acc = it.type == BK_ITEM_FWD ? (fits ? sw + nown : accg) : nullptr;
            if (it.type == BK_ITEM_BLOCK || it.type == BK_ITEM_FWD) {
                for (int kk = T.lo + lane; kk < T.hi; kk += 32) wl[kk - T.lo] = init_row(d, s, kk, q, b, ldb);
                if (acc)
                    for (int a = lane; a < na; a += 32) acc[a] = 0.0;
                __syncwarp();
                if (it.type == BK_ITEM_FWD) {
                    // contributions of every descendant (fixed order: postorder)
                    for (int u = it.desc_beg; u < it.desc_end; u++) {
                        const int ut = s.desc[u];
                        load_task(U, d.tasks + ut, lane);
                        const double *au = s.acc + (int64_t)q * s.acc_stride + s.acc_off[ut];
                        for (int kk = T.lo + lane; kk < T.hi; kk += 32) {
                            const int a = anc_slot(U, kk);
                            if (a >= 0) wl[kk - T.lo] -= __ldcg(au + a);
                        }
                        __syncwarp();
                    }
                }
                forward_sweep(d, s, T, wl, acc, lane);
                if (it.type == BK_ITEM_BLOCK) backward_sweep(d, s, T, wl, w, lane);
                if (fits && acc)
                    for (int a = lane; a < na; a += 32) accg[a] = acc[a];
            } else {
                // own rows were written by other warps: read them through L2 (and
                // rewrite them in place when they stay in global memory)
                for (int kk = T.lo + lane; kk < T.hi; kk += 32) wl[kk - T.lo] = __ldcg(w + kk);
                __syncwarp();
                backward_sweep(d, s, T, wl, w, lane);
            }
            __syncwarp();
            if (fits)
                for (int kk = T.lo + lane; kk < T.hi; kk += 32) w[kk] = wl[kk - T.lo];
            if (it.type != BK_ITEM_FWD)
                for (int kk = T.lo + lane; kk < T.hi; kk += 32) x[(int64_t)q * ldx + d.Q[kk]] = wl[kk - T.lo];
            __syncwarp();
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(s.item_done + k, epoch);
    }
}

// L's row indices as pivot steps (for the solve), after every factorization.
__global__ void bk_lsteps_kernel(bk_dev d, int *Ls)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < d.n; c += nwarps) {
        const int64_t lb = d.Lbeg[c];
        const int lc = d.Lcnt[c];
        for (int t = lane; t < lc; t += 32) Ls[lb + t] = d.pinv[d.Li[lb + t]];
    }
}

}  // namespace

void bk_launch_solve(const bk_dev &d, const bk_solve_dev &s, int32_t nrhs, const double *b, int32_t ldb,
                     double *x, int32_t ldx, int32_t epoch, long long budget, void *stream)
{
    if (s.nitems <= 0) return;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    static int attr_set = -1;
    if (attr_set != (int)s.smem_bytes) {
        cudaFuncSetAttribute(bk_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem_bytes);
        attr_set = (int)s.smem_bytes;
    }
    const int per_sm = s.smem_bytes > 0 ? std::max<int>(1, std::min<int>(16, (int)(200 * 1024 / s.smem_bytes))) : 16;
    const int ctas = std::min<int>(s.nitems, std::max(1, sms) * per_sm);
    bk_solve_kernel<<<ctas, 32, (size_t)s.smem_bytes, (cudaStream_t)stream>>>(d, s, nrhs, b, ldb, x, ldx, epoch,
                                                                               budget);
}

void bk_launch_lsteps(const bk_dev &d, int *Ls, void *stream)
{
    if (d.n <= 0) return;
    const int blocks = std::max(1, std::min((d.n + 7) / 8, 152 * 8));
    bk_lsteps_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(d, Ls);
}
