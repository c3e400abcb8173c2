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

__device__ void forward_sweep(const bk_dev &d, const bk_solve_dev &s, const bk_task &T, int q,
                              double *acc, int lane)
{
    double *w = s.w + (int64_t)q * d.n;
    for (int k = T.lo; k < T.hi; k++) {
        const double wk = __ldcg(w + k);
        const int64_t lb = d.Lbeg[k];
        const int lc = d.Lcnt[k];
        for (int t = lane; t < lc; t += 32) {
            const int i = d.pinv[d.Li[lb + t]];
            const double l = d.Lx[lb + t];
            if (i > k && i < T.hi) {
                w[i] = fma(-l, wk, __ldcg(w + i));
            } else {
                const int a = acc ? anc_slot(T, i) : -1;
                if (a >= 0) acc[a] = fma(l, wk, acc[a]);
                else report_internal(d.status, k, 51);
            }
        }
        __syncwarp();
    }
}

__device__ void backward_sweep(const bk_dev &d, const bk_solve_dev &s, const bk_task &T, int q,
                               double *x, int ldx, int lane)
{
    double *w = s.w + (int64_t)q * d.n;
    for (int k = T.hi - 1; k >= T.lo; k--) {
        const int64_t ub = d.Ubeg[k];
        const int uc = d.Ucnt[k];
        const double zk = __ldcg(w + k) / d.Ux[ub + uc - 1];
        for (int t = lane; t < uc - 1; t += 32) {
            const int i = d.Ui[ub + t];
            w[i] = fma(-d.Ux[ub + t], zk, __ldcg(w + i));
        }
        __syncwarp();
        if (lane == 0) w[k] = zk;
        __syncwarp();
    }
    for (int k = T.lo + lane; k < T.hi; k += 32) x[(int64_t)q * ldx + d.Q[k]] = __ldcg(w + k);
}

__global__ void __launch_bounds__(128) bk_solve_kernel(bk_dev d, bk_solve_dev s, int32_t nrhs,
                                                       const double *__restrict__ b, int32_t ldb,
                                                       double *x, int32_t ldx, int32_t epoch,
                                                       long long budget)
{
    __shared__ bk_task Ts[4];
    __shared__ bk_task Us[4];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    bk_task &T = Ts[wib];
    bk_task &U = Us[wib];
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(d.counter + 2, 1);
        k = __shfl_sync(BK_FULL, k, 0);
        if (k >= s.nitems) break;
        const bk_sitem it = s.items[k];
        if (!wait_items(d, s, it, epoch, budget, lane)) return;
        load_task(T, d.tasks + it.task, lane);
        for (int q = 0; q < nrhs; q++) {
            double *w = s.w + (int64_t)q * d.n;
            if (it.type == BK_ITEM_BLOCK || it.type == BK_ITEM_FWD) {
                for (int kk = T.lo + lane; kk < T.hi; kk += 32) {
                    double v = init_row(d, s, kk, q, b, ldb);
                    w[kk] = v;
                }
                double *acc = nullptr;
                if (it.type == BK_ITEM_FWD) {
                    acc = s.acc + (int64_t)q * s.acc_stride + s.acc_off[it.task];
                    const int na = T.lspace - (T.hi - T.lo);
                    for (int a = lane; a < na; a += 32) acc[a] = 0.0;
                    __syncwarp();
                    // contributions of every descendant (fixed order: postorder)
                    for (int u = it.desc_beg; u < it.desc_end; u++) {
                        const int ut = s.desc[u];
                        load_task(U, d.tasks + ut, lane);
                        const double *au = s.acc + (int64_t)q * s.acc_stride + s.acc_off[ut];
                        for (int kk = T.lo + lane; kk < T.hi; kk += 32) {
                            const int a = anc_slot(U, kk);
                            if (a >= 0) w[kk] -= __ldcg(au + a);
                        }
                        __syncwarp();
                    }
                }
                __syncwarp();
                forward_sweep(d, s, T, q, acc, lane);
                if (it.type == BK_ITEM_BLOCK) backward_sweep(d, s, T, q, x, ldx, lane);
            } else {
                backward_sweep(d, s, T, q, x, ldx, lane);
            }
            __syncwarp();
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(s.item_done + k, epoch);
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
    int warps = std::min<int>(s.nitems, std::max(1, sms) * 8);
    bk_solve_kernel<<<(warps + 3) / 4, 128, 0, (cudaStream_t)stream>>>(d, s, nrhs, b, ldb, x, ldx, epoch,
                                                                        budget);
}
