// kernels_solve.cu -- x = A^{-1} b with the factors of the BTF diagonal blocks.
//
// BTF back-substitution (Sec. II and III-B: only the diagonal blocks are
// factored; the off-diagonal blocks keep A's values and enter through a
// product): blocks from last to first, c_d -= sum_{e>d} B_de z_e, then
// L_d w = P_d c_d and U_d z_d = w.  Evaluated by rows in pivot-step space, one
// warp per row and direction, claimed in a topological order:
//   forward row i   w_i = c(prow i) - sum_k L(i,k) w_k, k ascending, after the
//                   coupling terms of row prow i (later blocks' final z_j)
//   backward row i  z_i = (w_i - sum_k U(i,k) z_k) / U(i,i), k descending
// Each term waits for the flag of the row it reads (point-to-point
// synchronisation, Sec. IV) with a bounded wait.  Per solution entry the fma
// sequence is the one of the column sweeps (ascending steps for L, descending for
// U), so the result does not depend on the schedule.
//
// The factors are kept by columns; after every factorization bk_launch_rows
// transposes them into rows (count, scan, scatter, and a rank sort per row).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "basker_internal.h"
#include "device_util.cuh"
#include "solve_internal.h"

using namespace bk;

namespace {

// ---------------------------------------------------------------- factors by rows

template <typename V>
__global__ void bk_rows_count(bk_dev d, bk_rows r)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int32_t *lc = r.cnt, *uc = r.cnt + d.n + 1;
    for (int c = warp; c < d.n; c += nwarps) {
        const int64_t lb = d.Lbeg[c];
        const int ln = d.Lcnt[c];
        for (int t = lane; t < ln; t += 32) atomicAdd(lc + d.pinv[d.Li[lb + t]], 1);
        const int64_t ub = d.Ubeg[c];
        const int un = d.Ucnt[c];
        for (int t = lane; t < un - 1; t += 32) atomicAdd(uc + d.Ui[ub + t], 1);
        if (lane == 0) vals<V>(r.Ud)[c] = vals<V>(d.Ux)[ub + un - 1];
    }
}

// Exclusive scan of m counts into m + 1 starts: per-block sums, a scan of the
// block sums, then each block's scan plus its offset.
__device__ __forceinline__ int64_t block_exscan(int64_t v, int64_t *warp_tot, int64_t &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(BK_FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(BK_FULL, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[lane] = ti - t;
        if (lane == 31) warp_tot[32] = ti;
    }
    __syncthreads();
    const int64_t ex = inc - v + warp_tot[wid];
    total = warp_tot[32];
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(1024) bk_scan_sums(const int32_t *cnt, int32_t m, int64_t *part)
{
    __shared__ int64_t wt[33];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    int64_t total;
    block_exscan(i < m ? cnt[i] : 0, wt, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) bk_scan_parts(int64_t *part, int32_t nb)
{
    __shared__ int64_t wt[33];
    int64_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const int64_t v = i < nb ? part[i] : 0;
        int64_t total;
        const int64_t ex = block_exscan(v, wt, total);
        if (i < nb) part[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

__global__ void __launch_bounds__(1024) bk_scan_apply(const int32_t *cnt, int32_t m, const int64_t *part,
                                                      int64_t *out)
{
    __shared__ int64_t wt[33];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    int64_t total;
    const int64_t ex = block_exscan(i < m ? cnt[i] : 0, wt, total);
    if (i < m) out[i] = part[blockIdx.x] + ex;
    if (i == 0) out[m] = part[gridDim.x];
}

// Entries of L (which = 0) or U (which = 1) into the unsorted row buffer.
template <typename V>
__global__ void bk_rows_scatter(bk_dev d, bk_rows r, int which)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int32_t *cur = r.cnt + (which ? d.n + 1 : 0);
    const int64_t *rp = which ? r.Urp : r.Lrp;
    for (int c = warp; c < d.n; c += nwarps) {
        if (which == 0) {
            const int64_t lb = d.Lbeg[c];
            const int ln = d.Lcnt[c];
            for (int t = lane; t < ln; t += 32) {
                const int i = d.pinv[d.Li[lb + t]];
                const int64_t pos = rp[i] + atomicAdd(cur + i, 1);
                r.tk[pos] = c;
                vals<V>(r.tx)[pos] = vals<V>(d.Lx)[lb + t];
            }
        } else {
            const int64_t ub = d.Ubeg[c];
            const int un = d.Ucnt[c];
            for (int t = lane; t < un - 1; t += 32) {
                const int i = d.Ui[ub + t];
                const int64_t pos = rp[i] + atomicAdd(cur + i, 1);
                r.tk[pos] = c;
                vals<V>(r.tx)[pos] = vals<V>(d.Ux)[ub + t];
            }
        }
    }
}

// Each row's entries in ascending (L) or descending (U) column order: the rank of
// an entry is the number of entries of its row that come before it.
template <typename V>
__global__ void bk_rows_sort(int32_t n, const int64_t *rp, const int32_t *tk, const V *tx, int32_t *ok, V *ox,
                             int desc)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int sentinel = desc ? INT_MIN : INT_MAX;
    for (int i = warp; i < n; i += nwarps) {
        const int64_t p0 = rp[i];
        const int len = (int)(rp[i + 1] - p0);
        for (int e0 = 0; e0 < len; e0 += 32) {
            const bool mine = e0 + lane < len;
            const int myk = mine ? tk[p0 + e0 + lane] : sentinel;
            const V myx = mine ? tx[p0 + e0 + lane] : V(0);
            int rank = 0;
            for (int f0 = 0; f0 < len; f0 += 32) {
                const int other = f0 + lane < len ? tk[p0 + f0 + lane] : sentinel;
#pragma unroll 8
                for (int t = 0; t < 32; t++) {
                    const int kk = __shfl_sync(BK_FULL, other, t);
                    rank += desc ? (kk > myk) : (kk < myk);
                }
            }
            if (mine) {
                ok[p0 + rank] = myk;
                ox[p0 + rank] = myx;
            }
        }
    }
}

// ---------------------------------------------------------------- the solve

// Bounded wait until flags[j] == epoch for every lane with want.  Each lane
// checks its flag once; lane 0 alone then polls the flags still unset, in lane
// order (one poller per warp, and no rereads of the other flags meanwhile), and
// finally each of those lanes rereads its own flag with an acquiring load, which
// orders its later reads.  False if a wait ran out (the timeout status is then
// set).
__device__ __forceinline__ bool lane0_poll(const bk_dev &d, const int32_t *flag, int epoch, long long budget)
{
    const long long t0 = clock64();
    unsigned ns = 32;
    while (ld_acquire(flag) != epoch) {
        if (*reinterpret_cast<const volatile int *>(&d.status->timeout) || clock64() - t0 > budget) {
            atomicExch(&d.status->timeout, 1);
            return false;
        }
        __nanosleep(ns);
        ns = min(ns * 2, 256u);
    }
    return true;
}

__device__ __forceinline__ bool wait_flags(const bk_dev &d, const int32_t *flags, int j, bool want, int epoch,
                                           long long budget)
{
    const int lane = threadIdx.x & 31;
    const uint32_t pending = __ballot_sync(BK_FULL, want && ld_acquire(flags + j) != epoch);
    if (!pending) return true;
    int ok = 1;
    for (uint32_t p = pending; p; p &= p - 1) {
        const int jt = __shfl_sync(BK_FULL, j, __ffs(p) - 1);
        if (lane == 0 && ok) ok = lane0_poll(d, flags + jt, epoch, budget);
    }
    if (!__shfl_sync(BK_FULL, ok, 0)) return false;
    int mine = 1;
    if ((pending >> lane) & 1u) mine = lane0_poll(d, flags + j, epoch, budget);
    return __all_sync(BK_FULL, mine);
}

// z -= sum over up to 32 terms a_t * v_t, in lane order (every lane computes the
// same chain).
template <typename V>
__device__ __forceinline__ V chain(V z, V a, V v, int cnt)
{
    for (int t = 0; t < cnt; t++) z = fma(-__shfl_sync(BK_FULL, a, t), __shfl_sync(BK_FULL, v, t), z);
    return z;
}

template <typename V>
__global__ void __launch_bounds__(128) bk_solve_kernel(bk_dev d, bk_solve_dev s, int32_t nrhs,
                                                       const double *__restrict__ b, int32_t ldb, double *x,
                                                       int32_t ldx, int32_t epoch, long long budget,
                                                       const int32_t *__restrict__ Pin,
                                                       const int32_t *__restrict__ Qout)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = d.n;
    const V *const Bx = vals<V>(d.Bx);
    const V *const Lrx = vals<V>(s.r.Lrx);
    const V *const Urx = vals<V>(s.r.Urx);
    const V *const Ud = vals<V>(s.r.Ud);
    V *const w = vals<V>(s.w);
    V *const zz = vals<V>(s.z);
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(d.counter + 2, 1);
        k = __shfl_sync(BK_FULL, k, 0);
        if (k >= s.nitems) break;
        const int it = s.items[k];
        if (it >= 0) {
            // forward row i: coupling terms of row prow i, then L(i,:)
            const int i = it;
            const int r = d.prow[i];
            const int e0 = s.offp[r], e1 = s.offp[r + 1];
            const int64_t l0 = s.r.Lrp[i], l1 = s.r.Lrp[i + 1];
            for (int q = 0; q < nrhs; q++) {
                V z = (V)b[(int64_t)q * ldb + (Pin ? Pin[r] : r)];
                for (int e = e0; e < e1; e += 32) {
                    const int cnt = min(32, e1 - e);
                    const bool have = lane < cnt;
                    const int j = have ? s.offj[e + lane] : 0;
                    const V a = have ? Bx[s.offpos[e + lane]] : V(0);
                    if (!wait_flags(d, s.bdone, j, have, epoch, budget)) return;
                    const V v = have ? __ldcg(zz + q * n + j) : V(0);
                    z = chain(z, a, v, cnt);
                }
                for (int64_t e = l0; e < l1; e += 32) {
                    const int cnt = (int)min((int64_t)32, l1 - e);
                    const bool have = lane < cnt;
                    const int j = have ? s.r.Lrk[e + lane] : 0;
                    const V a = have ? Lrx[e + lane] : V(0);
                    if (!wait_flags(d, s.fdone, j, have, epoch, budget)) return;
                    const V v = have ? __ldcg(w + q * n + j) : V(0);
                    z = chain(z, a, v, cnt);
                }
                if (lane == 0) w[q * n + i] = z;
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release(s.fdone + i, epoch);
        } else {
            // backward row i: its forward result, then U(i,:), then the diagonal
            const int i = ~it;
            if (!wait_flags(d, s.fdone, i, lane == 0, epoch, budget)) return;
            const int64_t u0 = s.r.Urp[i], u1 = s.r.Urp[i + 1];
            const V ud = Ud[i];
            for (int q = 0; q < nrhs; q++) {
                V z = __shfl_sync(BK_FULL, lane == 0 ? __ldcg(w + q * n + i) : V(0), 0);
                for (int64_t e = u0; e < u1; e += 32) {
                    const int cnt = (int)min((int64_t)32, u1 - e);
                    const bool have = lane < cnt;
                    const int j = have ? s.r.Urk[e + lane] : 0;
                    const V a = have ? Urx[e + lane] : V(0);
                    if (!wait_flags(d, s.bdone, j, have, epoch, budget)) return;
                    const V v = have ? __ldcg(zz + q * n + j) : V(0);
                    z = chain(z, a, v, cnt);
                }
                z = z / ud;
                if (lane == 0) {
                    zz[q * n + i] = z;
                    x[(int64_t)q * ldx + (Qout ? Qout[i] : i)] = (double)z;
                }
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release(s.bdone + i, epoch);
        }
    }
}

int solve_blocks()
{
    static int blocks = 0;
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bk_solve_kernel<double>, 128, 0);
        blocks = std::max(1, sms) * std::max(1, std::min(per, 8));
    }
    return blocks;
}

void launch_scan(const int32_t *cnt, int32_t m, int64_t *part, int64_t *out, cudaStream_t st)
{
    const int nb = std::max(1, (m + 1023) / 1024);
    bk_scan_sums<<<nb, 1024, 0, st>>>(cnt, m, part);
    bk_scan_parts<<<1, 1024, 0, st>>>(part, nb);
    bk_scan_apply<<<nb, 1024, 0, st>>>(cnt, m, part, out);
}

}  // namespace

void bk_launch_rows(const bk_dev &d, const bk_rows &r, void *stream)
{
    if (d.n <= 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = d.n;
    const int blocks = std::max(1, std::min((n + 7) / 8, 152 * 8));
    cudaMemsetAsync(r.cnt, 0, sizeof(int32_t) * 2 * ((size_t)n + 1), st);
    if (d.prec)
        bk_rows_count<float><<<blocks, 256, 0, st>>>(d, r);
    else
        bk_rows_count<double><<<blocks, 256, 0, st>>>(d, r);
    launch_scan(r.cnt, n, r.part, r.Lrp, st);
    launch_scan(r.cnt + n + 1, n, r.part, r.Urp, st);
    cudaMemsetAsync(r.cnt, 0, sizeof(int32_t) * 2 * ((size_t)n + 1), st);
    if (d.prec) {
        bk_rows_scatter<float><<<blocks, 256, 0, st>>>(d, r, 0);
        bk_rows_sort<float><<<blocks, 256, 0, st>>>(n, r.Lrp, r.tk, vals<float>(r.tx), r.Lrk, vals<float>(r.Lrx), 0);
        bk_rows_scatter<float><<<blocks, 256, 0, st>>>(d, r, 1);
        bk_rows_sort<float><<<blocks, 256, 0, st>>>(n, r.Urp, r.tk, vals<float>(r.tx), r.Urk, vals<float>(r.Urx), 1);
    } else {
        bk_rows_scatter<double><<<blocks, 256, 0, st>>>(d, r, 0);
        bk_rows_sort<double><<<blocks, 256, 0, st>>>(n, r.Lrp, r.tk, r.tx, r.Lrk, r.Lrx, 0);
        bk_rows_scatter<double><<<blocks, 256, 0, st>>>(d, r, 1);
        bk_rows_sort<double><<<blocks, 256, 0, st>>>(n, r.Urp, r.tk, r.tx, r.Urk, r.Urx, 1);
    }
}

void bk_launch_solve(const bk_dev &d, const bk_solve_dev &s, int32_t nrhs, const double *b, int32_t ldb,
                     double *x, int32_t ldx, int32_t epoch, long long budget, void *stream, bool permute)
{
    const int32_t *Pin = permute ? d.P : nullptr, *Qout = permute ? d.Q : nullptr;
    if (s.nitems <= 0) return;
    const int ctas = std::min<int>((s.nitems + 3) / 4, solve_blocks());
    if (d.prec)
        bk_solve_kernel<float><<<ctas, 128, 0, (cudaStream_t)stream>>>(d, s, nrhs, b, ldb, x, ldx, epoch, budget, Pin,
                                                                        Qout);
    else
        bk_solve_kernel<double><<<ctas, 128, 0, (cudaStream_t)stream>>>(d, s, nrhs, b, ldb, x, ldx, epoch, budget, Pin,
                                                                         Qout);
}
