// kernels_static.cu -- refactorization on a known pattern (the matrix-sequence
// case of Sec. V: same pattern, new values, previous pivots preferred).
//
//   bk_static_kernel   persistent; each warp claims columns in a topological order
//                      of the column DAG (column c waits for every step of
//                      U(:,c)) and recomputes the column on the stored pattern:
//                      x = B(:,c); for each step j of U(:,c), lowest first:
//                      x -= L(:,j) x(prow j); then L(:,c) = x / pivot.  The
//                      preferred pivot is validated as Algorithm 1's pivot selection would
//                      decide it (|x_pref| >= tau * max over the node's candidate
//                      rows); a column that would pick another row is reported for
//                      the reach-based path.  Waits are point-to-point flags (the
//                      paper's volatile-flag synchronisation, Sec. IV) with an
//                      iteration budget: a wait that runs out sets the timeout
//                      status and every warp returns.
//   bk_levels_kernel   the same dataflow over the current pattern, computing each
//                      column's DAG level; a counting sort then gives the claim
//                      order for the next static pass.
#include <cuda_runtime.h>

#include <algorithm>

#include "basker_internal.h"
#include "column_static.cuh"
#include "device_util.cuh"
#include "trace.cuh"

using namespace bk;

namespace {

template <typename V>
__global__ void __launch_bounds__(128) bk_static_kernel(bk_dev d, int32_t ncols, double tau, int32_t epoch,
                                                        long long budget)
{
    __shared__ bk_task Ts[4];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * 4 + wib;
    if (gw >= d.sx_warps) return;
    bk_task &T = Ts[wib];
    V *x = vals<V>(d.sx) + (int64_t)gw * d.sx_stride;
    int cur = -1;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(d.counter, 1);
        k = __shfl_sync(BK_FULL, k, 0);
        if (k >= ncols) break;
        const int c = d.order[k];
        BK_TSTART(t0);
        const int tid = d.col_task[c];
        if (tid != cur) {
            load_task(T, d.tasks + tid, lane);
            cur = tid;
        }
        if (T.dense) {
            // a separator recomputed afterwards by the dense elimination
            if (lane == 0) st_release(d.done + c, epoch);
            continue;
        }
        bool ok = false, bad = false, broken = false;
        if (!pattern_column(d, T, tid, x, c, epoch, budget, tau, lane, true, 0, ok, bad, broken)) return;
        if (broken && lane == 0) report_internal(d.status, c, 41);
        __syncwarp();
        __threadfence();
        if (lane == 0) {
            d.col_fail[c] = ok ? 0 : 1;
            if (!ok) {
                atomicMin(d.task_fail + tid, c);
                atomicAdd(&d.status->static_fail, 1);
            }
            st_release(d.done + c, epoch);
            BK_TREC(d.trace, BK_TR_STATIC, ok ? 0 : 1, c, t0);
        }
    }
}

// The stored levels are still a topological order of the current pattern if
// every step of every U(:,c) has a lower level than c; any violation sets *stale.
__global__ void bk_level_check_kernel(bk_dev d, int32_t *stale)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < d.n; c += warps) {
        const int64_t ub = d.Ubeg[c];
        const int uc = d.Ucnt[c];
        const int lc = __ldg(d.level + c);
        for (int q = lane; q < uc - 1; q += 32) {
            const int j = d.Ui[ub + q];
            if ((unsigned)j >= (unsigned)d.n || __ldg(d.level + j) >= lc) bad = true;
        }
    }
    if (__any_sync(BK_FULL, bad) && lane == 0) atomicExch(stale, 1);
}

__global__ void __launch_bounds__(128) bk_levels_kernel(bk_dev d, int32_t epoch, long long budget,
                                                        int32_t *maxlev, const int32_t *stale)
{
    if (!*stale) return;                 // the stored levels still hold
    const int lane = threadIdx.x & 31;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(d.counter + 1, 1);
        c = __shfl_sync(BK_FULL, c, 0);
        if (c >= d.n) break;
        c = d.iorder[c];
        BK_TSTART(t0);
        const int64_t ub = d.Ubeg[c];
        const int uc = d.Ucnt[c];
        int lv = 0;
        int ok = 1;
        for (int q = lane; q < uc - 1; q += 32) {
            const int j = d.Ui[ub + q];
            const int *flag = d.done + j;
            if (ld_relaxed(flag) != epoch) {
                const long long t0 = clock64();
                while (ld_relaxed(flag) != epoch) {
                    if (*reinterpret_cast<const volatile int *>(&d.status->timeout) || clock64() - t0 > budget) {
                        atomicExch(&d.status->timeout, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (!ok) break;
            fence_acquire();
            lv = max(lv, __ldcg(d.level + j) + 1);
        }
        if (__any_sync(BK_FULL, !ok)) return;
        lv = warp_max_i(lv);
        if (lane == 0) {
            d.level[c] = lv;
            atomicMax(maxlev, lv);
            st_release(d.done + c, epoch);          // orders this thread's write of the level
            BK_TREC(d.trace, BK_TR_LEVELS, 0, c, t0);
        }
        __syncwarp();
    }
}

__global__ void bk_level_count(const int32_t *__restrict__ level, int32_t n, int32_t *cnt, const int32_t *stale)
{
    if (!*stale) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        atomicAdd(cnt + level[c], 1);
}

// Exclusive scan of cnt[0..m) in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) bk_level_scan(int32_t *cnt, int32_t m, const int32_t *stale)
{
    if (!*stale) return;
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int chunk = (m + 1023) / 1024;
    const int a = min(m, t * chunk), b = min(m, a + chunk);
    int s = 0;
    for (int i = a; i < b; i++) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = a; i < b; i++) {
        const int v = cnt[i];
        cnt[i] = run;
        run += v;
    }
}

__global__ void bk_level_scatter(const int32_t *__restrict__ level, int32_t n, int32_t *cursor,
                                 int32_t *order, const int32_t *stale)
{
    if (!*stale) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        order[atomicAdd(cursor + level[c], 1)] = c;
}

}  // namespace

int bk_static_blocks()
{
    // computed once, thread-safely (a function-local static)
    static const int blocks = [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bk_static_kernel<double>, 128, 0);
        return std::max(1, sms) * std::max(1, std::min(per, 4));
    }();
    return blocks;
}

void bk_launch_static(const bk_dev &d, int32_t ncols, double tau, int32_t epoch, long long budget,
                      int blocks, void *stream)
{
    if (ncols <= 0) return;
    if (d.prec)
        bk_static_kernel<float><<<blocks, 128, 0, (cudaStream_t)stream>>>(d, ncols, tau, epoch, budget);
    else
        bk_static_kernel<double><<<blocks, 128, 0, (cudaStream_t)stream>>>(d, ncols, tau, epoch, budget);
}

// Levels of the current pattern's column DAG and the claim order sorted by level.
// scratch: n + 2 ints (counts), last one receives the maximum level.  With
// check, the stored levels are kept (and nothing else runs) when they are still
// a topological order of the pattern; the decision stays on the device.
void bk_launch_levels(const bk_dev &d, int32_t epoch, long long budget, int blocks, void *stream, bool check)
{
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *cnt = d.level + d.n;               // level array holds n + (n + 2) ints
    int32_t *maxlev = cnt + d.n + 1;
    int32_t *stale = d.counter + 6;
    int g = std::max(1, std::min((d.n + 255) / 256, 152 * 8));
    if (check) {
        cudaMemsetAsync(stale, 0, sizeof(int32_t), s);
        bk_level_check_kernel<<<std::max(1, std::min((d.n + 7) / 8, 152 * 16)), 256, 0, s>>>(d, stale);
    } else {
        cudaMemsetAsync(stale, 0xff, sizeof(int32_t), s);
    }
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)d.n + 2), s);
    cudaMemsetAsync(d.counter + 1, 0, sizeof(int32_t), s);
    bk_levels_kernel<<<blocks, 128, 0, s>>>(d, epoch, budget, maxlev, stale);
    bk_level_count<<<g, 256, 0, s>>>(d.level, d.n, cnt, stale);
    bk_level_scan<<<1, 1024, 0, s>>>(cnt, d.n + 1, stale);
    bk_level_scatter<<<g, 256, 0, s>>>(d.level, d.n, cnt, d.order, stale);
}
