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
#include "trace.cuh"

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
        for (int t = lane; t < ln; t += 32) {
            const int i = d.pinv[d.Li[lb + t]];
            r.Ls[lb + t] = i;
            atomicAdd(lc + i, 1);
        }
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
        if (len > BK_LONG_ROW) continue;          // bk_rows_sort_long
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

__global__ void bk_rows_long_list(int32_t n, const int64_t *rp, int32_t *longs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (rp[i + 1] - rp[i] > BK_LONG_ROW) longs[1 + atomicAdd(longs, 1)] = i;
}

// Long rows, one block a row: the row's columns (distinct) set bits of a bitmap
// over [cmin, cmax]; an entry's rank is the number of set bits before its own,
// a prefix sum of the words' popcounts plus the popcount within its word.
// Linear in the row's length and its column range.
template <typename V>
__global__ void __launch_bounds__(1024) bk_rows_sort_long(const int64_t *rp, const int32_t *tk, const V *tx,
                                                          int32_t *ok, V *ox, int desc, const int32_t *longs,
                                                          uint32_t *sbits, int32_t *spre, int64_t swords)
{
    __shared__ int64_t wt[33];
    __shared__ int red[2][32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint32_t *bm = sbits + (int64_t)blockIdx.x * swords;
    int32_t *pre = spre + (int64_t)blockIdx.x * swords;
    const int nlong = longs[0];
    for (int q = blockIdx.x; q < nlong; q += gridDim.x) {
        const int i = longs[1 + q];
        const int64_t p0 = rp[i];
        const int len = (int)(rp[i + 1] - p0);
        int lo = INT_MAX, hi = -1;
        for (int e = tid; e < len; e += blockDim.x) {
            const int c = tk[p0 + e];
            lo = min(lo, c);
            hi = max(hi, c);
        }
        lo = warp_min(lo);
        hi = warp_max_i(hi);
        if (lane == 0) { red[0][wid] = lo; red[1][wid] = hi; }
        __syncthreads();
        if (wid == 0) {
            lo = lane < (int)(blockDim.x >> 5) ? red[0][lane] : INT_MAX;
            hi = lane < (int)(blockDim.x >> 5) ? red[1][lane] : -1;
            lo = warp_min(lo);
            hi = warp_max_i(hi);
            if (lane == 0) { red[0][0] = lo; red[1][0] = hi; }
        }
        __syncthreads();
        const int cmin = red[0][0];
        const int W = ((red[1][0] - cmin) >> 5) + 1;
        for (int w = tid; w < W; w += blockDim.x) bm[w] = 0u;
        __syncthreads();
        for (int e = tid; e < len; e += blockDim.x) {
            const int off = tk[p0 + e] - cmin;
            atomicOr(bm + (off >> 5), 1u << (off & 31));
        }
        __syncthreads();
        int64_t carry = 0;
        for (int w0 = 0; w0 < W; w0 += blockDim.x) {
            const int w = w0 + tid;
            const int64_t v = w < W ? __popc(bm[w]) : 0;
            int64_t total;
            const int64_t ex = block_exscan(v, wt, total);
            if (w < W) pre[w] = (int32_t)(carry + ex);
            carry += total;
        }
        __syncthreads();
        for (int e = tid; e < len; e += blockDim.x) {
            const int c = tk[p0 + e];
            const int off = c - cmin;
            const int r = pre[off >> 5] + __popc(bm[off >> 5] & ((1u << (off & 31)) - 1u));
            const int rank = desc ? len - 1 - r : r;
            ok[p0 + rank] = c;
            ox[p0 + rank] = tx[p0 + e];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- leaf order

// Orders of an ND leaf's rows.  Backward: U(i,k) != 0 makes column k depend on
// step i in the factorization, so the factorization's column levels (d.level,
// longest chain from a source, counting only the leaf's steps for a leaf
// column) taken in decreasing order are a valid order, and one with the most
// rows at each level.  Forward: the same levels in increasing order are valid
// when every L(i,k) != 0 of the leaf has level(k) < level(i) (true for
// symmetric patterns); a leaf where that fails keeps its step order.  Each leaf's
// rows are split over `chunks` blocks (block b: leaf b / chunks, chunk b % chunks).
__global__ void bk_leaf_check(bk_dev d, bk_solve_dev s, int chunks)
{
    const int leaf = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bk_task &T = d.tasks[s.leaf_tasks[leaf]];
    int bad = 0;
    for (int i = T.lo + chunk * nw + wid; i < T.hi; i += nw * chunks) {
        const int li = d.level[i];
        for (int64_t e = s.r.Lrp[i] + lane; e < s.r.Lrp[i + 1]; e += 32)
            if (d.level[s.r.Lrk[e]] >= li) bad = 1;
    }
    if (__any_sync(BK_FULL, bad) && lane == 0) s.leaf_bad[leaf] = 1;
}

// Sort key of leaf row i (both below the leaf's size).
__device__ __forceinline__ int leaf_key(const bk_dev &d, const bk_solve_dev &s, int leaf, int lo, int hi, int i,
                                        int dir)
{
    if (dir == 0) return s.leaf_bad[leaf] ? i - lo : d.level[i];
    return s.leaf_maxrows - d.level[i];
}

// Counting sort of all leaf rows by level into their places of the claim order
// (a thread a row; rows of one level take their places in any order).
__global__ void bk_leaf_count(bk_dev d, bk_solve_dev s, int chunks)
{
    const int leaf = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
    const bk_task &T = d.tasks[s.leaf_tasks[leaf]];
    for (int i = T.lo + chunk * blockDim.x + threadIdx.x; i < T.hi; i += blockDim.x * chunks) {
        atomicAdd(s.lcnt + leaf_key(d, s, leaf, T.lo, T.hi, i, 0), 1);
        atomicAdd(s.lcnt + (s.leaf_maxrows + 1) + leaf_key(d, s, leaf, T.lo, T.hi, i, 1), 1);
    }
}

__global__ void __launch_bounds__(1024) bk_leaf_scan(bk_solve_dev s)
{
    // exclusive scan of both count arrays (one block; counts of at most leaf_maxrows levels)
    __shared__ int64_t wt[33];
    const int m = s.leaf_maxrows + 1;
    for (int dir = 0; dir < 2; dir++) {
        int32_t *c = s.lcnt + dir * m;
        int64_t carry = 0;
        for (int b0 = 0; b0 < m; b0 += 1024) {
            const int i = b0 + threadIdx.x;
            const int64_t v = i < m ? c[i] : 0;
            int64_t total;
            const int64_t ex = block_exscan(v, wt, total);
            if (i < m) c[i] = (int32_t)(carry + ex);
            carry += total;
        }
        __syncthreads();
    }
}

__global__ void bk_leaf_scatter(bk_dev d, bk_solve_dev s, int chunks)
{
    const int leaf = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
    const bk_task &T = d.tasks[s.leaf_tasks[leaf]];
    const int m = s.leaf_maxrows + 1;
    for (int i = T.lo + chunk * blockDim.x + threadIdx.x; i < T.hi; i += blockDim.x * chunks) {
        s.items[s.leaf_f0 + atomicAdd(s.lcnt + leaf_key(d, s, leaf, T.lo, T.hi, i, 0), 1)] = i;
        s.items[s.leaf_b0 + atomicAdd(s.lcnt + m + leaf_key(d, s, leaf, T.lo, T.hi, i, 1), 1)] = ~i;
    }
}

// ---------------------------------------------------------------- the solve

// One lane's bounded wait until *flag == epoch (an acquiring load, which orders
// the lane's later reads), sleeping between polls.  False if the wait ran out
// (the timeout status is then set).
__device__ __forceinline__ bool poll_flag(const bk_dev &d, const int32_t *flag, int epoch, long long budget)
{
    const long long t0 = clock64();
    unsigned ns = 32;
    while (ld_acquire(flag) != epoch) {
        if (*reinterpret_cast<const volatile int *>(&d.status->timeout) || clock64() - t0 > budget) {
            atomicExch(&d.status->timeout, 1);
            return false;
        }
        __nanosleep(ns);
        ns = min(ns * 2, 128u);
    }
    return true;
}

// Bounded wait until flags[j] == epoch for every lane with want.  Each lane
// checks its flag once; lane 0 alone then polls the flags still unset, in lane
// order (one poller per warp, and no rereads of the other flags meanwhile), and
// finally each of those lanes rereads its own flag with an acquiring load, which
// orders its later reads.  False if a wait ran out.
__device__ __forceinline__ bool wait_flags(const bk_dev &d, const int32_t *flags, int j, bool want, int epoch,
                                           long long budget)
{
    const int lane = threadIdx.x & 31;
    const uint32_t pending = __ballot_sync(BK_FULL, want && ld_acquire(flags + j) != epoch);
    if (!pending) return true;
    int ok = 1;
    for (uint32_t p = pending; p; p &= p - 1) {
        const int jt = __shfl_sync(BK_FULL, j, __ffs(p) - 1);
        if (lane == 0 && ok) ok = poll_flag(d, flags + jt, epoch, budget);
    }
    if (!__shfl_sync(BK_FULL, ok, 0)) return false;
    int mine = 1;
    if ((pending >> lane) & 1u) mine = poll_flag(d, flags + j, epoch, budget);
    return __all_sync(BK_FULL, mine);
}

// z -= sum over up to 32 terms a_t * v_t, v_t = vals[j_t] once flags[j_t] ==
// epoch, in lane order (every lane computes the same chain).  The terms whose
// flags are set are applied as soon as every earlier term is, and the first term
// still waited for is polled by its own lane: the term that arrives last (in a
// chain of rows, the previous row) costs one fma after its flag, not a batch.
// False if a wait ran out (the timeout status is then set).
template <typename V>
__device__ __forceinline__ bool chain_wait(const bk_dev &d, const int32_t *flags, const V *vals, int j, bool have,
                                           V a, int cnt, int epoch, long long budget, V &z)
{
    const int lane = threadIdx.x & 31;
    bool ready = !have || ld_acquire(flags + j) == epoch;
    V v = (have && ready) ? __ldcg(vals + j) : V(0);
    for (int done = 0;;) {
        const uint32_t nr = __ballot_sync(BK_FULL, !ready);
        const int upto = nr ? __ffs(nr) - 1 : cnt;
        for (int t = done; t < upto; t++) z = fma(-__shfl_sync(BK_FULL, a, t), __shfl_sync(BK_FULL, v, t), z);
        if (upto >= cnt) return true;
        done = upto;
        int ok = 1;
        if (lane == done) {
            ok = poll_flag(d, flags + j, epoch, budget);
            if (ok) {
                v = __ldcg(vals + j);
                ready = true;
            }
        }
        if (!__shfl_sync(BK_FULL, ok, done)) return false;
        if (!ready && ld_acquire(flags + j) == epoch) {
            v = __ldcg(vals + j);
            ready = true;
        }
    }
}

// ---------------------------------------------------------------- separator sweeps
//
// One block solves a separator's own triangle, its rows' outside terms already
// applied (the rows' values in zs, in shared memory or in place in global
// memory).  Forward: for k ascending, w_k = zs[k] is final and L(i,k) w_k is
// subtracted from the node's rows i > k; backward: for k descending, z_k =
// zs[k] / U(k,k) is final and U(j,k) z_k is subtracted from the node's rows
// j < k.  Per row the terms come in the order of the row sweeps (ascending k
// forward, descending backward), after the outside terms; each step's terms go
// to distinct rows, spread over the block's threads, with one barrier a step.
// A column's own entries (the first ones of L(:,k), the last ones above the
// diagonal of U(:,k)) are copied into shared memory SW_P - 1 steps ahead
// (cp.async, a ring of SW_P stages of sw_win entries), and the columns' extents
// 2 SW_P steps ahead, so that a step waits for no global load.
constexpr int SW_NT = 128;     // threads of a block (the kernel's block size)
constexpr int SW_P = 8;        // pipeline stages
constexpr int SW_MR = 4 * SW_P;  // ring of column extents
constexpr int SW_WMAX = 448;   // most entries of a column a stage holds
constexpr int SW_MAXB = 64;    // most sweeper blocks
constexpr int SEP_SMEM_ROWS = 1024;   // most rows of a node swept in shared memory

__host__ __device__ constexpr size_t sw_align(size_t b) { return (b + 15) & ~(size_t)15; }

struct SwLayout {
    size_t ri, rv, rd, mb, mc, total;
};

__host__ __device__ inline SwLayout sw_layout(int win, int zrows, size_t vsize)
{
    SwLayout L;
    L.ri = sw_align((size_t)zrows * vsize);
    L.rv = L.ri + (size_t)SW_P * win * 4;
    L.rd = L.rv + (size_t)SW_P * win * vsize;
    L.mb = L.rd + sw_align((size_t)SW_P * vsize);
    L.mc = L.mb + (size_t)SW_MR * 8;
    L.total = L.mc + (size_t)SW_MR * 4;
    return L;
}

__device__ __forceinline__ void sw_cp4(void *dst, const void *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
}

__device__ __forceinline__ void sw_cp8(void *dst, const void *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}

template <typename V>
__device__ __forceinline__ void sw_cpv(V *dst, const V *src)
{
    if (sizeof(V) == 8) sw_cp8(dst, src);
    else sw_cp4(dst, src);
}

__device__ __forceinline__ void sw_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void sw_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename V>
__device__ void sep_sweep_block(const bk_dev &d, const bk_solve_dev &s, int it, int nrhs, double *x, int ldx,
                                int epoch, long long budget, const int32_t *Qout, unsigned char *smem)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = d.n;
    const bool fwd = it >= 0;
    const int t = (fwd ? it : ~it) - (int)n;
    const int lo = d.tasks[t].lo, hi = d.tasks[t].hi, m = hi - lo;
    const int W = s.sw_win;
    const V *const Lx = vals<V>(d.Lx);
    const V *const Ux = vals<V>(d.Ux);
    V *const w = vals<V>(s.w);
    V *const zz = vals<V>(s.z);
    const SwLayout Ly = sw_layout(W, s.sw_zrows, sizeof(V));
    V *const zsm = reinterpret_cast<V *>(smem);
    int32_t *const ri = reinterpret_cast<int32_t *>(smem + Ly.ri);
    V *const rv = reinterpret_cast<V *>(smem + Ly.rv);
    V *const rd = reinterpret_cast<V *>(smem + Ly.rd);
    int64_t *const mb = reinterpret_cast<int64_t *>(smem + Ly.mb);
    int32_t *const mc = reinterpret_cast<int32_t *>(smem + Ly.mc);
    BK_TSTART(t0);
    int32_t *flags = fwd ? s.fdone : s.bdone;
    bool ok = true;
    for (int r0 = lo + 32 * warp; r0 < hi && ok; r0 += SW_NT)
        ok = wait_flags(d, flags, r0 + lane, r0 + lane < hi, -epoch, budget);
    if (__syncthreads_or(!ok)) return;
    BK_TPHASE0(tp);
    // the column at sweep position p, and its own entries held by a stage
    auto col_of = [&](int p) { return lo + (fwd ? p : m - 1 - p); };
    auto own_win = [&](int p, int cnt) {
        const int kl = fwd ? p : m - 1 - p;
        return fwd ? min(min(cnt, m - 1 - kl), W) : min(min(cnt - 1, kl), W);
    };
    auto issue = [&](int p) {
        const int slot = p % SW_MR, st = p % SW_P;
        const int64_t beg = mb[slot];
        const int cnt = mc[slot];
        const int wn = own_win(p, cnt);
        const int64_t g0 = fwd ? beg : beg + cnt - 1 - wn;
        for (int e = tid; e < wn; e += SW_NT) {
            sw_cp4(ri + st * W + e, (fwd ? s.r.Ls : d.Ui) + g0 + e);
            sw_cpv(rv + st * W + e, (fwd ? Lx : Ux) + g0 + e);
        }
        if (!fwd && tid == 0) sw_cpv(rd + st, Ux + beg + cnt - 1);
    };
    for (int q = 0; q < nrhs; q++) {
        V *vq = (fwd ? w : zz) + q * n;
        V *zs = m <= s.sw_zrows ? zsm : vq + lo;
        if (zs == zsm)
            for (int r = tid; r < m; r += SW_NT) zs[r] = __ldcg(vq + lo + r);
        for (int p = tid; p < min(2 * SW_P, m); p += SW_NT) {
            const int c = col_of(p);
            mb[p % SW_MR] = fwd ? d.Lbeg[c] : d.Ubeg[c];
            mc[p % SW_MR] = fwd ? d.Lcnt[c] : d.Ucnt[c];
        }
        __syncthreads();
        for (int p = 0; p < SW_P - 1; p++) {
            if (p < m) issue(p);
            sw_commit();
        }
        V zprev = V(0);
        int kprev = -1;
        for (int p = 0; p < m; p++) {
            sw_wait<SW_P - 2>();
            __syncthreads();
            // the previous step's z (backward) is stored once every thread read it
            if (kprev >= 0 && tid == 0) zs[kprev] = zprev;
            const int kl = fwd ? p : m - 1 - p;
            const int st = p % SW_P, slot = p % SW_MR;
            const int cnt = mc[slot];
            const int64_t beg = mb[slot];
            V v = zs[kl];
            if (!fwd) v = v / rd[st];
            const int wn = own_win(p, cnt);
            for (int e = tid; e < wn; e += SW_NT) {
                const int r = ri[st * W + e];
                if (fwd ? r < hi : r >= lo) zs[r - lo] = fma(-rv[st * W + e], v, zs[r - lo]);
            }
            // own entries past the stage's window, read directly
            const int own = fwd ? min(cnt, m - 1 - kl) : min(cnt - 1, kl);
            for (int e = W + tid; e < own; e += SW_NT) {
                const int64_t g = fwd ? beg + e : beg + cnt - 2 - e;
                const int r = fwd ? s.r.Ls[g] : d.Ui[g];
                if (fwd ? r >= hi : r < lo) break;
                zs[r - lo] = fma(-(fwd ? Lx[g] : Ux[g]), v, zs[r - lo]);
            }
            if (!fwd) {
                zprev = v;
                kprev = kl;
            }
            // extents 2 SW_P positions ahead; entries SW_P - 1 positions ahead (into
            // the stage every thread finished reading in the previous step)
            if (tid == 0 && p + 2 * SW_P < m) {
                const int pn = p + 2 * SW_P, c = col_of(pn);
                sw_cp8(mb + pn % SW_MR, fwd ? d.Lbeg + c : d.Ubeg + c);
                sw_cp4(mc + pn % SW_MR, fwd ? d.Lcnt + c : d.Ucnt + c);
            }
            if (p + SW_P - 1 < m) issue(p + SW_P - 1);
            sw_commit();
        }
        sw_wait<0>();
        __syncthreads();
        if (kprev >= 0 && tid == 0) zs[kprev] = zprev;
        __syncthreads();
        for (int r = tid; r < m; r += SW_NT) {
            const V v = zs[r];
            vq[lo + r] = v;
            if (!fwd) x[(int64_t)q * ldx + (Qout ? Qout[lo + r] : lo + r)] = (double)v;
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    for (int r = lo + tid; r < hi; r += SW_NT) st_release(flags + r, epoch);
    if (tid == 0) BK_TREC(d.trace, BK_TR_SOLVE, fwd ? 2 : 3, t, t0);
    BK_TPHASE(d.trace, tp, fwd ? 10 : 11, t);     // the sweep itself
}

template <typename V>
__global__ void __launch_bounds__(128) bk_solve_kernel(bk_dev d, bk_solve_dev s, int32_t nrhs,
                                                       const double *__restrict__ b, int32_t ldb, double *x,
                                                       int32_t ldx, int32_t epoch, long long budget,
                                                       const int32_t *__restrict__ Pin,
                                                       const int32_t *__restrict__ Qout)
{
    extern __shared__ __align__(16) double solve_smem[];
    const int lane = threadIdx.x & 31;
    const int64_t n = d.n;
    // the first blocks sweep the separators' own triangles, in claim order
    const int nsb = min(s.nsweeps, SW_MAXB);
    if ((int)blockIdx.x < nsb) {
        for (int k = blockIdx.x; k < s.nsweeps; k += nsb) {
            sep_sweep_block<V>(d, s, s.sweeps[k], nrhs, x, ldx, epoch, budget, Qout,
                               reinterpret_cast<unsigned char *>(solve_smem));
            if (__syncthreads_or(*reinterpret_cast<const volatile int *>(&d.status->timeout) != 0)) return;
        }
        return;
    }
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
        BK_TSTART(t0);
        const bool fwd = it >= 0;
        const int i = fwd ? it : ~it;
        if (i >= n) continue;     // a separator's sweep (the sweeper blocks take it)
        // a separator's row takes only the terms from outside its node
        const int clo = s.cutlo[i], chi = s.cuthi[i];
        const bool part = clo >= 0;
        if (fwd) {
            // forward row i: coupling terms of row prow i, then L(i,k) for k < clo (or all)
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
                    if (!chain_wait(d, s.bdone, zz + q * n, j, have, a, cnt, epoch, budget, z)) return;
                }
                for (int64_t e = l0; e < l1; e += 32) {
                    int cnt = (int)min((int64_t)32, l1 - e);
                    const int j0 = lane < cnt ? s.r.Lrk[e + lane] : 0;
                    if (part) cnt = __popc(__ballot_sync(BK_FULL, lane < cnt && j0 < clo));
                    const bool have = lane < cnt;
                    const int j = have ? j0 : 0;
                    const V a = have ? Lrx[e + lane] : V(0);
                    if (!chain_wait(d, s.fdone, w + q * n, j, have, a, cnt, epoch, budget, z)) return;
                    if (cnt < 32) break;
                }
                if (lane == 0) w[q * n + i] = z;
            }
            // lane 0 alone wrote what the flag publishes: its release store orders it
            __syncwarp();
            if (lane == 0) st_release(s.fdone + i, part ? -epoch : epoch);
            if (lane == 0) BK_TREC(d.trace, BK_TR_SOLVE, 0, i, t0);
        } else {
            // backward row i: its forward result, then U(i,k) for k >= chi (or all), then the diagonal
            if (!wait_flags(d, s.fdone, i, lane == 0, epoch, budget)) return;
            const int64_t u0 = s.r.Urp[i], u1 = s.r.Urp[i + 1];
            const V ud = Ud[i];
            for (int q = 0; q < nrhs; q++) {
                V z = __shfl_sync(BK_FULL, lane == 0 ? __ldcg(w + q * n + i) : V(0), 0);
                for (int64_t e = u0; e < u1; e += 32) {
                    int cnt = (int)min((int64_t)32, u1 - e);
                    const int j0 = lane < cnt ? s.r.Urk[e + lane] : 0;
                    if (part) cnt = __popc(__ballot_sync(BK_FULL, lane < cnt && j0 >= chi));
                    const bool have = lane < cnt;
                    const int j = have ? j0 : 0;
                    const V a = have ? Urx[e + lane] : V(0);
                    if (!chain_wait(d, s.bdone, zz + q * n, j, have, a, cnt, epoch, budget, z)) return;
                    if (cnt < 32) break;
                }
                if (!part) z = z / ud;
                if (lane == 0) {
                    zz[q * n + i] = z;
                    if (!part) x[(int64_t)q * ldx + (Qout ? Qout[i] : i)] = (double)z;
                }
            }
            __syncwarp();
            if (lane == 0) st_release(s.bdone + i, part ? -epoch : epoch);
            if (lane == 0) BK_TREC(d.trace, BK_TR_SOLVE, 1, i, t0);
        }
    }
}

}  // namespace

int bk_solve_blocks()
{
    // computed once, thread-safely (a function-local static)
    static const int blocks = [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bk_solve_kernel<double>, 128,
                                                      4 * SEP_SMEM_ROWS * sizeof(double));
        return std::max(1, sms) * std::max(1, std::min(per, 8));
    }();
    return blocks;
}

void bk_solve_sweep_setup(bk_solve_dev &s, int32_t sw_maxm)
{
    const int own = std::max(1, sw_maxm - 1);
    s.sw_win = std::min(SW_WMAX, (own + 3) & ~3);
    s.sw_zrows = std::min(std::max(sw_maxm, 1), SEP_SMEM_ROWS);
    // the FP64 layout, the larger one, serves both kernels
    s.sw_smem = sw_layout(s.sw_win, s.sw_zrows, sizeof(double)).total;
    int dev = 0, sms = 0, per[2] = {0, 0};
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the function attribute is shared by every handle: the largest layout, once
    static const bool raised = [] {
        const int most = (int)sw_layout(SW_WMAX, SEP_SMEM_ROWS, sizeof(double)).total;
        cudaFuncSetAttribute(bk_solve_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        cudaFuncSetAttribute(bk_solve_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        return true;
    }();
    (void)raised;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], bk_solve_kernel<double>, SW_NT, s.sw_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], bk_solve_kernel<float>, SW_NT, s.sw_smem);
    for (int k = 0; k < 2; k++) s.sw_cap[k] = std::max(1, sms) * std::max(1, std::min(per[k], 8));
}

namespace {

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
    const int lblocks = std::max(1, std::min((n + 255) / 256, 152 * 8));
    for (int which = 0; which < 2; which++) {
        const int64_t *rp = which ? r.Urp : r.Lrp;
        int32_t *ok = which ? r.Urk : r.Lrk;
        double *ox = which ? r.Urx : r.Lrx;
        cudaMemsetAsync(r.longs, 0, sizeof(int32_t), st);
        bk_rows_long_list<<<lblocks, 256, 0, st>>>(n, rp, r.longs);
        if (d.prec) {
            bk_rows_scatter<float><<<blocks, 256, 0, st>>>(d, r, which);
            bk_rows_sort<float><<<blocks, 256, 0, st>>>(n, rp, r.tk, vals<float>(r.tx), ok, vals<float>(ox), which);
            bk_rows_sort_long<float><<<BK_LONG_CTAS, 1024, 0, st>>>(rp, r.tk, vals<float>(r.tx), ok, vals<float>(ox),
                                                                     which, r.longs, r.sbits, r.spre, r.swords);
        } else {
            bk_rows_scatter<double><<<blocks, 256, 0, st>>>(d, r, which);
            bk_rows_sort<double><<<blocks, 256, 0, st>>>(n, rp, r.tk, r.tx, ok, ox, which);
            bk_rows_sort_long<double><<<BK_LONG_CTAS, 1024, 0, st>>>(rp, r.tk, r.tx, ok, ox, which, r.longs, r.sbits,
                                                                      r.spre, r.swords);
        }
    }
}

void bk_launch_leaf_order(const bk_dev &d, const bk_solve_dev &s, void *stream)
{
    if (s.nleaves <= 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    // each leaf's rows over up to 32 blocks of 256 threads
    const int chunks = std::max(1, std::min((s.leaf_maxrows + 255) / 256, 32));
    const unsigned grid = (unsigned)s.nleaves * (unsigned)chunks;
    cudaMemsetAsync(s.leaf_bad, 0, sizeof(int32_t) * (size_t)s.nleaves, st);
    bk_leaf_check<<<grid, 256, 0, st>>>(d, s, chunks);
    cudaMemsetAsync(s.lcnt, 0, sizeof(int32_t) * 2 * ((size_t)s.leaf_maxrows + 1), st);
    bk_leaf_count<<<grid, 256, 0, st>>>(d, s, chunks);
    bk_leaf_scan<<<1, 1024, 0, st>>>(s);
    bk_leaf_scatter<<<grid, 256, 0, st>>>(d, s, chunks);
}

void bk_launch_solve(const bk_dev &d, const bk_solve_dev &s, int32_t nrhs, const double *b, int32_t ldb,
                     double *x, int32_t ldx, int32_t epoch, long long budget, void *stream, bool permute,
                     int max_ctas)
{
    const int32_t *Pin = permute ? d.P : nullptr, *Qout = permute ? d.Q : nullptr;
    if (s.nitems <= 0) return;
    // sweeper blocks first, then the row warps' blocks; every block co-resident
    const int nsb = std::min(s.nsweeps, SW_MAXB);
    const int cap = s.sw_cap[d.prec ? 1 : 0];
    const int limit = max_ctas > 0 ? std::min(max_ctas, cap) : cap;
    const int ctas = nsb + std::max(1, std::min<int>((s.nitems + 3) / 4, limit - nsb));
    const size_t smem = s.sw_smem;
    if (d.prec)
        bk_solve_kernel<float><<<ctas, SW_NT, smem, (cudaStream_t)stream>>>(d, s, nrhs, b, ldb, x, ldx, epoch, budget, Pin,
                                                                        Qout);
    else
        bk_solve_kernel<double><<<ctas, SW_NT, smem, (cudaStream_t)stream>>>(d, s, nrhs, b, ldb, x, ldx, epoch, budget, Pin,
                                                                         Qout);
}
