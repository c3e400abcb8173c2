// kernels_dd.cu -- the rounds of a refactorization after the stored-pattern pass.
//
// The stored-pattern pass computes every column with the previous pivots and
// flags the columns whose preferred pivot Algorithm 1's pivot selection would
// reject.  Within a task (BTF block or ND node) everything before the first such
// column f is exact.  A round then processes each active task from its start
// column s (one warp per column, claimed in ascending order within a task, the
// tasks interleaved; flags per column):
//   * resolve (s = f): column s is recomputed by the reach of Algorithm 1 and
//     takes the pivot the selection rule gives; its previous and new pivot rows
//     are marked "touched" in this round;
//   * every other column is classified from its stored pattern: kept if no row of
//     it was touched and none of its stored steps was recomputed (in this round,
//     or, in a separator's first round, anywhere below it during this
//     refactorization) and it had not rejected its pivot; recomputed on its
//     stored pattern if only values can differ (a step was recomputed with an
//     unchanged pattern, or it rejected its pivot); recomputed by the reach if
//     a row was touched or a step's pattern may have changed;
//   * a recomputed column (other than the resolve column) keeps its previous
//     pivot if the selection rule still accepts it; otherwise it is flagged and
//     the next round resolves the task's first flagged column.
// Recomputation uses the reach over the task's whole space (descendant steps and
// own steps, ascending; own steps of this round are waited for), with a row
// counted as pivoted at column c when 0 <= pinv[row] < c.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "basker_internal.h"
#include "column_static.cuh"
#include "device_util.cuh"
#include "trace.cuh"

using namespace bk;

// Per-column phase clocks of the reach path, kept only in trace builds: the
// cycles from the last wait to the end of the step loop, of the pivot selection,
// of the L write and of the epilogue, and the cycles spent waiting.
#ifdef BK_TRACE
#define DD_CLK(v) v = clock64()
#else
#define DD_CLK(v)
#endif

namespace {

__device__ __forceinline__ void set_bit(volatile uint32_t *bm, int i)
{
    atomicOr(const_cast<uint32_t *>(bm) + (i >> 5), 1u << (i & 31));
}

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

// Bounded wait of one lane on a flag; false if the budget ran out (or another
// warp already gave up).  dist: how many columns the waiting column lies past
// the one it waits for.  Along a chain of columns, every column still to come
// polls the flag of the chain's head; the far ones poll it less often (their
// wait is about dist links long), which keeps the head's flag from being the
// point every waiter's requests queue at.
__device__ __forceinline__ bool lane_wait(const bk_dev &d, const int *flag, int epoch, long long budget, int dist = 1)
{
    if (ld_relaxed(flag) != epoch) {
        const unsigned nap = (unsigned)min(max(dist, 1), 32) * 32u;
        const long long t0 = clock64();
        while (ld_relaxed(flag) != epoch) {
            if (*reinterpret_cast<const volatile int *>(&d.status->timeout) || clock64() - t0 > budget) {
                atomicExch(&d.status->timeout, 1);
                return false;
            }
            __nanosleep(nap);
        }
    }
    fence_acquire();
    return true;
}

// Row slots of the pattern, listed in ascending order: one segment of set bits
// of rb starting at word wcur (advanced past the words listed).  A segment holds
// whole groups of 32 words, at most RLIST slots; 32 words hold at most RLIST.
// A lane lists the bits of its own word when they are few; words with more than
// LIST_DENSE bits (the runs of consecutive rows a separator brings) are listed by
// the whole warp, one word at a time, one bit a lane.  Either way a slot's
// position is its word's offset plus its rank in the word.
constexpr int RLIST = 1024;
constexpr int RL_PF = 8;
constexpr int LIST_DENSE = 8;

__device__ __forceinline__ int build_list(const volatile uint32_t *rb, int nrw, int &wcur, int *list, int lane)
{
    int filled = 0;
    const uint32_t below = (1u << lane) - 1u;
    while (wcur < nrw) {
        const int w = wcur + lane;
        const uint32_t bits = w < nrw ? rb[w] : 0u;
        if (!__any_sync(BK_FULL, bits != 0u)) {      // 32 empty words: nothing to list
            wcur += 32;
            continue;
        }
        const int cnt = __popc(bits);
        const int pre = warp_exscan(cnt, lane);
        const int tot = __shfl_sync(BK_FULL, pre + cnt, 31);
        if (filled + tot > RLIST) break;
        const int q0 = filled + pre;
        uint32_t mine = cnt > LIST_DENSE ? 0u : bits;
        int q = q0;
        while (mine) {
            const int b = __ffs(mine) - 1;
            mine &= mine - 1;
            list[q++] = (w << 5) + b;
        }
        uint32_t dense = __ballot_sync(BK_FULL, cnt > LIST_DENSE);
        while (dense) {
            const int src = __ffs(dense) - 1;
            dense &= dense - 1;
            const uint32_t bw = __shfl_sync(BK_FULL, bits, src);
            const int qb = __shfl_sync(BK_FULL, q0, src);
            if ((bw >> lane) & 1u) list[qb + __popc(bw & below)] = ((wcur + src) << 5) + lane;
        }
        filled += tot;
        wcur += 32;
    }
    __syncwarp();
    return filled;
}

// One step of the reach, read ahead: its pivot slot, L(:,j)'s extent, and the
// first RSTEP_PF * 32 entries of L(:,j) with their slots, values and what each
// row adds (a step bit >= 0, a row bit encoded -2 - bit, or -1).  Entries are
// read only when column j is final in this round (full); pinv of the rows is
// final for every column after the round's resolve column.
constexpr int RSTEP_PF = 4;
template <typename V>
struct RStep {
    int sp, jc, why;
    int64_t jl;
    bool full;
    int s[RSTEP_PF], bit[RSTEP_PF];
    V l[RSTEP_PF];
};

template <typename V>
__device__ __forceinline__ void read_step(const bk_dev &d, const bk_task &T, RStep<V> &st, int j, int c, int s0,
                                          int epoch, int lane, int ndesc, bool after_wait = false)
{
    const int base = T.sp_lo;
    const bool inround = j >= s0 && j < T.hi;
    int dn = 1;
    if (inround && !after_wait) {
        dn = 0;
        if (lane == 0 && ld_relaxed(d.done + j) == epoch) {
            fence_acquire();
            dn = 1;
        }
        dn = __shfl_sync(BK_FULL, dn, 0);
    }
    // after the wait, L(:,j)'s entries are read where the extent read before the
    // wait put them, together with the extent itself (one round trip instead of
    // two); entries the final extent places elsewhere are read again
    int rg[RSTEP_PF];
    V lg[RSTEP_PF];
    const int64_t jl_g = st.jl;
    const int jc_g = after_wait ? st.jc : 0;
#pragma unroll
    for (int u = 0; u < RSTEP_PF; u++) {
        const int q = lane + 32 * u;
        rg[u] = q < jc_g ? __ldcg(d.Li + jl_g + q) : -1;
        lg[u] = q < jc_g ? __ldcg(vals<V>(d.Lx) + jl_g + q) : V(0);
    }
    st.sp = slot_of(T, base, __ldcg(d.prow + j));
    st.jl = __ldcg(d.Lbeg + j);
    st.jc = __ldcg(d.Lcnt + j);
    st.full = dn != 0;
    st.why = 0;
    const bool moved = st.jl != jl_g;
#pragma unroll
    for (int u = 0; u < RSTEP_PF; u++) {
        const int q = lane + 32 * u;
        st.s[u] = -1;
        st.bit[u] = -1;
        st.l[u] = 0.0;
        if (!dn || q >= st.jc) continue;
        const bool have = !moved && q < jc_g;
        const int r = have ? rg[u] : __ldcg(d.Li + st.jl + q);
        st.l[u] = have ? lg[u] : __ldcg(vals<V>(d.Lx) + st.jl + q);
        const int s = slot_of(T, base, r);
        if (s < 0) { st.why = 65; continue; }
        st.s[u] = s;
        const int p = s < T.hi - base ? __ldcg(d.pinv + r) : -1;
        if (p >= 0 && p < c) {
            if (p > j) st.bit[u] = p - base;
            else st.why = 66;
        } else if (s >= ndesc) {
            st.bit[u] = -2 - (s - ndesc);
        } else {
            st.why = 67;
        }
    }
}

// A step waited for: L(:,j) copied into the warp's staging area in shared
// memory (16-byte copies at L2 only, from the 16-byte boundary below the column;
// the arrays carry 16 bytes of padding), started where the extent read before
// the wait puts it while the extent itself is read again; then the rows' slots
// and, for rows of the node, the steps that pivot them, read with the x values
// under the rows, RS_PF entries a lane in flight.  Each entry leaves its slot in
// srow, what it adds in sadd (a step bit >= 0, a row bit encoded -2 - bit, or -1)
// and x at its slot in sxv.  Returns the number of entries,
// or -1 when L(:,j) has more than BK_DD_SCAP entries (read the usual way).
constexpr int RS_PF = 8;

__device__ __forceinline__ void dd_cp16(void *dst, const void *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void dd_cp_wait()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ int stage_range(T *dst, const T *src, int64_t e0, int cnt, int lane)
{
    constexpr int per = 16 / (int)sizeof(T);
    const int64_t a0 = e0 & ~(int64_t)(per - 1);
    const int off = (int)(e0 - a0);
    const int chunks = (off + cnt + per - 1) / per;
    for (int k = lane; k < chunks; k += 32) dd_cp16(dst + k * per, src + a0 + (int64_t)k * per);
    return off;
}

// The rows rows[ro + q], q < n, of L(:,j): each one's slot (sslot), what it
// adds to the reach (sadd) and x at its slot (sxv), RS_PF rows a lane at a time
// (their pivot steps and x values read together).
template <typename V>
__device__ __forceinline__ void classify_rows(const bk_dev &d, const bk_task &T, int j, int c, int ndesc, const V *x,
                                              const int *rows, int ro, int n, int *sslot, int *sadd, V *sxv,
                                              int &why, int lane)
{
    const int base = T.sp_lo;
    for (int q0 = 0; q0 < n; q0 += 32 * RS_PF) {
        int rr[RS_PF], sl[RS_PF], pp[RS_PF];
        V xv[RS_PF];
#pragma unroll
        for (int u = 0; u < RS_PF; u++) {
            const int q = q0 + lane + 32 * u;
            rr[u] = q < n ? rows[ro + q] : -1;
            sl[u] = rr[u] >= 0 ? slot_of(T, base, rr[u]) : -1;
            pp[u] = (sl[u] >= 0 && sl[u] < T.hi - base) ? __ldcg(d.pinv + rr[u]) : -1;
            xv[u] = sl[u] >= 0 ? x[sl[u]] : V(0);
        }
#pragma unroll
        for (int u = 0; u < RS_PF; u++) {
            const int q = q0 + lane + 32 * u;
            if (q >= n) continue;
            int add = -1;
            if (sl[u] < 0) {
                if (!why) why = 65;
            } else if (pp[u] >= 0 && pp[u] < c) {
                if (pp[u] > j) add = pp[u] - base;
                else if (!why) why = 66;
            } else if (sl[u] >= ndesc) {
                add = -2 - (sl[u] - ndesc);
            } else if (!why) {
                why = 67;
            }
            sslot[q] = sl[u];
            sadd[q] = add;
            sxv[q] = xv[u];
        }
    }
    __syncwarp();
}

// Before waiting for step j: its rows where the extent read earlier puts them
// (a guess: the step may still change them) into sgr, classified into sslot,
// sadd and sxv while the wait goes on.  x is final for step j already (every
// earlier step is applied).  Returns the offset of the first row in sgr, or -1
// when the guess is not usable.
template <typename V>
__device__ __forceinline__ int prestage_step(const bk_dev &d, const bk_task &T, const RStep<V> &st, int j, int c,
                                             int ndesc, const V *x, int *sgr, int *sslot, int *sadd, V *sxv,
                                             int &why_pre, int lane)
{
    if (st.jc < 0 || st.jc > BK_DD_SCAP || st.jl < 0 || st.jl + st.jc > d.lpool_end) return -1;
    const int go = stage_range(sgr, d.Li, st.jl, st.jc, lane);
    dd_cp_wait();
    __syncwarp();
    classify_rows(d, T, j, c, ndesc, x, sgr, go, st.jc, sslot, sadd, sxv, why_pre, lane);
    return go;
}

// After the wait: L(:,j)'s rows and values copied again, with its extent read
// again (one round trip); when the extent is the guessed one and the rows are
// the prestaged rows, their classification stands; otherwise the rows are
// classified now.  Returns the number of entries, or -1 when L(:,j) has more
// than BK_DD_SCAP entries (read the usual way).
template <typename V>
__device__ __forceinline__ int stage_step(const bk_dev &d, const bk_task &T, RStep<V> &st, int j, int c, int lane,
                                          int ndesc, const V *x, int *srow, V *sval, int *sadd, V *sxv, int *sslot,
                                          const int *sgr, int go, int why_pre, int &vo, int &why)
{
    const int base = T.sp_lo;
    const V *const Lx = vals<V>(d.Lx);
    if (st.jc > BK_DD_SCAP) return -1;
    // the extent read before the wait is a guess (its two words may come from
    // either side of a move of the column): copied only inside the arrays
    const bool guess = st.jl >= 0 && st.jc >= 0 && st.jl + st.jc <= d.lpool_end;
    int ro = 0;
    if (guess) {
        ro = stage_range(srow, d.Li, st.jl, st.jc, lane);
        vo = stage_range(sval, Lx, st.jl, st.jc, lane);
    }
    const int pr = __ldcg(d.prow + j);
    const int64_t jl = __ldcg(d.Lbeg + j);
    const int jc = __ldcg(d.Lcnt + j);
    dd_cp_wait();
    const bool kept = go >= 0 && guess && jl == st.jl && jc == st.jc;
    if (!guess || jl != st.jl || jc > st.jc) {
        st.jl = jl;
        st.jc = jc;
        if (jc > BK_DD_SCAP || jl < 0 || jl + jc > d.lpool_end) return -1;
        __syncwarp();
        ro = stage_range(srow, d.Li, jl, jc, lane);
        vo = stage_range(sval, Lx, jl, jc, lane);
        dd_cp_wait();
    }
    st.jl = jl;
    st.jc = jc;
    st.sp = slot_of(T, base, pr);
    __syncwarp();
    bool same = kept;
    if (kept)
        for (int q = lane; q < jc; q += 32)
            if (srow[ro + q] != sgr[go + q]) same = false;
    if (__all_sync(BK_FULL, same)) {
        if (!why) why = why_pre;
        return jc;
    }
    classify_rows(d, T, j, c, ndesc, x, srow, ro, jc, sslot, sadd, sxv, why, lane);
    return jc;
}

template <typename V>
__global__ void __launch_bounds__(128) bk_dd_kernel(bk_dev d, const int32_t *__restrict__ cols, int32_t ncols,
                                                    int32_t *counter, double tau, int32_t epoch, long long budget,
                                                    int32_t refno)
{
    const V *const Bx = vals<V>(d.Bx);
    V *const Lx = vals<V>(d.Lx);
    V *const Ux = vals<V>(d.Ux);
    __shared__ bk_task Ts[4];
    __shared__ int rlist[4 * RLIST];
    extern __shared__ __align__(16) uint32_t dd_bits[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * 4 + wib;
    if (gw >= d.wsd_warps) return;
    bk_task &T = Ts[wib];
    unsigned char *slice = d.wsd + (int64_t)gw * d.wsd_slice;
    // the reach's bitmaps, when they fit in shared memory; zero between columns
    uint32_t *wbits = dd_bits + (int64_t)wib * d.dd_words;
    for (int i = lane; i < d.dd_words; i += 32) wbits[i] = 0u;
    // the staging area of a waited-for step (rows, values, what each row adds)
    unsigned char *const stg = reinterpret_cast<unsigned char *>(dd_bits + 4 * (int64_t)d.dd_words) +
                               (int64_t)wib * BK_DD_STAGE_BYTES;
    int *const srow = reinterpret_cast<int *>(stg);
    V *const sval = reinterpret_cast<V *>(stg + (BK_DD_SCAP + 16) * 4);
    int *const sadd = reinterpret_cast<int *>(stg + (BK_DD_SCAP + 16) * 12);
    V *const sxv = reinterpret_cast<V *>(stg + (BK_DD_SCAP + 16) * 12 + BK_DD_SCAP * 4);
    int *const sold = reinterpret_cast<int *>(stg + (BK_DD_SCAP + 16) * 12 + BK_DD_SCAP * 12);
    int *const sgr = sold + (BK_DD_SCAP + 16);
    int *const sslot = sgr + (BK_DD_SCAP + 16);

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
        if (__shfl_sync(BK_FULL, (int)should_stop(d, tid, c), 0)) {
            if (lane == 0) st_release(d.done + c, epoch);
            continue;
        }
        if (tid != cur_task) {
            load_task(T, d.tasks + tid, lane);
            cur_task = tid;
        }
        const int s0 = d.dd_start[tid];
        const int fl = d.dd_flags[tid];
        const bool resolve = (fl & BK_DD_RESOLVE) && c == s0;
        // the resolve column's touched rows must be visible before deciding
        if ((fl & BK_DD_RESOLVE) && c > s0) {
            int ok = lane == 0 ? (int)lane_wait(d, d.done + s0, epoch, budget, c - s0) : 1;
            if (!__shfl_sync(BK_FULL, ok, 0)) return;
        }
        int64_t ub = d.Ubeg[c], ue = d.Uend[c];
        int64_t lb = d.Lbeg[c], le = d.Lend[c];
        // A column is kept (resolve rounds), recomputed on its stored pattern, or
        // recomputed by the reach when its pattern may change: a row of it was
        // touched (this round; or, in a separator's first round, anywhere below
        // during this refactorization), or one of its steps was recomputed by the
        // reach (checked as the steps are reached).
        int mode = resolve ? 2 : ((fl & BK_DD_DESC) ? 1 : 0);
        if (!resolve) {
            if (lane == 0) {
                const int r = d.prow[c];
                if (__ldcg(d.touch + r) == epoch) mode = 2;
                if ((fl & BK_DD_DESC) && __ldcg(d.touch_ref + r) == refno) mode = 2;
            }
            const int uc = d.Ucnt[c];
            for (int q = lane; q < uc - 1; q += 32) {
                const int j = d.Ui[ub + q];
                const int r = __ldcg(d.prow + j);
                if (__ldcg(d.touch + r) == epoch) mode = 2;
                if ((fl & BK_DD_DESC) && (__ldcg(d.touch_ref + r) == refno ||
                                          (d.col_task[j] != tid && __ldcg(d.pchg_ref + j) == refno)))
                    mode = 2;
            }
            const int lc = d.Lcnt[c];
            for (int q = lane; q < lc; q += 32) {
                const int r = d.Li[lb + q];
                if (__ldcg(d.touch + r) == epoch) mode = 2;
                if ((fl & BK_DD_DESC) && __ldcg(d.touch_ref + r) == refno) mode = 2;
            }
            mode = warp_max_i(mode);
            // a column that rejected its pivot in the previous round is revalidated
            if (mode == 0 && __shfl_sync(BK_FULL, lane == 0 ? d.col_fail[c] : 0, 0)) mode = 1;
            if (mode == 0 && (fl & BK_DD_RESOLVE)) {
                // keep the column unless a step of it recomputed in this round; its
                // steps are examined lowest first, deciding at the first done step
                // that was recomputed, waiting only for the lowest unfinished one
                int verdict = 0;                      // 0 keep, 1 stored pattern, 2 reach
                for (int k0 = 0; k0 < uc - 1 && verdict == 0; k0 += 32) {
                    const int q = k0 + lane;
                    int j = -1;
                    if (q < uc - 1) {
                        const int jj = d.Ui[ub + q];
                        if (jj >= s0 && jj < c && d.col_task[jj] == tid) j = jj;
                    }
                    uint32_t todo = __ballot_sync(BK_FULL, j >= 0);
                    while (todo && verdict == 0) {
                        bool done = false;
                        int v = 0;
                        if ((todo >> lane) & 1u) {
                            done = ld_relaxed(d.done + j) == epoch;
                            if (done) fence_acquire();
                            if (done) v = __ldcg(d.pchg_ep + j) == epoch ? 2 : (__ldcg(d.dirty_ep + j) == epoch ? 1 : 0);
                        }
                        verdict = warp_max_i(v);
                        if (verdict) break;
                        todo &= ~__ballot_sync(BK_FULL, done);
                        if (todo) {
                            const int first = __ffs(todo) - 1;
                            const int jw = __shfl_sync(BK_FULL, j, first);
                            int okw = lane == 0 ? (int)lane_wait(d, d.done + jw, epoch, budget, c - jw) : 1;
                            if (!__shfl_sync(BK_FULL, okw, 0)) return;
                        }
                    }
                }
                mode = verdict;
                if (mode == 0) {
                    __syncwarp();
                    if (lane == 0) {
                        st_release(d.done + c, epoch);
                        BK_TREC(d.trace, BK_TR_ROUND, 0, c, t0);
                    }
                    continue;
                }
            }
            if (mode == 1) {
                bool ok = false, bad = false, broken = false, aborted = false;
                V *xs = reinterpret_cast<V *>(slice);
                if (!pattern_column(d, T, tid, xs, c, epoch, budget, tau, lane, false, s0, ok, bad, broken,
                                   d.pchg_ep, &aborted))
                    return;
                if (!aborted) {
                    __syncwarp();
                    if (lane == 0) {
                        if (broken) report_internal(d.status, c, 68);
                        d.col_fail[c] = ok ? 0 : 1;
                        if (!ok) atomicMin(d.task_fail + tid, c);
                        d.dirty_ep[c] = epoch;
                        d.dirty_ref[c] = refno;
                        __threadfence();
                        st_release(d.done + c, epoch);
                        BK_TREC(d.trace, BK_TR_ROUND, 1, c, t0);
                    }
                    __syncwarp();
                    if (broken) return;
                    continue;
                }
            }
        }

        // ---- recompute column c by the reach over the task's space
        const int base = T.sp_lo;
        const int nsteps = T.hi - T.sp_lo;
        const int ndesc = T.lo - T.sp_lo;
        const int nown = T.hi - T.lo;
        const int lsp = T.lspace;
        const int nsw = (nsteps + 31) >> 5;
        const int nrw = (lsp + 31) >> 5;
        V *x = reinterpret_cast<V *>(slice);
        volatile uint32_t *sb = d.dd_words ? wbits : reinterpret_cast<uint32_t *>(x + T.space);
        volatile uint32_t *rb = sb + nsw;
        bool bad = false, overflow = false;
        int why = 0;
        int nu = 0;
        // the stored pattern, to tell whether the recomputed one differs
        const int old_uc = d.Ucnt[c], old_lc = d.Lcnt[c];
        const int64_t old_ub = ub, old_lb = lb;
        bool same = true;
        // the column's previous L rows, copied on chip while the steps run (the L
        // write compares the new rows with them)
        int so_old = -1;
        if (old_lc <= BK_DD_SCAP && old_lb >= 0 && old_lb + old_lc <= d.lpool_end) {
            so_old = stage_range(sold, d.Li, old_lb, old_lc, lane);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        auto old_row = [&](int64_t q) -> int { return so_old >= 0 ? sold[so_old + (int)(q - old_lb)] : d.Li[q]; };

        const int e1 = d.Bp[c + 1];
        for (int e = d.dstart[c] + lane; e < e1; e += 32) {
            const int r = d.Bi[e];
            const int s = slot_of(T, base, r);
            if (s < 0) { if (!why) why = 61; continue; }
            x[s] = Bx[e];
            const int p = s < T.hi - base ? __ldcg(d.pinv + r) : -1;
            if (p >= 0 && p < c && p >= base) set_bit(sb, p - base);
            else if (s >= ndesc) set_bit(rb, s - ndesc);
            else if (!why) why = 62;                 // a descendant row is always pivoted
        }
        __syncwarp();
        // Steps in ascending order: the lowest set bit of sb.  The step after the
        // current one is predicted (the lowest set bit once the current one is
        // cleared) and its data read while the current step is applied; a step
        // that the current one adds below the prediction is read when it is found.
#ifdef BK_TRACE
        long long ck_wait = 0, ck_last = 0, ck_a = 0, ck_b = 0, ck_c = 0, ck_stg = 0, ck_app = 0;
        int steps_after = 0;
#endif
        DD_CLK(ck_last);
        int w0 = 0;
        int jb = next_step_bit(sb, nsw, w0, lane);
        RStep<V> cur, nxt;
        if (jb >= 0) read_step(d, T, cur, base + jb, c, s0, epoch, lane, ndesc);
        for (int iter = 0; jb >= 0; iter++) {
            const int j = base + jb;
            int nstaged = -1, so_v = 0;
            if (iter > nsteps || j >= c) { if (!why) why = 63; break; }
            if (lane == 0) atomicAnd(const_cast<uint32_t *>(sb) + (jb >> 5), ~(1u << (jb & 31)));
            __syncwarp();
            int wp = w0;
            const int jbp = next_step_bit(sb, nsw, wp, lane);
            if (jbp >= 0 && base + jbp < c) read_step(d, T, nxt, base + jbp, c, s0, epoch, lane, ndesc);
            if (!cur.full) {
#ifdef BK_TRACE
                const long long cw0 = clock64();
#endif
                // a step still being computed: its rows prestaged while it runs
                int set = 0;
                if (lane == 0) set = ld_relaxed(d.done + j) == epoch;
                set = __shfl_sync(BK_FULL, set, 0);
                int go = -1, why_pre = 0;
                if (!set) go = prestage_step(d, T, cur, j, c, ndesc, x, sgr, sslot, sadd, sxv, why_pre, lane);
                int ok = 1;
                if (lane == 0) {
                    if (set) fence_acquire();
                    else ok = (int)lane_wait(d, d.done + j, epoch, budget, c - j);
                }
                if (!__shfl_sync(BK_FULL, ok, 0)) {
                    asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy left in flight
                    return;
                }
                DD_CLK(ck_last);
#ifdef BK_TRACE
                ck_wait += ck_last - cw0;
#endif
                nstaged = stage_step(d, T, cur, j, c, lane, ndesc, x, srow, sval, sadd, sxv, sslot, sgr, go, why_pre,
                                     so_v, why);
#ifdef BK_TRACE
                ck_stg = clock64() - ck_last;
                steps_after = 0;
#endif
                if (nstaged < 0) {
                    read_step(d, T, cur, j, c, s0, epoch, lane, ndesc, true);
                } else {
                    cur.full = true;
                    cur.why = 0;
                    cur.jc = 0;          // the entries are applied from the staging area
#pragma unroll
                    for (int u = 0; u < RSTEP_PF; u++) cur.s[u] = -1;
                }
            }
            const int sp = cur.sp;
            if (sp < 0) { if (!why) why = 64; break; }
            const V m = x[sp];
            V xv[RSTEP_PF];
#pragma unroll
            for (int u = 0; u < RSTEP_PF; u++) xv[u] = cur.s[u] >= 0 ? x[cur.s[u]] : 0.0;
            const int oldu = (lane == 0 && ub == old_ub && nu < old_uc - 1) ? d.Ui[ub + nu] : -1;
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
                    for (int q = lane; q < nu; q += 32) {
                        d.Ui[nb + q] = d.Ui[ub + q];
                        Ux[nb + q] = Ux[ub + q];
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
#pragma unroll
            for (int u = 0; u < RSTEP_PF; u++) {
                if (cur.s[u] < 0) continue;
                x[cur.s[u]] = fma(-cur.l[u], m, xv[u]);
                if (cur.bit[u] >= 0) set_bit(sb, cur.bit[u]);
                else if (cur.bit[u] <= -2) set_bit(rb, -2 - cur.bit[u]);
            }
            if (cur.why && !why) why = cur.why;
            // entries past the read-ahead window, RSTEP_PF a lane at a time: their
            // rows, values, x and pinv loads issued together (the rows of L(:,j)
            // are distinct, so the batch's updates do not alias)
            for (int q0 = 32 * RSTEP_PF; q0 < cur.jc; q0 += 32 * RSTEP_PF) {
                int rq[RSTEP_PF], sq[RSTEP_PF], pq[RSTEP_PF];
                V lq[RSTEP_PF], xq[RSTEP_PF];
#pragma unroll
                for (int u = 0; u < RSTEP_PF; u++) {
                    const int q = q0 + lane + 32 * u;
                    rq[u] = q < cur.jc ? __ldcg(d.Li + cur.jl + q) : -1;
                    lq[u] = q < cur.jc ? __ldcg(Lx + cur.jl + q) : V(0);
                }
#pragma unroll
                for (int u = 0; u < RSTEP_PF; u++) {
                    sq[u] = rq[u] >= 0 ? slot_of(T, base, rq[u]) : -1;
                    if (rq[u] >= 0 && sq[u] < 0 && !why) why = 65;
                    pq[u] = (sq[u] >= 0 && sq[u] < T.hi - base) ? __ldcg(d.pinv + rq[u]) : -1;
                    xq[u] = sq[u] >= 0 ? x[sq[u]] : V(0);
                }
#pragma unroll
                for (int u = 0; u < RSTEP_PF; u++) {
                    if (sq[u] < 0) continue;
                    x[sq[u]] = fma(-lq[u], m, xq[u]);
                    const int p = pq[u];
                    if (p >= 0 && p < c) {
                        if (p > j) set_bit(sb, p - base);
                        else if (!why) why = 66;
                    } else if (sq[u] >= ndesc) {
                        set_bit(rb, sq[u] - ndesc);
                    } else if (!why) {
                        why = 67;
                    }
                }
            }
            // the staged entries
#ifdef BK_TRACE
            const long long ck_ap0 = clock64();
            steps_after++;
#endif
            for (int q0 = 0; q0 < nstaged; q0 += 32 * RSTEP_PF) {
                int sq[RSTEP_PF], aq[RSTEP_PF];
                V lq[RSTEP_PF], xq[RSTEP_PF];
#pragma unroll
                for (int u = 0; u < RSTEP_PF; u++) {
                    const int q = q0 + lane + 32 * u;
                    sq[u] = q < nstaged ? sslot[q] : -1;
                    lq[u] = q < nstaged ? sval[so_v + q] : V(0);
                    aq[u] = q < nstaged ? sadd[q] : -1;
                    xq[u] = q < nstaged ? sxv[q] : V(0);
                }
#pragma unroll
                for (int u = 0; u < RSTEP_PF; u++) {
                    if (sq[u] < 0) continue;
                    x[sq[u]] = fma(-lq[u], m, xq[u]);
                    if (aq[u] >= 0) set_bit(sb, aq[u]);
                    else if (aq[u] <= -2) set_bit(rb, -2 - aq[u]);
                }
            }
#ifdef BK_TRACE
            if (nstaged >= 0) ck_app = clock64() - ck_ap0;
#endif
            if (lane == 0 && oldu != j) same = false;
            nu++;
            __syncwarp();
            jb = next_step_bit(sb, nsw, w0, lane);
            if (jb >= 0) {
                if (jb == jbp) cur = nxt;
                else read_step(d, T, cur, base + jb, c, s0, epoch, lane, ndesc);
            }
        }
        why = warp_max_i(why);
        DD_CLK(ck_a);
        // Algorithm 1's pivot selection among the node's unpivoted rows.  The
        // pattern's row slots are listed in ascending order, a segment of at most
        // RLIST at a time, and their values read eight per lane at once.
        int *list = rlist + wib * RLIST;
        unsigned long long km = 0;          // largest own magnitude, as a key
        int ncand = 0, nrows = 0, nseg = 0;
        const int pcur = __ldcg(d.prow + c);
        auto in_pattern = [&](int r) -> bool {
            const int ls = r - T.lo;
            return (unsigned)ls < (unsigned)nown && ((rb[ls >> 5] >> (ls & 31)) & 1u);
        };
        // L(:,c) goes to its region, or to a larger one from the pool
        auto place_l = [&](int cnt_all) {
            if (!overflow && lb + cnt_all > le) {
                const int64_t cap = max((long long)cnt_all,
                                        min((long long)(2 * (int64_t)cnt_all + 16),
                                            (long long)((T.hi - c - 1) + (lsp - nown))));
                int64_t nb = 0;
                if (lane == 0) nb = pool_alloc(d.pool, d.lpool_end, cap);
                nb = __shfl_sync(BK_FULL, nb, 0);
                if (nb < 0) {
                    overflow = true;
                } else {
                    lb = nb;
                    le = nb + cap;
                    if (lane == 0) {
                        d.Lbeg[c] = lb;
                        d.Lend[c] = le;
                    }
                }
            }
            if (lb + cnt_all > le) overflow = true;
        };
        if (so_old >= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
        int wfirst = 0;
        const int filled0 = build_list(rb, nrw, wfirst, list, lane);
        int piv = -1;
        bool ok = false;
        int pls = 0;
        bool pin = false;
        V xp = V(0);
        if (!resolve && wfirst >= nrw) {
            // every column but the round's resolve column keeps its pivot row, so
            // with the pattern listed in one segment the selection's check and the
            // L write share one pass over the values
            nrows = filled0;
            piv = pcur;
            pls = piv - T.lo;
            pin = in_pattern(piv);
            xp = pin ? x[ndesc + pls] : V(0);
            DD_CLK(ck_b);
            place_l(nrows - (pin ? 1 : 0));
            for (int i0 = 0; i0 < nrows; i0 += 32 * RL_PF) {
                int ls[RL_PF], oldr[RL_PF];
                int64_t qq[RL_PF];
                V v[RL_PF];
#pragma unroll
                for (int u = 0; u < RL_PF; u++) {
                    const int i = i0 + lane + 32 * u;
                    ls[u] = i < nrows ? list[i] : -1;
                    const bool isp = pin && ls[u] == pls;
                    qq[u] = lb + i - ((pin && ls[u] > pls) ? 1 : 0);
                    v[u] = ls[u] >= 0 ? x[ndesc + ls[u]] : V(0);
                    oldr[u] = (ls[u] >= 0 && !isp && !overflow && lb == old_lb && qq[u] - lb < old_lc) ? old_row(qq[u])
                                                                                                      : -1;
                }
#pragma unroll
                for (int u = 0; u < RL_PF; u++) {
                    if (ls[u] < 0) continue;
                    if (!isfinite(v[u])) bad = true;
                    if (ls[u] < nown) {
                        ncand++;
                        km = key_max(km, mag_key(v[u]));
                    }
                    if (pin && ls[u] == pls) continue;            // the pivot row: cleared below
                    if (!overflow) {
                        const int r = row_of_lslot(T, ls[u]);
                        if (oldr[u] != r) same = false;
                        d.Li[qq[u]] = r;
                        Lx[qq[u]] = v[u] / xp;
                    }
                    x[ndesc + ls[u]] = 0.0;
                }
            }
            __syncwarp();
            km = warp_max_key(km);
            const V amax = key_value<V>(km);
            ncand = warp_sum(ncand);
            bad = __any_sync(BK_FULL, bad);
            ok = !bad && ncand > 0 && amax > 0.0 && pin && (double)fabs(xp) >= tau * (double)amax;
        } else {
            int wcur = wfirst, filled = filled0;
            for (;;) {
                nrows += filled;
                nseg++;
                for (int i0 = 0; i0 < filled; i0 += 32 * RL_PF) {
                    int ls[RL_PF];
                    V v[RL_PF];
#pragma unroll
                    for (int u = 0; u < RL_PF; u++) {
                        const int i = i0 + lane + 32 * u;
                        ls[u] = i < filled ? list[i] : -1;
                        v[u] = ls[u] >= 0 ? x[ndesc + ls[u]] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < RL_PF; u++) {
                        if (ls[u] < 0) continue;
                        if (!isfinite(v[u])) bad = true;
                        if (ls[u] < nown) {
                            ncand++;
                            km = key_max(km, mag_key(v[u]));
                        }
                    }
                }
                __syncwarp();
                if (wcur >= nrw) break;
                filled = build_list(rb, nrw, wcur, list, lane);
            }
            km = warp_max_key(km);
            const V amax = key_value<V>(km);
            ncand = warp_sum(ncand);
            bad = __any_sync(BK_FULL, bad);
            const int pref = resolve ? d.pref[c] : pcur;
            if (!bad && ncand > 0 && amax > 0.0) {
                if (in_pattern(pref) && (double)fabs(x[ndesc + pref - T.lo]) >= tau * (double)amax) {
                    piv = pref;
                    ok = true;
                } else if (resolve) {
                    // the lowest own row reaching the maximum (the list is rebuilt over
                    // the own rows: the L write below lists the pattern again)
                    nseg = 0;
                    int best = INT_MAX;
                    const int nw_own = (nown + 31) >> 5;
                    for (int wc = 0; wc < nw_own && best == INT_MAX;) {
                        const int fo = build_list(rb, nw_own, wc, list, lane);
                        for (int i0 = 0; i0 < fo; i0 += 32 * RL_PF) {
                            int ls[RL_PF];
                            V v[RL_PF];
#pragma unroll
                            for (int u = 0; u < RL_PF; u++) {
                                const int i = i0 + lane + 32 * u;
                                ls[u] = i < fo ? list[i] : -1;
                                v[u] = ls[u] >= 0 ? x[ndesc + ls[u]] : 0.0;
                            }
#pragma unroll
                            for (int u = 0; u < RL_PF; u++)
                                if (ls[u] >= 0 && ls[u] < nown && mag_key(v[u]) == km) best = min(best, ls[u]);
                        }
                        best = warp_min(best);
                        __syncwarp();
                    }
                    piv = T.lo + best;
                    ok = true;
                }
            }
            if (resolve && piv < 0) {
                // no acceptable pivot at an exact column: the matrix is singular here
                if (lane == 0) report_fail(d.status, c, bad ? BK_CODE_NAN : BK_CODE_SINGULAR);
            }
            if (piv < 0) piv = pcur;                     // keep the speculation consistent
            DD_CLK(ck_b);
            pls = piv - T.lo;
            pin = in_pattern(piv);
            xp = pin ? x[ndesc + pls] : 0.0;
            // L(:,c) = x / pivot over the pattern's unpivoted rows; clear the state
            place_l(nrows - (pin ? 1 : 0));
            int rank0 = 0;
            // a pattern listed in one segment by the selection above is still listed
            const bool listed = nseg == 1;
            for (int wc = 0; wc < nrw;) {
                int fl2 = nrows;
                if (listed) wc = nrw;
                else fl2 = build_list(rb, nrw, wc, list, lane);
                for (int i0 = 0; i0 < fl2; i0 += 32 * RL_PF) {
                    int ls[RL_PF], oldr[RL_PF];
                    int64_t qq[RL_PF];
                    V v[RL_PF];
#pragma unroll
                    for (int u = 0; u < RL_PF; u++) {
                        const int i = i0 + lane + 32 * u;
                        ls[u] = i < fl2 ? list[i] : -1;
                        if (ls[u] == pls && pin) ls[u] = -2;          // the pivot row: cleared below
                        qq[u] = lb + rank0 + i - ((pin && ls[u] > pls) ? 1 : 0);
                        v[u] = ls[u] >= 0 ? x[ndesc + ls[u]] : 0.0;
                        oldr[u] = (ls[u] >= 0 && !overflow && lb == old_lb && qq[u] - lb < old_lc) ? old_row(qq[u])
                                                                                                  : -1;
                    }
#pragma unroll
                    for (int u = 0; u < RL_PF; u++) {
                        if (ls[u] < 0) continue;
                        if (!overflow) {
                            const int r = row_of_lslot(T, ls[u]);
                            if (oldr[u] != r) same = false;
                            d.Li[qq[u]] = r;
                            Lx[qq[u]] = v[u] / xp;
                        }
                        x[ndesc + ls[u]] = 0.0;
                    }
                }
                rank0 += fl2;
                __syncwarp();
            }
        }
        int64_t lpos = lb;
        DD_CLK(ck_c);
        lpos = lb + nrows - (pin ? 1 : 0);
        for (int w = lane; w < nrw; w += 32) rb[w] = 0u;
        overflow = __any_sync(BK_FULL, overflow);
        same = __all_sync(BK_FULL, same) && !overflow && nu + 1 == old_uc && lpos - lb == old_lc;
        __syncwarp();
        if (lane == 0) {
            if (pin) x[ndesc + pls] = 0.0;
            if (why) report_internal(d.status, c, why);
            if (!overflow) {
                d.Ui[ub + nu] = c;
                Ux[ub + nu] = xp;
                d.Ucnt[c] = nu + 1;
                d.Lcnt[c] = (int)(lpos - lb);
            } else {
                report_overflow(d, T, tid, c, 3);
            }
            if (resolve && piv != pcur) {
                if (__ldcg(d.pinv + pcur) == c) d.pinv[pcur] = -1;
                d.pinv[piv] = c;
                d.prow[c] = piv;
                d.touch[pcur] = epoch;
                d.touch[piv] = epoch;
                d.touch_ref[pcur] = refno;
                d.touch_ref[piv] = refno;
                if (piv != c) atomicAdd(&d.status->offdiag, 1);
            }
            d.col_fail[c] = ok ? 0 : 1;
            if (!ok && !resolve) atomicMin(d.task_fail + tid, c);
            d.dirty_ep[c] = epoch;
            d.dirty_ref[c] = refno;
            // dependents take the reach only if this column's pattern or pivot changed
            if (!same || (resolve && piv != pcur)) {
                d.pchg_ep[c] = epoch;
                d.pchg_ref[c] = refno;
            }
            // the release orders this lane's writes and, through the warp barrier
            // above, the other lanes' L entries before the flag
            st_release(d.done + c, epoch);
            BK_TREC(d.trace, BK_TR_ROUND, resolve ? 3 : 2, c, t0);
#ifdef BK_TRACE
            const long long ck_d = clock64();
            bk_trace_raw(d.trace, BK_TR_PHASE, 50, c, (unsigned long long)(ck_a - ck_last),
                         (unsigned long long)(ck_b - ck_a));
            bk_trace_raw(d.trace, BK_TR_PHASE, 51, c, (unsigned long long)(ck_c - ck_b),
                         (unsigned long long)(ck_d - ck_c));
            bk_trace_raw(d.trace, BK_TR_PHASE, 52, c, (unsigned long long)ck_wait, (unsigned long long)nu);
            bk_trace_raw(d.trace, BK_TR_PHASE, 53, c, (unsigned long long)ck_stg,
                         (unsigned long long)ck_app | ((unsigned long long)steps_after << 40));
#endif
        }
        __syncwarp();
        if (why) return;      // the workspace slice may hold stale values; the host clears it
    }
}

}  // namespace

void bk_launch_dd(const bk_dev &d, const int32_t *cols, int32_t ncols, int32_t *counter, double tau,
                  int32_t epoch, long long budget, int32_t refno, void *stream, int max_warps)
{
    if (ncols <= 0) return;
    int warps = std::min<int>(ncols, max_warps > 0 ? std::min<int>(max_warps, d.wsd_warps) : d.wsd_warps);
    const size_t smem = (size_t)4 * d.dd_words * sizeof(uint32_t) + (size_t)4 * BK_DD_STAGE_BYTES;
    const int grid = (warps + 3) / 4;
    // the limit is a property of the kernel shared by every handle and thread:
    // raise it once to the largest footprint the plan allows (160 KB)
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(bk_dd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        cudaFuncSetAttribute(bk_dd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    if (d.prec)
        bk_dd_kernel<float><<<grid, 128, smem, (cudaStream_t)stream>>>(d, cols, ncols, counter, tau, epoch, budget,
                                                                        refno);
    else
        bk_dd_kernel<double><<<grid, 128, smem, (cudaStream_t)stream>>>(d, cols, ncols, counter, tau, epoch, budget,
                                                                         refno);
}
