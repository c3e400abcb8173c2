// kernels_repair.cu -- the rejected pivots of a refactorization, resolved in
// column order on the device (the matrix sequence of Sec. V, previous pivots
// preferred).
//
// The stored-pattern pass computes every column of the ND leaves and BTF blocks
// with its previous pivot and flags the columns whose pivot Algorithm 1's
// selection would reject; task_fail[t] is the first such column f of task t.
// Everything of the task before f is exact.  One warp then walks the task's
// columns c = f, f+1, ..., hi-1 in order, so that every column before c is final
// when c is examined:
//   * c is dirty if it is f, if the pass flagged it, if a step of its stored
//     U(:,c) was recomputed here, or if a row of its stored pattern (the pivot
//     rows of those steps, its own pivot row, the rows of L(:,c)) changed its
//     pivot status here.  Otherwise the pass's result for c is exact: its reach,
//     its values and its pivot are those Algorithm 1 gives, and c is kept.
//   * A dirty column is recomputed by Algorithm 1 itself: the reach of B(:,c) in
//     the graph of the final L(:, <c), the update x -= L(:,j) x(prow j) for its
//     steps in ascending order (one fma per entry), and the pivot rule (the
//     previous pivot if it is a candidate and |x| >= tau * max, else the lowest
//     candidate row holding the maximum).  A changed pivot marks both rows.
// A rejection is so resolved where it occurs, and a cascade of rejections costs
// one pass instead of one pass per rejection.  Tasks are independent (pivots are
// confined to the task), one warp each; x and the bitmaps live in shared memory
// when the task's space fits, else x lives in the warp's global workspace slice.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "basker_internal.h"
#include "column_fast.cuh"
#include "device_util.cuh"
#include "trace.cuh"

using namespace bk;

namespace {

constexpr int RP_LIST = 1024;   // row slots listed per segment
constexpr int RP_PF = 4;        // L entries per lane read ahead for the next step
constexpr int RP_RL = 8;        // listed rows per lane read at once

__device__ __forceinline__ bool get_bit(const uint32_t *bm, int i) { return (bm[i >> 5] >> (i & 31)) & 1u; }

__device__ __forceinline__ void set_bit_s(uint32_t *bm, int i) { atomicOr(bm + (i >> 5), 1u << (i & 31)); }

// Lowest set bit at or after word w0 (advanced to the word holding it), or -1.
__device__ __forceinline__ int next_bit(const volatile uint32_t *bm, int nw, int &w0, int lane)
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

// Slots of the set bits of rb from word wcur on, ascending, at most RP_LIST
// (whole groups of 32 words); wcur advances past the words listed.
__device__ __forceinline__ int list_rows(const volatile uint32_t *rb, int nrw, int &wcur, int *list, int lane)
{
    int filled = 0;
    while (wcur < nrw) {
        const int w = wcur + lane;
        uint32_t bits = w < nrw ? rb[w] : 0u;
        const int cnt = __popc(bits);
        const int pre = warp_exscan(cnt, lane);
        const int tot = __shfl_sync(BK_FULL, pre + cnt, 31);
        if (filled + tot > RP_LIST) break;
        int q = filled + pre;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            list[q++] = (w << 5) + b;
        }
        filled += tot;
        wcur += 32;
    }
    __syncwarp();
    return filled;
}

// One step of the reach, read before it is applied: the slot of its pivot row,
// L(:,j)'s extent and its first RP_PF * 32 entries (slot, value, and the bit the
// entry adds: a step bit >= 0, a row bit encoded -2 - slot, or -1).
template <typename V>
struct RpStep {
    int sp, jc, why;
    int64_t jl;
    int s[RP_PF], bit[RP_PF];
    V l[RP_PF];
};

template <typename V>
__device__ __forceinline__ void rp_read_step(const bk_dev &d, const bk_task &T, RpStep<V> &st, int j, int c, int lane)
{
    const int base = T.sp_lo;
    st.sp = slot_of(T, base, __ldcg(d.prow + j));
    st.jl = __ldcg(d.Lbeg + j);
    st.jc = __ldcg(d.Lcnt + j);
    st.why = 0;
#pragma unroll
    for (int u = 0; u < RP_PF; u++) {
        const int q = lane + 32 * u;
        st.s[u] = -1;
        st.bit[u] = -1;
        st.l[u] = V(0);
        if (q >= st.jc) continue;
        const int r = __ldcg(d.Li + st.jl + q);
        st.l[u] = __ldcg(vals<V>(d.Lx) + st.jl + q);
        const int s = slot_of(T, base, r);
        if (s < 0) { st.why = 71; continue; }
        st.s[u] = s;
        const int p = s < T.hi - base ? __ldcg(d.pinv + r) : -1;
        if (p >= 0 && p < c) {
            if (p > j) st.bit[u] = p - base;
            else st.why = 72;
        } else {
            st.bit[u] = -2 - s;
        }
    }
}

constexpr int RP_NT = 128;     // threads of a repair block (four warps)

template <typename V>
__global__ void __launch_bounds__(RP_NT, 1) bk_repair_kernel(bk_dev d, const int32_t *__restrict__ tasks,
                                                          int32_t ntasks, int32_t *counter, double tau,
                                                          int32_t smem_bytes)
{
    const V *const Bx = vals<V>(d.Bx);
    V *const Lx = vals<V>(d.Lx);
    V *const Ux = vals<V>(d.Ux);
    extern __shared__ __align__(16) uint32_t rp_smem[];
    __shared__ bk_task T;
    __shared__ int list[RP_LIST];
    __shared__ int red[RP_NT / 32 + 1];
    __shared__ int ctl[4];             // [0] claimed task index, [1] why, [2] stop
    __shared__ FcSmem<V> fcs;
    const int tid_x = threadIdx.x, lane = tid_x & 31, warp = tid_x >> 5;
    for (;;) {
        if (tid_x == 0) ctl[0] = atomicAdd(counter, 1);
        __syncthreads();
        const int k = ctl[0];
        if (k >= ntasks) break;
        const int tid = tasks[k];
        if (warp == 0) load_task(T, d.tasks + tid, lane);
        __syncthreads();
        const int f = __ldcg(d.task_fail + tid);
        bool skip = f < T.lo || f >= T.hi;
        if (!skip && T.sp_lo != T.lo) {           // only tasks without descendants come here
            if (tid_x == 0) report_internal(d.status, f, 70);
            skip = true;
        }
        if (skip) {
            __syncthreads();
            continue;
        }
        const int base = T.sp_lo;          // = lo: a leaf or a BTF block has no descendants
        const int nown = T.hi - T.lo;
        const int nsp = T.hi - base;       // slots below this are rows pivoted in the task
        const int lsp = T.lspace;
        const int nsw = (nsp + 31) >> 5, nrw = (lsp + 31) >> 5, nbw = (nown + 31) >> 5;
        uint32_t *const sb = rp_smem;      // steps of the reach (pivot steps - base)
        uint32_t *const rb = sb + nsw;     // unpivoted rows of the pattern (slots)
        uint32_t *const rec = rb + nrw;    // columns recomputed here (c - lo)
        uint32_t *const tch = rec + nbw;   // rows whose pivot status changed here (r - lo)
        uint32_t *const sset = tch + nbw;  // the stored steps of the column at hand (j - lo)
        const int words = (2 * nsw + nrw + 2 * nbw + 3) & ~3;
        // then the pivot steps of the task's rows (a copy of pinv kept up to date
        // here), a byte per slot marking the stored-pattern update's pattern, and x
        int32_t *const spv = reinterpret_cast<int32_t *>(rp_smem + words);
        unsigned char *const mark = reinterpret_cast<unsigned char *>(spv + ((nown + 3) & ~3));
        const int mbytes = (T.space + 15) & ~15;
        const int64_t fixed = (int64_t)words * 4 + (int64_t)((nown + 3) & ~3) * 4 + mbytes;
        const bool xsh = fixed + (int64_t)T.space * 8 <= smem_bytes;
        const bool vsp = fixed <= smem_bytes;     // the stored-pattern update needs the marks
        V *const x = xsh ? reinterpret_cast<V *>(mark + mbytes)
                         : reinterpret_cast<V *>(d.wsd + (int64_t)blockIdx.x * d.wsd_slice);
        for (int i = tid_x; i < words; i += RP_NT) rp_smem[i] = 0u;
        if (vsp) {
            for (int i = tid_x; i < nown; i += RP_NT) spv[i] = __ldcg(d.pinv + T.lo + i);
            for (int i = tid_x; i < mbytes / 4; i += RP_NT) reinterpret_cast<uint32_t *>(mark)[i] = 0u;
        }
        if (xsh)
            for (int i = tid_x; i < T.space; i += RP_NT) x[i] = V(0);
        if (tid_x == 0) ctl[1] = ctl[2] = 0;
        __syncthreads();
        for (int c = f; c < T.hi; c++) {
            BK_TSTART(t0);
            BK_TPHASE0(tp);
            // ---- dirty?  (every column before c is final)
            const bool d0 = c == f || __ldcg(d.col_fail + c) != 0;
            bool hit = false;
            if (!d0) {
                const int64_t ub0 = __ldcg(d.Ubeg + c), lb0 = __ldcg(d.Lbeg + c);
                const int uc0 = __ldcg(d.Ucnt + c), lc0 = __ldcg(d.Lcnt + c);
                for (int q = tid_x; q < uc0; q += RP_NT) {
                    const int j = __ldcg(d.Ui + ub0 + q);
                    if (j >= T.lo && j < c && get_bit(rec, j - T.lo)) hit = true;
                    const int r = __ldcg(d.prow + j) - T.lo;
                    if ((unsigned)r < (unsigned)nown && get_bit(tch, r)) hit = true;
                }
                for (int q = tid_x; q < lc0; q += RP_NT) {
                    const int r = __ldcg(d.Li + lb0 + q) - T.lo;
                    if ((unsigned)r < (unsigned)nown && get_bit(tch, r)) hit = true;
                }
            }
            if (!__syncthreads_or(d0 || hit)) continue;
            if (__syncthreads_or(tid_x == 0 && should_stop(d, tid, c))) break;
            if (tid_x == 0) BK_TPHASE(d.trace, tp, 0, c);       // dirty check

            // ---- recompute column c by Algorithm 1.  First on its stored pattern
            // (its steps known in advance, the update dealt over the block and
            // streamed through shared memory), verified against the pivots now in
            // place: the stored steps are the reach if each has its pivot row in
            // the pattern the update builds and each pivoted row of that pattern is
            // the pivot row of a stored step.  Otherwise by the reach itself.
            int64_t ub = d.Ubeg[c], ue = d.Uend[c];
            int64_t lb = d.Lbeg[c], le = d.Lend[c];
            const int e1 = d.Bp[c + 1];
            const int ns = __ldcg(d.Ucnt + c) - 1;
            bool stored_ok = false, vbad_all = false;
            if (vsp) {
                bool ok = ns >= 0;
                for (int q = tid_x; q < ns; q += RP_NT) {
                    const int j = __ldcg(d.Ui + ub + q);
                    if (j < base || j >= c) ok = false;
                    else set_bit_s(sset, j - base);
                }
                for (int e = d.dstart[c] + tid_x; e < e1; e += RP_NT) {
                    const int sl = slot_of(T, base, d.Bi[e]);
                    if (sl < 0) { ok = false; continue; }     // reported by the reach below
                    x[sl] = Bx[e];
                    mark[sl] = 1;
                }
                ok = __syncthreads_and(ok);
                if (tid_x == 0) BK_TPHASE(d.trace, tp, 1, c);   // stored steps, B scattered
                bool vbad = false;
                if (ok)
                    ok = column_fast_update_cta<V, true, RP_NT>(d, T, base, d.Ui + ub, ns, Ux + ub, x, fcs, mark,
                                                                red, tid_x, vbad);
                if (tid_x == 0) BK_TPHASE(d.trace, tp, 2, c);   // the update
                int nin = 0;
                for (int w4 = tid_x; w4 < mbytes / 16; w4 += RP_NT) {
                    const uint4 mv = reinterpret_cast<const uint4 *>(mark)[w4];
                    const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        uint32_t bytes = mw[h];
                        while (bytes) {
                            const int bi = (__ffs(bytes) - 1) >> 3;
                            bytes &= ~(0xffu << (8 * bi));
                            const int sl = 16 * w4 + 4 * h + bi;
                            const int p = sl < nown ? spv[sl] : -1;
                            if (p >= 0 && p < c) {
                                x[sl] = V(0);                    // a pivot row: its value went to U
                                if (p >= base && get_bit(sset, p - base)) nin++;
                                else ok = false;
                            } else {
                                set_bit_s(rb, sl);
                            }
                        }
                    }
                }
                nin = warp_sum(nin);
                if (lane == 0) red[warp] = nin;
                ok = __syncthreads_and(ok);
                int nin_all = 0;
#pragma unroll
                for (int w = 0; w < RP_NT / 32; w++) nin_all += red[w];
                ok = ok && nin_all == ns;
                if (tid_x == 0) BK_TPHASE(d.trace, tp, 3, c);   // the pattern checked
                // clear the marks (and, if the stored steps are not the reach, x and rb)
                for (int w4 = tid_x; w4 < mbytes / 16; w4 += RP_NT) {
                    uint4 *const mp = reinterpret_cast<uint4 *>(mark) + w4;
                    const uint4 mv = *mp;
                    if (!(mv.x | mv.y | mv.z | mv.w)) continue;
                    if (!ok) {
                        const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
                        for (int h = 0; h < 4; h++)
#pragma unroll
                            for (int bi = 0; bi < 4; bi++)
                                if ((mw[h] >> (8 * bi)) & 0xffu) x[16 * w4 + 4 * h + bi] = V(0);
                    }
                    *mp = make_uint4(0u, 0u, 0u, 0u);
                }
                if (!ok)
                    for (int w = tid_x; w < nrw; w += RP_NT) rb[w] = 0u;
                for (int w = tid_x; w < nsw; w += RP_NT) sset[w] = 0u;
                vbad_all = __syncthreads_or(vbad);
                stored_ok = ok;
            }
            if (warp == 0) {
            int why = ctl[1];
            bool bad = stored_ok && vbad_all, overflow = false;
            int nu = stored_ok ? ns : 0;
                if (!stored_ok && !why) {
                for (int e = d.dstart[c] + lane; e < e1; e += 32) {
                    const int r = d.Bi[e];
                    const int s = slot_of(T, base, r);
                    if (s < 0) { if (!why) why = 73; continue; }
                    x[s] = Bx[e];
                    const int p = s < nsp ? __ldcg(d.pinv + r) : -1;
                    if (p >= 0 && p < c) set_bit_s(sb, p - base);
                    else set_bit_s(rb, s);
                }
                __syncwarp();
                // steps in ascending order (lowest set bit); the next one is predicted
                // and read while the current one is applied
                int w0 = 0;
                int jb = next_bit(sb, nsw, w0, lane);
                RpStep<V> cur, nxt;
                if (jb >= 0) rp_read_step(d, T, cur, base + jb, c, lane);
                for (int iter = 0; jb >= 0; iter++) {
                    const int j = base + jb;
                    if (iter > nsp || j >= c) { if (!why) why = 74; break; }
                    if (lane == 0) sb[jb >> 5] &= ~(1u << (jb & 31));
                    __syncwarp();
                    int wp = w0;
                    const int jbp = next_bit(sb, nsw, wp, lane);
                    if (jbp >= 0 && base + jbp < c) rp_read_step(d, T, nxt, base + jbp, c, lane);
                    const int sp = cur.sp;
                    if (sp < 0) { if (!why) why = 75; break; }
                    const V m = x[sp];
                    V xv[RP_PF];
    #pragma unroll
                    for (int u = 0; u < RP_PF; u++) xv[u] = cur.s[u] >= 0 ? x[cur.s[u]] : V(0);
                    __syncwarp();
                    if (lane == 0) x[sp] = V(0);
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
                    for (int u = 0; u < RP_PF; u++) {
                        if (cur.s[u] < 0) continue;
                        x[cur.s[u]] = fma(-cur.l[u], m, xv[u]);
                        if (cur.bit[u] >= 0) set_bit_s(sb, cur.bit[u]);
                        else if (cur.bit[u] <= -2) set_bit_s(rb, -2 - cur.bit[u]);
                    }
                    if (cur.why && !why) why = cur.why;
                    for (int q = 32 * RP_PF + lane; q < cur.jc; q += 32) {
                        const int r = __ldcg(d.Li + cur.jl + q);
                        const V l = __ldcg(Lx + cur.jl + q);
                        const int s1 = slot_of(T, base, r);
                        if (s1 < 0) { if (!why) why = 71; continue; }
                        x[s1] = fma(-l, m, x[s1]);
                        const int p = s1 < nsp ? __ldcg(d.pinv + r) : -1;
                        if (p >= 0 && p < c) {
                            if (p > j) set_bit_s(sb, p - base);
                            else if (!why) why = 72;
                        } else {
                            set_bit_s(rb, s1);
                        }
                    }
                    nu++;
                    __syncwarp();
                    jb = next_bit(sb, nsw, w0, lane);
                    if (jb >= 0) {
                        if (jb == jbp) cur = nxt;
                        else rp_read_step(d, T, cur, base + jb, c, lane);
                    }
                }
                }
            why = warp_max_i(why);
            if (lane == 0) BK_TPHASE(d.trace, tp, 4, c);       // the reach (if needed)
                // the pivot rule over the task's unpivoted rows of the pattern
                unsigned long long km = 0;      // largest own magnitude, as a key
                int ncand = 0, nrows = 0;
                for (int wcur = 0; wcur < nrw;) {
                    const int filled = list_rows(rb, nrw, wcur, list, lane);
                    nrows += filled;
                    for (int i0 = 0; i0 < filled; i0 += 32 * RP_RL) {
                        int ls[RP_RL];
                        V v[RP_RL];
    #pragma unroll
                        for (int u = 0; u < RP_RL; u++) {
                            const int i = i0 + lane + 32 * u;
                            ls[u] = i < filled ? list[i] : -1;
                            v[u] = ls[u] >= 0 ? x[ls[u]] : V(0);
                        }
    #pragma unroll
                        for (int u = 0; u < RP_RL; u++) {
                            if (ls[u] < 0) continue;
                            if (!isfinite(v[u])) bad = true;
                            if (ls[u] < nown) {
                                ncand++;
                                km = key_max(km, mag_key(v[u]));
                            }
                        }
                    }
                    __syncwarp();
                }
                km = warp_max_key(km);
                const V amax = key_value<V>(km);
                ncand = warp_sum(ncand);
                bad = __any_sync(BK_FULL, bad);
                const int pcur = __ldcg(d.prow + c);
                const int pref = d.pref[c];
                auto in_pattern = [&](int r) -> bool {
                    const int ls = r - T.lo;
                    return (unsigned)ls < (unsigned)nown && get_bit(rb, ls);
                };
                int piv = -1;
                if (!bad && ncand > 0 && amax > V(0)) {
                    if (in_pattern(pref) && (double)fabs(x[pref - T.lo]) >= tau * (double)amax) {
                        piv = pref;
                    } else {
                        int best = INT_MAX;
                        for (int wcur = 0; wcur < nbw && best == INT_MAX;) {
                            const int filled = list_rows(rb, nbw, wcur, list, lane);
                            for (int i0 = 0; i0 < filled; i0 += 32) {
                                const int i = i0 + lane;
                                const int ls = i < filled ? list[i] : -1;
                                if (ls >= 0 && ls < nown && mag_key(x[ls]) == km) best = min(best, ls);
                            }
                            best = warp_min(best);
                            __syncwarp();
                        }
                        piv = best == INT_MAX ? -1 : T.lo + best;
                        if (piv < 0 && !why) why = 76;     // amax is one of the listed values
                    }
                }
                if (piv < 0) {
                    // no acceptable pivot at an exact column: the matrix is singular here
                    if (lane == 0 && !why) report_fail(d.status, c, bad ? BK_CODE_NAN : BK_CODE_SINGULAR);
                    piv = pcur;
                }
                const int pls = piv - T.lo;
                const bool pin = in_pattern(piv);
                const V xp = pin ? x[pls] : V(0);
                BK_TPHASE(d.trace, tp, 5, c);       // the pivot
                // L(:,c) = x / pivot over the pattern's unpivoted rows; x and rb cleared
                const int cnt_all = nrows - (pin ? 1 : 0);
                if (!overflow && lb + cnt_all > le) {
                    const int64_t cap = max((long long)cnt_all, min((long long)(2 * (int64_t)cnt_all + 16),
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
                int rank0 = 0;
                for (int wcur = 0; wcur < nrw;) {
                    const int filled = list_rows(rb, nrw, wcur, list, lane);
                    for (int i0 = 0; i0 < filled; i0 += 32 * RP_RL) {
                        int ls[RP_RL];
                        int64_t qq[RP_RL];
                        V v[RP_RL];
    #pragma unroll
                        for (int u = 0; u < RP_RL; u++) {
                            const int i = i0 + lane + 32 * u;
                            ls[u] = i < filled ? list[i] : -1;
                            if (ls[u] == pls && pin) ls[u] = -2;      // the pivot row: cleared below
                            qq[u] = lb + rank0 + i - ((pin && ls[u] > pls) ? 1 : 0);
                            v[u] = ls[u] >= 0 ? x[ls[u]] : V(0);
                        }
    #pragma unroll
                        for (int u = 0; u < RP_RL; u++) {
                            if (ls[u] < 0) continue;
                            if (!overflow) {
                                d.Li[qq[u]] = row_of_lslot(T, ls[u]);
                                Lx[qq[u]] = v[u] / xp;
                            }
                            x[ls[u]] = V(0);
                        }
                    }
                    rank0 += filled;
                    __syncwarp();
                }
                for (int w = lane; w < nrw; w += 32) rb[w] = 0u;
                overflow = __any_sync(BK_FULL, overflow);
                __syncwarp();
                if (lane == 0) {
                    if (pin) x[pls] = V(0);
                    if (why) report_internal(d.status, c, why);
                    if (!overflow) {
                        d.Ui[ub + nu] = c;
                        Ux[ub + nu] = xp;
                        d.Ucnt[c] = nu + 1;
                        d.Lcnt[c] = cnt_all;
                    } else {
                        report_overflow(d, T, tid, c, 3);
                    }
                    if (piv != pcur) {
                        if (__ldcg(d.pinv + pcur) == c) {
                            d.pinv[pcur] = -1;
                            if (vsp) spv[pcur - T.lo] = -1;
                        }
                        d.pinv[piv] = c;
                        if (vsp) spv[pls] = c;
                        d.prow[c] = piv;
                        if ((unsigned)(pcur - T.lo) < (unsigned)nown) tch[(pcur - T.lo) >> 5] |= 1u << ((pcur - T.lo) & 31);
                        tch[pls >> 5] |= 1u << (pls & 31);
                        if (piv != c) atomicAdd(&d.status->offdiag, 1);
                    }
                    rec[(c - T.lo) >> 5] |= 1u << ((c - T.lo) & 31);
                    d.col_fail[c] = 0;
                    atomicAdd(&d.status->repaired, 1);
                    BK_TREC(d.trace, BK_TR_REPAIR, (piv != pcur ? 1 : 0) | (stored_ok ? 2 : 0), c, t0);
                    BK_TPHASE(d.trace, tp, 6, c);   // L written
                }
            __syncwarp();
            if (lane == 0) {
                ctl[1] = why;
                ctl[2] = (why || overflow) ? 1 : 0;
            }
            }
            __syncthreads();
            if (ctl[2]) break;
        }
        if (ctl[1]) return;      // the workspace may hold stale values; the host clears it
        __syncthreads();
    }
}

}  // namespace

// Dynamic shared memory of the repair kernel for the tasks it serves: the bitmaps
// of the largest, and x as well when that fits in limit bytes.
size_t bk_repair_smem(const bk_task *tasks, const int32_t *ids, int32_t count, size_t limit)
{
    size_t bits = 16, full = 16;
    for (int32_t i = 0; i < count; i++) {
        const bk_task &T = tasks[ids[i]];
        const size_t nown = (size_t)(T.hi - T.lo);
        const size_t words = (2 * (((size_t)(T.hi - T.sp_lo) + 31) / 32) + ((size_t)T.lspace + 31) / 32 +
                              2 * ((nown + 31) / 32) + 3) & ~(size_t)3;
        const size_t fixed = words * 4 + ((nown + 3) & ~(size_t)3) * 4 + (((size_t)T.space + 15) & ~(size_t)15);
        bits = std::max(bits, fixed);
        full = std::max(full, fixed + (size_t)T.space * 8);
    }
    return full <= limit ? full : bits;
}

void bk_launch_repair(const bk_dev &d, const int32_t *tasks, int32_t ntasks, int32_t *counter, double tau,
                      size_t smem, int ctas, void *stream)
{
    if (ntasks <= 0) return;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(bk_repair_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024);
        cudaFuncSetAttribute(bk_repair_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024);
    });
    const int grid = std::max(1, std::min<int>(ntasks, ctas));
    cudaStream_t s = (cudaStream_t)stream;
    if (d.prec)
        bk_repair_kernel<float><<<grid, RP_NT, smem, s>>>(d, tasks, ntasks, counter, tau, (int32_t)smem);
    else
        bk_repair_kernel<double><<<grid, RP_NT, smem, s>>>(d, tasks, ntasks, counter, tau, (int32_t)smem);
}
