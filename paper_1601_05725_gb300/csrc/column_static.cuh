// column_static.cuh -- one column recomputed on its stored pattern (one warp).
//
// x = B(:,c); for each step j of the stored U(:,c), lowest first: U(j,c) is
// x(prow j), then x -= L(:,j) U(j,c); finally U(c,c) = x(prow c) and
// L(:,c) = x / U(c,c) over the stored rows of L(:,c).  x is the warp's dense slice
// over the task's space (base = sp_lo); it is zero outside the column before and
// after.  Used by the stored-pattern pass of a refactorization and by the rounds
// that follow it (pattern_column below).
#pragma once

#include "basker_internal.h"
#include "device_util.cuh"

namespace bk {

// Bounded wait of lane 0 on a flag, the warp told the outcome.  dist: how many
// columns the waiting column lies past the one it waits for; the farther, the
// less often it polls (a chain's head is polled by every column still to come).
__device__ __forceinline__ bool flag_wait(const bk_dev &d, const int *flag, int epoch, long long budget, int lane,
                                          int dist = 1)
{
    int ok = 1;
    if (lane == 0) {
        if (ld_relaxed(flag) != epoch) {
            const unsigned nap = (unsigned)min(max(dist, 1), 32) * 32u;
            const long long t0 = clock64();
            while (ld_relaxed(flag) != epoch) {
                if (*reinterpret_cast<const volatile int *>(&d.status->timeout) || clock64() - t0 > budget) {
                    atomicExch(&d.status->timeout, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(nap);
            }
        }
        if (ok) fence_acquire();
    }
    return __shfl_sync(BK_FULL, ok, 0) != 0;
}

// Zero x over column c's stored pattern (its rows of B are a subset).
template <typename V>
__device__ __forceinline__ void clear_stored(const bk_dev &d, const bk_task &T, V *x, int c, int lane)
{
    const int base = T.sp_lo;
    const int64_t ub = d.Ubeg[c];
    const int uc = d.Ucnt[c];
    for (int q = lane; q < uc; q += 32) {
        const int s = slot_of(T, base, __ldcg(d.prow + d.Ui[ub + q]));
        if (s >= 0) x[s] = 0.0;
    }
    const int64_t lb = d.Lbeg[c];
    const int lc = d.Lcnt[c];
    for (int q = lane; q < lc; q += 32) {
        const int s = slot_of(T, base, d.Li[lb + q]);
        if (s >= 0) x[s] = 0.0;
    }
    __syncwarp();
}


// Column c on its stored pattern.  Within a pass no stored pattern changes
// except, in a refactorization round, that of a step recomputed by the reach,
// which is flagged (pchg[j] == epoch) before its done flag is released.  So the
// rows of every L(:,j) and of L(:,c) are read ahead, and the only reads that must
// follow a step's flag are its values L(j+1:n, j); a flagged step stops the
// computation instead (x is cleared over the stored pattern, aborted is set).
// Per step: the rows of L(:,j) (read during the previous step), their x values
// and x(prow j) are loaded together once the previous step's updates are stored;
// after the flag, L(:,j)'s values; then one fma per entry in ascending step order
// (the same per-entry operation order as Algorithm 1's update).  The first
// FIX_PF * 32 entries of a column live in registers; longer columns take the rest
// in batches.  A step is waited for (done[j] == epoch) when wait_all, or when it
// is a column of the same task at or after wait_lo.  Returns false when a wait
// ran out of budget.  Outputs: ok (Algorithm 1's pivot selection keeps prow[c]),
// bad (a non-finite value), broken (an index outside the space; never valid
// input).
constexpr int FIX_PF = 8;

template <typename V>
__device__ __forceinline__ bool pattern_column(const bk_dev &d, const bk_task &T, int tid, V *x, int c,
                                               int epoch, long long budget, double tau, int lane, bool wait_all,
                                               int wait_lo, bool &ok_out, bool &bad_out, bool &broken_out,
                                               const int *pchg = nullptr, bool *aborted = nullptr)
{
    const V *const Bx = vals<V>(d.Bx);
    V *const Lx = vals<V>(d.Lx);
    V *const Ux = vals<V>(d.Ux);
    const int base = T.sp_lo;
    const int own_lo = T.lo - base, own_hi = T.hi - base;
    bool broken = false, bad = false;
    const int e1 = d.Bp[c + 1];
    for (int e = d.dstart[c] + lane; e < e1; e += 32) {
        const int s = slot_of(T, base, d.Bi[e]);
        if (s < 0) { broken = true; continue; }
        x[s] = Bx[e];
    }
    // rows of L(:,c) and the pivot row, for the selection at the end
    const int64_t lb = d.Lbeg[c];
    const int lc = d.Lcnt[c];
    int fs[FIX_PF];
#pragma unroll
    for (int u = 0; u < FIX_PF; u++) {
        const int q = lane + 32 * u;
        fs[u] = -2;
        if (q < lc) {
            fs[u] = slot_of(T, base, d.Li[lb + q]);
            if (fs[u] < 0) broken = true;
        }
    }
    int sp_c = slot_of(T, base, __ldcg(d.prow + c));
    if (sp_c < 0) { broken = true; sp_c = 0; }
    __syncwarp();
    const int64_t ub = d.Ubeg[c];
    const int nsteps = d.Ucnt[c] - 1;
    for (int k0 = 0; k0 < nsteps; k0 += 32) {
        const int nin = min(32, nsteps - k0);
        int j_l = 0, sp_l = -1, jc_l = 0;
        int64_t jl_l = 0;
        bool done_l = true, changed = false;
        if (lane < nin) {
            j_l = d.Ui[ub + k0 + lane];
            const bool must = wait_all || (j_l >= wait_lo && d.col_task[j_l] == tid);
            done_l = !must || ld_relaxed(d.done + j_l) == epoch;
            if (must && done_l) fence_acquire();
            if (pchg && must && done_l && __ldcg(pchg + j_l) == epoch) changed = true;
            sp_l = slot_of(T, base, __ldcg(d.prow + j_l));
            jl_l = __ldcg(d.Lbeg + j_l);
            jc_l = __ldcg(d.Lcnt + j_l);
            if (sp_l < 0) broken = true;
        }
        const uint32_t pending = __ballot_sync(BK_FULL, !done_l);
        if (__any_sync(BK_FULL, changed)) {
            clear_stored(d, T, x, c, lane);
            *aborted = true;
            return true;
        }
        // rows (and, for a finished step, values) of the chunk's first step
        int rr[FIX_PF];
        V ll[FIX_PF];
        {
            const int64_t jl0 = __shfl_sync(BK_FULL, jl_l, 0);
            const int jc0 = __shfl_sync(BK_FULL, jc_l, 0);
#pragma unroll
            for (int u = 0; u < FIX_PF; u++) {
                const int q = lane + 32 * u;
                rr[u] = q < jc0 ? __ldcg(d.Li + jl0 + q) : -1;
                ll[u] = (q < jc0 && !(pending & 1u)) ? __ldcg(Lx + jl0 + q) : 0.0;
            }
        }
        for (int t = 0; t < nin; ++t) {
            const int j = __shfl_sync(BK_FULL, j_l, t);
            const int sp = __shfl_sync(BK_FULL, sp_l, t);
            const int64_t jl = __shfl_sync(BK_FULL, jl_l, t);
            const int jc = __shfl_sync(BK_FULL, jc_l, t);
            // x(prow j) and the x values under L(:,j); all earlier steps are stored
            int ss[FIX_PF];
            V xv[FIX_PF];
            const V m = sp >= 0 ? x[sp] : 0.0;
#pragma unroll
            for (int u = 0; u < FIX_PF; u++) {
                ss[u] = rr[u] >= 0 ? slot_of(T, base, rr[u]) : -1;
                if (rr[u] >= 0 && ss[u] < 0) broken = true;
                xv[u] = ss[u] >= 0 ? x[ss[u]] : 0.0;
            }
            if ((pending >> t) & 1u) {
                if (!flag_wait(d, d.done + j, epoch, budget, lane, c - j)) return false;
                if (pchg && __ldcg(pchg + j) == epoch) {
                    clear_stored(d, T, x, c, lane);
                    *aborted = true;
                    return true;
                }
#pragma unroll
                for (int u = 0; u < FIX_PF; u++) {
                    const int q = lane + 32 * u;
                    if (q < jc) ll[u] = __ldcg(Lx + jl + q);
                }
            }
            // the next step's rows and, if it has finished, values
            int rn[FIX_PF];
            V ln[FIX_PF];
            {
                const int tn = t + 1 < nin ? t + 1 : t;
                const int64_t jln = __shfl_sync(BK_FULL, jl_l, tn);
                const int jcn = t + 1 < nin ? __shfl_sync(BK_FULL, jc_l, tn) : 0;
                const bool pn = (pending >> tn) & 1u;
#pragma unroll
                for (int u = 0; u < FIX_PF; u++) {
                    const int q = lane + 32 * u;
                    rn[u] = q < jcn ? __ldcg(d.Li + jln + q) : -1;
                    ln[u] = (q < jcn && !pn) ? __ldcg(Lx + jln + q) : 0.0;
                }
            }
            if (sp >= 0) {
                __syncwarp();
                if (lane == 0) {
                    x[sp] = 0.0;
                    Ux[ub + k0 + t] = m;
                }
                if (!isfinite(m)) bad = true;
#pragma unroll
                for (int u = 0; u < FIX_PF; u++)
                    if (ss[u] >= 0) x[ss[u]] = fma(-ll[u], m, xv[u]);
                // entries past the register window, in batches
                for (int q0 = 32 * FIX_PF; q0 < jc; q0 += 32 * FIX_PF) {
                    int sb[FIX_PF];
                    V lb2[FIX_PF], xb[FIX_PF];
#pragma unroll
                    for (int u = 0; u < FIX_PF; u++) {
                        const int q = q0 + lane + 32 * u;
                        sb[u] = -1;
                        lb2[u] = 0.0;
                        if (q < jc) {
                            sb[u] = slot_of(T, base, __ldcg(d.Li + jl + q));
                            lb2[u] = __ldcg(Lx + jl + q);
                            if (sb[u] < 0) broken = true;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < FIX_PF; u++) xb[u] = sb[u] >= 0 ? x[sb[u]] : 0.0;
#pragma unroll
                    for (int u = 0; u < FIX_PF; u++)
                        if (sb[u] >= 0) x[sb[u]] = fma(-lb2[u], m, xb[u]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < FIX_PF; u++) {
                rr[u] = rn[u];
                ll[u] = ln[u];
            }
        }
    }
    // Algorithm 1's pivot selection, validated for the stored pivot row
    const V xp = x[sp_c];
    unsigned long long km = mag_key(xp);
    if (!isfinite(xp)) bad = true;
    V v[FIX_PF];
#pragma unroll
    for (int u = 0; u < FIX_PF; u++) v[u] = fs[u] >= 0 ? x[fs[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < FIX_PF; u++) {
        if (fs[u] < 0) continue;
        if (!isfinite(v[u])) bad = true;
        if (fs[u] >= own_lo && fs[u] < own_hi) km = key_max(km, mag_key(v[u]));
        x[fs[u]] = 0.0;
        Lx[lb + lane + 32 * u] = v[u] / xp;
    }
    for (int t = 32 * FIX_PF + lane; t < lc; t += 32) {
        const int s = slot_of(T, base, d.Li[lb + t]);
        if (s < 0) { broken = true; continue; }
        const V w = x[s];
        x[s] = 0.0;
        if (!isfinite(w)) bad = true;
        if (s >= own_lo && s < own_hi) km = key_max(km, mag_key(w));
        Lx[lb + t] = w / xp;
    }
    km = warp_max_key(km);
    const V amax = key_value<V>(km);
    bad = __any_sync(BK_FULL, bad);
    broken = __any_sync(BK_FULL, broken);
    __syncwarp();
    if (lane == 0) {
        x[sp_c] = 0.0;
        Ux[ub + nsteps] = xp;
    }
    __syncwarp();
    ok_out = !bad && !broken && amax > V(0) && (double)fabs(xp) >= tau * (double)amax;
    bad_out = bad;
    broken_out = broken;
    return true;
}

}  // namespace bk
