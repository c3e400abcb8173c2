// column_fast.cuh -- the update loop of one column over a known list of steps
// (one warp), with the factors' data streamed through shared memory.
//
// Algorithm 1's update of column c, for a list S of pivot steps in ascending
// order: for each j in S, U(j,c) = x(prow j), then x -= L(:,j) U(j,c) (one fma
// per entry).  When S is a stored pattern the steps are known before the loop
// starts, so nothing of step j+1 has to wait for step j: the steps' metadata
// (pivot-row slot, extent of L(:,j)) are read for a segment of steps at once,
// and the entries of L(:,j) are copied into one of two shared-memory buffers by
// cp.async while the other buffer's entries are applied.  The per-step chain is
// then x(prow j) in the dense column, the fmas and a warp barrier.
//
// Verification (MARK): S is the reach of the column only if every step of S has
// its pivot row in the column's pattern and every pivoted row of the pattern is
// the pivot row of a step of S (a row pivoted at step p enters the pattern only
// through steps before p, so the final pattern decides it as well as the
// step-by-step one).  The loop marks every slot it touches in a byte array (B's
// rows are marked by the caller), from which the caller decides.
#pragma once

#include "basker_internal.h"
#include "device_util.cuh"
#include "trace.cuh"

namespace bk {

constexpr int FC_SEG = 128;    // steps whose metadata sit in shared memory at once
constexpr int FC_CAP = 1024;   // L entries per buffer (two buffers)

template <typename V, int CAP = FC_CAP>
struct FcSmem {
    int32_t j[FC_SEG], sp[FC_SEG], jc[FC_SEG], off[FC_SEG + 1];
    int64_t jl[FC_SEG];
    V u[FC_SEG];               // U(j,c) of the segment's steps, written out after it
    int32_t bi[2][CAP];
    V bv[2][CAP];
};

__device__ __forceinline__ void fc_cp4(void *dst, const void *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
}

__device__ __forceinline__ void fc_cp8(void *dst, const void *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}

__device__ __forceinline__ void fc_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void fc_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fc_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void fc_set(uint32_t *bm, int i) { atomicOr(bm + (i >> 5), 1u << (i & 31)); }

// Copy the entries [e0, e1) of the segment (concatenated L columns of its
// steps, offsets in S.off) into buffer b.  t: this lane's step cursor, at or
// before the step holding its first entry (entries only grow, chunk to chunk).
template <typename V>
__device__ __forceinline__ void fc_issue(const bk_dev &d, FcSmem<V> &S, int nseg, int e0, int e1, int b, int lane,
                                         int &t)
{
    const V *const Lx = vals<V>(d.Lx);
    // the step holding entry e; lanes advance by 32 entries at a time
    for (int e = e0 + lane; e < e1; e += 32) {
        while (t + 1 < nseg && S.off[t + 1] <= e) t++;
        const int64_t g = S.jl[t] + (e - S.off[t]);
        fc_cp4(&S.bi[b][e - e0], d.Li + g);
        if (sizeof(V) == 8) fc_cp8(&S.bv[b][e - e0], Lx + g);
        else fc_cp4(&S.bv[b][e - e0], Lx + g);
    }
    fc_commit();
}

// The update of column c over the steps Ulist[0..ns) (ascending).  U(j,c) is
// written to Uout[k] for the k-th step.  x is the dense column over the slots of
// slot_of(T, base, .), holding B(:,c) scattered by the caller.  MARK sets
// mark[s] = 1 for every slot an entry touches.  Returns false if an index fell
// outside the space (never valid input); bad: a non-finite U value.
template <typename V, bool MARK>
__device__ __forceinline__ bool column_fast_update(const bk_dev &d, const bk_task &T, int base,
                                                   const int32_t *Ulist, int ns, V *Uout, V *x, FcSmem<V> &S,
                                                   unsigned char *mark, int lane, bool &bad)
{
    bool broken = false;
    for (int k0 = 0; k0 < ns; k0 += FC_SEG) {
        const int nseg = min(FC_SEG, ns - k0);
        // ---- metadata of the segment's steps: four consecutive steps a lane
        int cnt4 = 0;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int t = 4 * lane + u;
            if (t >= nseg) continue;
            S.j[t] = __ldcg(Ulist + k0 + t);
        }
        __syncwarp();
        int jc4[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int t = 4 * lane + u;
            jc4[u] = 0;
            if (t >= nseg) continue;
            const int j = S.j[t];
            const int64_t jl = __ldcg(d.Lbeg + j);
            const int jc = __ldcg(d.Lcnt + j);
            const int sp = slot_of(T, base, __ldcg(d.prow + j));
            if (sp < 0) broken = true;
            S.jl[t] = jl;
            S.jc[t] = jc;
            S.sp[t] = sp;
            jc4[u] = jc;
            cnt4 += jc;
        }
        const int pre = warp_exscan(cnt4, lane);
        {
            int run = pre;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int t = 4 * lane + u;
                if (t < nseg) S.off[t] = run;
                run += jc4[u];
            }
            if (lane == 31) S.off[nseg] = run;
        }
        __syncwarp();
        const int E = S.off[nseg];
        const int nchunks = (E + FC_CAP - 1) / FC_CAP;
        // ---- entries in chunks of FC_CAP, copied one chunk ahead
        int tcp = 0;           // this lane's cursor over the steps, for the copies
        if (nchunks > 0) fc_issue(d, S, nseg, 0, min(E, FC_CAP), 0, lane, tcp);
        int t = 0;             // next step to start
        V m = V(0);            // the current step's U(j,c)
        for (int ch = 0; ch <= nchunks; ch++) {
            const int e0 = ch * FC_CAP, e1 = min(E, e0 + FC_CAP);
            if (ch < nchunks) {
                if (ch + 1 < nchunks) {
                    fc_issue(d, S, nseg, e1, min(E, e1 + FC_CAP), (ch + 1) & 1, lane, tcp);
                    fc_wait_prev();
                } else {
                    fc_wait_all();
                }
            }
            __syncwarp();
            const int b = ch & 1;
            // steps whose entries start in this chunk (the steps after the last
            // entry, which have none, belong to the pseudo-chunk ch == nchunks),
            // and the tail of a step begun in an earlier chunk
            int tc = t > 0 ? t - 1 : 0;
            while (tc < nseg) {
                const int s0 = S.off[tc], s1 = S.off[tc + 1];
                if (tc == t) {
                    if (ch < nchunks ? s0 >= e1 : s0 < E) break;
                    // start step tc: its U value, and its pivot row leaves x
                    const int sp = S.sp[tc];
                    m = sp >= 0 ? x[sp] : V(0);
                    __syncwarp();
                    if (lane == 0) {
                        if (sp >= 0) x[sp] = V(0);
                        S.u[tc] = m;
                    }
                    if (!isfinite(m)) bad = true;
                    t++;
                }
                // entries of step tc inside [e0, e1)
                const int a = max(s0, e0), z = min(s1, e1);
                const V *const bv = S.bv[b];
                const int32_t *const bi = S.bi[b];
                int q = a + lane;
                for (; q + 96 < z; q += 128) {
                    int sl[4];
                    V lv[4], xv[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        sl[u] = slot_of(T, base, bi[q + 32 * u - e0]);
                        lv[u] = bv[q + 32 * u - e0];
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++) xv[u] = sl[u] >= 0 ? x[sl[u]] : V(0);
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        if (sl[u] < 0) { broken = true; continue; }
                        x[sl[u]] = fma(-lv[u], m, xv[u]);
                        if (MARK) mark[sl[u]] = 1;
                    }
                }
                for (; q < z; q += 32) {
                    const int s = slot_of(T, base, bi[q - e0]);
                    if (s < 0) { broken = true; continue; }
                    x[s] = fma(-bv[q - e0], m, x[s]);
                    if (MARK) mark[s] = 1;
                }
                __syncwarp();
                if (s1 > e1) break;      // step tc continues in the next chunk
                tc++;
            }
            __syncwarp();
        }
        // the segment's U values, one coalesced store (no global store inside the
        // step chain, whose warp barriers would wait for it)
        for (int q = lane; q < nseg; q += 32) Uout[k0 + q] = S.u[q];
        __syncwarp();
    }
    return !__any_sync(BK_FULL, broken);
}

// Non-finite test on the bit pattern (integer operations only: FP64 issue is the
// scarce resource of these loops).
__device__ __forceinline__ bool fc_nonfinite(double v)
{
    return (__double_as_longlong(v) & 0x7ff0000000000000ll) == 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool fc_nonfinite(float v) { return (__float_as_int(v) & 0x7f800000) == 0x7f800000; }

// The same update by a whole block of NT threads (NT / 32 warps, so that the
// steps' fmas use every FP64 unit of the SM): the entries of each step are
// dealt over the block and one block barrier separates the steps.  The steps
// of a segment go in batches whose entries fit one buffer (a step with more
// entries than a buffer holds is applied from global memory), the next batch
// copied while one is applied, its rows turned into slots once it has landed;
// inside a batch the next step's metadata and first entry are read ahead, so
// that a step's chain is x(prow j), the fmas and the barrier.  x(prow j) is not cleared
// here (no later step reads it; the caller clears the pattern).  red: shared
// scratch of NT / 32 ints.  allow (if not null): an entry whose slot lies below
// nallow must have its bit set there, else vfail is set (the stored steps are
// not the reach; the caller falls back).  map (if not null): x and mark are
// indexed by a compact index instead of the slot: map.find(slot) for slots below
// nallow (-1: not there, vfail), map.shift + slot for the others.
// An open-addressing table from slot to position: each entry packs the slot
// (above FC_POS_BITS) and the position (below); -1 is empty.
constexpr int FC_POS_BITS = 11;
constexpr int FC_POS_MASK = (1 << FC_POS_BITS) - 1;

__device__ __forceinline__ int fc_hash(int s, int mask) { return (int)(((unsigned)s * 2654435761u) >> 7) & mask; }

struct FcMap {
    const int32_t *tab;
    int mask, shift;
    __device__ __forceinline__ int find(int s) const
    {
        int h = fc_hash(s, mask);
        for (int probe = 0; probe <= mask; probe++) {
            const int k = tab[h];
            if (k < 0) return -1;
            if ((k >> FC_POS_BITS) == s) return k & FC_POS_MASK;
            h = (h + 1) & mask;
        }
        return -1;
    }
};

template <typename V, bool MARK, int NT, int CAP = FC_CAP>
__device__ __forceinline__ bool column_fast_update_cta(const bk_dev &d, const bk_task &T, int base,
                                                       const int32_t *Ulist, int ns, V *Uout, V *x,
                                                       FcSmem<V, CAP> &S, unsigned char *mark, int *red, int tid,
                                                       bool &bad, const uint32_t *allow = nullptr, int nallow = 0,
                                                       bool *vfail = nullptr, const FcMap *map = nullptr)
{
#ifdef BK_TRACE
    long long cy[6] = {0, 0, 0, 0, 0, 0};   // metadata, batch bounds + copies, wait, conversion, apply, tail
    long long cyt = clock64();
#define FC_LAP(i)                        \
    do {                                 \
        const long long now = clock64(); \
        cy[i] += now - cyt;              \
        cyt = now;                       \
    } while (0)
#else
#define FC_LAP(i)
#endif
    auto remap = [&](int sl, bool &vf) -> int {
        if (!map || sl < 0) return sl;
        if (sl >= nallow) return map->shift + sl;
        const int ix = map->find(sl);
        if (ix < 0) vf = true;
        return ix;
    };
    static_assert(NT == FC_SEG, "one step's metadata a thread");
    const int lane = tid & 31, warp = tid >> 5;
    const V *const Lx = vals<V>(d.Lx);
    bool broken = false;
    for (int k0 = 0; k0 < ns; k0 += FC_SEG) {
        const int nseg = min(FC_SEG, ns - k0);
        int jc = 0;
        if (tid < nseg) {
            const int j = __ldcg(Ulist + k0 + tid);
            const int64_t jl = __ldcg(d.Lbeg + j);
            jc = __ldcg(d.Lcnt + j);
            int sp = slot_of(T, base, __ldcg(d.prow + j));
            if (sp < 0) broken = true;
            bool vf = false;
            sp = remap(sp, vf);
            if (vf) *vfail = true;
            S.j[tid] = j;
            S.jl[tid] = jl;
            S.jc[tid] = jc;
            S.sp[tid] = sp;
        }
        const int pre = warp_exscan(jc, lane);
        if (lane == 31) red[warp] = pre + jc;
        __syncthreads();
        int wofs = 0, E = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; w++) {
            if (w < warp) wofs += red[w];
            E += red[w];
        }
        if (tid < nseg) S.off[tid] = wofs + pre;
        if (tid == 0) S.off[nseg] = E;
        __syncthreads();
        FC_LAP(0);
        // the batch starting at step bs: as many steps as fit one buffer (at least
        // one); the steps that fit form a prefix, so their count decides
        auto batch_end = [&](int bs) {
            const bool fits = tid >= bs && tid < nseg && S.off[tid + 1] - S.off[bs] <= CAP;
            return bs + max(1, __syncthreads_count(fits));
        };
        // copies of a batch's entries: steps dealt to the warps, entries to the lanes
        auto issue = [&](int bs, int be, int b) {
            const int e0 = S.off[bs];
            if (S.off[be] - e0 <= CAP) {
                for (int t = bs + warp; t < be; t += NT / 32) {
                    const int a = S.off[t], cnt = S.off[t + 1] - a;
                    const int64_t g = S.jl[t];
                    for (int q = lane; q < cnt; q += 32) {
                        fc_cp4(&S.bi[b][a - e0 + q], d.Li + g + q);
                        if (sizeof(V) == 8) fc_cp8(&S.bv[b][a - e0 + q], Lx + g + q);
                        else fc_cp4(&S.bv[b][a - e0 + q], Lx + g + q);
                    }
                }
            }
            fc_commit();
        };
        int bs = 0, be = batch_end(0), buf = 0;
        issue(bs, be, 0);
        while (bs < nseg) {
            const int nbs = be, nbe = nbs < nseg ? batch_end(nbs) : nbs;
            if (nbs < nseg) issue(nbs, nbe, buf ^ 1);
            FC_LAP(1);
            if (nbs < nseg) fc_wait_prev();
            else fc_wait_all();
            __syncthreads();
            FC_LAP(2);
            const int e0 = S.off[bs], e1 = S.off[be];
            const bool direct = e1 - e0 > CAP;
            int32_t *const bi = S.bi[buf];
            const V *const bv = S.bv[buf];
            if (!direct) {
                // the batch's rows become slots (once, all threads), so that the
                // step chain below has no slot search in it
                bool vf = false;
                for (int e = e0 + tid; e < e1; e += NT) {
                    const int sl = slot_of(T, base, bi[e - e0]);
                    if (sl < 0) broken = true;
                    else if (allow && sl < nallow && !((allow[sl >> 5] >> (sl & 31)) & 1u)) vf = true;
                    bi[e - e0] = remap(sl, vf);
                }
                if (vf) *vfail = true;
                __syncthreads();
                FC_LAP(3);
                // steps; the next step's metadata and this thread's first entry of
                // it are read while the current step is applied
                int sp_n = S.sp[bs], a_n = S.off[bs], z_n = S.off[bs + 1];
                int s_n = a_n + tid < z_n ? bi[a_n + tid - e0] : -1;
                V l_n = a_n + tid < z_n ? bv[a_n + tid - e0] : V(0);
                for (int t = bs; t < be; t++) {
                    const int sp = sp_n, a = a_n, z = z_n, s0 = s_n;
                    const V l0 = l_n;
                    if (t + 1 < be) {
                        sp_n = S.sp[t + 1];
                        a_n = z;
                        z_n = S.off[t + 2];
                        s_n = a_n + tid < z_n ? bi[a_n + tid - e0] : -1;
                        l_n = a_n + tid < z_n ? bv[a_n + tid - e0] : V(0);
                    }
                    const V m = sp >= 0 ? x[sp] : V(0);
                    if (tid == 0) S.u[t] = m;
                    if (fc_nonfinite(m)) bad = true;
                    if (s0 >= 0) {
                        const V xv = x[s0];
                        x[s0] = fma(-l0, m, xv);
                        if (MARK) mark[s0] = 1;
                    }
                    int q = a + tid + NT;
                    for (; q + NT < z; q += 2 * NT) {
                        const int sa = bi[q - e0], sb = bi[q + NT - e0];
                        const V la = bv[q - e0], lb = bv[q + NT - e0];
                        if (sa >= 0) {
                            const V xa = x[sa];
                            x[sa] = fma(-la, m, xa);
                            if (MARK) mark[sa] = 1;
                        }
                        if (sb >= 0) {
                            const V xb = x[sb];
                            x[sb] = fma(-lb, m, xb);
                            if (MARK) mark[sb] = 1;
                        }
                    }
                    if (q < z) {
                        const int sa = bi[q - e0];
                        if (sa >= 0) {
                            x[sa] = fma(-bv[q - e0], m, x[sa]);
                            if (MARK) mark[sa] = 1;
                        }
                    }
                    __syncthreads();
                }
            } else {
                // one step with more entries than a buffer holds: from global memory
                const int t = bs;
                const int sp = S.sp[t], a = S.off[t], z = S.off[t + 1];
                const int64_t gl = S.jl[t] - a;
                const V m = sp >= 0 ? x[sp] : V(0);
                if (tid == 0) S.u[t] = m;
                if (fc_nonfinite(m)) bad = true;
                for (int q = a + tid; q < z; q += NT) {
                    int sq = slot_of(T, base, __ldcg(d.Li + gl + q));
                    const V lq = __ldcg(Lx + gl + q);
                    if (sq < 0) { broken = true; continue; }
                    if (allow && sq < nallow && !((allow[sq >> 5] >> (sq & 31)) & 1u)) *vfail = true;
                    bool vf = false;
                    sq = remap(sq, vf);
                    if (vf) { *vfail = true; continue; }
                    x[sq] = fma(-lq, m, x[sq]);
                    if (MARK) mark[sq] = 1;
                }
                __syncthreads();
            }
            FC_LAP(4);
            bs = nbs;
            be = nbe;
            buf ^= 1;
        }
        for (int q = tid; q < nseg; q += NT) Uout[k0 + q] = S.u[q];
        __syncthreads();
        FC_LAP(5);
    }
#ifdef BK_TRACE
    if (tid == 0)
        for (int i = 0; i < 6; i++) bk_trace_raw(d.trace, BK_TR_PHASE, 20 + i, ns, 0ull, (unsigned long long)cy[i]);
#endif
#undef FC_LAP
    return !__syncthreads_or(broken);
}
}  // namespace bk
