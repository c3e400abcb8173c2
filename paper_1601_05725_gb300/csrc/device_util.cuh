// device_util.cuh -- small device helpers shared by the library's kernels.
#pragma once

#include <cstdint>

#include "basker_internal.h"

#define BK_FULL 0xffffffffu

namespace bk {

// Slot of row r in a task's dense column space.  The space lists the rows
// [base, hi) (base = sp_lo: subtree and own rows; base = lo: own rows only) and
// then each ancestor node's rows, ancestors in ascending row order; so slots are
// ascending in r.  Returns -1 for a row outside the space.  Ancestor rows (all
// above hi) are found by a fixed binary search over the padded table anc_lo
// (k = number of ranges starting at or below r), without a data-dependent loop.
__device__ __forceinline__ int slot_of(const bk_task &T, int base, int r)
{
    if (r < T.anc_lo[0]) return (r >= base && r < T.hi) ? r - base : -1;
    int k = T.anc_lo[7] <= r ? 8 : 0;
    k += T.anc_lo[k + 3] <= r ? 4 : 0;
    k += T.anc_lo[k + 1] <= r ? 2 : 0;
    k += T.anc_lo[k] <= r ? 1 : 0;
    const int a = k - 1;                       // r >= anc_lo[0], so k >= 1
    return r < T.anc_hi[a] ? r + (T.hi - base) + T.anc_sh[a] : -1;
}

// Row of an index of the L-space (own rows [lo, hi), then the ancestors' rows).
__device__ __forceinline__ int row_of_lslot(const bk_task &T, int ls)
{
    const int own = T.hi - T.lo;
    if (ls < own) return T.lo + ls;
    const int v = ls - own;
    int k = T.anc_cum[7] <= v ? 8 : 0;
    k += T.anc_cum[k + 3] <= v ? 4 : 0;
    k += T.anc_cum[k + 1] <= v ? 2 : 0;
    k += T.anc_cum[k] <= v ? 1 : 0;
    const int a = k - 1;                       // anc_cum[0] = 0 <= v when nanc > 0
    return (a >= 0 && v - T.anc_cum[a] < T.anc_hi[a] - T.anc_lo[a]) ? v - T.anc_sh[a] : -1;
}

// |v| as an unsigned integer key (the bits with the sign cleared): over the
// finite values and the infinities the keys are ordered as the magnitudes, so a
// largest magnitude, and the rows that reach it, are found with integer
// instructions only (NaNs, above the infinities, are caught as non-finite first)
__device__ __forceinline__ unsigned long long mag_key(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long mag_key(float v)
{
    return (unsigned long long)((unsigned)__float_as_int(v) & 0x7fffffffu);
}
template <typename V> __device__ __forceinline__ V key_value(unsigned long long k);
template <> __device__ __forceinline__ double key_value<double>(unsigned long long k)
{
    return __longlong_as_double((long long)k);
}
template <> __device__ __forceinline__ float key_value<float>(unsigned long long k)
{
    return __int_as_float((int)(unsigned)k);
}
template <typename V> __device__ __forceinline__ unsigned long long key_inf();
template <> __device__ __forceinline__ unsigned long long key_inf<double>() { return 0x7ff0000000000000ull; }
template <> __device__ __forceinline__ unsigned long long key_inf<float>() { return 0x7f800000ull; }

__device__ __forceinline__ unsigned long long key_max(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k = key_max(k, __shfl_xor_sync(BK_FULL, k, o));
    return k;
}

template <typename V>
__device__ __forceinline__ V warp_max(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(BK_FULL, v, o));
    return v;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(BK_FULL, v, o);
    return v;
}

__device__ __forceinline__ int warp_min(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(BK_FULL, v, o));
    return v;
}

__device__ __forceinline__ int warp_max_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(BK_FULL, v, o));
    return v;
}

// Exclusive prefix sum over the warp.
__device__ __forceinline__ int warp_exscan(int v, int lane)
{
    int s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(BK_FULL, s, o);
        if (lane >= o) s += t;
    }
    return s - v;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Waits poll a flag with relaxed loads and, once it holds the value waited for,
// take one fence: a relaxed load followed by fence.acq_rel is an acquire pattern,
// so the reads after the wait are ordered after the writes released before the
// flag, while the polls themselves order nothing (one fence a wait, not one
// acquire a poll).
__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Copy a task descriptor into shared memory (all lanes of the warp).
__device__ __forceinline__ void load_task(bk_task &dst, const bk_task *src, int lane)
{
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int i = lane; i < (int)(sizeof(bk_task) / 4); i += 32) d[i] = s[i];
    __syncwarp();
}

// A failure (SINGULAR / NAN) at column c; the smallest column wins, as in a
// column-by-column factorization that stops at its first failure.
__device__ __forceinline__ void report_fail(bk_status *st, int c, int code)
{
    atomicMin(&st->first_fail, ((unsigned long long)(unsigned)c << 8) | (unsigned)code);
}

// An index outside its space (never valid input): record where, then fail.
__device__ __forceinline__ void report_internal(bk_status *st, int c, int site)
{
    if (atomicCAS(&st->internal_site, 0, site) == 0) st->internal_col = c;
    report_fail(st, c, BK_CODE_INTERNAL);
}

// Stop work on column c of task tid if an earlier (or the same) column already
// failed, a wait gave up, or this task or one of its descendants ran out of L/U
// room (the host regrows and starts over; independent tasks run on, so one
// attempt finds the first overflow of every task).
__device__ __forceinline__ bool should_stop(const bk_dev &d, int tid, int c)
{
    const unsigned long long f = *reinterpret_cast<const volatile unsigned long long *>(&d.status->first_fail);
    const int to = *reinterpret_cast<const volatile int *>(&d.status->timeout);
    const int ts = *reinterpret_cast<const volatile int *>(d.task_stop + tid);
    return ts != 0 || to != 0 || (long long)(f >> 8) <= (long long)c;
}

// A region of count entries from a spill pool; -1 if the pool is exhausted.
__device__ __forceinline__ int64_t pool_alloc(unsigned long long *next, int64_t end, int64_t count)
{
    const unsigned long long cnt = (unsigned long long)((count + 3) & ~(int64_t)3);
    const unsigned long long b = atomicAdd(next, cnt);
    return (int64_t)(b + cnt) <= end ? (int64_t)b : -1;
}

// Room for a U column that outgrew its region after nu entries: twice what it
// holds so far (a column may move again; the copies add up to at most twice its
// final size), never more than its largest possible size.
__device__ __forceinline__ int64_t grown_ucap(int nu, int64_t bound)
{
    return min((long long)bound, (long long)(2 * ((int64_t)nu + 2) + 16));
}

// Column c of task T ran out of room (what: 1 = L, 2 = U): flag it for the
// host, and stop the task and every ND ancestor (their input is incomplete).
__device__ __forceinline__ void report_overflow(const bk_dev &d, const bk_task &T, int tid, int c, int what)
{
    atomicOr(d.col_over + c, what);
    atomicExch(&d.status->capacity, 1);
    atomicExch(d.task_stop + tid, 1);
    for (int a = 0; a < T.nanc; a++) atomicExch(d.task_stop + d.col_task[T.anc_lo[a]], 1);
}

}  // namespace bk
