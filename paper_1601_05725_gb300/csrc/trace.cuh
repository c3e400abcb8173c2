// trace.cuh -- optional per-item timeline of the persistent kernels.
//
// Built only with -DBK_TRACE (never in the library's normal build): each warp
// that finishes an item (a column of the stored-pattern pass, of a round, of the
// descendant phase; a separator's dense elimination; a solve item; a column
// level) appends one record {kind | mode | id, start ns, end ns, SM | warp} to
// bk_dev::trace, whose first word counts the records.  The timeline shows the
// chains of dependent items that set each kernel's duration.
#pragma once

#include <cstdint>

#define BK_TRACE_CAP (1 << 22)     // records kept (32 bytes each)

enum { BK_TR_STATIC = 1, BK_TR_ROUND = 2, BK_TR_DESC = 3, BK_TR_DENSE = 4, BK_TR_SOLVE = 5, BK_TR_LEVELS = 6, BK_TR_REPAIR = 7, BK_TR_PHASE = 8 };

#ifdef BK_TRACE
__device__ __forceinline__ unsigned long long bk_gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bk_trace_rec(unsigned long long *buf, int kind, int mode, int id,
                                             unsigned long long t0)
{
    if (!buf) return;
    const unsigned long long t1 = bk_gtime();
    const unsigned long long i = atomicAdd(buf, 1ull);
    if (i >= BK_TRACE_CAP) return;
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    unsigned long long *r = buf + 4 + 4 * i;
    r[0] = ((unsigned long long)kind << 56) | ((unsigned long long)(mode & 0xff) << 48) | (unsigned)id;
    r[1] = t0;
    r[2] = t1;
    r[3] = ((unsigned long long)sm << 32) | ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
}
// a record whose two time fields carry other numbers (cycle counts)
__device__ __forceinline__ void bk_trace_raw(unsigned long long *buf, int kind, int mode, int id,
                                             unsigned long long a, unsigned long long b)
{
    if (!buf) return;
    const unsigned long long i = atomicAdd(buf, 1ull);
    if (i >= BK_TRACE_CAP) return;
    unsigned long long *r = buf + 4 + 4 * i;
    r[0] = ((unsigned long long)kind << 56) | ((unsigned long long)(mode & 0xff) << 48) | (unsigned)id;
    r[1] = a;
    r[2] = b;
    r[3] = 0;
}
#define BK_TSTART(v) const unsigned long long v = bk_gtime()
#define BK_TREC(buf, kind, mode, id, t0) bk_trace_rec(buf, kind, mode, id, t0)
// phases inside one item: v holds the start of the current phase
#define BK_TPHASE0(v) unsigned long long v = bk_gtime()
#define BK_TPHASE(buf, v, phase, id)                                   \
    do {                                                               \
        if ((threadIdx.x & 31) == 0) bk_trace_rec(buf, BK_TR_PHASE, phase, id, v); \
        v = bk_gtime();                                                \
    } while (0)
#else
#define BK_TSTART(v)
#define BK_TREC(buf, kind, mode, id, t0)
#define BK_TPHASE0(v)
#define BK_TPHASE(buf, v, phase, id)
#endif
