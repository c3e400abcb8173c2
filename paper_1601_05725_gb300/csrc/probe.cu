// probe.cu -- the latencies that set the floor of the dependency chains.
//
// The factorization and the solve advance along chains of columns or rows, each
// link a point-to-point handoff through a flag in global memory (Sec. IV: a
// thread waits for the columns it reads instead of a barrier), followed by the
// link's own arithmetic.  Three numbers bound a link from below: one flag handoff
// between two blocks (release store, acquire load), one dependent FP64 fma, and
// one FP64 division (a backward solve's diagonal, a column's pivot reciprocal).
#include <cuda_runtime.h>

#include "basker.h"
#include "basker_internal.h"
#include "device_util.cuh"

using namespace bk;

namespace {

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Two blocks (one thread each) pass a counter back and forth `hops` times; the
// handoffs take out[0] ns.  Every wait is bounded: past `budget` cycles the
// block sets *err and returns.
__global__ void bk_probe_hop_kernel(int *flags, int hops, long long budget, unsigned long long *out, int *err)
{
    if (threadIdx.x != 0) return;
    const int me = blockIdx.x;
    int *mine = flags + me, *theirs = flags + (1 - me);
    const unsigned long long t0 = global_ns();
    for (int i = 1; i <= hops; i++) {
        if (me == 0) st_release(mine, i);
        const long long c0 = clock64();
        while (ld_acquire(theirs) != i) {
            if (*reinterpret_cast<volatile int *>(err) || clock64() - c0 > budget) {
                atomicExch(err, 1);
                return;
            }
        }
        if (me == 1) st_release(mine, i);
    }
    if (me == 0) out[0] = global_ns() - t0;
}

// One thread: `n` dependent fmas, then `n` dependent divisions; ns of each run.
__global__ void bk_probe_fp64_kernel(double a, double b, int n, unsigned long long *out, double *sink)
{
    double x = a;
    unsigned long long t0 = global_ns();
    for (int i = 0; i < n; i++) x = fma(x, b, a);
    unsigned long long t1 = global_ns();
    double y = x + 1.5;
    for (int i = 0; i < n; i++) y = b / y;
    unsigned long long t2 = global_ns();
    out[1] = t1 - t0;
    out[2] = t2 - t1;
    sink[0] = x + y;
}

}  // namespace

extern "C" int basker_probe_latency(double *ns_out)
{
    if (!ns_out) return BASKER_ERR_INVALID_ARG;
    int *flags = nullptr, *err = nullptr;
    unsigned long long *out = nullptr;
    double *sink = nullptr;
    constexpr int HOPS = 2000, FMAS = 4096;
    int status = BASKER_OK;
    if (cudaMalloc((void **)&flags, 4 * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&out, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&sink, sizeof(double)) != cudaSuccess) {
        status = BASKER_ERR_OOM;
    } else {
        err = flags + 2;
        cudaMemset(flags, 0, 4 * sizeof(int));
        cudaMemset(out, 0, 4 * sizeof(unsigned long long));
        // warm-up launches, then the measured ones
        for (int rep = 0; rep < 2 && status == BASKER_OK; rep++) {
            cudaMemset(flags, 0, 4 * sizeof(int));
            bk_probe_hop_kernel<<<2, 32>>>(flags, HOPS, 2000000000LL, out, err);
            bk_probe_fp64_kernel<<<1, 1>>>(1.0000001, 0.9999999, FMAS, out, sink);
            if (cudaDeviceSynchronize() != cudaSuccess) status = BASKER_ERR_CUDA;
        }
        unsigned long long h[4] = {0, 0, 0, 0};
        int herr = 0;
        if (status == BASKER_OK && (cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess ||
                                    cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess))
            status = BASKER_ERR_CUDA;
        if (status == BASKER_OK && herr) status = BASKER_ERR_TIMEOUT;
        if (status == BASKER_OK) {
            ns_out[0] = (double)h[0] / (2.0 * HOPS);
            ns_out[1] = (double)h[1] / FMAS;
            ns_out[2] = (double)h[2] / FMAS;
        }
    }
    cudaFree(flags);
    cudaFree(out);
    cudaFree(sink);
    return status;
}
