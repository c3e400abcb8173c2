// noalloc.cu -- basker_solve_noalloc: the solve of basker_solve with its two work
// vectors (forward results and solution, indexed by pivot step) in a fixed array
// of this library's device memory, so that the call allocates nothing.  Host
// code only sees the array's name as a host-side stand-in; its device address
// is looked up once per device (cudaGetSymbolAddress, with that device current)
// and passed to the kernel.
#include <cuda_runtime.h>

#include <mutex>

#include "basker_internal.h"

int bk_handle_device(basker_t h);
int32_t bk_handle_n(basker_t h);
int64_t bk_solve_scratch_doubles(basker_t h, int32_t nrhs);
int bk_solve_on_scratch(basker_t h, int32_t nrhs, const double *b_dev, int32_t ldb, double *x_dev, int32_t ldx,
                        double *scratch, void *stream);

// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) double bk_noalloc_scratch[BASKER_NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_scratch[kMaxDevices] = {};

// Device address of the array on device dev (dev must be current).
int scratch_on(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return BASKER_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, bk_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return BASKER_ERR_CUDA;
        }
        g_scratch[dev] = static_cast<double *>(p);
    }
    *out = g_scratch[dev];
    return BASKER_OK;
}

}  // namespace

extern "C" int basker_solve_noalloc(basker_t h, int32_t nrhs, const double *b_dev, int32_t ldb, double *x_dev,
                                    int32_t ldx, void *stream)
{
    if (!h || nrhs < 0) return BASKER_ERR_INVALID_ARG;
    const int dev = bk_handle_device(h);
    const int32_t n = bk_handle_n(h);
    if (nrhs > 0 && (!b_dev || !x_dev || ldb < n || ldx < n)) return BASKER_ERR_INVALID_ARG;
    if (bk_solve_scratch_doubles(h, nrhs) > (int64_t)BASKER_NOALLOC_SCRATCH_DOUBLES)
        return BASKER_ERR_INVALID_ARG;          // larger than the fixed array
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return BASKER_ERR_CUDA;
    }
    double *scratch = nullptr;
    const int st = scratch_on(dev, &scratch);
    if (st != BASKER_OK) return st;
    return bk_solve_on_scratch(h, nrhs, b_dev, ldb, x_dev, ldx, scratch, stream);
}
