// refine.cu -- FP64 iterative refinement of the solves.
//
// With FP32 factors (options.precision 1) the triangular solves run in FP32;
// with FP64 factors (precision 2) in FP64.  FP64 holds the residual
// r = c - B z, the update z += dz and the norms of the backward error, all in
// B's row/column space (c = b(P), x(Q) = z):
//   eta = ||c - B z||_inf / (||B||_inf ||z||_inf + ||c||_inf)
// The pivot growth max|U_d| / max|B_d| of every BTF block decides, after each
// factorization, whether the FP32 factors are used at all.
#include <cuda_runtime.h>

#include <algorithm>

#include "basker_internal.h"
#include "device_util.cuh"
#include "refine_internal.h"

using namespace bk;

namespace {

// Maxima of nonnegative doubles through their bit patterns (monotone as integers).
__device__ __forceinline__ void max_nonneg(double *dst, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)__double_as_longlong(v));
}

__global__ void bk_gather64(double *__restrict__ Bx64, const double *__restrict__ vals,
                            const int32_t *__restrict__ bmap, int64_t nnz)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        Bx64[e] = __ldg(vals + bmap[e]);
}

// ||B||_inf (row sums of |B| over the rows of B in CSR order) into norms[0], and
// the per-block maxima of |B| and |U| into bmax / umax.
__global__ void bk_norms_kernel(bk_dev d, bk_refine_dev rf, double *norms)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const float *Ux = vals<float>(d.Ux);
    for (int i = warp; i < d.n; i += nwarps) {
        double s = 0.0, bm = 0.0;
        for (int64_t e = rf.Brp[i] + lane; e < rf.Brp[i + 1]; e += 32) {
            const double v = fabs(rf.Bx64[rf.Brpos[e]]);
            s += v;
            bm = fmax(bm, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(BK_FULL, s, o);
            bm = fmax(bm, __shfl_xor_sync(BK_FULL, bm, o));
        }
        // column i of U (its block is the block of row i: diagonal blocks are square)
        float um = 0.0f;
        if (d.prec) {
            const int64_t ub = d.Ubeg[i];
            const int uc = d.Ucnt[i];
            for (int t = lane; t < uc; t += 32) um = fmaxf(um, fabsf(Ux[ub + t]));
        }
        um = warp_max(um);
        if (lane == 0) {
            max_nonneg(norms, s);
            max_nonneg(rf.bmax + rf.blk[i], bm);
            max_nonneg(rf.umax + rf.blk[i], (double)um);
        }
    }
}

// growth = max over blocks of max|U_d| / max|B_d| into norms[1]
__global__ void bk_growth_kernel(bk_refine_dev rf, int32_t nblocks, double *norms)
{
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < nblocks; d += gridDim.x * blockDim.x) {
        const double b = rf.bmax[d], u = rf.umax[d];
        const double g = b > 0.0 ? u / b : (u > 0.0 ? INFINITY : 0.0);
        max_nonneg(norms + 1, g);
    }
}

// c = b(P) for every right-hand side; ||c||_inf per right-hand side into cmax
__global__ void bk_ir_start(int32_t n, int32_t nrhs, const int32_t *__restrict__ P, const double *__restrict__ b,
                            int32_t ldb, double *c, double *r, double *z, double *cmax)
{
    const int64_t total = (int64_t)n * nrhs;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(k / n), i = (int)(k % n);
        const double v = b[(int64_t)q * ldb + P[i]];
        c[k] = v;
        r[k] = v;
        z[k] = 0.0;
        max_nonneg(cmax + q, fabs(v));
    }
}

// z += dz; ||z||_inf per right-hand side into zmax
__global__ void bk_ir_update(int64_t total, int32_t n, double *z, const double *__restrict__ dz, double *zmax)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double v = z[k] + dz[k];
        z[k] = v;
        max_nonneg(zmax + (int)(k / n), fabs(v));
    }
}

// r = c - B z by rows (one warp a row, the row's terms summed lane-wise then in a
// fixed tree), ||r||_inf per right-hand side into rmax
__global__ void bk_ir_residual(bk_refine_dev rf, int32_t n, int32_t nrhs, const double *__restrict__ c,
                               const double *__restrict__ z, double *r, double *rmax)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp; k < (int64_t)n * nrhs; k += nwarps) {
        const int q = (int)(k / n), i = (int)(k % n);
        const double *zq = z + (int64_t)q * n;
        double s = 0.0;
        for (int64_t e = rf.Brp[i] + lane; e < rf.Brp[i + 1]; e += 32) s = fma(rf.Bx64[rf.Brpos[e]], zq[rf.Brj[e]], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(BK_FULL, s, o);
        if (lane == 0) {
            const double v = c[k] - s;
            r[k] = v;
            max_nonneg(rmax + q, fabs(v));
        }
    }
}

// x(Q) = z
__global__ void bk_ir_finish(int32_t n, int32_t nrhs, const int32_t *__restrict__ Q, const double *__restrict__ z,
                             double *x, int32_t ldx)
{
    const int64_t total = (int64_t)n * nrhs;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(k / n), j = (int)(k % n);
        x[(int64_t)q * ldx + Q[j]] = z[k];
    }
}

int grid_for(int64_t work, int per_block)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + per_block - 1) / per_block, 152 * 16));
}

}  // namespace

void bk_launch_gather64(const bk_dev &d, const bk_refine_dev &rf, const double *values, int64_t nnz, void *stream)
{
    if (nnz <= 0) return;
    bk_gather64<<<grid_for(nnz, 256), 256, 0, (cudaStream_t)stream>>>(rf.Bx64, values, d.bmap, nnz);
}

void bk_launch_norms(const bk_dev &d, const bk_refine_dev &rf, double *norms, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(norms, 0, 2 * sizeof(double), st);
    cudaMemsetAsync(rf.bmax, 0, sizeof(double) * (size_t)std::max(d.nblocks, 1), st);
    cudaMemsetAsync(rf.umax, 0, sizeof(double) * (size_t)std::max(d.nblocks, 1), st);
    if (d.n > 0) bk_norms_kernel<<<grid_for((int64_t)d.n * 32, 256), 256, 0, st>>>(d, rf, norms);
    if (d.nblocks > 0) bk_growth_kernel<<<grid_for(d.nblocks, 256), 256, 0, st>>>(rf, d.nblocks, norms);
}

void bk_launch_ir_start(const bk_dev &d, int32_t nrhs, const double *b, int32_t ldb, double *c, double *r,
                        double *z, double *cmax, void *stream)
{
    const int64_t total = (int64_t)d.n * nrhs;
    if (total <= 0) return;
    bk_ir_start<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(d.n, nrhs, d.P, b, ldb, c, r, z, cmax);
}

void bk_launch_ir_step(const bk_dev &d, const bk_refine_dev &rf, int32_t nrhs, const double *c, double *z,
                       const double *dz, double *r, double *zmax, double *rmax, void *stream)
{
    const int64_t total = (int64_t)d.n * nrhs;
    if (total <= 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    bk_ir_update<<<grid_for(total, 256), 256, 0, st>>>(total, d.n, z, dz, zmax);
    bk_ir_residual<<<grid_for(total * 32, 256), 256, 0, st>>>(rf, d.n, nrhs, c, z, r, rmax);
}

void bk_launch_ir_finish(const bk_dev &d, int32_t nrhs, const double *z, double *x, int32_t ldx, void *stream)
{
    const int64_t total = (int64_t)d.n * nrhs;
    if (total <= 0) return;
    bk_ir_finish<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(d.n, nrhs, d.Q, z, x, ldx);
}
