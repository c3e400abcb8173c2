// refine_internal.h -- FP64 refinement of FP32 solves (refine.cu).
#pragma once

#include <cstdint>

#include "basker_internal.h"

struct bk_refine_dev {
    double *Bx64;                // B's values in FP64, CSC order (as Bx)
    const int64_t *Brp;          // B by rows: n + 1 starts
    const int32_t *Brj;          // column of each entry
    const int32_t *Brpos;        // position of each entry in B's CSC arrays
    const int32_t *blk;          // BTF block of each row / column
    double *bmax, *umax;         // per block: max |B_d|, max |U_d|
};

void bk_launch_gather64(const bk_dev &d, const bk_refine_dev &rf, const double *values, int64_t nnz, void *stream);
// norms[0] = ||B||_inf, norms[1] = max over blocks of max|U_d| / max|B_d|
void bk_launch_norms(const bk_dev &d, const bk_refine_dev &rf, double *norms, void *stream);
void bk_launch_ir_start(const bk_dev &d, int32_t nrhs, const double *b, int32_t ldb, double *c, double *r,
                        double *z, double *cmax, void *stream);
void bk_launch_ir_step(const bk_dev &d, const bk_refine_dev &rf, int32_t nrhs, const double *c, double *z,
                       const double *dz, double *r, double *zmax, double *rmax, void *stream);
void bk_launch_ir_finish(const bk_dev &d, int32_t nrhs, const double *z, double *x, int32_t ldx, void *stream);
