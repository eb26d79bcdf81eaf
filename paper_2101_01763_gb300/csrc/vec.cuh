// Declarations of the vector / tall-skinny helpers shared by GMRES and SpMV.
#pragma once
#include <cstdint>

#include "internal.h"

namespace spand {

int spmv_fused(const bsr_matrix* A, const double* x, double* y, int transpose, double sa, double a1,
               const double* u1, double a2, const double* u2, cudaStream_t st);
// spmv_fused with x in FP32 (x_is_float) or FP64
int spmv_fused_x(const bsr_matrix* A, const void* x, int x_is_float, double* y, int transpose, double sa, double a1,
                 const double* u1, double a2, const double* u2, cudaStream_t st);
int gram(int64_t N, int nz, const double* const* dZ, int ny, const double* const* dY, double* part, int nblk,
         double* G, int ldg, cudaStream_t st);
int block_update(int64_t N, int s, int ny, const double* Y, int64_t ldy, const double* Sinv, int nz,
                 const double* Z, int64_t ldz, const double* C, int ldc, double* X, int64_t ldx, int accumulate,
                 cudaStream_t st);
int scale_copy(int64_t N, const double* a, double* b, const double* scal, int invert, cudaStream_t st);
int axpy_dev(int64_t N, const double* coef, double sign, const double* x, double* y, cudaStream_t st);
// direct = true runs the apply's launches one by one on st, never through the
// factor's CUDA graph (building a graph allocates; see the no-allocation solve)
int factor_apply(spand_factor_t F, const double* r, double* z, int transpose, cudaStream_t st, bool direct = false);
int factor_size(spand_factor_t F);
// The preconditioner's sweeps on r without the final conversion: *w receives
// the factor's own output vector (device, N values in the DOF order, FP32 when
// *w_is_float, else FP64), valid until the factor's next apply.
int factor_apply_slot(spand_factor_t F, const double* r, int transpose, cudaStream_t st, bool direct, const void** w,
                      int* w_is_float);

}  // namespace spand
