// Block-CSR SpMV (FP64) and the tall-skinny vector kernels of s-step GMRES.
//
// bsr_spmv: y = A x for the DG block pattern (Algorithm 2, the SpMV of the
// matrix-powers step).  Blocks are column-major so for a fixed block column
// consecutive rows are consecutive doubles.  The fused form y = sa*(A x) + a1*u1 + a2*u2 also gives residuals and the Newton
// recurrence v_{k+1} = A M^-1 v_k - theta v_k (+ Im(theta)^2 v_{k-1}).
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "vec.cuh"

namespace spand {

// y = sa * A x + a1 * u1 + a2 * u2 (u1, u2 optional).  Each row's columns are
// split over the 8 warps of a CTA: a CTA owns 32 consecutive rows (lane = row,
// so a warp reads 32 consecutive entries of a block column), warp w sums block
// columns w*cs .. w*cs+cs-1 of every block of the row, and warp 0 adds the 8
// partial sums: eight times as many threads as rows and an eighth of the
// dependent loads per thread.
// x may be FP64 or FP32 (the FP32 preconditioner's own output vector, read in
// place by the matrix-powers step); the products are accumulated in FP64.
template <typename TX>
__global__ void __launch_bounds__(256) k_bsr_spmv(int K, int B, const int* __restrict__ row_ptr,
                                                        const int* __restrict__ col, const double* __restrict__ val,
                                                        const TX* __restrict__ x, double* __restrict__ y,
                                                        double sa, double a1, const double* __restrict__ u1,
                                                        double a2, const double* __restrict__ u2) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * 32 + lane;
  const int64_t N = (int64_t)K * B;
  double s = 0;
  if (g < N) {
    const int e = (int)(g / B), r = (int)(g % B);
    const size_t bb = (size_t)B * B;
    const int cs = (B + 7) / 8, c0 = w * cs, c1 = min(B, c0 + cs);
    double s1 = 0;
    for (int k = row_ptr[e]; k < row_ptr[e + 1]; ++k) {
      const double* blk = val + (size_t)k * bb + r;
      const TX* xv = x + (size_t)col[k] * B;
      int c = c0;
      for (; c + 2 <= c1; c += 2) {
        s += __ldg(blk + (size_t)c * B) * (double)__ldg(xv + c);
        s1 += __ldg(blk + (size_t)(c + 1) * B) * (double)__ldg(xv + c + 1);
      }
      if (c < c1) s += __ldg(blk + (size_t)c * B) * (double)__ldg(xv + c);
    }
    s += s1;
  }
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && g < N) {
    double t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][lane];
    double v = sa * t;
    if (u1) v += a1 * u1[g];
    if (u2) v += a2 * u2[g];
    y[g] = v;
  }
}

// y = A^T x: row e' of A^T gathers block (e, e') of every neighbour e (symmetric pattern)
template <typename TX>
__global__ void __launch_bounds__(256) k_bsr_spmv_t(int K, int B, const int* __restrict__ row_ptr,
                                                    const int* __restrict__ col, const double* __restrict__ val,
                                                    const TX* __restrict__ x, double* __restrict__ y, double sa,
                                                    double a1, const double* __restrict__ u1, double a2,
                                                    const double* __restrict__ u2) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)K * B) return;
  const int ep = (int)(g / B), c = (int)(g % B);
  const size_t bb = (size_t)B * B;
  double s = 0;
  for (int j = row_ptr[ep]; j < row_ptr[ep + 1]; ++j) {
    const int e = col[j];
    int kk = -1;
    for (int k = row_ptr[e]; k < row_ptr[e + 1]; ++k)
      if (col[k] == ep) kk = k;
    if (kk < 0) continue;
    const double* blk = val + (size_t)kk * bb + (size_t)c * B;   // column c of block (e, e')
    const TX* xv = x + (size_t)e * B;
    for (int r = 0; r < B; ++r) s += blk[r] * (double)xv[r];
  }
  double v = sa * s;
  if (u1) v += a1 * u1[g];
  if (u2) v += a2 * u2[g];
  y[g] = v;
}

template <typename TX>
static int spmv_launch(const bsr_matrix* A, const TX* x, double* y, int transpose, double sa, double a1,
                       const double* u1, double a2, const double* u2, cudaStream_t st) {
  const int64_t n = (int64_t)A->K * A->B;
  const unsigned g = (unsigned)((n + 255) / 256);
  note_launch();
  if (!transpose)
    k_bsr_spmv<TX><<<(unsigned)((n + 31) / 32), 256, 0, st>>>(A->K, A->B, A->row_ptr, A->col, A->val, x, y, sa,
                                                                   a1, u1, a2, u2);
  else
    k_bsr_spmv_t<TX><<<g, 256, 0, st>>>(A->K, A->B, A->row_ptr, A->col, A->val, x, y, sa, a1, u1, a2, u2);
  return cudaGetLastError() == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
}

int spmv_fused(const bsr_matrix* A, const double* x, double* y, int transpose, double sa, double a1,
               const double* u1, double a2, const double* u2, cudaStream_t st) {
  return spmv_launch<double>(A, x, y, transpose, sa, a1, u1, a2, u2, st);
}

int spmv_fused_x(const bsr_matrix* A, const void* x, int x_is_float, double* y, int transpose, double sa, double a1,
                 const double* u1, double a2, const double* u2, cudaStream_t st) {
  if (x_is_float)
    return spmv_launch<float>(A, static_cast<const float*>(x), y, transpose, sa, a1, u1, a2, u2, st);
  return spmv_launch<double>(A, static_cast<const double*>(x), y, transpose, sa, a1, u1, a2, u2, st);
}

// ------------------------------------------------------------------ Gram: G = Z^T Y
// Z: nz columns given by pointers, Y: ny <= 32 columns given by pointers.
// Each CTA covers a row range and writes partial sums; a second kernel adds
// the partials in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_gram_partial(int64_t N, int nz, const double* const* Z, int ny,
                                                      const double* const* Y, double* part) {
  __shared__ double ys[32][129];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = min(N, lo + per);
  double* P = part + (size_t)blockIdx.x * nz * ny;
  // accumulators: warp w handles z columns w, w+8, ...; each lane keeps ny partial dots
  for (int a0 = 0; a0 < nz; a0 += 8) {
    const int a = a0 + wid;
    double acc[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) acc[b] = 0;
    for (int64_t r0 = lo; r0 < hi; r0 += 128) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < ny * 128; idx += 256) {
        const int b = idx / 128, rr = idx % 128;
        ys[b][rr] = (r0 + rr < hi) ? Y[b][r0 + rr] : 0.0;
      }
      __syncthreads();
      if (a < nz) {
        for (int rr = lane; rr < 128; rr += 32) {
          const double zv = (r0 + rr < hi) ? Z[a][r0 + rr] : 0.0;
#pragma unroll
          for (int b = 0; b < 32; ++b)
            if (b < ny) acc[b] += zv * ys[b][rr];
        }
      }
    }
    if (a < nz) {
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        if (b >= ny) break;
        double v = acc[b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) P[a * ny + b] = v;
      }
    }
  }
}

__global__ void k_gram_reduce(int nblk, int nz, int ny, const double* part, double* G, int ldg) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nz * ny) return;
  const int a = t / ny, b = t % ny;
  double s = 0;
  for (int k = 0; k < nblk; ++k) s += part[(size_t)k * nz * ny + t];
  G[a + (size_t)b * ldg] = s;   // column-major nz x ny
}

int gram(int64_t N, int nz, const double* const* dZ, int ny, const double* const* dY, double* part, int nblk,
         double* G, int ldg, cudaStream_t st) {
  if (ny > 32 || nz <= 0 || ny <= 0) return SPAND_ERR_ARG;
  note_launch();
  k_gram_partial<<<nblk, 256, 0, st>>>(N, nz, dZ, ny, dY, part);
  note_launch();
  k_gram_reduce<<<(nz * ny + 127) / 128, 128, 0, st>>>(nblk, nz, ny, part, G, ldg);
  return cudaGetLastError() == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
}

// ------------------------------------------------------------------ block update
// X[:, j] = sum_b Y[:, b] Sinv[b, j] - sum_a Z[:, a] C[a, j]   (j < s), column-major
// coefficient matrices Sinv (ny x s, ld ny) and C (nz x s, ld ldc) in device memory.
__global__ void __launch_bounds__(256) k_block_update(int64_t N, int s, int ny, const double* Y, int64_t ldy,
                                                      const double* Sinv, int nz, const double* Z, int64_t ldz,
                                                      const double* C, int ldc, double* X, int64_t ldx,
                                                      int accumulate) {
  extern __shared__ double cs[];
  double* sS = cs;                 // ny * s
  double* sC = cs + ny * s;        // nz * s
  for (int i = threadIdx.x; i < ny * s; i += blockDim.x) sS[i] = Sinv[i];
  for (int i = threadIdx.x; i < nz * s; i += blockDim.x) sC[i] = C[(i % nz) + (size_t)(i / nz) * ldc];
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    double out[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = 0;
    for (int b = 0; b < ny; ++b) {
      const double yv = Y[r + b * ldy];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < s) out[j] += yv * sS[b + j * ny];
    }
    for (int a = 0; a < nz; ++a) {
      const double zv = Z[r + a * ldz];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < s) out[j] -= zv * sC[a + j * nz];
    }
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < s) {
        if (accumulate) X[r + j * ldx] += out[j];
        else X[r + j * ldx] = out[j];
      }
  }
}

int block_update(int64_t N, int s, int ny, const double* Y, int64_t ldy, const double* Sinv, int nz,
                 const double* Z, int64_t ldz, const double* C, int ldc, double* X, int64_t ldx, int accumulate,
                 cudaStream_t st) {
  if (s > 16) return SPAND_ERR_ARG;
  const size_t sm = (size_t)(ny + nz) * s * sizeof(double);
  static std::atomic<uint64_t> attr{0};
  once_per_device(attr, [] { set_dyn_smem((const void*)k_block_update, 200 * 1024); });
  const unsigned g = (unsigned)std::min<int64_t>(152 * 8, (N + 255) / 256);
  note_launch();
  k_block_update<<<g, 256, sm, st>>>(N, s, ny, Y, ldy, Sinv, nz, Z, ldz, C, ldc, X, ldx, accumulate);
  return cudaGetLastError() == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
}

__global__ void k_scale_copy(int64_t N, const double* a, double* b, const double* scal, int invert) {
  const double s = invert ? 1.0 / *scal : *scal;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i] * s;
}

int scale_copy(int64_t N, const double* a, double* b, const double* scal, int invert, cudaStream_t st) {
  const unsigned g = (unsigned)std::min<int64_t>(152 * 8, (N + 255) / 256);
  note_launch();
  k_scale_copy<<<g, 256, 0, st>>>(N, a, b, scal, invert);
  return cudaGetLastError() == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
}

__global__ void k_axpy_dev(int64_t N, const double* coef, double sign, const double* x, double* y) {
  const double a = sign * *coef;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

int axpy_dev(int64_t N, const double* coef, double sign, const double* x, double* y, cudaStream_t st) {
  const unsigned g = (unsigned)std::min<int64_t>(152 * 8, (N + 255) / 256);
  note_launch();
  k_axpy_dev<<<g, 256, 0, st>>>(N, coef, sign, x, y);
  return cudaGetLastError() == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
}

// out[k] = alpha * u_row(k) v_col(k)^T for every stored block k (column-major)
__global__ void __launch_bounds__(256) k_pattern_outer(int K, int B, const int* __restrict__ row_ptr,
                                                       const int* __restrict__ col, const double* __restrict__ u,
                                                       const double* __restrict__ v, double alpha,
                                                       double* __restrict__ out) {
  const int e = blockIdx.x;
  if (e >= K) return;
  const size_t bb = (size_t)B * B;
  for (int k = row_ptr[e]; k < row_ptr[e + 1]; ++k) {
    const double* ue = u + (size_t)e * B;
    const double* vc = v + (size_t)col[k] * B;
    double* o = out + (size_t)k * bb;
    for (int idx = threadIdx.x; idx < B * B; idx += blockDim.x) {
      const int r = idx % B, c = idx / B;
      o[idx] = alpha * ue[r] * vc[c];
    }
  }
}

}  // namespace spand

extern "C" int bsr_pattern_outer(const bsr_matrix* A, const double* u, const double* v, double alpha, double* out,
                                 cudaStream_t stream) {
  if (!A || !u || !v || !out || !A->row_ptr || !A->col || A->K <= 0 || A->B <= 0) return SPAND_ERR_ARG;
  spand::note_launch();
  spand::k_pattern_outer<<<A->K, 256, 0, stream>>>(A->K, A->B, A->row_ptr, A->col, u, v, alpha, out);
  return cudaGetLastError() == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
}

extern "C" int bsr_spmv(const bsr_matrix* A, const double* x, double* y, int transpose, cudaStream_t stream) {
  if (!A || !x || !y || x == y || !A->row_ptr || !A->col || !A->val || A->K <= 0 || A->B <= 0) return SPAND_ERR_ARG;
  return spand::spmv_fused(A, x, y, transpose, 1.0, 0.0, nullptr, 0.0, nullptr, stream);
}
