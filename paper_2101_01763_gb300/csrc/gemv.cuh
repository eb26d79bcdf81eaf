// Batched gather-GEMV used by the spaND apply sweeps (Sec. 2.2.1: the
// preconditioner is the product of the stored elimination, scaling and
// orthogonal operators).  Every operator application is
//     y[yidx[i]] = base[bidx[i]] + alpha * sum_t (op(M_t) x_t)[i]
// with x_t[j] = src[xidx[j]] - xsub[j]; M null means the identity.  Matrices
// are column-major; tri marks a stored lower (1) / upper (2) triangle so the
// kernel skips the zero half.  One CTA per 64 output rows of a task; the x
// vectors are staged in shared memory.  The sweeps alternate two vectors so
// no launch reads what another CTA of the same launch writes.
#pragma once
#include <cuda_runtime.h>

namespace spand {

template <typename T>
struct GvTerm {
  const T* M;
  const T* x;
  const int* xidx;
  const T* xsub;
  int ld, k, trans, tri;
};

template <typename T>
struct GvTask {
  T* y;
  const int* yidx;
  const T* base;
  const int* bidx;
  T* y2;
  T alpha;
  int m, t0, t1;
};

struct GvTile {
  int task, r0;
};

constexpr int GV_ROWS = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_gemv(const GvTask<T>* tasks, const GvTerm<T>* terms,
                                              const GvTile* tiles) {
  extern __shared__ unsigned char gv_smem[];
  T* xs = reinterpret_cast<T*>(gv_smem);
  __shared__ T part[4][GV_ROWS];
  const GvTile tl = tiles[blockIdx.x];
  const GvTask<T> tk = tasks[tl.task];
  const int r0 = tl.r0, rows = min(GV_ROWS, tk.m - r0);
  const int tid = threadIdx.x;
  T acc = 0;                                       // threads 0..63 own the output rows
  for (int t = tk.t0; t < tk.t1; ++t) {
    const GvTerm<T> tm = terms[t];
    __syncthreads();
    for (int j = tid; j < tm.k; j += blockDim.x) {
      T v = tm.xidx ? tm.x[tm.xidx[j]] : tm.x[j];
      if (tm.xsub) v -= tm.xsub[j];
      xs[j] = v;
    }
    __syncthreads();
    if (!tm.M) {
      if (tid < rows) acc += xs[r0 + tid];
      continue;
    }
    // column range with possibly non-zero entries for this row tile
    int jlo = 0, jhi = tm.k;
    const bool lower_eff = (tm.tri == 1 && !tm.trans) || (tm.tri == 2 && tm.trans);
    const bool upper_eff = (tm.tri == 2 && !tm.trans) || (tm.tri == 1 && tm.trans);
    if (lower_eff) jhi = min(tm.k, r0 + GV_ROWS);
    if (upper_eff) jlo = min(tm.k, r0);
    if (!tm.trans) {
      const int r = tid & 63, sl = tid >> 6;        // 64 rows x 4 column slices
      T s = 0;
      if (r < rows) {
        const T* Mp = tm.M + (r0 + r);
        for (int j = jlo + sl; j < jhi; j += 4) s += Mp[(size_t)j * tm.ld] * xs[j];
      }
      part[sl][r] = s;
    } else {
      const int lane = tid & 31, w = tid >> 5;      // warp per output row
      for (int r = w; r < GV_ROWS; r += 8) {
        T s = 0;
        if (r < rows) {
          const T* col = tm.M + (size_t)(r0 + r) * tm.ld;
          for (int j = jlo + lane; j < jhi; j += 32) s += col[j] * xs[j];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
          part[0][r] = s;
          part[1][r] = 0;
          part[2][r] = 0;
          part[3][r] = 0;
        }
      }
    }
    __syncthreads();
    if (tid < rows) acc += part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid];
  }
  if (tid < rows) {
    const int i = r0 + tid;
    T v = tk.alpha * acc;
    if (tk.base) v += tk.bidx ? tk.base[tk.bidx[i]] : tk.base[i];
    if (tk.yidx) tk.y[tk.yidx[i]] = v;
    else tk.y[i] = v;
    if (tk.y2) tk.y2[i] = v;
  }
}

}  // namespace spand
