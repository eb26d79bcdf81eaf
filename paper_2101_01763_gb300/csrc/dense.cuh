// Batched dense kernels on variable-size column-major matrices (FP64 / FP32).
//
// These carry the per-level block operations of spaND (Sec. 2.2.1):
//   * getrf: right-looking blocked LU with partial pivoting (Eq. 10, Eq. 11);
//     one launch per 32-column panel (one CTA per matrix) followed by a
//     grouped GEMM for the trailing update;
//   * grouped GEMM: C = beta C + alpha sum_t op(A_t) op(B_t), one CTA per
//     64x64 output tile, all terms of a target accumulated by that CTA
//     (Schur updates of Eq. 10 without atomics);
//   * triangular inverses: L^-1 P^T and U^-1 (optionally with the scaling
//     split of Eq. 11), one CTA per 32-column tile;
//   * column-pivoted Householder QR truncated at |R_kk| <= eps |R_00| (the
//     rank-revealing QR of Eq. 12) and the explicit Q_c it defines;
//   * block copies / transposed copies / identity fills for gathers and merges.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

namespace spand {

constexpr int LU_NB = 32;
constexpr int LU_NB2 = 128;   // columns per block of the two-level LU

template <typename T>
struct MatRef {      // square matrix for getrf / inverses
  T* A;
  int n;
  int* ipiv;         // n pivots (absolute 0-based rows)
  int* perm;         // n: (P^T b)[k] = b[perm[k]]
  int* aff;          // getrf scratch: per matrix of a batch, the rows a panel moves (1 + 4 LU_NB ints)
};

template <typename T>
struct GemmTask {
  T* C;
  int ldc, m, n;
  T alpha, beta;
  int t0, t1;        // term range
};

template <typename T>
struct GemmTerm {
  const T* A;
  const T* B;
  int lda, ldb, k, ta, tb;
  int tri;           // 1: op(A) lower triangular, 2: op(B) upper triangular (zero k-chunks skipped)
};

// number of k values of term t that can be non-zero for the output tile at (i0, j0)
template <typename T>
__device__ inline int term_klim(const GemmTerm<T>& tm, int i0, int j0, int BM, int BN) {
  if (tm.tri == 1) return min(tm.k, i0 + BM);
  if (tm.tri == 2) return min(tm.k, j0 + BN);
  return tm.k;
}

struct TileItem {
  int task, tm, tn;
};

template <typename T>
struct CopyTask {    // dst[r + c*ldd] = trans ? src[c + r*lds] : src[r + c*lds]
  const T* src;
  T* dst;
  int lds, ldd, rows, cols, trans;
};

struct CopyTile {
  int task, tr, tc;
};

template <typename T>
struct QrTask {
  T* W;              // n x c ROW-major (element (i, j) at i*c + j); overwritten
  T* V;              // n x min(n,c) column-major: reflector k in column k, rows k..n-1 (v_k[k] = 1)
  T* tau;            // min(n, c)
  T* norm2;          // c scratch
  T* Q;              // explicit Q_c output (n x r, ld = n)
  int n, c;
  int* rank;         // output
};

// ------------------------------------------------------------------ reductions
template <typename T>
__device__ inline void argmax_pair(T& v, int& i, T v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

// argmax over the 32 lanes of a warp (largest value, lowest index on ties)
template <typename T>
__device__ inline void warp_argmax(T& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    argmax_pair(v, i, v2, i2);
  }
}

template <typename T>
__device__ inline void block_argmax(T& v, int& idx, T* sv, int* si) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    T v2 = __shfl_down_sync(0xffffffffu, v, o);
    int i2 = __shfl_down_sync(0xffffffffu, idx, o);
    argmax_pair(v, idx, v2, i2);
  }
  if (lane == 0) {
    sv[wid] = v;
    si[wid] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T bv = sv[0];
    int bi = si[0];
    for (int w = 1; w < nw; ++w) argmax_pair(bv, bi, sv[w], si[w]);
    sv[0] = bv;
    si[0] = bi;
  }
  __syncthreads();
  v = sv[0];
  idx = si[0];
  __syncthreads();
}

template <typename T>
__device__ inline T block_sum(T v, T* sv) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sv[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T s = 0;
    for (int w = 0; w < nw; ++w) s += sv[w];
    sv[0] = s;
  }
  __syncthreads();
  v = sv[0];
  __syncthreads();
  return v;
}

template <typename T>
__device__ inline T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ getrf panel
// Factor columns k0..k0+jb-1 of every matrix (rows k0..n-1) with partial
// pivoting, swap whole rows, then U12 = L11^-1 A12.  flags[0] |= 1 on an exact
// zero pivot, flags[0] |= 2 on a non-finite pivot.
// Row interchanges reach every column; U12 = L11^-1 A12 is formed for the
// columns in [k0 + jb, tcol) (the rest wait for the end of their block).
template <typename T>
__global__ void __launch_bounds__(256) k_getrf_panel(const MatRef<T>* mats, int nmat, int k0, int tcol, int* flags) {
  __shared__ T sv[32];
  __shared__ int si[32];
  __shared__ T L11[LU_NB][LU_NB + 1];
  __shared__ T urow[LU_NB];                 // pivot row segment of the panel
  const int b = blockIdx.x;
  if (b >= nmat) return;
  const MatRef<T> M = mats[b];
  const int n = M.n;
  if (k0 >= n) return;
  T* A = M.A;
  const size_t ld = n;
  const int jb = min(LU_NB, n - k0);
  for (int j = k0; j < k0 + jb; ++j) {
    T best = -1;
    int bi = n;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
      T a = fabs(A[i + j * ld]);
      if (a != a) a = (T)INFINITY;        // NaN ranks first so it is caught
      argmax_pair(best, bi, a, i);
    }
    block_argmax(best, bi, sv, si);
    const int p = bi;
    if (threadIdx.x == 0) M.ipiv[j] = p;
    if (p != j)
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        T t = A[j + c * ld];
        A[j + c * ld] = A[p + c * ld];
        A[p + c * ld] = t;
      }
    __syncthreads();
    const T piv = A[j + j * ld];
    for (int c = j + 1 + threadIdx.x; c < k0 + jb; c += blockDim.x) urow[c - k0] = A[j + c * ld];
    __syncthreads();
    if (!(piv == piv) || isinf(piv)) {
      if (threadIdx.x == 0) atomicOr(flags, 2);
    } else if (piv == (T)0) {
      if (threadIdx.x == 0) atomicOr(flags, 1);
    } else {
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
        // the row's panel segment is loaded before any store so the loads overlap
        const T a = A[i + j * ld];
        T x[LU_NB];
#pragma unroll
        for (int c = 0; c < LU_NB; ++c) x[c] = (c > j - k0 && c < jb) ? A[i + (size_t)(k0 + c) * ld] : (T)0;
        const T l = a / piv;
        A[i + j * ld] = l;
#pragma unroll
        for (int c = 0; c < LU_NB; ++c)
          if (c > j - k0 && c < jb) A[i + (size_t)(k0 + c) * ld] = x[c] - l * urow[c];
      }
    }
    __syncthreads();
  }
  // U12 = L11^-1 A12
  for (int t = threadIdx.x; t < jb * jb; t += blockDim.x) {
    const int r = t % jb, c = t / jb;
    L11[r][c] = A[(k0 + r) + (size_t)(k0 + c) * ld];
  }
  __syncthreads();
  const int cend = min(n, tcol);
  for (int c = k0 + jb + threadIdx.x; c < cend; c += blockDim.x) {
    T x[LU_NB];
    T* col = A + (size_t)c * ld + k0;
#pragma unroll
    for (int r = 0; r < LU_NB; ++r) x[r] = (r < jb) ? col[r] : (T)0;
#pragma unroll
    for (int r = 1; r < LU_NB; ++r) {
      T s = x[r];
#pragma unroll
      for (int q = 0; q < r; ++q) s -= L11[r][q] * x[q];
      x[r] = s;
    }
#pragma unroll
    for (int r = 0; r < LU_NB; ++r)
      if (r < jb) col[r] = x[r];
  }
}

// The panel's interchanges as one row gather for the columns outside it:
// after the swaps, row pos[i] holds what row src[i] held (rows relative to k0;
// at most 2 jb rows move).  rec[0] = count, rec[1..] = pos, rec[1 + 2 LU_NB..]
// = src.  One thread.
__device__ inline void lu_record_interchanges(int* rec, const int* piv_loc, int jb) {
  int pos[2 * LU_NB], src[2 * LU_NB];
  int cnt = 0;
  for (int j = 0; j < jb; ++j) {
    pos[cnt] = j;
    src[cnt] = j;
    ++cnt;
  }
  for (int j = 0; j < jb; ++j) {
    const int pj = piv_loc[j];
    if (pj == j) continue;
    int a = -1, b = -1;
    for (int t = 0; t < cnt; ++t) {
      if (pos[t] == j) a = t;
      if (pos[t] == pj) b = t;
    }
    if (b < 0) {                     // first time row pj moves
      pos[cnt] = pj;
      src[cnt] = pj;
      b = cnt++;
    }
    const int t = src[a];
    src[a] = src[b];
    src[b] = t;
  }
  rec[0] = cnt;
  for (int t = 0; t < cnt; ++t) {
    rec[1 + t] = pos[t];
    rec[1 + 2 * LU_NB + t] = src[t];
  }
}

// The panel step of k_getrf_panel with the panel (rows k0..n-1 of the 32 panel
// columns) staged in shared memory: pivot search, interchanges, scaling and the
// rank-1 updates run on-chip; afterwards the panel is written back and the rows
// its interchanges move are recorded for k_getrf_swap_trsm, which updates the
// columns outside the panel.  Used when (n - k0) * 32 values fit the shared
// budget.
constexpr int LU_SMEM_BYTES = 200 * 1024;

template <typename T>
__global__ void __launch_bounds__(512) k_getrf_panel_smem(const MatRef<T>* mats, int nmat, int k0, int* flags) {
  extern __shared__ unsigned char lu_smem[];
  T* P = reinterpret_cast<T*>(lu_smem);          // panel, column-major m x jb (ld m)
  __shared__ T sv[32];
  __shared__ int si[32];
  __shared__ int piv_loc[LU_NB];
  const int b = blockIdx.x;
  if (b >= nmat) return;
  const MatRef<T> M = mats[b];
  const int n = M.n;
  if (k0 >= n) return;
  T* A = M.A;
  const size_t ld = n;
  const int jb = min(LU_NB, n - k0), m = n - k0;
  if ((size_t)m * jb * sizeof(T) > (size_t)LU_SMEM_BYTES) return;   // host routes these elsewhere
  for (int idx = threadIdx.x; idx < m * jb; idx += blockDim.x) {
    const int r = idx % m, c = idx / m;
    P[idx] = A[(k0 + r) + (size_t)(k0 + c) * ld];
  }
  __syncthreads();
  // pivot of column 0; later columns get theirs from the rank-1 update pass
  // (each thread tracks |P(i, j+1)| of its rows as it updates them)
  int p;
  {
    T best = -1;
    int bi = m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      T a = fabs(P[i]);
      if (a != a) a = (T)INFINITY;
      argmax_pair(best, bi, a, i);
    }
    block_argmax(best, bi, sv, si);
    p = bi;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < jb; ++j) {
    if (threadIdx.x == 0) {
      M.ipiv[k0 + j] = k0 + p;
      piv_loc[j] = p;
    }
    if (p != j && threadIdx.x < jb) {
      const int c = threadIdx.x;
      const T t = P[j + c * m];
      P[j + c * m] = P[p + c * m];
      P[p + c * m] = t;
    }
    __syncthreads();
    const T pv = P[j + j * m];
    const bool bad = !(pv == pv) || isinf(pv) || pv == (T)0;
    if (threadIdx.x == 0 && bad) atomicOr(flags, (pv == (T)0) ? 1 : 2);
    T best = -1;
    int bi = m;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
      if (!bad) {
        const T l = P[i + j * m] / pv;
        P[i + j * m] = l;
        for (int c = j + 1; c < jb; ++c) P[i + c * m] -= l * P[j + c * m];
      }
      if (j + 1 < jb) {
        T a = fabs(P[i + (j + 1) * m]);
        if (a != a) a = (T)INFINITY;
        argmax_pair(best, bi, a, i);
      }
    }
    warp_argmax(best, bi);
    if (lane == 0) {
      sv[wid] = best;
      si[wid] = bi;
    }
    __syncthreads();
    // every thread combines the warps' candidates (read before the next
    // iteration's first barrier, written only after it)
    T b2 = -1;
    int i2 = m;
    for (int w = 0; w < nw; ++w) argmax_pair(b2, i2, sv[w], si[w]);
    p = i2;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * jb; idx += blockDim.x) {
    const int r = idx % m, c = idx / m;
    A[(k0 + r) + (size_t)(k0 + c) * ld] = P[idx];
  }
  // the panel's interchanges as one row gather for the columns outside it:
  // after the swaps, row pos[i] holds what row src[i] held (rows relative to
  // k0; at most 2 jb rows move).  Applied by k_getrf_swap_trsm.
  if (threadIdx.x == 0) lu_record_interchanges(M.aff + (size_t)b * (1 + 4 * LU_NB), piv_loc, jb);
}

// The panel step with the panel's rows spread over the CTAs of a thread-block
// cluster: CTA `rank` holds panel rows [rank R, rank R + R) (R = ceil(m / C),
// m = n - k0) in its shared memory.  For tall panels, or too few matrices to
// fill the GPU with one CTA each.  Per column j:
//  * every CTA publishes its best candidate (largest |value| in column j among
//    its rows >= j, lowest row on ties) with the candidate row's panel values
//    into every CTA's shared memory, and the owner of row j publishes row j;
//  * one cluster barrier; every CTA then picks the same pivot row p, the owners
//    of rows j and p write the interchanged rows from the published copies, and
//    every CTA applies the rank-1 update to its rows below j with the pivot row
//    (now row j), tracking the next column's candidate.
// Same pivots and arithmetic as k_getrf_panel_smem, and the same interchange
// record for k_getrf_swap_trsm.  The published copies are double-buffered by
// the parity of j: a CTA writes column j+2's copies only after the barrier of
// column j+1, which every CTA reaches after it has read column j's.
constexpr int LU_CL_MAX = 16;
template <typename T>
__host__ __device__ constexpr size_t lu_cl_smem(int R) {
  return ((size_t)R * LU_NB + (size_t)2 * (LU_CL_MAX + 1) * LU_NB) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(512) k_getrf_panel_cl(const MatRef<T>* mats, int nmat, int k0, int* flags) {
  namespace cg = cooperative_groups;
  extern __shared__ unsigned char lu_smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  __shared__ T cand_v[2][LU_CL_MAX];
  __shared__ int cand_i[2][LU_CL_MAX];
  __shared__ T sv[32];
  __shared__ int si[32];
  __shared__ int piv_loc[LU_NB];
  const int b = blockIdx.x / C;                 // one cluster per matrix (uniform exits below)
  if (b >= nmat) return;
  const MatRef<T> M = mats[b];
  const int n = M.n;
  if (k0 >= n) return;
  T* A = M.A;
  const size_t ld = n;
  const int jb = min(LU_NB, n - k0), m = n - k0;
  const int R = (m + C - 1) / C;
  T* P = reinterpret_cast<T*>(lu_smem);         // my rows, column-major R x jb (ld R)
  T* pub = P + (size_t)R * LU_NB;               // [2][LU_CL_MAX + 1][LU_NB] published rows
  const int r0 = rank * R, nr = max(0, min(R, m - r0));
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int idx = tid; idx < nr * jb; idx += bd) {
    const int r = idx % nr, c = idx / nr;
    P[r + c * R] = A[(k0 + r0 + r) + (size_t)(k0 + c) * ld];
  }
  __syncthreads();
  T best = -1;
  int bi = m;
  for (int r = tid; r < nr; r += bd) {
    T a = fabs(P[r]);
    if (a != a) a = (T)INFINITY;
    argmax_pair(best, bi, a, r0 + r);
  }
  block_argmax(best, bi, sv, si);
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    T* slot = pub + (size_t)par * (LU_CL_MAX + 1) * LU_NB;
    // publish my candidate (and row j if it is mine) into every CTA
    for (int t = tid; t < C * jb; t += bd) {
      const int d = t / jb, c = t % jb;
      *cl.map_shared_rank(slot + (size_t)rank * LU_NB + c, d) = (bi < m) ? P[(bi - r0) + c * R] : (T)0;
    }
    if (tid < C) {
      *cl.map_shared_rank(&cand_v[par][rank], tid) = best;
      *cl.map_shared_rank(&cand_i[par][rank], tid) = bi;
    }
    if (j / R == rank)
      for (int t = tid; t < C * jb; t += bd) {
        const int d = t / jb, c = t % jb;
        *cl.map_shared_rank(slot + (size_t)LU_CL_MAX * LU_NB + c, d) = P[(j - r0) + c * R];
      }
    cl.sync();
    T bv = -1;
    int p = m, pc = 0;
    for (int q = 0; q < C; ++q) {
      const T v2 = cand_v[par][q];
      const int i2 = cand_i[par][q];
      if (v2 > bv || (v2 == bv && i2 < p)) {
        bv = v2;
        p = i2;
        pc = q;
      }
    }
    if (rank == 0 && tid == 0) {
      M.ipiv[k0 + j] = k0 + p;
      piv_loc[j] = p;
    }
    const T* urow = slot + (size_t)pc * LU_NB;           // old row p: the new row j
    const T* jrow = slot + (size_t)LU_CL_MAX * LU_NB;    // old row j
    if (p != j && tid < jb) {
      if (j / R == rank) P[(j - r0) + tid * R] = urow[tid];
      if (p / R == rank) P[(p - r0) + tid * R] = jrow[tid];
    }
    __syncthreads();
    const T pv = urow[j];
    const bool bad = !(pv == pv) || isinf(pv) || pv == (T)0;
    if (rank == 0 && tid == 0 && bad) atomicOr(flags, (pv == (T)0) ? 1 : 2);
    best = -1;
    bi = m;
    for (int r = tid; r < nr; r += bd) {
      const int i = r0 + r;
      if (i <= j) continue;
      if (!bad) {
        const T l = P[r + j * R] / pv;
        P[r + j * R] = l;
        for (int c = j + 1; c < jb; ++c) P[r + c * R] -= l * urow[c];
      }
      if (j + 1 < jb) {
        T a = fabs(P[r + (j + 1) * R]);
        if (a != a) a = (T)INFINITY;
        argmax_pair(best, bi, a, i);
      }
    }
    block_argmax(best, bi, sv, si);
  }
  for (int idx = tid; idx < nr * jb; idx += bd) {
    const int r = idx % nr, c = idx / nr;
    A[(k0 + r0 + r) + (size_t)(k0 + c) * ld] = P[r + c * R];
  }
  if (rank == 0 && tid == 0) lu_record_interchanges(M.aff + (size_t)b * (1 + 4 * LU_NB), piv_loc, jb);
  cl.sync();                                    // no CTA leaves while a peer may still address it
}

// The columns outside the panel of every matrix: apply the panel's row
// interchanges (one gather of at most 2 jb rows per column) and, right of the
// panel, form U12 = L11^-1 A12 by forward substitution.  A CTA handles 32
// columns of one matrix, a warp one column at a time (lane r holds row k0+r).
struct LuColTile {
  int mat, c0;
};

template <typename T>
__global__ void __launch_bounds__(256) k_getrf_swap_trsm(const MatRef<T>* mats, const LuColTile* tiles, int k0,
                                                         int tcol) {
  __shared__ T L11[LU_NB][LU_NB + 1];
  __shared__ int s_pos[2 * LU_NB], s_src[2 * LU_NB];
  __shared__ int s_cnt;
  const LuColTile tl = tiles[blockIdx.x];
  const MatRef<T> M = mats[tl.mat];
  const int n = M.n;
  const size_t ld = n;
  const int jb = min(LU_NB, n - k0);
  const int* rec = M.aff + (size_t)tl.mat * (1 + 4 * LU_NB);
  if (threadIdx.x == 0) s_cnt = rec[0];
  for (int t = threadIdx.x; t < 2 * LU_NB; t += blockDim.x) {
    s_pos[t] = rec[1 + t];
    s_src[t] = rec[1 + 2 * LU_NB + t];
  }
  for (int t = threadIdx.x; t < LU_NB * LU_NB; t += blockDim.x) {
    const int r = t % LU_NB, c = t / LU_NB;
    L11[r][c] = (r < jb && c < jb) ? M.A[(k0 + r) + (size_t)(k0 + c) * ld] : (T)0;
  }
  __syncthreads();
  const int cnt = s_cnt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int cc = wid; cc < 32; cc += 8) {
    const int c = tl.c0 + cc;                       // column index among the n - jb outside ones
    if (c >= n - jb) break;
    const int col = (c < k0) ? c : c + jb;
    T* colp = M.A + (size_t)col * ld + k0;
    // gather the moved rows: read all sources first, then write
    T v0 = 0, v1 = 0;
    if (lane < cnt) v0 = colp[s_src[lane]];
    if (lane + 32 < cnt) v1 = colp[s_src[lane + 32]];
    __syncwarp();
    if (lane < cnt) colp[s_pos[lane]] = v0;
    if (lane + 32 < cnt) colp[s_pos[lane + 32]] = v1;
    __syncwarp();
    if (col >= k0 + jb && col < tcol) {
      // U12 column: x = L11^-1 x over rows k0 .. k0+jb-1
      T x = (lane < jb) ? colp[lane] : (T)0;
      for (int q = 0; q < jb - 1; ++q) {
        const T xq = __shfl_sync(0xffffffffu, x, q);
        if (lane > q) x -= L11[lane][q] * xq;
      }
      if (lane < jb) colp[lane] = x;
    }
  }
}

// The end of a block of panels: rows k0 .. k0+jb-1 of the columns right of
// the block become U12 = L11^-1 A12 (the row interchanges have already
// reached them).  tiles[].c0: first column of a 32-column tile.
template <typename T>
__global__ void __launch_bounds__(256) k_lu_trsm_cols(const MatRef<T>* mats, const LuColTile* tiles, int k0) {
  __shared__ T L11[LU_NB][LU_NB + 1];
  const LuColTile tl = tiles[blockIdx.x];
  const MatRef<T> M = mats[tl.mat];
  const int n = M.n;
  const size_t ld = n;
  const int jb = min(LU_NB, n - k0);
  for (int t = threadIdx.x; t < LU_NB * LU_NB; t += blockDim.x) {
    const int r = t % LU_NB, c = t / LU_NB;
    L11[r][c] = (r < jb && c < jb) ? M.A[(k0 + r) + (size_t)(k0 + c) * ld] : (T)0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int cc = wid; cc < 32; cc += 8) {
    const int col = tl.c0 + cc;
    if (col >= n) break;
    T* colp = M.A + (size_t)col * ld + k0;
    T x = (lane < jb) ? colp[lane] : (T)0;
    for (int q = 0; q < jb - 1; ++q) {
      const T xq = __shfl_sync(0xffffffffu, x, q);
      if (lane > q) x -= L11[lane][q] * xq;
    }
    if (lane < jb) colp[lane] = x;
  }
}

// permutation from LAPACK-style interchanges: (P^T b)[k] = b[perm[k]];
// one CTA per matrix, the sequential swaps run in shared memory
template <typename T>
__global__ void k_ipiv_to_perm(const MatRef<T>* mats, int nmat) {
  extern __shared__ int pm_s[];
  const int b = blockIdx.x;
  if (b >= nmat) return;
  const MatRef<T> M = mats[b];
  for (int k = threadIdx.x; k < M.n; k += blockDim.x) pm_s[k] = k;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < M.n; ++k) {
      const int p = M.ipiv[k];
      const int t = pm_s[k];
      pm_s[k] = pm_s[p];
      pm_s[p] = t;
    }
  __syncthreads();
  for (int k = threadIdx.x; k < M.n; k += blockDim.x) M.perm[k] = pm_s[k];
}

// ------------------------------------------------------------------ grouped GEMM
template <typename T>
struct GemmCfg;
template <>
struct GemmCfg<double> {
  static constexpr int BK = 8;
};
template <>
struct GemmCfg<float> {
  static constexpr int BK = 16;
};

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmTask<T>* tasks, const GemmTerm<T>* terms,
                                              const TileItem* tiles) {
  constexpr int BM = 64, BN = 64, BK = GemmCfg<T>::BK;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const TileItem it = tiles[blockIdx.x];
  const GemmTask<T> tk = tasks[it.task];
  const int i0 = it.tm * BM, j0 = it.tn * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0;
  for (int t = tk.t0; t < tk.t1; ++t) {
    const GemmTerm<T> tm = terms[t];
    const int klim = term_klim(tm, i0, j0, BM, BN);
    for (int l0 = 0; l0 < klim; l0 += BK) {
      for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
        int i, l;
        if (!tm.ta) { i = idx % BM; l = idx / BM; }
        else { l = idx % BK; i = idx / BK; }
        const int gi = i0 + i, gl = l0 + l;
        T v = 0;
        if (gi < tk.m && gl < tm.k)
          v = tm.ta ? tm.A[gl + (size_t)gi * tm.lda] : tm.A[gi + (size_t)gl * tm.lda];
        As[l][i] = v;
      }
      for (int idx = threadIdx.x; idx < BN * BK; idx += 256) {
        int j, l;
        if (!tm.tb) { l = idx % BK; j = idx / BK; }
        else { j = idx % BN; l = idx / BN; }
        const int gj = j0 + j, gl = l0 + l;
        T v = 0;
        if (gj < tk.n && gl < tm.k)
          v = tm.tb ? tm.B[gj + (size_t)gl * tm.ldb] : tm.B[gl + (size_t)gj * tm.ldb];
        Bs[l][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int l = 0; l < BK; ++l) {
        T a[4], bb[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[l][ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bb[c] = Bs[l][tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * bb[c];
      }
      __syncthreads();
    }
  }
  // all loads of C before any store, so they overlap
  T cv[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gi = i0 + ty * 4 + r, gj = j0 + tx * 4 + c;
      cv[r][c] = (tk.beta != (T)0 && gi < tk.m && gj < tk.n) ? tk.C[gi + (size_t)gj * tk.ldc] : (T)0;
    }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int gj = j0 + tx * 4 + c;
    if (gj >= tk.n) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gi = i0 + ty * 4 + r;
      if (gi >= tk.m) continue;
      tk.C[gi + (size_t)gj * tk.ldc] = tk.alpha * acc[r][c] + tk.beta * cv[r][c];
    }
  }
}

// ------------------------------------------------------------------ grouped GEMM, FP32 on tensor cores
// Same task/term/tile contract as k_gemm<float>.  128 threads = 4 warps, a
// 64 x 64 output tile, each warp a 32 x 32 sub-tile of m16n8k8 TF32 MMAs with
// FP32 accumulation.  SPLIT = 3: error-compensated 3xTF32 (each operand split
// into a TF32 high part and a TF32 remainder; hi*hi + hi*lo + lo*hi), which
// keeps the products at about FP32 accuracy; SPLIT = 1: plain TF32.
__device__ inline uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ inline void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ inline void cp_async4(void* smem, const void* g, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 4 : 0;                      // 0 bytes read -> zero fill
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(g), "r"(sz));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int SPLIT>
__global__ void __launch_bounds__(128) k_gemm_tc(const GemmTask<float>* tasks, const GemmTerm<float>* terms,
                                                 const TileItem* tiles) {
  constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
  __shared__ float As[2][BK][BM + PAD];   // k-major: As[s][l][i] = op(A)[i0+i, l0+l]
  __shared__ float Bs[2][BK][BN + PAD];   // Bs[s][l][j] = op(B)[l0+l, j0+j]
  const TileItem it = tiles[blockIdx.x];
  const GemmTask<float> tk = tasks[it.task];
  const int i0 = it.tm * BM, j0 = it.tn * BN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t4 = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  // flattened (term, k-chunk) sequence
  int cur_t = tk.t0, cur_l = 0;
  auto advance = [&](int& t, int& l) {
    l += BK;
    while (t < tk.t1 && l >= term_klim(terms[t], i0, j0, BM, BN)) {
      ++t;
      l = 0;
    }
  };
  while (cur_t < tk.t1 && term_klim(terms[cur_t], i0, j0, BM, BN) <= 0) ++cur_t;
  auto issue = [&](int stage, int t, int l0) {
    const GemmTerm<float> tm = terms[t];
    for (int idx = threadIdx.x; idx < BM * BK; idx += 128) {
      int i, l;
      if (!tm.ta) { i = idx % BM; l = idx / BM; }
      else { l = idx % BK; i = idx / BK; }
      const int gi = i0 + i, gl = l0 + l;
      const bool ok = gi < tk.m && gl < tm.k;
      const float* src = ok ? (tm.ta ? tm.A + gl + (size_t)gi * tm.lda : tm.A + gi + (size_t)gl * tm.lda) : tm.A;
      cp_async4(&As[stage][l][i], src, ok);
    }
    for (int idx = threadIdx.x; idx < BN * BK; idx += 128) {
      int j, l;
      if (!tm.tb) { l = idx % BK; j = idx / BK; }
      else { j = idx % BN; l = idx / BN; }
      const int gj = j0 + j, gl = l0 + l;
      const bool ok = gj < tk.n && gl < tm.k;
      const float* src = ok ? (tm.tb ? tm.B + gj + (size_t)gl * tm.ldb : tm.B + gl + (size_t)gj * tm.ldb) : tm.B;
      cp_async4(&Bs[stage][l][j], src, ok);
    }
  };
  int stage = 0;
  if (cur_t < tk.t1) issue(0, cur_t, cur_l);
  cp_async_commit();
  while (cur_t < tk.t1) {
    int nt = cur_t, nl = cur_l;
    advance(nt, nl);
    if (nt < tk.t1) issue(stage ^ 1, nt, nl);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 8) {
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = wm + a * 16 + g;
        const float x0 = As[stage][kk + t4][r], x1 = As[stage][kk + t4][r + 8];
        const float x2 = As[stage][kk + t4 + 4][r], x3 = As[stage][kk + t4 + 4][r + 8];
        ah[a][0] = to_tf32(x0);
        ah[a][1] = to_tf32(x1);
        ah[a][2] = to_tf32(x2);
        ah[a][3] = to_tf32(x3);
        if (SPLIT == 3) {
          al[a][0] = to_tf32(x0 - __uint_as_float(ah[a][0]));
          al[a][1] = to_tf32(x1 - __uint_as_float(ah[a][1]));
          al[a][2] = to_tf32(x2 - __uint_as_float(ah[a][2]));
          al[a][3] = to_tf32(x3 - __uint_as_float(ah[a][3]));
        }
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int cidx = wn + b * 8 + g;
        const float y0 = Bs[stage][kk + t4][cidx], y1 = Bs[stage][kk + t4 + 4][cidx];
        bh[b][0] = to_tf32(y0);
        bh[b][1] = to_tf32(y1);
        if (SPLIT == 3) {
          bl[b][0] = to_tf32(y0 - __uint_as_float(bh[b][0]));
          bl[b][1] = to_tf32(y1 - __uint_as_float(bh[b][1]));
        }
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (SPLIT == 3) {
            mma_tf32(acc[a][b], al[a], bh[b]);
            mma_tf32(acc[a][b], ah[a], bl[b]);
          }
          mma_tf32(acc[a][b], ah[a], bh[b]);
        }
    }
    __syncthreads();
    stage ^= 1;
    cur_t = nt;
    cur_l = nl;
  }
  cp_async_wait<0>();
  // epilogue: c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1); all
  // loads of C before any store, so they overlap
  float cv[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int gi = i0 + wm + a * 16 + g + ((e >= 2) ? 8 : 0);
        const int gj = j0 + wn + b * 8 + 2 * t4 + (e & 1);
        cv[a][b][e] = (tk.beta != 0.f && gi < tk.m && gj < tk.n) ? tk.C[gi + (size_t)gj * tk.ldc] : 0.f;
      }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int gi = i0 + wm + a * 16 + g + ((e >= 2) ? 8 : 0);
        const int gj = j0 + wn + b * 8 + 2 * t4 + (e & 1);
        if (gi < tk.m && gj < tk.n) tk.C[gi + (size_t)gj * tk.ldc] = tk.alpha * acc[a][b][e] + tk.beta * cv[a][b][e];
      }
}

// ------------------------------------------------------------------ triangular inverses
// A triangular inverse task: the LU factors, the n x n output and an optional
// diagonal scale (rows of L^-1 by 1/d_i, columns of U^-1 by d_j).  perm is
// unused here (the row permutation is folded into gather indices elsewhere).
template <typename T>
struct InvTask {
  const T* LU;       // n x n factors
  T* out;            // n x n output
  const int* perm;
  const T* dscale;
  int n;
};

struct InvTile {
  int task, j0;
};

// Column tile [j0, j0+32) of U^-1 (non-unit upper), column j scaled by dscale[j].
template <typename T>
__global__ void __launch_bounds__(256) k_inv_upper(const InvTask<T>* tasks, const InvTile* tiles) {
  __shared__ T Us[32][33];
  __shared__ T Xs[32][33];
  __shared__ T Acc[32][33];
  const InvTile tl = tiles[blockIdx.x];
  const InvTask<T> tk = tasks[tl.task];
  const int n = tk.n, j0 = tl.j0, jb = min(32, n - j0);
  const size_t ld = n;
  T* X = tk.out;
  // zero rows below the tile's diagonal block
  for (int idx = threadIdx.x; idx < (n - (j0 + 32 < n ? j0 + 32 : n)) * jb; idx += blockDim.x) {
    const int nz = n - min(n, j0 + 32);
    const int r = min(n, j0 + 32) + idx % nz, c = idx / nz;
    X[r + (size_t)(j0 + c) * ld] = 0;
  }
  // row blocks from the diagonal block (starting at j0) upward, aligned to j0
  for (int r0 = j0; r0 >= 0; r0 -= 32) {
    const int rb = min(32, n - r0);
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) Acc[idx % 32][idx / 32] = 0;
    __syncthreads();
    for (int q0 = r0 + 32; q0 < j0 + jb; q0 += 32) {
      const int qb = min(32, n - q0);
      for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
        const int r = idx % 32, c = idx / 32;
        Us[r][c] = (r < rb && c < qb) ? tk.LU[(r0 + r) + (size_t)(q0 + c) * ld] : (T)0;
        Xs[r][c] = (r < qb && c < jb) ? X[(q0 + r) + (size_t)(j0 + c) * ld] : (T)0;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
        const int r = idx % 32, c = idx / 32;
        T s = 0;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) s += Us[r][q] * Xs[q][c];
        Acc[r][c] += s;
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx % 32, c = idx / 32;
      Us[r][c] = (r < rb && c < rb) ? tk.LU[(r0 + r) + (size_t)(r0 + c) * ld] : (T)1;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int c = threadIdx.x;
      if (c < jb) {
        const T dsc = tk.dscale ? tk.dscale[j0 + c] : (T)1;
        T x[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) x[r] = ((r0 + r == j0 + c) ? dsc : (T)0) - Acc[r][c];
#pragma unroll
        for (int r = 31; r >= 0; --r) {
          T s = x[r];
#pragma unroll
          for (int q = r + 1; q < 32; ++q) s -= Us[r][q] * x[q];
          x[r] = (r < rb) ? s / Us[r][r] : (T)0;
        }
#pragma unroll
        for (int r = 0; r < 32; ++r)
          if (r < rb) X[(r0 + r) + (size_t)(j0 + c) * ld] = x[r];
      }
    }
    __syncthreads();
    if (r0 == 0) break;
  }
}

// Inverse of one 32 x 32 diagonal block of the LU factors: lower = unit lower
// L (strict lower part of LU), upper = U (upper part of LU).  One warp per
// block, a lane per column; the block of the output is overwritten.
template <typename T>
struct DiagInvTask {
  const T* LU;
  T* out;
  int n, p, lower;   // block p covers rows/cols [32p, min(n, 32p+32))
};

template <typename T>
__global__ void __launch_bounds__(32) k_inv_diag(const DiagInvTask<T>* tasks) {
  __shared__ T Bl[32][33];
  const DiagInvTask<T> tk = tasks[blockIdx.x];
  const int n = tk.n, o = 32 * tk.p, b = min(32, n - o);
  const int c = threadIdx.x;
  for (int r = 0; r < 32; ++r) Bl[r][c] = (r < b && c < b) ? tk.LU[(o + r) + (size_t)(o + c) * n] : (T)0;
  __syncwarp();
  if (c < b) {
    T x[32];
    if (tk.lower) {
#pragma unroll
      for (int r = 0; r < 32; ++r) x[r] = (r == c) ? (T)1 : (T)0;
#pragma unroll
      for (int r = 1; r < 32; ++r) {
        T s = x[r];
#pragma unroll
        for (int q = 0; q < r; ++q) s -= Bl[r][q] * x[q];
        x[r] = (r < b) ? s : (T)0;
      }
    } else {
#pragma unroll
      for (int r = 0; r < 32; ++r) x[r] = (r == c) ? (T)1 : (T)0;
#pragma unroll
      for (int r = 31; r >= 0; --r) {
        T s = x[r];
#pragma unroll
        for (int q = r + 1; q < 32; ++q) s -= Bl[r][q] * x[q];
        x[r] = (r < b) ? s / Bl[r][r] : (T)0;
      }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (r < b) tk.out[(o + r) + (size_t)(o + c) * n] = x[r];
  }
}

// zero a batch of n x n matrices
template <typename T>
__global__ void k_zero_mats(T* const* ptr, const int* nn) {
  T* p = ptr[blockIdx.y];
  const size_t tot = (size_t)nn[blockIdx.y] * nn[blockIdx.y];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x)
    p[i] = (T)0;
}

// columns of out scaled by dscale[j]  (U^-1 |d|^1/2)
template <typename T>
__global__ void k_scale_cols(const InvTask<T>* tasks, const InvTile* tiles) {
  const InvTile tl = tiles[blockIdx.x];
  const InvTask<T> tk = tasks[tl.task];
  if (!tk.dscale) return;
  const int n = tk.n, jb = min(32, n - tl.j0);
  for (int idx = threadIdx.x; idx < n * jb; idx += blockDim.x) {
    const int r = idx % n, c = tl.j0 + idx / n;
    tk.out[r + (size_t)c * n] *= tk.dscale[c];
  }
}

// rows of out scaled by 1 / dscale[i]  (diag(|d|^-1/2) applied to L^-1 P^T)
template <typename T>
__global__ void k_scale_rows(const InvTask<T>* tasks, const InvTile* tiles) {
  const InvTile tl = tiles[blockIdx.x];
  const InvTask<T> tk = tasks[tl.task];
  if (!tk.dscale) return;
  const int n = tk.n, jb = min(32, n - tl.j0);
  for (int idx = threadIdx.x; idx < n * jb; idx += blockDim.x) {
    const int r = idx % n, c = tl.j0 + idx / n;
    tk.out[r + (size_t)c * n] /= tk.dscale[r];
  }
}

// d[i] = sqrt(|U_ii|)
template <typename T>
__global__ void k_diag_sqrt(const MatRef<T>* mats, T* const* dout, int nmat) {
  const int b = blockIdx.x;
  if (b >= nmat) return;
  const MatRef<T> M = mats[b];
  for (int i = threadIdx.x; i < M.n; i += blockDim.x) dout[b][i] = sqrt(fabs(M.A[i + (size_t)i * M.n]));
}

// ------------------------------------------------------------------ copies
template <typename T>
__global__ void __launch_bounds__(256) k_copy_tiles(const CopyTask<T>* tasks, const CopyTile* tiles) {
  __shared__ T tile[32][33];
  const CopyTile ct = tiles[blockIdx.x];
  const CopyTask<T> tk = tasks[ct.task];
  const int r0 = ct.tr * 32, c0 = ct.tc * 32;
  if (!tk.trans) {
    // 256 threads, 4 elements each, all loaded before any store
    const int r = r0 + (threadIdx.x & 31), cq = c0 + (threadIdx.x >> 5);
    T v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = cq + 8 * e;
      v[e] = (r < tk.rows && c < tk.cols) ? tk.src[r + (size_t)c * tk.lds] : T(0);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = cq + 8 * e;
      if (r < tk.rows && c < tk.cols) tk.dst[r + (size_t)c * tk.ldd] = v[e];
    }
  } else {
    // dst (rows x cols) = src^T, src is cols x rows
    for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) {
      const int sr = c0 + (idx & 31), sc = r0 + (idx >> 5);
      if (sr < tk.cols && sc < tk.rows) tile[idx >> 5][idx & 31] = tk.src[sr + (size_t)sc * tk.lds];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) {
      const int r = r0 + (idx & 31), c = c0 + (idx >> 5);
      if (r < tk.rows && c < tk.cols) tk.dst[r + (size_t)c * tk.ldd] = tile[idx & 31][idx >> 5];
    }
  }
}

// dst = I_r at (dst, ldd)
template <typename T>
struct EyeTask {
  T* dst;
  int ldd, r;
  int rows;        // 0: write the r diagonal ones only; else write all rows x r entries ([I_r; 0])
};

template <typename T>
__global__ void k_eye(const EyeTask<T>* tasks, int ntask) {
  for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
    const EyeTask<T> tk = tasks[t];
    if (tk.rows == 0) {
      for (int i = threadIdx.x; i < tk.r; i += blockDim.x) tk.dst[i + (size_t)i * tk.ldd] = (T)1;
    } else {
      for (int j = 0; j < tk.r; ++j)
        for (int i = threadIdx.x; i < tk.rows; i += blockDim.x) tk.dst[i + (size_t)j * tk.ldd] = (T)(i == j);
    }
  }
}

// ------------------------------------------------------------------ RRQR
// Column-pivoted Householder QR of W (n x c, row-major) by the CTAs of one
// exchange group (a thread-block cluster of 1 to 16 CTAs, or a group of a
// cooperative launch) that split the columns into contiguous chunks.  Each
// step: every CTA proposes its best remaining column (largest residual norm,
// lowest index on ties); after one barrier every CTA knows the winner, reads
// its column from the owner and builds the same Householder vector; every CTA
// updates its own remaining columns and their norms.  Columns are not moved: a
// used flag (norm set to -1) replaces the swap, which leaves the reflectors and
// hence Q unchanged.  The factorization stops at the first k with
// |R_kk| <= eps |R_00| (or R_00 = 0); columns whose initial norm is already
// <= eps |R_00| can never be chosen before that and are dropped.
constexpr int QR_CS = 8;
constexpr int QR_THREADS = 512;

// How the CTAs that share one interface exchange the pivot proposals and the
// winner's column.  ClusterX: one thread-block cluster, distributed shared
// memory and cluster barriers.  GroupX: a group of CTAs of a cooperative
// launch, global memory (read past L1) and a counting barrier per group whose
// wait is bounded (on timeout it raises bit 4 of the error flags and the CTAs
// leave).
template <typename T, int CS>
struct ClusterX {
  static constexpr int kMax = CS;
  static constexpr bool kPublishCol = false;
  cooperative_groups::cluster_group cl;
  T* cand_v;                              // [2]: proposals double-buffered by step parity
  int* cand_i;
  int par = 0;
  __device__ int rank() const { return (int)cl.block_rank(); }
  __device__ int size() const { return CS; }
  __device__ bool sync() {
    cl.sync();
    return true;
  }
  __device__ void publish(T v, int i) {   // thread 0
    cand_v[par] = v;
    cand_i[par] = i;
  }
  __device__ void gather(int r, T& v, int& i) {
    v = *cl.map_shared_rank(cand_v + par, r);
    i = *cl.map_shared_rank(cand_i + par, r);
  }
  __device__ void next_step() { par ^= 1; }
  template <typename U>
  __device__ U* remote(U* p, int r) { return cl.map_shared_rank(p, r); }

  __device__ void finish() { cl.sync(); }   // no CTA leaves while another may read its shared memory
};

struct GroupSync {
  unsigned count, gen;
};

constexpr int QR_GMAX = 256;     // largest CTA group of the cooperative variants

template <typename T>
struct GroupX {
  // One barrier per pivot step: each CTA also writes its candidate column to a
  // global slot before the barrier, so after it every CTA reads the winner's
  // column and builds the reflector itself.  Proposals and slots are
  // double-buffered by step parity.
  static constexpr int kMax = QR_GMAX;
  static constexpr bool kPublishCol = true;
  int q, G;
  T* prop_v;                 // [2][QR_GMAX] proposals of this group (global)
  int* prop_i;
  GroupSync* gs;
  int* err;
  T* slot;                   // [2][G][ns] candidate columns of this group (global)
  int ns;
  int par = 0;
  long poll_limit = 1l << 22;  // polls before a barrier wait gives up (well under a second)
  __device__ int rank() const { return q; }
  __device__ int size() const { return G; }
  __device__ bool sync() {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      s_ok = 1;
      volatile unsigned* vgen = &gs->gen;
      const unsigned g = *vgen;
      __threadfence();
      if (atomicAdd(&gs->count, 1u) == (unsigned)G - 1) {
        gs->count = 0;
        __threadfence();
        atomicAdd(&gs->gen, 1u);
      } else {
        long it = 0;
        while (*vgen == g) {
          if (++it > poll_limit) {          // bounded: the back-off below keeps this under a second
            atomicOr(err, 16);
            s_ok = 0;
            break;
          }
          if (it > 2048) __nanosleep(64);   // spin first: the partners are resident and close
        }
      }
      __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
  }
  __device__ void publish(T v, int i) {
    prop_v[par * QR_GMAX + q] = v;
    prop_i[par * QR_GMAX + q] = i;
  }
  __device__ void gather(int r, T& v, int& i) {
    v = __ldcg(prop_v + par * QR_GMAX + r);
    i = __ldcg(prop_i + par * QR_GMAX + r);
  }
  __device__ T* col_out() { return slot + ((size_t)par * G + q) * ns; }
  __device__ const T* col_in(int r) { return slot + ((size_t)par * G + r) * ns; }
  __device__ void next_step() { par ^= 1; }
  template <typename U>
  __device__ U* remote(U* p, int) { return p; }

  __device__ void finish() {}
};

// sum over aligned groups of L lanes (L a power of two <= 32)
template <typename T>
__device__ inline T group_sum(T x, int L) {
  for (int o = L >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// The factorization of one interface by the CTAs of one exchange group X
// (rank q of X.size() CTAs; columns split in contiguous chunks).  Inside a
// CTA a column is handled by L consecutive lanes of one warp (L chosen so
// that one pass covers the chunk), which combine their row partial sums with
// shuffles: the column pass of a pivot step needs no block barrier, and it
// also yields the CTA's proposal for the next step.
template <typename T, bool SMEM, int NT, typename X>
__device__ void qrcp_group(const QrTask<T>& tk, T eps, X& xc, unsigned char* smem_raw, T* cand_v, int* cand_i,
                           int* err) {
  constexpr int CSM = X::kMax;
  T* v = reinterpret_cast<T*>(smem_raw);           // n: current reflector (local copy)
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T allc_v[CSM];
  __shared__ int allc_i[CSM];
  __shared__ T s_scal[4];                          // [0] tau, [1] winner norm^2
  __shared__ int s_win;
  __shared__ T s_prop_v;                           // this CTA's proposal for the next step
  __shared__ int s_prop_i;
  const int q = xc.rank(), CS = xc.size();
  const int n = tk.n, c = tk.c;
  const int chunk = (c + CS - 1) / CS;
  const int j0 = min(c, q * chunk), j1 = min(c, j0 + chunk);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int wdt = j1 - j0;
  int L = 1;                                       // lanes per column
  while (L < 32 && (NT / (2 * L)) >= wdt) L *= 2;
  const int slots = NT / L;                        // columns per pass
  const int cs_ = tid / L, li = tid % L;
  T* Wg = tk.W;
  T* Ws = v + ((n + 31) & ~31);
  const size_t ldg = (size_t)c;
  auto at = [&](int i, int j) -> T& {
    if (SMEM) return Ws[(size_t)i * chunk + (j - j0)];
    return Wg[(size_t)i * ldg + j];
  };
  if (SMEM) {
    for (int idx = tid; idx < n * wdt; idx += NT) {
      const int i = idx / wdt, jj = idx % wdt;
      Ws[(size_t)i * chunk + jj] = Wg[(size_t)i * ldg + j0 + jj];
    }
    __syncthreads();
  }
  // ---- initial column norms
  for (int g = j0; g < j1; g += slots) {
    const int j = g + cs_;
    T sum = 0;
    if (j < j1)
      for (int i = li; i < n; i += L) {
        const T a = at(i, j);
        sum += a * a;
      }
    sum = group_sum(sum, L);
    if (li == 0 && j < j1) tk.norm2[j] = sum;
  }
  __syncthreads();
  const int kmax = min(n, c);
  int rank = kmax;
  T nrm0 = 0;
  bool ok = true;
  for (int k = 0; k < kmax; ++k) {
    // ---- this CTA's proposal (from the norms at k = 0, else from the last column pass)
    if (k == 0) {
      T best = -1;
      int bi = c;
      for (int j = j0 + tid; j < j1; j += NT) argmax_pair(best, bi, tk.norm2[j], j);
      block_argmax(best, bi, red_v, red_i);
      if constexpr (X::kPublishCol) {
        if (bi < c) {
          T* out = xc.col_out();
          for (int i = tid; i < n; i += NT) out[i] = at(i, bi);
        }
      }
      if (tid == 0) xc.publish(best, bi);
    } else if (tid == 0) {
      xc.publish(s_prop_v, s_prop_i);
    }
    if (!(ok = xc.sync())) break;
    // ---- group-wide winner: one read per thread, in parallel
    if (tid < CS) xc.gather(tid, allc_v[tid], allc_i[tid]);
    __syncthreads();
    if (tid == 0) {
      T gb = -1;
      int gi = c;
      for (int r = 0; r < CS; ++r) argmax_pair(gb, gi, allc_v[r], allc_i[r]);
      s_scal[1] = gb;
      s_win = gi;
    }
    __syncthreads();
    const int gi = s_win;
    const T nrm = sqrt(fmax(s_scal[1], (T)0));
    if (k == 0) {
      nrm0 = nrm;
      // drop columns that can never be chosen before the stopping test
      const T cut = eps * nrm0;
      for (int j = j0 + tid; j < j1; j += NT)
        if (tk.norm2[j] >= 0 && sqrt(tk.norm2[j]) <= cut) tk.norm2[j] = -1;
    }
    const bool stop = (nrm0 == (T)0) || nrm <= eps * nrm0 || gi >= c;
    if (stop) {
      rank = k;
      break;
    }
    const int p = gi;
    const bool owner = (p >= j0 && p < j1);
    const int orank = p / chunk;
    // every CTA builds the same reflector from column p, read from the owner
    // (its shared memory through the cluster, its published slot in a group,
    // or W in global memory); the owner never touches a used column again, so
    // no second barrier is needed
    {
      if constexpr (X::kPublishCol) {
        const T* src = xc.col_in(orank);
        for (int i = k + tid; i < n; i += NT) v[i] = owner ? at(i, p) : __ldcg(src + i);
      } else if (SMEM) {
        const T* ws_o = xc.remote(Ws, orank);
        const int pj = p - orank * chunk;
        for (int i = k + tid; i < n; i += NT) v[i] = ws_o[(size_t)i * chunk + pj];
      } else {
        for (int i = k + tid; i < n; i += NT) v[i] = owner ? at(i, p) : __ldcg(Wg + (size_t)i * ldg + p);
      }
      __syncthreads();
      T prt = 0;
      for (int i = k + 1 + tid; i < n; i += NT) prt += v[i] * v[i];
      const T sigma = block_sum(prt, red_v);
      const T alpha = v[k];
      T tau = 2, beta = -alpha, scale = 0;          // column already reduced: H = I - 2 e_k e_k^T
      if (sigma > (T)0) {
        beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
        tau = (beta - alpha) / beta;
        scale = (T)1 / (alpha - beta);
      }
      __syncthreads();
      for (int i = k + tid; i < n; i += NT) {
        const T vi = (i == k) ? (T)1 : v[i] * scale;
        v[i] = vi;
        if (owner) tk.V[(size_t)i + (size_t)k * n] = vi;
      }
      if (tid == 0) {
        s_scal[0] = tau;
        if (owner) {
          tk.tau[k] = tau;
          tk.norm2[p] = -1;                // used
        }
      }
      __syncthreads();
    }
    const T tau = s_scal[0];
    // ---- update the own remaining columns and their norms; track the best
    T best = -1;
    int bi = c;
    for (int g = j0; g < j1; g += slots) {
      const int j = g + cs_;
      const bool act = j < j1 && tk.norm2[j] >= 0;
      T d0 = 0, d1 = 0;
      if (act) {
        int i = k + li;
        for (; i + L < n; i += 2 * L) {
          d0 += v[i] * at(i, j);
          d1 += v[i + L] * at(i + L, j);
        }
        if (i < n) d0 += v[i] * at(i, j);
      }
      const T dt = group_sum(d0 + d1, L) * tau;
      T s0 = 0;
      if (act) {
        int i = k + li;
        for (; i + L < n; i += 2 * L) {
          T& a = at(i, j);
          T& b = at(i + L, j);
          a -= dt * v[i];
          b -= dt * v[i + L];
          if (i > k) s0 += a * a;
          s0 += b * b;
        }
        if (i < n) {
          T& a = at(i, j);
          a -= dt * v[i];
          if (i > k) s0 += a * a;
        }
      }
      s0 = group_sum(s0, L);
      if (li == 0 && act) {
        tk.norm2[j] = s0;
        argmax_pair(best, bi, s0, j);
      }
    }
    warp_argmax(best, bi);
    if (lane == 0) {
      red_v[wid] = best;
      red_i[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      T b2 = -1;
      int i2 = c;
      for (int w = 0; w < NT / 32; ++w) argmax_pair(b2, i2, red_v[w], red_i[w]);
      s_prop_v = b2;
      s_prop_i = i2;
    }
    xc.next_step();
    if constexpr (X::kPublishCol) {
      // the candidate column for the next step, rows k+1.., into this step
      // parity's slot (read by the others after the next barrier)
      __syncthreads();
      const int jn = s_prop_i;
      if (jn < c) {
        T* out = xc.col_out();
        for (int i = k + 1 + tid; i < n; i += NT) out[i] = at(i, jn);
      }
    }
  }
  if (q == 0 && tid == 0) *tk.rank = ok ? rank : 0;
  if (ok) xc.finish();
}

template <typename T, bool SMEM, int CS, int NT>
__global__ void __launch_bounds__(NT, 1) k_qrcp_cluster(const QrTask<T>* tasks, T eps) {
  extern __shared__ unsigned char qr_smem2[];
  __shared__ T cand_v[2];
  __shared__ int cand_i[2];
  ClusterX<T, CS> xc{cooperative_groups::this_cluster(), cand_v, cand_i};
  const QrTask<T> tk = tasks[blockIdx.x / CS];
  qrcp_group<T, SMEM, NT>(tk, eps, xc, qr_smem2, cand_v, cand_i, nullptr);
}

// Interfaces too large for one cluster: a cooperative launch in which group t
// (G <= QR_GMAX CTAs, one per SM) factors task t.  SMEM = true: each CTA holds
// its column chunk in shared memory; SMEM = false: W streams from L2 / HBM,
// spread over as many SMs as the group has CTAs.
struct QrGroupDesc {
  int task, q, G, pad;
};

template <typename T, bool SMEM, int NT>
__global__ void __launch_bounds__(NT, 1) k_qrcp_group(const QrTask<T>* tasks, const QrGroupDesc* desc,
                                                      T* prop_v, int* prop_i, GroupSync* gs, int* err, T* slots,
                                                      int ns, T eps) {
  extern __shared__ unsigned char qr_smem3[];
  const QrGroupDesc d = desc[blockIdx.x];
  // a group's CTAs are consecutive in the launch: its slots start at its first CTA
  T* gslot = slots + (size_t)(blockIdx.x - d.q) * 2 * ns;
  GroupX<T> xc{d.q, d.G, prop_v + (size_t)d.task * 2 * QR_GMAX, prop_i + (size_t)d.task * 2 * QR_GMAX,
               gs + d.task, err, gslot, ns};
  const QrTask<T> tk = tasks[d.task];
  qrcp_group<T, SMEM, NT>(tk, eps, xc, qr_smem3, nullptr, nullptr, err);
}

// bytes of dynamic shared memory the SMEM variant needs for an n x c problem
template <typename T>
inline size_t qrcp_smem_bytes(int n, int c, int cs) {
  const size_t chunk = (size_t)(c + cs - 1) / cs;
  return (((size_t)n + 31) & ~(size_t)31) * sizeof(T) + (size_t)n * chunk * sizeof(T);
}

// compact-WY form of the explicit Q_c = H_0 ... H_{r-1} [I_r; 0] = [I_r; 0] - V T V_top^T,
// with T upper triangular and T^-1 = striu(V^T V) + diag(1/tau) (Householder
// reflectors, tau = 2 / v^T v).  This kernel turns the Gram G = V^T V (r x r,
// ld r) into T^-1 in place: diagonal 1/tau, strictly lower part zero.
template <typename T>
struct WyTask {
  T* G;
  const T* tau;
  int r;
};

template <typename T>
__global__ void k_wy_tinv(const WyTask<T>* tasks) {
  const WyTask<T> tk = tasks[blockIdx.x];
  const int r = tk.r;
  for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
    const int i = idx % r, j = idx / r;
    if (i == j) tk.G[idx] = (T)1 / tk.tau[i];
    else if (i > j) tk.G[idx] = 0;
  }
}

}  // namespace spand
