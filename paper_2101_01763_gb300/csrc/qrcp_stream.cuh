// Column-pivoted Householder QR truncated at |R_kk| <= eps |R_00| (the RRQR of
// Eq. 12) for interfaces whose W = [A_sn A_ns^T] is too large for on-chip
// memory: W (n x c) streams from L2 / HBM at every pivot step.
//
// Layout and work split.  W is column-major (column j at W + j*ldw, ldw a
// multiple of 16 bytes), so a column is one contiguous run.  The CTAs of a
// group (a cooperative launch; one CTA per SM) own the columns j = q (mod G),
// interleaved so that strong and weak neighbour blocks spread evenly over the
// group; inside a CTA the columns are dealt round-robin to the warps.  A warp
// processes one column at a time: it loads rows floor(k)..n-1 into registers
// with 16-byte loads (NV vectors per lane, all in flight at once), forms the
// reflector dot product with a shuffle reduction, updates the column in
// registers, stores it back and recomputes its residual norm exactly (columns
// of up to 32 x 16 x NV bytes go 16 / NV at a time, so that a warp always has
// 16 vector loads per lane in flight).  One read and one write of every live
// column per pivot step.
//
// Columns that can no longer be pivots are dropped for good: the residual norm
// of a column never grows, and the factorization stops at the first step whose
// largest residual norm is <= eps |R_00|, so a column whose residual norm has
// fallen to that cut is never chosen and never needed again (only Q is kept).
// Each warp keeps its live columns in its own list in shared memory and
// compacts it as it goes; the rank, the pivots and Q are those of the plain
// column-pivoted QR.
//
// A pivot step: every CTA publishes its best live column (largest residual
// norm, lowest index on ties); after one group barrier every CTA reads the
// proposals, takes the winner, reads the winner's column from W (the owner
// wrote it before the barrier and never touches it again) and builds the same
// reflector; the owner writes it to V.
#pragma once
#include <type_traits>

#include "dense.cuh"

namespace spand {

template <typename T>
struct QrStreamTask {
  T* W;              // n x c column-major, leading dimension ldw; overwritten
  T* V;              // n x min(n,c) column-major: reflector k in column k, rows k..n-1 (v_k[k] = 1)
  T* tau;            // min(n, c)
  T* Q;              // explicit Q_c output (filled later; n x r, ld n)
  int n, c, ldw;
  int* rank;         // output
  unsigned long long* work;   // sum over steps of (rows k..n-1) x (live columns): elements streamed
};

constexpr int QRS_THREADS = 512;
constexpr int QRS_WARPS = QRS_THREADS / 32;

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int W = 4;
  __device__ static inline V load(const float* p) { return *reinterpret_cast<const float4*>(p); }
  __device__ static inline V ldcg(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
  __device__ static inline void store(float* p, const V& v) { *reinterpret_cast<float4*>(p) = v; }
  __device__ static inline float get(const V& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
  __device__ static inline void set(V& v, int i, float a) {
    if (i == 0) v.x = a;
    else if (i == 1) v.y = a;
    else if (i == 2) v.z = a;
    else v.w = a;
  }
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int W = 2;
  __device__ static inline V load(const double* p) { return *reinterpret_cast<const double2*>(p); }
  __device__ static inline V ldcg(const double* p) { return __ldcg(reinterpret_cast<const double2*>(p)); }
  __device__ static inline void store(double* p, const V& v) { *reinterpret_cast<double2*>(p) = v; }
  __device__ static inline double get(const V& v, int i) { return i == 0 ? v.x : v.y; }
  __device__ static inline void set(V& v, int i, double a) {
    if (i == 0) v.x = a;
    else v.y = a;
  }
};

// Dynamic shared memory: the reflector (ldw values) and the warps' column lists.
template <typename T>
inline size_t qrcp_stream_smem(int ldw, int c, int G) {
  const int per_cta = (c + G - 1) / G;
  const int per_warp = (per_cta + QRS_WARPS - 1) / QRS_WARPS;
  return (size_t)ldw * sizeof(T) + (size_t)QRS_WARPS * per_warp * sizeof(int);
}

// One column pass at step k on column j: y = tau (v^T w); w -= y v; returns the
// residual norm^2 over rows k+1..n-1.  Rows [kb, n) are processed (kb = k
// rounded down to a vector boundary; v is zero on rows < k, so those rows are
// unchanged).  With n - kb <= 32 NV VW the column stays in registers between
// the two halves; otherwise it is read twice.
template <typename T, int NV>
__device__ inline T qrs_column(T* __restrict__ col, const T* __restrict__ v, T tau, int k, int kb, int n, int lane) {
  using VT = Vec16<T>;
  constexpr int VW = VT::W;
  const int span = 32 * VW * NV;            // rows per register pass
  if (n - kb <= span) {
    typename VT::V r[NV];
    T d = 0;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int i0 = kb + (lane + 32 * t) * VW;
      if (i0 < n) r[t] = VT::load(col + i0);
    }
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int i0 = kb + (lane + 32 * t) * VW;
      if (i0 < n) {
        const typename VT::V vv = VT::load(v + i0);
#pragma unroll
        for (int e = 0; e < VW; ++e) d += VT::get(vv, e) * VT::get(r[t], e);
      }
    }
    d = warp_sum(d) * tau;
    T s = 0;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int i0 = kb + (lane + 32 * t) * VW;
      if (i0 < n) {
        const typename VT::V vv = VT::load(v + i0);
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const T a = VT::get(r[t], e) - d * VT::get(vv, e);
          VT::set(r[t], e, a);
          if (i0 + e > k) s += a * a;
        }
        VT::store(col + i0, r[t]);
      }
    }
    return warp_sum(s);
  }
  // tall column: dot product pass, then update pass (rows re-read)
  T d = 0;
  for (int i0 = kb + lane * VW; i0 < n; i0 += 32 * VW) {
    const typename VT::V a = VT::load(col + i0), vv = VT::load(v + i0);
#pragma unroll
    for (int e = 0; e < VW; ++e) d += VT::get(vv, e) * VT::get(a, e);
  }
  d = warp_sum(d) * tau;
  T s = 0;
  for (int i0 = kb + lane * VW; i0 < n; i0 += 32 * VW) {
    typename VT::V a = VT::load(col + i0);
    const typename VT::V vv = VT::load(v + i0);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const T x = VT::get(a, e) - d * VT::get(vv, e);
      VT::set(a, e, x);
      if (i0 + e > k) s += x * x;
    }
    VT::store(col + i0, a);
  }
  return warp_sum(s);
}

// CB columns at once (register path only: n - kb <= 32 NV VW): all their
// loads are in flight together, so a warp keeps CB x NV 16-byte loads per lane
// outstanding.  act[b] = false skips column b.  sres[b]: residual norm^2.
template <typename T, int NV, int CB>
__device__ inline void qrs_columns(T* const (&col)[CB], const bool (&act)[CB], const T* __restrict__ v, T tau,
                                   int k, int kb, int n, int lane, T (&sres)[CB]) {
  using VT = Vec16<T>;
  constexpr int VW = VT::W;
  typename VT::V r[CB][NV];
#pragma unroll
  for (int b = 0; b < CB; ++b)
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int i0 = kb + (lane + 32 * t) * VW;
      if (act[b] && i0 < n) r[b][t] = VT::load(col[b] + i0);
    }
  T d[CB];
#pragma unroll
  for (int b = 0; b < CB; ++b) d[b] = 0;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const int i0 = kb + (lane + 32 * t) * VW;
    if (i0 < n) {
      const typename VT::V vv = VT::load(v + i0);
#pragma unroll
      for (int b = 0; b < CB; ++b)
        if (act[b])
#pragma unroll
          for (int e = 0; e < VW; ++e) d[b] += VT::get(vv, e) * VT::get(r[b][t], e);
    }
  }
#pragma unroll
  for (int b = 0; b < CB; ++b) d[b] = warp_sum(d[b]) * tau;
  T sq[CB];
#pragma unroll
  for (int b = 0; b < CB; ++b) sq[b] = 0;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const int i0 = kb + (lane + 32 * t) * VW;
    if (i0 < n) {
      const typename VT::V vv = VT::load(v + i0);
#pragma unroll
      for (int b = 0; b < CB; ++b)
        if (act[b]) {
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            const T a = VT::get(r[b][t], e) - d[b] * VT::get(vv, e);
            VT::set(r[b][t], e, a);
            if (i0 + e > k) sq[b] += a * a;
          }
          VT::store(col[b] + i0, r[b][t]);
        }
    }
  }
#pragma unroll
  for (int b = 0; b < CB; ++b) sres[b] = warp_sum(sq[b]);
}

// squared norm of rows [kb, n) of a column (kb vector-aligned)
template <typename T>
__device__ inline T qrs_norm2(const T* __restrict__ col, int kb, int n, int lane) {
  using VT = Vec16<T>;
  constexpr int VW = VT::W;
  T s = 0;
  for (int i0 = kb + lane * VW; i0 < n; i0 += 32 * VW) {
    const typename VT::V a = VT::load(col + i0);
#pragma unroll
    for (int e = 0; e < VW; ++e) s += VT::get(a, e) * VT::get(a, e);
  }
  return warp_sum(s);
}

// FP32 groups exchange their pivot proposals in one word per CTA and step:
// the proposal's residual norm^2 (float bits, high half) and column index
// (bits 8..31) with the step's tag (k mod 256, bits 0..7).  A CTA makes its
// column updates visible, then stores its word; the others poll every word of
// the group until all carry this step's tag, which is the step's barrier and
// the proposals' gather in one L2 round trip.  Words are double-buffered by
// step parity (a CTA is at most one step ahead of the slowest).
__device__ inline unsigned long long qrs_pack(float v, int i, int k) {
  return ((unsigned long long)__float_as_uint(v) << 32) | ((unsigned long long)(unsigned)i << 8) |
         (unsigned long long)(k & 255);
}

// The factorization of one interface by the CTA of rank q in a group of G
// (G = 1: a CTA alone, no group barrier).  Gx is the group size the barrier
// waits for (G, or G + 1 when a test makes the wait run out).
template <typename T, int NV>
__device__ bool qrs_task(const QrStreamTask<T>& tk, int q, int G, int Gx, T* prop_v, int* prop_i, GroupSync* gs,
                         unsigned long long* words, int* err, T eps, long poll_limit, unsigned char* smem) {
  using VT = Vec16<T>;
  constexpr int VW = VT::W;
  __shared__ T red_v[QRS_WARPS];
  __shared__ int red_i[QRS_WARPS];
  __shared__ T s_scal[2];
  __shared__ int s_win;
  __shared__ int s_ok;
  constexpr bool kWords = std::is_same<T, float>::value;
  GroupX<T> xc{q, Gx, prop_v, prop_i, gs, err, nullptr, 0};
  xc.poll_limit = poll_limit;
  const int n = tk.n, c = tk.c, ldw = tk.ldw;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  T* v = reinterpret_cast<T*>(smem);
  const int per_cta = (c + G - 1) / G;
  const int per_warp = (per_cta + QRS_WARPS - 1) / QRS_WARPS;
  int* list = reinterpret_cast<int*>(smem + (size_t)ldw * sizeof(T)) + wid * per_warp;
  // this warp's columns: local index m = wid + QRS_WARPS t, global j = q + G m
  int cnt = 0;
  for (int t = 0; t < per_warp; ++t) {
    const long long j = q + (long long)G * (wid + (long long)QRS_WARPS * t);
    if (j >= c) break;
    if (lane == 0) list[t] = (int)j;
    ++cnt;
  }
  // the reflector buffer past row n stays zero (padding rows of W are zero)
  for (int i = tid; i < ldw; i += QRS_THREADS) v[i] = 0;
  __syncthreads();
  // ---- initial column norms; the warp's best
  T best = -1;
  int bi = c;
  for (int t = 0; t < cnt; ++t) {
    const int j = list[t];
    const T s = qrs_norm2<T>(tk.W + (size_t)j * ldw, 0, n, lane);
    argmax_pair(best, bi, s, j);
  }
  const int kmax = min(n, c);
  int rank = kmax;
  T nrm0 = 0, cut2 = 0;
  bool ok = true;
  unsigned long long work = 0;
  for (int k = 0; k < kmax; ++k) {
    // ---- this CTA's proposal
    if (lane == 0) {
      red_v[wid] = best;
      red_i[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      T b2 = -1;
      int i2 = c;
      for (int w = 0; w < QRS_WARPS; ++w) argmax_pair(b2, i2, red_v[w], red_i[w]);
      if (Gx == 1) {
        s_scal[1] = b2;
        s_win = i2;
      } else if (kWords) {
        __threadfence();                    // this CTA's column updates before its word
        volatile unsigned long long* wq = words + (size_t)(k & 1) * QR_GMAX + q;
        *wq = qrs_pack((float)b2, i2, k);
      } else {
        xc.publish(b2, i2);
      }
    }
    if (Gx > 1 && kWords) {
      __syncthreads();
      if (tid < 32) {
        T gb = -1;
        int gi = c;
        bool wok = true;
        for (int r = lane; r < Gx && wok; r += 32) {
          volatile unsigned long long* wr = words + (size_t)(k & 1) * QR_GMAX + r;
          unsigned long long w = 0;
          long it = 0;
          while (true) {
            w = *wr;
            if ((int)(w & 255ull) == (k & 255)) break;
            if (++it > poll_limit) {
              wok = false;
              break;
            }
            if (it > 2048) __nanosleep(64);
          }
          if (wok) argmax_pair(gb, gi, (T)__uint_as_float((unsigned)(w >> 32)), (int)((w >> 8) & 0xFFFFFFull));
        }
        wok = __all_sync(0xffffffffu, wok);
        __threadfence();                    // the others' column updates are visible from here on
        warp_argmax(gb, gi);
        if (lane == 0) {
          s_scal[1] = gb;
          s_win = gi;
          s_ok = wok ? 1 : 0;
          if (!wok) atomicOr(err, 16);
        }
      }
      __syncthreads();
      if (!s_ok) {
        ok = false;
        break;
      }
    } else if (Gx > 1) {
      if (!(ok = xc.sync())) break;
      // ---- group-wide winner
      if (tid < 32) {
        T gb = -1;
        int gi = c;
        for (int r = lane; r < G; r += 32) {
          T pv;
          int pi;
          xc.gather(r, pv, pi);
          argmax_pair(gb, gi, pv, pi);
        }
        warp_argmax(gb, gi);
        if (lane == 0) {
          s_scal[1] = gb;
          s_win = gi;
        }
      }
    }
    __syncthreads();
    const int p = s_win;
    const T nrm = sqrt(fmax(s_scal[1], (T)0));
    if (k == 0) {
      nrm0 = nrm;
      cut2 = (eps * nrm0) * (eps * nrm0);
    }
    if ((nrm0 == (T)0) || nrm <= eps * nrm0 || p >= c) {
      rank = k;
      break;
    }
    const bool owner = (p % G) == q;
    const int kb = k & ~(VW - 1);
    // ---- the reflector from column p (rows k..n-1), identical in every CTA
    const T* colp = tk.W + (size_t)p * ldw;
    for (int i = kb + tid; i < n; i += QRS_THREADS) v[i] = (i < k) ? (T)0 : __ldcg(colp + i);
    __syncthreads();
    T prt = 0;
    for (int i = k + 1 + tid; i < n; i += QRS_THREADS) prt += v[i] * v[i];
    const T alpha = v[k];                   // read before the barriers: thread 0 rewrites v[k] below
    const T sigma = block_sum(prt, red_v);
    T tau = 2, scale = 0;                   // column already reduced: H = I - 2 e_k e_k^T
    if (sigma > (T)0) {
      const T beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
      tau = (beta - alpha) / beta;
      scale = (T)1 / (alpha - beta);
    }
    for (int i = k + tid; i < n; i += QRS_THREADS) {
      const T vi = (i == k) ? (T)1 : v[i] * scale;
      v[i] = vi;
      if (owner) tk.V[(size_t)i + (size_t)k * n] = vi;
    }
    if (owner && tid == 0) tk.tau[k] = tau;
    __syncthreads();
    // ---- every live column of this warp: update, exact residual norm, keep or drop
    best = -1;
    bi = c;
    int kept = 0;
    constexpr int CB = (NV >= 16) ? 1 : 16 / NV;   // columns in flight per warp on the register path
    if (CB > 1 && n - kb <= 32 * VW * NV) {
      for (int t = 0; t < cnt; t += CB) {
        int js[CB];
        bool act[CB];
        T* cols[CB];
#pragma unroll
        for (int b = 0; b < CB; ++b) {
          js[b] = (t + b < cnt) ? list[t + b] : -1;
          act[b] = js[b] >= 0 && js[b] != p;  // the pivot column is done (warp-uniform)
          cols[b] = tk.W + (size_t)(act[b] ? js[b] : 0) * ldw;
        }
        T sres[CB];
        qrs_columns<T, NV, CB>(cols, act, v, tau, k, kb, n, lane, sres);
        __syncwarp();
#pragma unroll
        for (int b = 0; b < CB; ++b)
          if (act[b] && sres[b] > cut2) {
            if (lane == 0) list[kept] = js[b];   // kept <= t + b: compacted in place, in order
            ++kept;
            argmax_pair(best, bi, sres[b], js[b]);
          }
        __syncwarp();
      }
    } else {
      for (int t = 0; t < cnt; ++t) {
        const int j = list[t];
        if (j == p) continue;                 // the pivot column is done (warp-uniform)
        const T s = qrs_column<T, NV>(tk.W + (size_t)j * ldw, v, tau, k, kb, n, lane);
        __syncwarp();
        if (s > cut2) {
          if (lane == 0) list[kept] = j;      // kept <= t: compacted in place, in order
          ++kept;
          argmax_pair(best, bi, s, j);
        }
        __syncwarp();
      }
    }
    work += (unsigned long long)(n - k) * (unsigned long long)cnt;
    cnt = kept;
    xc.next_step();
  }
  if (work && lane == 0 && tk.work) atomicAdd(tk.work, work);
  if (q == 0 && tid == 0) *tk.rank = ok ? rank : 0;
  __syncthreads();                          // smem is reused by the next task
  return ok;
}

// A cooperative launch of one CTA per SM.  CTAs [0, n_group_ctas) run the
// groups of desc (large interfaces); every CTA then takes single-CTA
// interfaces from a shared queue until it is empty.  prop_v / prop_i / gs hold
// one slot per task.  fault_task >= 0: that task's barrier waits for one CTA
// more than it has (a test of the bounded wait).
template <typename T, int NV>
__global__ void __launch_bounds__(QRS_THREADS, 1)
    k_qrcp_stream(const QrStreamTask<T>* tasks, const QrGroupDesc* desc, int n_group_ctas, const int* solo,
                  int n_solo, int* queue, T* prop_v, int* prop_i, GroupSync* gs, unsigned long long* words,
                  int* err, T eps, int poll_log2, int fault_task) {
  extern __shared__ __align__(16) unsigned char qrs_smem[];
  __shared__ int s_next;
  const long poll_limit = 1l << poll_log2;
  bool ok = true;
  if ((int)blockIdx.x < n_group_ctas) {
    const QrGroupDesc d = desc[blockIdx.x];
    const int Gx = d.G + (d.task == fault_task ? 1 : 0);
    ok = qrs_task<T, NV>(tasks[d.task], d.q, d.G, Gx, prop_v + (size_t)d.task * 2 * QR_GMAX,
                         prop_i + (size_t)d.task * 2 * QR_GMAX, gs + d.task, words + (size_t)d.task * 2 * QR_GMAX,
                         err, eps, poll_limit, qrs_smem);
  }
  while (ok) {
    if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
    __syncthreads();
    const int t = s_next;
    __syncthreads();
    if (t >= n_solo) break;
    const int task = solo[t];
    const int Gx = 1 + (task == fault_task ? 1 : 0);
    ok = qrs_task<T, NV>(tasks[task], 0, 1, Gx, prop_v + (size_t)task * 2 * QR_GMAX,
                         prop_i + (size_t)task * 2 * QR_GMAX, gs + task, words + (size_t)task * 2 * QR_GMAX, err,
                         eps, poll_limit, qrs_smem);
  }
}

}  // namespace spand
