// Grouped FP32 GEMM on the 5th-generation tensor cores with warp-specialised
// roles (same task / term / tile contract as k_gemm_umma:
// C = alpha * sum_t op(A_t) op(B_t) + beta * C, column-major, 128 x 64 tiles,
// 16-wide k-chunks, error-compensated 3xTF32 with FP32 accumulation).
//
//  * producer warps (0-1) copy raw FP32 operand tiles from global memory into a
//    4-deep ring of shared-memory stages with cp.async, 16 bytes at a time
//    along whichever dimension is contiguous in memory (column-major A runs
//    along m, row-major A along k; the same for B), zero filling past the
//    matrix edges; each producer's copies arrive on the stage's "full"
//    mbarrier when they land (cp.async.mbarrier.arrive);
//  * converter warps (2-5) split each raw value into a TF32 high part
//    (truncated) and an exact FP32 remainder and write both in the K-major
//    core-matrix layout the MMA reads, into a 2-deep ring;
//  * one thread of warp 6 issues lo*hi + hi*lo + hi*hi per 8-wide k-step
//    (tcgen05.mma.kind::tf32, accumulator in tensor memory) and commits each
//    chunk to the converted stage's "empty" mbarrier;
//  * the converter warps then read the accumulator (tcgen05.ld, warp w owns
//    the lanes of quarter w % 4) and apply alpha / beta.
// Every wait is bounded (about one second); on timeout the CTA sets
// g_umma_fail, skips its epilogue, waits for its copies and frees its tensor
// memory.
#pragma once
#include <cstdint>

#include "umma.cuh"

namespace spand {

constexpr int U3_BM = 128, U3_BN = 64, U3_BK = 16;
static_assert(U3_BM == UM_BM && U3_BN == UM_BN && U3_BK == UM_BK, "tiles shared with k_gemm_umma");
constexpr int U3_RS = 4, U3_CS = 2;                  // raw and converted ring depths
constexpr int U3_THREADS = 224;                      // 7 warps
constexpr int U3_PROD = 64, U3_CONV = 128;           // producer / converter threads
constexpr int U3_KPAD = U3_BK + 4;                   // row stride (floats) of K-contiguous raw tiles
constexpr int U3_RAW_A = (U3_BM * U3_KPAD > U3_BK * U3_BM) ? U3_BM * U3_KPAD : U3_BK * U3_BM;   // floats
constexpr int U3_RAW_B = (U3_BN * U3_KPAD > U3_BK * U3_BN) ? U3_BN * U3_KPAD : U3_BK * U3_BN;
constexpr int U3_RAW_BYTES = (U3_RAW_A + U3_RAW_B) * 4;
constexpr int U3_CA = U3_BM * U3_BK * 4, U3_CB = U3_BN * U3_BK * 4;   // one converted operand part (bytes)
constexpr int U3_CONV_BYTES = 2 * U3_CA + 2 * U3_CB;
constexpr int U3_SMEM_BYTES = U3_RS * U3_RAW_BYTES + U3_CS * U3_CONV_BYTES + 1024;
constexpr int U3_TMEM_COLS = 64;

// bounded wait on an mbarrier phase: gives up after about one second of
// global-timer time (no wait of a healthy tile comes near that)
__device__ inline bool u3_wait(uint32_t bar, uint32_t parity) {
  uint64_t t0 = 0;
  for (long it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 0) {
      uint64_t now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (it == 0)
        t0 = now;
      else if (now - t0 > 1000000000ull || it > (1l << 26))
        return false;
    }
  }
}
__device__ inline void u3_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ inline void u3_cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ inline void u3_cp4(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

// The tile's flattened (term, k-chunk) sequence, walked identically by every role.
struct U3Cursor {
  int t, l;
};
__device__ inline void u3_first(U3Cursor& c, const GemmTerm<float>* terms, const GemmTask<float>& tk, int i0, int j0) {
  c.t = tk.t0;
  c.l = 0;
  while (c.t < tk.t1 && term_klim(terms[c.t], i0, j0, U3_BM, U3_BN) <= 0) ++c.t;
}
__device__ inline void u3_next(U3Cursor& c, const GemmTerm<float>* terms, const GemmTask<float>& tk, int i0, int j0) {
  c.l += U3_BK;
  while (c.t < tk.t1 && c.l >= term_klim(terms[c.t], i0, j0, U3_BM, U3_BN)) {
    ++c.t;
    c.l = 0;
  }
}

// Raw tile of an operand: `rows` rows (m or n) x 16 k values starting at
// (r0, l0) of op(X) (op(X)[r, l] = X[r + l ld] when contiguous along r, i.e.
// "rowc", else X[l + r ld]).  Contiguous along r: stored [k][rows]; contiguous
// along k: stored [rows][U3_KPAD].  Thread p of np copies 16-byte groups.
template <int ROWS>
__device__ inline void u3_copy(uint32_t dst, const float* X, int ld, bool rowc, int r0, int nr, int l0, int kl, int p,
                               int np) {
  const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (rowc) {
    // groups of 4 consecutive rows at one k: ROWS / 4 x 16 groups
    constexpr int NG = ROWS / 4 * U3_BK;
    for (int g = p; g < NG; g += np) {
      const int lk = g / (ROWS / 4), rr = (g % (ROWS / 4)) * 4;
      const int l = l0 + lk, r = r0 + rr;
      const uint32_t d = dst + (uint32_t)((lk * ROWS + rr) * 4);
      if (vec) {
        const int nb = (l < kl) ? max(0, min(4, nr - r)) * 4 : 0;
        u3_cp16(d, nb ? X + r + (size_t)l * ld : X, nb);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool ok = l < kl && r + e < nr;
          u3_cp4(d + 4 * e, ok ? X + (r + e) + (size_t)l * ld : X, ok);
        }
      }
    }
  } else {
    // groups of 4 consecutive k at one row: ROWS x 4 groups
    constexpr int NG = ROWS * (U3_BK / 4);
    for (int g = p; g < NG; g += np) {
      const int rr = g / (U3_BK / 4), lq = (g % (U3_BK / 4)) * 4;
      const int r = r0 + rr, l = l0 + lq;
      const uint32_t d = dst + (uint32_t)((rr * U3_KPAD + lq) * 4);
      if (vec) {
        const int nb = (r < nr) ? max(0, min(4, kl - l)) * 4 : 0;
        u3_cp16(d, nb ? X + l + (size_t)r * ld : X, nb);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool ok = r < nr && l + e < kl;
          u3_cp4(d + 4 * e, ok ? X + (l + e) + (size_t)r * ld : X, ok);
        }
      }
    }
  }
}

// 4 raw values (k = kq..kq+3 of row r) of a raw tile
template <int ROWS>
__device__ inline float4 u3_raw4(const float* raw, bool rowc, int r, int kq) {
  if (rowc)
    return make_float4(raw[(kq + 0) * ROWS + r], raw[(kq + 1) * ROWS + r], raw[(kq + 2) * ROWS + r],
                       raw[(kq + 3) * ROWS + r]);
  return *reinterpret_cast<const float4*>(raw + r * U3_KPAD + kq);
}

__device__ inline void u3_split_store(unsigned char* hi_base, unsigned char* lo_base, uint32_t off, float4 x) {
  uint4 h;
  float4 lo;
  h.x = __float_as_uint(x.x) & 0xFFFFE000u;
  h.y = __float_as_uint(x.y) & 0xFFFFE000u;
  h.z = __float_as_uint(x.z) & 0xFFFFE000u;
  h.w = __float_as_uint(x.w) & 0xFFFFE000u;
  lo.x = x.x - __uint_as_float(h.x);
  lo.y = x.y - __uint_as_float(h.y);
  lo.z = x.z - __uint_as_float(h.z);
  lo.w = x.w - __uint_as_float(h.w);
  *reinterpret_cast<uint4*>(hi_base + off) = h;
  *reinterpret_cast<float4*>(lo_base + off) = lo;
}

__global__ void __launch_bounds__(U3_THREADS, 2) k_gemm_umma3(const GemmTask<float>* tasks,
                                                               const GemmTerm<float>* terms, const TileItem* tiles) {
  extern __shared__ unsigned char u3_smem[];
  __shared__ uint64_t full_raw[U3_RS], empty_raw[U3_RS], full_conv[U3_CS], empty_conv[U3_CS], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  unsigned char* base = u3_smem + ((1024 - (smem_u32(u3_smem) & 1023)) & 1023);
  unsigned char* raw_base = base;
  unsigned char* conv_base = base + U3_RS * U3_RAW_BYTES;
  const TileItem it = tiles[blockIdx.x];
  const GemmTask<float> tk = tasks[it.task];
  const int i0 = it.tm * U3_BM, j0 = it.tn * U3_BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (warp == 6) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(U3_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < U3_RS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_raw[s])), "r"(U3_PROD));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty_raw[s])), "r"(U3_CONV));
    }
    for (int s = 0; s < U3_CS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_conv[s])), "r"(U3_CONV));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_conv[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // number of chunks of the tile
  int nch = 0;
  {
    U3Cursor c;
    u3_first(c, terms, tk, i0, j0);
    while (c.t < tk.t1) {
      ++nch;
      u3_next(c, terms, tk, i0, j0);
    }
  }

  if (warp < 2) {
    // ---------------- producers
    const int p = tid;
    U3Cursor c;
    u3_first(c, terms, tk, i0, j0);
    for (int i = 0; i < nch; ++i) {
      const int s = i % U3_RS;
      if (i >= U3_RS && !u3_wait(smem_u32(&empty_raw[s]), (uint32_t)(((i / U3_RS) - 1) & 1))) {
        atomicOr(&s_fail, 1);
        break;
      }
      if (s_fail) break;
      const GemmTerm<float> tm = terms[c.t];
      const uint32_t ra = smem_u32(raw_base + s * U3_RAW_BYTES), rb = ra + U3_RAW_A * 4;
      // op(A)[i, l]: ta = 0 -> A[i + l lda] (contiguous along m); op(B)[l, j]: tb = 1 -> contiguous along n
      u3_copy<U3_BM>(ra, tm.A, tm.lda, !tm.ta, i0, tk.m, c.l, tm.k, p, U3_PROD);
      u3_copy<U3_BN>(rb, tm.B, tm.ldb, tm.tb != 0, j0, tk.n, c.l, tm.k, p, U3_PROD);
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full_raw[s])) : "memory");
      u3_next(c, terms, tk, i0, j0);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp < 6) {
    // ---------------- converters
    const int cr = tid - U3_PROD;                 // A row; B row cr & 63, k half cr >> 6
    const int br = cr & 63, bh = cr >> 6;
    U3Cursor c;
    u3_first(c, terms, tk, i0, j0);
    for (int i = 0; i < nch; ++i) {
      const int s = i % U3_RS, t = i % U3_CS;
      bool ok = u3_wait(smem_u32(&full_raw[s]), (uint32_t)((i / U3_RS) & 1));
      if (ok && i >= U3_CS) ok = u3_wait(smem_u32(&empty_conv[t]), (uint32_t)(((i / U3_CS) - 1) & 1));
      if (!ok) {
        atomicOr(&s_fail, 1);
        break;
      }
      if (s_fail) break;
      const GemmTerm<float> tm = terms[c.t];
      const float* ra = reinterpret_cast<const float*>(raw_base + s * U3_RAW_BYTES);
      const float* rb = ra + U3_RAW_A;
      unsigned char* cv = conv_base + t * U3_CONV_BYTES;
#pragma unroll
      for (int kq = 0; kq < U3_BK; kq += 4)
        u3_split_store(cv, cv + U3_CA, umma_off_bk(cr, kq), u3_raw4<U3_BM>(ra, !tm.ta, cr, kq));
#pragma unroll
      for (int kq = 0; kq < U3_BK / 2; kq += 4)
        u3_split_store(cv + 2 * U3_CA, cv + 2 * U3_CA + U3_CB, umma_off_bk(br, bh * (U3_BK / 2) + kq),
                       u3_raw4<U3_BN>(rb, tm.tb != 0, br, bh * (U3_BK / 2) + kq));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      u3_arrive(smem_u32(&empty_raw[s]));
      u3_arrive(smem_u32(&full_conv[t]));
      u3_next(c, terms, tk, i0, j0);
    }
  } else if (lane == 0) {
    // ---------------- MMA issue (one thread)
    const uint32_t idesc = umma_idesc_tf32();
    int i = 0;
    for (; i < nch; ++i) {
      const int t = i % U3_CS;
      if (!u3_wait(smem_u32(&full_conv[t]), (uint32_t)((i / U3_CS) & 1))) {
        atomicOr(&s_fail, 1);
        break;
      }
      if (s_fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a_hi = smem_u32(conv_base + t * U3_CONV_BYTES), a_lo = a_hi + U3_CA;
      const uint32_t b_hi = a_hi + 2 * U3_CA, b_lo = b_hi + U3_CB;
#pragma unroll
      for (int ks = 0; ks < U3_BK / 8; ++ks) {
        const uint32_t ko = ks * 256;
        const uint64_t dah = umma_desc(a_hi + ko, 128, UM_SBO), dal = umma_desc(a_lo + ko, 128, UM_SBO);
        const uint64_t dbh = umma_desc(b_hi + ko, 128, UM_SBO), dbl = umma_desc(b_lo + ko, 128, UM_SBO);
        const uint32_t acc0 = (i > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(dal), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(dah), "l"(dbh), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty_conv[t])));
    }
    // the commit tracks every MMA issued above; with none issued, arrive directly
    if (i > 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&done_bar)));
    else
      u3_arrive(smem_u32(&done_bar));
  }
  // ---- epilogue by the converter warps
  if (warp >= 2 && warp < 6) {
    const bool ok = nch == 0 || u3_wait(smem_u32(&done_bar), 0u);
    if (!ok) atomicOr(&s_fail, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    // the warp decides as one (tcgen05.ld is warp-collective)
    if (!__any_sync(0xffffffffu, !ok || s_fail != 0)) {
      const int q = warp & 3, row = q * 32 + lane, gi = i0 + row;
#pragma unroll 1
      for (int cb = 0; cb < U3_BN; cb += 16) {
        uint32_t v[16];
        if (nch > 0) {
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cb;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0u;
        }
        if (gi < tk.m) {
          // all loads of C before any store, so they overlap (a load placed
          // after a store to C cannot be moved above it by the compiler)
          float cv[16];
#pragma unroll
          for (int e = 0; e < 16; ++e)
            cv[e] = (tk.beta != 0.f && j0 + cb + e < tk.n) ? tk.C[gi + (size_t)(j0 + cb + e) * tk.ldc] : 0.f;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int gj = j0 + cb + e;
            if (gj < tk.n) tk.C[gi + (size_t)gj * tk.ldc] = tk.alpha * __uint_as_float(v[e]) + tk.beta * cv[e];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (s_fail && tid == 0) atomicOr(&g_umma_fail, 1);
  if (warp == 6) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(U3_TMEM_COLS));
  }
}

}  // namespace spand
