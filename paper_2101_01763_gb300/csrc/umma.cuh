// Grouped FP32 GEMM on the 5th-generation tensor cores (tcgen05, sm_100 family).
//
// Same task / term / tile contract as k_gemm_tc (C = alpha * sum_t op(A_t) op(B_t)
// + beta * C, column-major), on 128 x 64 output tiles:
//  * 128 threads stage one 16-wide k-chunk of op(A) (128 x 16) and op(B)^T
//    (64 x 16) in shared memory, split into TF32 high parts (rounded) and the
//    exact FP32 remainders (of which the tensor core reads the top 19 bits),
//    in the K-major "core matrix" layout the MMA reads without swizzling
//    (8 rows x 16 bytes per core matrix);
//  * one thread issues tcgen05.mma.kind::tf32 with the accumulator in tensor
//    memory (128 lanes x 64 FP32 columns): hi*lo + lo*hi + hi*hi per 8-wide
//    k-step (error-compensated 3xTF32, about FP32 accuracy), and commits the
//    chunk to an mbarrier of its stage; two stages alternate so the staging
//    of chunk i+1 overlaps the MMAs of chunk i;
//  * the epilogue reads the accumulator with tcgen05.ld (warp w owns lanes
//    32w..32w+31 = rows of the tile) and applies alpha / beta.
// Every mbarrier wait is bounded; on timeout the CTA sets g_umma_fail (read by
// the host after the factorization), skips its epilogue and frees its tensor
// memory.
#pragma once
#include <cstdint>

#include "dense.cuh"

namespace spand {

constexpr int UM_BM = 128, UM_BN = 64, UM_BK = 16;
constexpr int UM_BH = UM_BK / 2;          // k values of a B column one thread stages
constexpr int UM_SBO = 8 * UM_BK * 4;     // bytes between 8-row groups of a K-major operand
constexpr int UM_TMEM_COLS = 64;
// bytes of one operand stage: A hi, A lo (128 x 32 x 4), B hi, B lo (64 x 32 x 4)
constexpr int UM_A_BYTES = UM_BM * UM_BK * 4, UM_B_BYTES = UM_BN * UM_BK * 4;
constexpr int UM_STAGE_BYTES = 2 * UM_A_BYTES + 2 * UM_B_BYTES;
constexpr int UM_SMEM_BYTES = 2 * UM_STAGE_BYTES + 1024;   // two stages + alignment slack

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte step between
// core matrices along K, sbo = byte step between 8-row groups
__device__ inline uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;                       // descriptor version of the sm_100 family
  return d;                                     // base offset 0, relative LBO, no swizzle
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 64
__host__ __device__ constexpr uint32_t umma_idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(UM_BN >> 3) << 17) | ((uint32_t)(UM_BM >> 4) << 24);
}

// byte offset of element (r, k) of a K-major operand of 32-wide k-chunks:
// core matrix (r/8, k/4) of 8 rows x 4 elements; k-neighbour core matrices
// 128 bytes apart, 8-row groups 1024 bytes apart
__device__ inline uint32_t umma_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
// the same for UM_BK-wide k-chunks (8-row groups UM_SBO bytes apart)
__device__ inline uint32_t umma_off_bk(int r, int k) {
  return (uint32_t)((r >> 3) * UM_SBO + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < (1l << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ int g_umma_fail;   // set when an MMA completion wait ran out of time

template <int DEPTH>
__global__ void __launch_bounds__(128, 4) k_gemm_umma(const GemmTask<float>* tasks, const GemmTerm<float>* terms,
                                                      const TileItem* tiles) {
  extern __shared__ unsigned char um_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  // 1024-byte aligned operand area
  unsigned char* um = um_raw + ((1024 - (smem_u32(um_raw) & 1023)) & 1023);
  const TileItem it = tiles[blockIdx.x];
  const GemmTask<float> tk = tasks[it.task];
  const int i0 = it.tm * UM_BM, j0 = it.tn * UM_BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(UM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // flattened (term, k-chunk) sequence, as in k_gemm_tc: nch chunks in all;
  // (pf_t, pf_l) is the next chunk to load
  int nch = 0;
  for (int t = tk.t0; t < tk.t1; ++t) {
    const int kl = term_klim(terms[t], i0, j0, UM_BM, UM_BN);
    if (kl > 0) nch += (kl + UM_BK - 1) / UM_BK;
  }
  // the term being loaded stays in registers (ct, its k limit ct_kl): a
  // global load of the term per chunk would put its latency on every chunk
  int pf_t = tk.t0, pf_l = 0;
  GemmTerm<float> ct{};
  int ct_kl = 0;
  auto seek = [&]() {     // first term from pf_t on with a non-empty k range
    for (; pf_t < tk.t1; ++pf_t) {
      ct = terms[pf_t];
      ct_kl = term_klim(ct, i0, j0, UM_BM, UM_BN);
      if (ct_kl > 0) break;
    }
  };
  seek();
  auto advance = [&]() {
    pf_l += UM_BK;
    if (pf_l >= ct_kl) {
      pf_l = 0;
      ++pf_t;
      seek();
    }
  };
  int item = 0;
  bool failed = false;
  // operand values of one k-chunk held in registers as pieces of 4 consecutive
  // k of one row: 4 pieces of op(A) (128 x UM_BK) and 2 of op(B)^T (64 x UM_BK).
  // An operand stored along k is read 8 rows x 64 bytes per warp instruction
  // (piece q of lane l: row kr + 32 q, k offset kk); one stored along m (n)
  // keeps a row (column) per thread and reads its k values one at a time, 32
  // consecutive rows per warp instruction.  DEPTH register sets: the loads of
  // chunk i + DEPTH are issued right after the MMAs of chunk i, so their
  // latency overlaps the staging and tensor-core work of DEPTH chunks.
  const int kr = 8 * warp + (lane & 7), kk = 4 * (lane >> 3);
  const int c = tid & 63, half = tid >> 6;
  const uint64_t desc0 = umma_desc(smem_u32(um), 128, UM_SBO), desc1 = umma_desc(smem_u32(um + UM_STAGE_BYTES), 128, UM_SBO);
  auto load_chunk = [&](int l_, float (&x)[UM_BK], float (&y)[UM_BH], bool& a_kc, bool& b_kc) {
    const GemmTerm<float>& tm = ct;
    a_kc = tm.ta != 0;
    b_kc = tm.tb == 0;
    if (a_kc) {
      const int gl = l_ + kk;
      const bool vec = ((tm.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(tm.A) & 15) == 0) && gl + 4 <= tm.k;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gi = i0 + kr + 32 * q;
        if (vec) {
          const float4 f = gi < tk.m ? *reinterpret_cast<const float4*>(tm.A + gl + (size_t)gi * tm.lda)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
          x[4 * q] = f.x;
          x[4 * q + 1] = f.y;
          x[4 * q + 2] = f.z;
          x[4 * q + 3] = f.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            x[4 * q + e] = (gi < tk.m && gl + e < tm.k) ? tm.A[gl + e + (size_t)gi * tm.lda] : 0.f;
        }
      }
    } else {
      const int gi = i0 + tid;
      const float* pa = tm.A + gi + (size_t)l_ * tm.lda;
      const int nk = gi < tk.m ? tm.k - l_ : 0;     // k values left in this row
#pragma unroll
      for (int e = 0; e < UM_BK; ++e) x[e] = e < nk ? pa[e * tm.lda] : 0.f;
    }
    if (b_kc) {
      const int gl = l_ + kk;
      const bool vec = ((tm.ldb & 3) == 0) && ((reinterpret_cast<uintptr_t>(tm.B) & 15) == 0) && gl + 4 <= tm.k;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int gj = j0 + kr + 32 * q;
        if (vec) {
          const float4 f = gj < tk.n ? *reinterpret_cast<const float4*>(tm.B + gl + (size_t)gj * tm.ldb)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
          y[4 * q] = f.x;
          y[4 * q + 1] = f.y;
          y[4 * q + 2] = f.z;
          y[4 * q + 3] = f.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            y[4 * q + e] = (gj < tk.n && gl + e < tm.k) ? tm.B[gl + e + (size_t)gj * tm.ldb] : 0.f;
        }
      }
    } else {
      const int gj = j0 + c, kb = l_ + half * UM_BH;
      const float* pb = tm.B + gj + (size_t)kb * tm.ldb;
      const int nk = gj < tk.n ? tm.k - kb : 0;
#pragma unroll
      for (int e = 0; e < UM_BH; ++e) y[e] = e < nk ? pb[e * tm.ldb] : 0.f;
    }
  };
  // stage chunk `item` from registers and issue its MMAs; false on a timed-out wait
  auto process = [&](const float (&x)[UM_BK], const float (&y)[UM_BH], bool a_kc, bool b_kc) -> bool {
    const int s = item & 1;
    unsigned char* st = um + s * UM_STAGE_BYTES;
    if (item >= 2) {
      // the MMAs that read this stage two chunks ago must be done; one thread
      // polls, the others wait at the barrier, and the outcome is uniform
      const bool ok = tid != 0 || mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((item >> 1) - 1) & 1));
      if (__syncthreads_or(!ok)) return false;
    }
    // ---- split the chunk's values into TF32 hi / lo in the core-matrix layout
    {
#pragma unroll
      for (int kq = 0; kq < UM_BK; kq += 4) {
        uint4 hi, lo;
        hi.x = to_tf32(x[kq]);
        hi.y = to_tf32(x[kq + 1]);
        hi.z = to_tf32(x[kq + 2]);
        hi.w = to_tf32(x[kq + 3]);
        lo.x = __float_as_uint(x[kq] - __uint_as_float(hi.x));
        lo.y = __float_as_uint(x[kq + 1] - __uint_as_float(hi.y));
        lo.z = __float_as_uint(x[kq + 2] - __uint_as_float(hi.z));
        lo.w = __float_as_uint(x[kq + 3] - __uint_as_float(hi.w));
        const uint32_t off = a_kc ? umma_off_bk(kr + 8 * kq, kk) : umma_off_bk(tid, kq);   // piece kq / 4
        *reinterpret_cast<uint4*>(st + off) = hi;
        *reinterpret_cast<uint4*>(st + UM_A_BYTES + off) = lo;
      }
#pragma unroll
      for (int kq = 0; kq < UM_BH; kq += 4) {
        uint4 hi, lo;
        hi.x = to_tf32(y[kq]);
        hi.y = to_tf32(y[kq + 1]);
        hi.z = to_tf32(y[kq + 2]);
        hi.w = to_tf32(y[kq + 3]);
        lo.x = __float_as_uint(y[kq] - __uint_as_float(hi.x));
        lo.y = __float_as_uint(y[kq + 1] - __uint_as_float(hi.y));
        lo.z = __float_as_uint(y[kq + 2] - __uint_as_float(hi.z));
        lo.w = __float_as_uint(y[kq + 3] - __uint_as_float(hi.w));
        const uint32_t off = b_kc ? umma_off_bk(kr + 8 * kq, kk) : umma_off_bk(c, half * UM_BH + kq);
        *reinterpret_cast<uint4*>(st + 2 * UM_A_BYTES + off) = hi;
        *reinterpret_cast<uint4*>(st + 2 * UM_A_BYTES + UM_B_BYTES + off) = lo;
      }
    }
    // the generic-proxy stores must be visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t idesc = umma_idesc_tf32();
      const uint64_t d0 = s ? desc1 : desc0;   // descriptor of the stage's A hi part
#pragma unroll
      for (int ks = 0; ks < UM_BK / 8; ++ks) {
        // two core matrices along K (256 bytes) per 8-wide step; descriptor
        // addresses are in 16-byte units in the low bits
        const uint64_t ko = (uint64_t)(ks * 256) >> 4;
        const uint64_t dah = d0 + ko, dal = d0 + ko + (UM_A_BYTES >> 4);
        const uint64_t dbh = d0 + ko + ((2 * UM_A_BYTES) >> 4), dbl = d0 + ko + ((2 * UM_A_BYTES + UM_B_BYTES) >> 4);
        const uint32_t acc0 = (item > 0 || ks > 0) ? 1u : 0u;
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
          smem_u32(&mbar[s])));
    }
    ++item;
    return true;
  };
  float x0[UM_BK], y0[UM_BH], x1[UM_BK], y1[UM_BH];
  bool ak0 = false, bk0 = false, ak1 = false, bk1 = false;
  if (pf_t < tk.t1) {
    load_chunk(pf_l, x0, y0, ak0, bk0);
    advance();
  }
  if (DEPTH == 2 && pf_t < tk.t1) {
    load_chunk(pf_l, x1, y1, ak1, bk1);
    advance();
  }
  while (item < nch) {
    if (!process(x0, y0, ak0, bk0)) {
      failed = true;
      break;
    }
    if (pf_t < tk.t1) {      // overlaps the MMAs just issued
      load_chunk(pf_l, x0, y0, ak0, bk0);
      advance();
    }
    if (DEPTH == 1 || item >= nch) continue;
    if (!process(x1, y1, ak1, bk1)) {
      failed = true;
      break;
    }
    if (pf_t < tk.t1) {
      load_chunk(pf_l, x1, y1, ak1, bk1);
      advance();
    }
  }
  // ---- wait for the last committed chunk (it tracks every earlier MMA of the thread)
  if (tid == 0 && item > 0 && !failed) {
    const int last = item - 1;
    if (!mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1))) failed = true;
  }
  if (failed) atomicOr(&s_fail, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (s_fail) {
    if (tid == 0) atomicOr(&g_umma_fail, 1);
  } else {
    // ---- epilogue: warp w holds rows 32w..32w+31 of the tile, 64 columns each
    const int row = warp * 32 + lane, gi = i0 + row;
#pragma unroll
    for (int cb = 0; cb < UM_BN; cb += 16) {
      uint32_t v[16];
      if (item > 0) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
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
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UM_TMEM_COLS));
  }
}

}  // namespace spand
