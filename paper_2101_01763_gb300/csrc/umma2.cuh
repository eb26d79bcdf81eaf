// Grouped FP32 GEMM on the 5th-generation tensor cores, pipelined through
// asynchronous copies (same task / term / tile contract as k_gemm_umma:
// C = alpha * sum_t op(A_t) op(B_t) + beta * C, column-major).
//
// 128 x 128 output tiles, 32-wide k-chunks, 128 threads:
//  * raw FP32 operand values go from global memory straight into a 4-deep ring
//    of shared-memory stages with cp.async (16-byte copies where 4 consecutive
//    k values are contiguous and aligned, 4-byte copies otherwise, zero fill
//    past the matrix edges), already in the K-major core-matrix layout that the
//    MMA reads (8 rows x 16 bytes per core matrix);
//  * a conversion pass splits each value in place: the stage keeps the high
//    part trunc_tf32(x) (the upper 19 bits, an exact TF32 value) and the
//    remainder x - trunc_tf32(x) (exact in FP32) goes to a second, 2-deep
//    buffer;
//  * one thread issues lo*hi + hi*lo + hi*hi per 8-wide k-step
//    (tcgen05.mma.kind::tf32, accumulator in tensor memory, 128 lanes x 128
//    FP32 columns) -- the error-compensated 3xTF32 product, about FP32
//    accuracy -- and commits the chunk to the mbarrier of its stage;
//  * copies run two chunks ahead of the MMAs; the epilogue reads the
//    accumulator with tcgen05.ld and applies alpha / beta.
// Every mbarrier wait is bounded; on timeout the CTA sets g_umma_fail, skips
// its epilogue, waits for its own copies and frees its tensor memory.
#pragma once
#include <cstdint>

#include "umma.cuh"

namespace spand {

constexpr int U2_BM = 128, U2_BN = 128, U2_BK = 32;
constexpr int U2_RAW = 4, U2_LO = 2;                 // ring depths
constexpr int U2_TMEM_COLS = 128;
constexpr int U2_A_BYTES = U2_BM * U2_BK * 4;        // 16 KB
constexpr int U2_B_BYTES = U2_BN * U2_BK * 4;        // 16 KB
constexpr int U2_STAGE = U2_A_BYTES + U2_B_BYTES;    // one raw or lo stage
constexpr int U2_SMEM_BYTES = (U2_RAW + U2_LO) * U2_STAGE + 1024;

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 128
__host__ __device__ constexpr uint32_t umma2_idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(U2_BN >> 3) << 17) | ((uint32_t)(U2_BM >> 4) << 24);
}

__device__ inline void u2_cp4(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ inline void u2_cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ inline void u2_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void u2_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One thread's share of a chunk: row r of op(A) (32 k values) and row r of
// op(B)^T (32 k values) into the raw stage at `st` (shared address).
__device__ inline void u2_load(uint32_t st, const GemmTerm<float>& tm, const GemmTask<float>& tk, int i0, int j0,
                               int l0, int r) {
  const int gi = i0 + r, gj = j0 + r;
  const int kl = tm.k;
  // op(A)[gi, l]: ta = 0 -> A[gi + l lda] (strided in l), ta = 1 -> A[l + gi lda] (contiguous in l)
  if (tm.ta && (tm.lda & 3) == 0 && (reinterpret_cast<uintptr_t>(tm.A) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < U2_BK / 4; ++q) {
      const int l = l0 + 4 * q;
      const int nb = (gi < tk.m) ? max(0, min(4, kl - l)) * 4 : 0;
      const float* src = nb ? tm.A + l + (size_t)gi * tm.lda : tm.A;
      u2_cp16(st + umma_off(r, 4 * q), src, nb);
    }
  } else {
#pragma unroll 8
    for (int e = 0; e < U2_BK; ++e) {
      const int l = l0 + e;
      const bool ok = gi < tk.m && l < kl;
      const float* src = ok ? (tm.ta ? tm.A + l + (size_t)gi * tm.lda : tm.A + gi + (size_t)l * tm.lda) : tm.A;
      u2_cp4(st + umma_off(r, e), src, ok);
    }
  }
  // op(B)[l, gj]: tb = 0 -> B[l + gj ldb] (contiguous in l), tb = 1 -> B[gj + l ldb]
  const uint32_t sb = st + U2_A_BYTES;
  if (!tm.tb && (tm.ldb & 3) == 0 && (reinterpret_cast<uintptr_t>(tm.B) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < U2_BK / 4; ++q) {
      const int l = l0 + 4 * q;
      const int nb = (gj < tk.n) ? max(0, min(4, kl - l)) * 4 : 0;
      const float* src = nb ? tm.B + l + (size_t)gj * tm.ldb : tm.B;
      u2_cp16(sb + umma_off(r, 4 * q), src, nb);
    }
  } else {
#pragma unroll 8
    for (int e = 0; e < U2_BK; ++e) {
      const int l = l0 + e;
      const bool ok = gj < tk.n && l < kl;
      const float* src = ok ? (tm.tb ? tm.B + gj + (size_t)l * tm.ldb : tm.B + l + (size_t)gj * tm.ldb) : tm.B;
      u2_cp4(sb + umma_off(r, e), src, ok);
    }
  }
}

__global__ void __launch_bounds__(128, 1) k_gemm_umma2(const GemmTask<float>* tasks, const GemmTerm<float>* terms,
                                                       const TileItem* tiles) {
  extern __shared__ unsigned char u2_raw[];
  __shared__ uint64_t mbar[U2_RAW];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  unsigned char* base = u2_raw + ((1024 - (smem_u32(u2_raw) & 1023)) & 1023);
  const uint32_t sbase = smem_u32(base);
  auto raw_st = [&](int i) { return sbase + (uint32_t)((i % U2_RAW) * U2_STAGE); };
  auto lo_st = [&](int i) { return sbase + (uint32_t)((U2_RAW + (i % U2_LO)) * U2_STAGE); };
  const TileItem it = tiles[blockIdx.x];
  const GemmTask<float> tk = tasks[it.task];
  const int i0 = it.tm * U2_BM, j0 = it.tn * U2_BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(U2_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < U2_RAW; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // the flattened (term, k-chunk) sequence of the tile, walked by the copy cursor
  int lt = tk.t0, ll = 0;          // copy cursor
  while (lt < tk.t1 && term_klim(terms[lt], i0, j0, U2_BM, U2_BN) <= 0) ++lt;
  auto advance = [&](int& t, int& l) {
    l += U2_BK;
    while (t < tk.t1 && l >= term_klim(terms[t], i0, j0, U2_BM, U2_BN)) {
      ++t;
      l = 0;
    }
  };
  int nchunks = 0;                 // chunks issued to the copy engine
  // prologue: chunks 0 and 1
  for (int p = 0; p < 2; ++p) {
    if (lt < tk.t1) {
      u2_load(raw_st(nchunks), terms[lt], tk, i0, j0, ll, tid);
      ++nchunks;
      advance(lt, ll);
    }
    u2_commit();
  }
  bool failed = false;
  int item = 0;
  for (; item < nchunks; ++item) {
    // ---- copies of chunk item+2 into raw stage (item+2) % 4, free once the
    // MMAs of chunk item-2 (same raw stage) are done; that also frees lo
    // stage item % 2
    if (item >= 2) {
      const int d = item - 2;
      const bool ok = mbar_wait(smem_u32(&mbar[d % U2_RAW]), (uint32_t)((d / U2_RAW) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    if (lt < tk.t1) {
      u2_load(raw_st(nchunks), terms[lt], tk, i0, j0, ll, tid);
      ++nchunks;
      advance(lt, ll);
    }
    u2_commit();
    u2_wait<2>();            // chunk `item` has landed (two newer groups may be pending)
    __syncthreads();
    // ---- remainders x - trunc_tf32(x) of chunk `item` into lo stage item % 2
    {
      unsigned char* rs = base + (item % U2_RAW) * U2_STAGE;
      unsigned char* ls = base + (U2_RAW + (item % U2_LO)) * U2_STAGE;
#pragma unroll
      for (int q = 0; q < 2 * U2_BK / 4; ++q) {
        // A row tid then B row tid: 8 core-matrix rows of 16 bytes each
        const uint32_t off = (q < U2_BK / 4) ? umma_off(tid, 4 * q) : U2_A_BYTES + umma_off(tid, 4 * (q - U2_BK / 4));
        const uint4 x = *reinterpret_cast<const uint4*>(rs + off);
        uint4 hi;
        float4 lo;
        hi.x = x.x & 0xFFFFE000u;
        hi.y = x.y & 0xFFFFE000u;
        hi.z = x.z & 0xFFFFE000u;
        hi.w = x.w & 0xFFFFE000u;
        lo.x = __uint_as_float(x.x) - __uint_as_float(hi.x);
        lo.y = __uint_as_float(x.y) - __uint_as_float(hi.y);
        lo.z = __uint_as_float(x.z) - __uint_as_float(hi.z);
        lo.w = __uint_as_float(x.w) - __uint_as_float(hi.w);
        *reinterpret_cast<uint4*>(rs + off) = hi;     // exact TF32 values: no reliance on how the MMA reads low bits
        *reinterpret_cast<float4*>(ls + off) = lo;
      }
    }
    // the copies (async proxy writes landed through the generic path) and the
    // remainders must be visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a_hi = raw_st(item), b_hi = a_hi + U2_A_BYTES;
      const uint32_t a_lo = lo_st(item), b_lo = a_lo + U2_A_BYTES;
      const uint32_t idesc = umma2_idesc_tf32();
#pragma unroll
      for (int ks = 0; ks < U2_BK / 8; ++ks) {
        const uint32_t ko = ks * 256;
        const uint64_t dah = umma_desc(a_hi + ko, 128, 1024), dal = umma_desc(a_lo + ko, 128, 1024);
        const uint64_t dbh = umma_desc(b_hi + ko, 128, 1024), dbl = umma_desc(b_lo + ko, 128, 1024);
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
          smem_u32(&mbar[item % U2_RAW])));
    }
  }
  u2_wait<0>();              // no copy may still target this CTA's shared memory
  // ---- the last committed chunk tracks every earlier MMA of the thread
  if (item > 0 && !failed) {
    const int last = item - 1;
    if (!mbar_wait(smem_u32(&mbar[last % U2_RAW]), (uint32_t)((last / U2_RAW) & 1))) failed = true;
  }
  if (failed) atomicOr(&s_fail, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (s_fail) {
    if (tid == 0) atomicOr(&g_umma_fail, 1);
  } else {
    // ---- epilogue: warp w holds rows 32w..32w+31 of the tile, 128 columns each
    const int row = warp * 32 + lane, gi = i0 + row;
#pragma unroll 1
    for (int cb = 0; cb < U2_BN; cb += 16) {
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
        // all loads of C before any store, so they overlap
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(U2_TMEM_COLS));
  }
}

}  // namespace spand
