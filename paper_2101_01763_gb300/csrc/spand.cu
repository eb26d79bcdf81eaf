// spaND factorization and apply on the GPU (Sec. 2.2.1, Eqs. 10-12).
//
// The host walks the levels of the plan; at each level every phase is one
// batched launch over all clusters of the level:
//   eliminate interiors   getrf (panel + grouped GEMM), L^-1 and U^-1,
//                         Y = L^-1 P^T A_sn, X = A_ns U^-1, Schur A_nn -= X Y
//   scale interfaces      getrf, |D|^-1/2 L^-1 and U^-1 |D|^1/2, A_ij <- SL_i A_ij SU_j
//   sparsify              W = [A_sn A_ns^T], column-pivoted QR truncated at eps,
//                         explicit Q_c; ranks are read back (one small copy)
//   compress + merge      A_ij <- Q_ic^T A_ij Q_jc written straight into the
//                         next level's merged blocks; identity on the diagonal
// Factors kept for the apply: L^-1 (permutation folded into the gather
// indices), U^-1, X, Y, the scaled triangular inverses and Q_c.  The apply is
// a fixed list of gather-GEMV launches built once per factorization.
#include <algorithm>
#include <stdexcept>
#include <array>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <memory>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "dense.cuh"
#include "qrcp_stream.cuh"
#include "gemv.cuh"
#include "umma.cuh"
#include "umma2.cuh"
#include "umma3.cuh"
#include "internal.h"

namespace spand {

// largest dynamic shared memory any kernel here asks for (x vectors, reflectors)
constexpr size_t kGemvSmemMax = 200 * 1024;
// dynamic shared memory of the RRQR cluster kernel (W chunk + reflector)
constexpr size_t kQrSmemMax = 224 * 1024;   // clamped per kernel to the opt-in limit minus its static shared memory

// ------------------------------------------------------------------ device memory
// host wall-clock milliseconds
static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

std::atomic<uint64_t> g_kernel_launches{0};

int debug_level() {
  static const int lv = [] {
    const char* v = std::getenv("SPAND_DEBUG");
    return v ? std::atoi(v) : 0;
  }();
  return lv;
}

void report_cuda_error(cudaError_t e, const char* expr, const char* file, int line) {
  const bool on = debug_level() >= 1;
  if (on) std::fprintf(stderr, "spand: %s:%d: %s -> %s (%s)\n", file, line, expr, cudaGetErrorName(e),
                       cudaGetErrorString(e));
}

// Pinned host staging for the small uploads of a factorization (task tables,
// slot lists): a copy from pinned memory is a plain DMA enqueue, where a copy
// from pageable memory is staged by the driver on every call.  The chunks come
// from a process-wide pool; a stage is reset only after its stream has been
// synchronised, so no queued copy still reads a reused chunk.
struct PinnedPool {
  std::mutex mu;
  std::vector<std::pair<char*, size_t>> free_chunks;
  static PinnedPool& get() {
    static PinnedPool* p = new PinnedPool();   // never destroyed: outlives every factor
    return *p;
  }
  std::pair<char*, size_t> take(size_t want) {
    {
      std::lock_guard<std::mutex> g(mu);
      for (size_t i = 0; i < free_chunks.size(); ++i)
        if (free_chunks[i].second >= want) {
          auto c = free_chunks[i];
          free_chunks.erase(free_chunks.begin() + i);
          return c;
        }
    }
    void* h = nullptr;
    if (cudaMallocHost(&h, want) != cudaSuccess) {
      cudaGetLastError();
      return {nullptr, 0};
    }
    return {static_cast<char*>(h), want};
  }
  void give(std::pair<char*, size_t> c) {
    std::lock_guard<std::mutex> g(mu);
    free_chunks.push_back(c);
  }
};

struct PinnedStage {
  static constexpr size_t kChunk = size_t(8) << 20;
  std::vector<std::pair<char*, size_t>> chunks;
  size_t ci = 0, off = 0;
  // host buffer for `bytes`, or nullptr (the caller then copies from pageable memory)
  char* get(size_t bytes) {
    bytes = (bytes + 63) & ~size_t(63);
    while (true) {
      if (ci < chunks.size() && off + bytes <= chunks[ci].second) {
        char* p = chunks[ci].first + off;
        off += bytes;
        return p;
      }
      if (ci < chunks.size() && off > 0) {
        ++ci;
        off = 0;
        continue;
      }
      if (ci >= chunks.size()) {
        auto c = PinnedPool::get().take(std::max(kChunk, bytes));
        if (!c.first) return nullptr;
        chunks.push_back(c);
        ci = chunks.size() - 1;
        off = 0;
        continue;
      }
      // current chunk is empty but too small: take a larger one after it
      auto c = PinnedPool::get().take(std::max(kChunk, bytes));
      if (!c.first) return nullptr;
      chunks.insert(chunks.begin() + ci, c);
      off = 0;
    }
  }
  void reset() {   // only after the stream that read the chunks has been synchronised
    ci = 0;
    off = 0;
  }
  ~PinnedStage() {
    for (auto& c : chunks) PinnedPool::get().give(c);
  }
};

// Stream-ordered device memory carved from 32 MB slabs (256-byte aligned
// pieces), so that the thousands of small arrays of a factorization cost a
// handful of allocator calls; large arrays get their own allocation.
struct DevMem {
  static constexpr size_t kSlab = size_t(32) << 20;
  std::vector<void*> ptrs;
  cudaStream_t st = nullptr;
  int err = 0;
  char* cur = nullptr;
  size_t left = 0;
  PinnedStage* stage = nullptr;   // optional pinned staging for uploads
  template <typename X>
  X* alloc(size_t n) {
    if (n == 0) n = 1;
    const size_t bytes = (n * sizeof(X) + 255) & ~size_t(255);
    void* p = nullptr;
    if (bytes > kSlab / 4) {
      if (pool_alloc(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        err = 1;
        return nullptr;
      }
      ptrs.push_back(p);
      return static_cast<X*>(p);
    }
    if (bytes > left) {
      if (pool_alloc(&p, kSlab, st) != cudaSuccess) {
        cudaGetLastError();
        err = 1;
        return nullptr;
      }
      ptrs.push_back(p);
      cur = static_cast<char*>(p);
      left = kSlab;
    }
    X* r = reinterpret_cast<X*>(cur);
    cur += bytes;
    left -= bytes;
    return r;
  }
  template <typename X>
  X* upload(const std::vector<X>& h) {
    X* d = alloc<X>(h.size());
    if (!d || h.empty()) return d;
    const size_t bytes = h.size() * sizeof(X);
    const void* src = h.data();
    if (stage) {
      char* p = stage->get(bytes);
      if (p) {
        memcpy(p, h.data(), bytes);
        src = p;
      }
    }
    if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) err = 1;
    return d;
  }
  void free_all() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
    cur = nullptr;
    left = 0;
  }
};

struct HostPack {
  std::vector<unsigned char> buf;
  template <typename X>
  size_t add(const std::vector<X>& v) {
    const size_t off = (buf.size() + 255) & ~size_t(255);
    buf.resize(off + std::max<size_t>(v.size(), 1) * sizeof(X));
    if (!v.empty()) memcpy(buf.data() + off, v.data(), v.size() * sizeof(X));
    return off;
  }
};

// a: first array, b: second (and c: third) -- one device allocation, one copy
template <typename A, typename B>
static void upload2(DevMem& m, const std::vector<A>& a, const std::vector<B>& b, A*& da, B*& db) {
  HostPack hp;
  const size_t oa = hp.add(a), ob = hp.add(b);
  unsigned char* d = m.upload(hp.buf);
  da = d ? reinterpret_cast<A*>(d + oa) : nullptr;
  db = d ? reinterpret_cast<B*>(d + ob) : nullptr;
}
template <typename A, typename B, typename C>
static void upload3(DevMem& m, const std::vector<A>& a, const std::vector<B>& b, const std::vector<C>& c, A*& da,
                    B*& db, C*& dc) {
  HostPack hp;
  const size_t oa = hp.add(a), ob = hp.add(b), oc = hp.add(c);
  unsigned char* d = m.upload(hp.buf);
  da = d ? reinterpret_cast<A*>(d + oa) : nullptr;
  db = d ? reinterpret_cast<B*>(d + ob) : nullptr;
  dc = d ? reinterpret_cast<C*>(d + oc) : nullptr;
}

// ------------------------------------------------------------------ launch helpers
// FP32 products: the tcgen05 kernel (128 x 64 tiles, tensor-memory accumulator)
// or the mma.sync kernel (64 x 64 tiles).  SPAND_GEMM=umma / mma forces one;
// by default an online tuner picks per class of launch (below).
static int gemm_mode() {   // 0: tuned, 1: tcgen05, 2: mma.sync
  static const int m = [] {
    const char* v = std::getenv("SPAND_GEMM");
    if (v && std::strcmp(v, "mma") == 0) return 2;
    if (v && (std::strcmp(v, "umma") == 0 || std::strcmp(v, "umma2") == 0 || std::strcmp(v, "umma3") == 0))
      return 1;
    return 0;
  }();
  return m;
}

// which tcgen05 kernel: 1 = the register-staged 128 x 64 one (default),
// 2 = the cp.async-pipelined 128 x 128 one (SPAND_GEMM=umma2; measured about 2x
// slower on the leaf-level elimination products, kept for measurement),
// 3 = the warp-specialised 128 x 64 one (SPAND_GEMM=umma3)
static int umma_variant() {
  static const int v = [] {
    const char* e = std::getenv("SPAND_GEMM");
    if (e && std::strcmp(e, "umma2") == 0) return 2;
    if (e && std::strcmp(e, "umma3") == 0) return 3;
    return 1;
  }();
  return v;
}

// register sets of operand prefetch in k_gemm_umma (SPAND_GEMM_DEPTH=1 or 2)
static int umma_depth() {
  static const int d = [] {
    const char* e = std::getenv("SPAND_GEMM_DEPTH");
    return (e && e[0] == '2') ? 2 : 1;
  }();
  return d;
}

// Online tuner for the choice of GEMM kernel (and with it the tile shape).
// Launches are grouped by device, the average number of 32-wide k-chunks per
// product (log2 bucket) and the logical flop count (log2 bucket).  The first
// launches of a class run each candidate once between two events; once both
// timings have completed (checked without waiting, at a later launch of the
// class) the candidate with the lower time per flop is used for the class for
// the rest of the process.  Until then -- and whenever a measurement is still
// in flight -- the rule "tcgen05 from four k-chunks per product on" decides.
// Either kernel computes the same products; only FP32 rounding order differs.
struct GemmTuner {
  struct Entry {
    int choice = -1;                 // decided: 0 tcgen05, 1 mma.sync
    bool pending[2] = {false, false};
    bool done[2] = {false, false};
    double per_flop[2] = {0, 0};
    double flops[2] = {0, 0};
    cudaEvent_t ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  };
  std::mutex mu;
  std::map<std::tuple<int, int, int>, Entry> table;
  static GemmTuner& get() {
    static GemmTuner* t = new GemmTuner();   // process lifetime
    return *t;
  }
};

// returns the kernel (0 tcgen05, 1 mma.sync) and, when this launch is to be
// timed, the two events to record around it
static int gemm_pick(double avg_chunks, double flops, cudaEvent_t& e0, cudaEvent_t& e1) {
  e0 = e1 = nullptr;
  const int rule = avg_chunks >= 4.0 ? 0 : 1;
  if (gemm_mode() == 1) return 0;
  if (gemm_mode() == 2) return 1;
  int dev = 0;
  cudaGetDevice(&dev);
  const int cb = std::min(6, (int)std::floor(std::log2(std::max(1.0, avg_chunks))));
  const int fb = std::min(12, (int)std::floor(std::log2(std::max(1.0, flops / 1e7))));
  GemmTuner& T = GemmTuner::get();
  std::lock_guard<std::mutex> g(T.mu);
  GemmTuner::Entry& E = T.table[std::make_tuple(dev, cb, fb)];
  if (E.choice >= 0) return E.choice;
  for (int c = 0; c < 2; ++c)
    if (E.pending[c] && !E.done[c]) {
      const cudaError_t q = cudaEventQuery(E.ev[c][1]);
      if (q == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, E.ev[c][0], E.ev[c][1]) == cudaSuccess && E.flops[c] > 0) {
          E.per_flop[c] = ms / E.flops[c];
          E.done[c] = true;
        }
        E.pending[c] = false;
      } else if (q == cudaErrorNotReady && cudaPeekAtLastError() == cudaErrorNotReady) {
        cudaGetLastError();          // a not-ready query is not an error of ours
      }
    }
  if (E.done[0] && E.done[1]) {
    E.choice = E.per_flop[0] <= E.per_flop[1] ? 0 : 1;
    for (auto& pr : E.ev)
      for (auto& e : pr)
        if (e) cudaEventDestroy(e);
    static const bool dbg = [] {
      const char* v = std::getenv("SPAND_DEBUG");
      return v && v[0] == '1';
    }();
    if (dbg)
      std::fprintf(stderr, "spand: GEMM class (k-chunks 2^%d, flops 2^%d x 1e7): tcgen05 %.3g, mma.sync %.3g ms/GF -> %s\n",
                   cb, fb, E.per_flop[0] * 1e9, E.per_flop[1] * 1e9, E.choice == 0 ? "tcgen05" : "mma.sync");
    return E.choice;
  }
  for (int c = 0; c < 2; ++c)
    if (!E.done[c] && !E.pending[c]) {
      if (!E.ev[c][0]) {
        if (cudaEventCreate(&E.ev[c][0]) != cudaSuccess || cudaEventCreate(&E.ev[c][1]) != cudaSuccess) {
          cudaGetLastError();
          return rule;
        }
      }
      E.pending[c] = true;
      E.flops[c] = flops;
      e0 = E.ev[c][0];
      e1 = E.ev[c][1];
      return c;
    }
  return rule;                       // both measurements still in flight
}

// SPAND_DEBUG=3: CUDA-event time, logical flops and kernel of every grouped
// GEMM launch, summed per purpose (tag) and printed when the factorization ends;
// SPAND_DEBUG=4 also prints every launch in order (index among the launches of
// its kernel, tag, tiles, time)
struct GemmLog {
  struct Rec {
    const char* tag;
    int kind;                // 0 tcgen05, 1 mma.sync, 2 FP64
    double flops;
    size_t tiles;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  static GemmLog& get() {
    static GemmLog* g = new GemmLog();
    return *g;
  }
  void print_and_clear() {
    std::map<std::string, std::array<double, 4>> agg;   // ms, flops, launches, tiles
    int nk[3] = {0, 0, 0};
    for (auto& r : recs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) cudaGetLastError();
      if (debug_level() >= 4)
        std::fprintf(stderr, "spand: GEMM launch %s #%d %-14s %8zu tiles %9.3f ms %7.1f TFLOP/s\n",
                     r.kind == 0 ? "tcgen05" : r.kind == 1 ? "mma.sync" : "fp64", nk[r.kind]++, r.tag, r.tiles, ms,
                     ms > 0 ? r.flops / (ms * 1e9) : 0.0);
      auto& a = agg[std::string(r.tag) + (r.kind == 0 ? " tcgen05" : r.kind == 1 ? " mma.sync" : " fp64")];
      a[0] += ms;
      a[1] += r.flops;
      a[2] += 1;
      a[3] += (double)r.tiles;
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    recs.clear();
    for (auto& kv : agg)
      std::fprintf(stderr, "spand: GEMM %-22s %8.2f ms %10.3g flops %6.0f launches %10.0f tiles %7.1f TFLOP/s\n",
                   kv.first.c_str(), kv.second[0], kv.second[1], kv.second[2], kv.second[3],
                   kv.second[0] > 0 ? kv.second[1] / (kv.second[0] * 1e9) : 0.0);
  }
};

template <typename T>
static void launch_gemm(DevMem& tmp, const std::vector<GemmTask<T>>& tasks, const std::vector<GemmTerm<T>>& terms,
                        cudaStream_t st, const char* tag = "") {
  bool umma = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (std::is_same<T, float>::value) {
    double chunks = 0, flops = 0;
    int ntask = 0;
    for (const auto& tk : tasks) {
      if (tk.m <= 0 || tk.n <= 0) continue;
      for (int t = tk.t0; t < tk.t1; ++t) {
        chunks += (terms[t].k + UM_BK - 1) / UM_BK;
        flops += 2.0 * tk.m * (double)tk.n * terms[t].k;
      }
      ++ntask;
    }
    if (ntask > 0) umma = gemm_pick(chunks / ntask, flops, e0, e1) == 0;
  }
  const int uv = umma_variant();
  const int BM = umma ? (uv == 2 ? U2_BM : UM_BM) : 64, BN = umma ? (uv == 2 ? U2_BN : UM_BN) : 64;
  std::vector<TileItem> tiles;
  for (int t = 0; t < (int)tasks.size(); ++t) {
    if (tasks[t].m <= 0 || tasks[t].n <= 0) continue;
    for (int a = 0; a < (tasks[t].m + BM - 1) / BM; ++a)
      for (int b = 0; b < (tasks[t].n + BN - 1) / BN; ++b) tiles.push_back({t, a, b});
  }
  if (tiles.empty()) return;
  GemmTask<T>* dt;
  GemmTerm<T>* dm;
  TileItem* dl;
  upload3(tmp, tasks, terms, tiles, dt, dm, dl);
  if (tmp.err) return;
  note_launch();
  GemmLog::Rec rec{tag, std::is_same<T, float>::value ? (umma ? 0 : 1) : 2, 0.0, tiles.size(), nullptr, nullptr};
  const bool logit = debug_level() >= 3 && cudaEventCreate(&rec.a) == cudaSuccess &&
                     cudaEventCreate(&rec.b) == cudaSuccess && cudaEventRecord(rec.a, st) == cudaSuccess;
  if (logit)
    for (const auto& tk : tasks)
      for (int t = tk.t0; t < tk.t1; ++t)   // a triangular operand halves the useful flops
        rec.flops += (terms[t].tri ? 1.0 : 2.0) * tk.m * (double)tk.n * terms[t].k;
  struct LogAtEnd {
    bool on;
    GemmLog::Rec& r;
    cudaStream_t s;
    ~LogAtEnd() {
      if (on && cudaEventRecord(r.b, s) == cudaSuccess) GemmLog::get().recs.push_back(r);
    }
  } log_at_end{logit, rec, st};
  if constexpr (std::is_same<T, float>::value) {
    if (e0) cudaEventRecord(e0, st);
    if (umma && uv == 1 && umma_depth() == 2) {
      static std::atomic<uint64_t> attr{0};
      once_per_device(attr, [] { set_dyn_smem((const void*)k_gemm_umma<2>, UM_SMEM_BYTES); });
      k_gemm_umma<2><<<(unsigned)tiles.size(), 128, UM_SMEM_BYTES, st>>>(dt, dm, dl);
    } else if (umma && uv == 1) {
      static std::atomic<uint64_t> attr1{0};
      once_per_device(attr1, [] { set_dyn_smem((const void*)k_gemm_umma<1>, UM_SMEM_BYTES); });
      k_gemm_umma<1><<<(unsigned)tiles.size(), 128, UM_SMEM_BYTES, st>>>(dt, dm, dl);
    } else if (umma && uv == 3) {
      static std::atomic<uint64_t> attr3{0};
      once_per_device(attr3, [] { set_dyn_smem((const void*)k_gemm_umma3, U3_SMEM_BYTES); });
      k_gemm_umma3<<<(unsigned)tiles.size(), U3_THREADS, U3_SMEM_BYTES, st>>>(dt, dm, dl);
    } else if (umma) {
      static std::atomic<uint64_t> attr2{0};
      once_per_device(attr2, [] { set_dyn_smem((const void*)k_gemm_umma2, U2_SMEM_BYTES); });
      k_gemm_umma2<<<(unsigned)tiles.size(), 128, U2_SMEM_BYTES, st>>>(dt, dm, dl);
    } else {
      k_gemm_tc<3><<<(unsigned)tiles.size(), 128, 0, st>>>(dt, dm, dl);   // 3xTF32 on mma.sync
    }
    if (e1) cudaEventRecord(e1, st);
  } else {
    k_gemm<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dt, dm, dl);
  }
}

template <typename T>
static void launch_copy(DevMem& tmp, const std::vector<CopyTask<T>>& tasks, cudaStream_t st) {
  std::vector<CopyTile> tiles;
  for (int t = 0; t < (int)tasks.size(); ++t)
    for (int a = 0; a < (tasks[t].rows + 31) / 32; ++a)
      for (int b = 0; b < (tasks[t].cols + 31) / 32; ++b) tiles.push_back({t, a, b});
  if (tiles.empty()) return;
  CopyTask<T>* dt;
  CopyTile* dl;
  upload2(tmp, tasks, tiles, dt, dl);
  if (tmp.err) return;
  note_launch();
  k_copy_tiles<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dt, dl);
}

// row-permuted copy: dst[r, c] = src[perm[r], c]; one CTA per 64 x 32 tile
// (rows x columns) of a task, a warp per column pair, lanes over rows
struct RowPermTask {
  const void* src;
  void* dst;
  const int* perm;
  int rows, cols;
};
struct RowPermTile {
  int task, r0, c0;
};

template <typename T>
__global__ void __launch_bounds__(256) k_row_perm(const RowPermTask* tasks, const RowPermTile* tiles) {
  const RowPermTile tl = tiles[blockIdx.x];
  const RowPermTask tk = tasks[tl.task];
  const T* s = static_cast<const T*>(tk.src);
  T* d = static_cast<T*>(tk.dst);
  const int n = tk.rows;
  // 8 elements per thread, all loaded before any store so the loads overlap
  const int r = tl.r0 + (threadIdx.x & 63), cq = tl.c0 + (threadIdx.x >> 6);
  if (r >= n) return;
  const int pr = tk.perm[r];
  T v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int c = cq + 4 * e;
    v[e] = (c < tk.cols) ? s[pr + (size_t)c * n] : T(0);
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int c = cq + 4 * e;
    if (c < tk.cols) d[r + (size_t)c * n] = v[e];
  }
}

template <typename T>
static void launch_row_perm(DevMem& tmp, const std::vector<const T*>& src, const std::vector<T*>& dst,
                            const std::vector<const int*>& perm, const std::vector<int>& rows,
                            const std::vector<int>& cols, cudaStream_t st) {
  if (src.empty()) return;
  std::vector<RowPermTask> tasks(src.size());
  std::vector<RowPermTile> tiles;
  for (size_t t = 0; t < src.size(); ++t) {
    tasks[t] = {src[t], dst[t], perm[t], rows[t], cols[t]};
    for (int r0 = 0; r0 < rows[t]; r0 += 64)
      for (int c0 = 0; c0 < cols[t]; c0 += 32) tiles.push_back({(int)t, r0, c0});
  }
  if (tiles.empty()) return;
  RowPermTask* dt;
  RowPermTile* dl;
  upload2(tmp, tasks, tiles, dt, dl);
  if (tmp.err) return;
  note_launch();
  k_row_perm<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dt, dl);
}

// ------------------------------------------------------------------ streaming RRQR launch
// SPAND_QR_STREAM=1 sends every interface with neighbours to the streaming
// kernel (a checking aid: the same factorization by the other code path);
// SPAND_QR_STREAM=0 never uses it.
static int stream_forced() {
  static const int m = [] {
    const char* v = std::getenv("SPAND_QR_STREAM");
    if (v && v[0] == '1') return 1;
    if (v && v[0] == '0') return -1;
    return 0;
  }();
  return m;
}

// SPAND_FAULT_GROUP_BARRIER=1: the first streaming RRQR launch of the process
// tells one group that it has one CTA more than is launched and shortens the
// barrier's poll limit to about a millisecond, so that the group's first
// barrier wait runs out; the factorization must then return SPAND_ERR_CUDA and
// leave the context usable.  A test of the bounded wait; one launch only.
static bool take_barrier_fault() {
  static const bool on = [] {
    const char* v = std::getenv("SPAND_FAULT_GROUP_BARRIER");
    return v && v[0] == '1';
  }();
  static std::atomic<int> used{0};
  return on && used.exchange(1) == 0;
}

// leading dimension of a column-major W: n rounded up to 16 bytes
template <typename T>
static int qrs_ldw(int n) {
  constexpr int vw = 16 / sizeof(T);
  return (n + vw - 1) / vw * vw;
}

// CTAs of the streaming kernel resident at once (one per SM)
template <typename T>
static int qrs_capacity() {
  int dev = 0, nsm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return coop ? std::min(nsm, QR_GMAX) : 0;
}

// register-resident rows of a column: 32 lanes x 16 bytes x NV
template <typename T>
static int qrs_pick_nv(int nmax) {
  constexpr int vw = 16 / sizeof(T);
  for (int nv : {4, 8}) if (nmax <= 32 * vw * nv) return nv;
  return 16;
}

// One cooperative launch of the streaming RRQR (one CTA per SM): the groups of
// desc first, then a queue of single-CTA interfaces drained by every CTA.
template <typename T, int NV>
static int launch_stream_once(DevMem& tmp, const QrStreamTask<T>* dt, size_t nt, const std::vector<QrStreamTask<T>>& tasks,
                              const std::vector<QrGroupDesc>& desc, const std::vector<int>& solo, int* d_flags, T eps,
                              cudaStream_t st) {
  auto kern = k_qrcp_stream<T, NV>;
  int dev = 0, nsm = 0, per_sm = 0;
  SPAND_CUDA_TRY(cudaGetDevice(&dev));
  SPAND_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int cap = std::min(nsm, QR_GMAX);
  size_t smem = 0;
  for (size_t d = 0; d < desc.size(); d += desc[d].G)
    smem = std::max(smem, qrcp_stream_smem<T>(tasks[desc[d].task].ldw, tasks[desc[d].task].c, desc[d].G));
  for (int i : solo) smem = std::max(smem, qrcp_stream_smem<T>(tasks[i].ldw, tasks[i].c, 1));
  if (debug_level() >= 2) {
    std::fprintf(stderr, "spand:   streaming launch: %zu group CTAs (", desc.size());
    for (size_t d = 0; d < desc.size(); d += desc[d].G)
      std::fprintf(stderr, " n%d c%d G%d", tasks[desc[d].task].n, tasks[desc[d].task].c, desc[d].G);
    std::fprintf(stderr, " ), %zu single-CTA interfaces\n", solo.size());
  }
  if (set_dyn_smem((const void*)kern, smem) < (long long)smem) return SPAND_ERR_UNSUPPORTED;
  SPAND_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, QRS_THREADS, smem));
  if (per_sm < 1 || (int)desc.size() > cap) return SPAND_ERR_UNSUPPORTED;
  QrGroupDesc* dd = desc.empty() ? nullptr : tmp.upload(desc);
  int* ds = solo.empty() ? nullptr : tmp.upload(solo);
  int* queue = tmp.alloc<int>(1);
  T* pv = tmp.alloc<T>(nt * 2 * QR_GMAX);
  int* pi = tmp.alloc<int>(nt * 2 * QR_GMAX);
  GroupSync* gs = tmp.alloc<GroupSync>(nt);
  unsigned long long* words = tmp.alloc<unsigned long long>(nt * 2 * QR_GMAX);
  if (tmp.err) return SPAND_ERR_NOMEM;
  SPAND_CUDA_TRY(cudaMemsetAsync(gs, 0, sizeof(GroupSync) * nt, st));
  SPAND_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), st));
  // every word starts with tag 255, which no word of steps 0 and 1 carries
  SPAND_CUDA_TRY(cudaMemsetAsync(words, 0xFF, sizeof(unsigned long long) * nt * 2 * QR_GMAX, st));
  int poll_log2 = 22, fault_task = -1;
  if (take_barrier_fault()) {
    fault_task = desc.empty() ? solo[0] : desc[0].task;   // a partner that never arrives
    poll_log2 = 14;
  }
  const int used = (int)desc.size();
  const int grid = std::max(1, std::min(cap, used + (int)solo.size()));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(QRS_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  SPAND_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, dt, (const QrGroupDesc*)dd, used, (const int*)ds, (int)solo.size(),
                                    queue, pv, pi, gs, words, d_flags, eps, poll_log2, fault_task));
  return SPAND_OK;
}

template <typename T>
static int launch_stream_nv(DevMem& tmp, const QrStreamTask<T>* dt, size_t nt, const std::vector<QrStreamTask<T>>& tasks,
                            const std::vector<QrGroupDesc>& desc, const std::vector<int>& solo, int* d_flags, T eps,
                            cudaStream_t st) {
  int nmax = 0;
  for (auto& d : desc) nmax = std::max(nmax, tasks[d.task].n);
  for (int i : solo) nmax = std::max(nmax, tasks[i].n);
  const int nv = qrs_pick_nv<T>(nmax);
  if (nv <= 4) return launch_stream_once<T, 4>(tmp, dt, nt, tasks, desc, solo, d_flags, eps, st);
  if (nv <= 8) return launch_stream_once<T, 8>(tmp, dt, nt, tasks, desc, solo, d_flags, eps, st);
  return launch_stream_once<T, 16>(tmp, dt, nt, tasks, desc, solo, d_flags, eps, st);
}

// The streaming RRQR of a level's interfaces.  Interfaces with more than twice
// a CTA's fair share of the work (estimated as n min(n, c) c: pivot steps x
// rows x columns) are the critical path: they run first, in groups that
// share every SM in proportion to their work; then every SM drains a queue of
// the remaining interfaces one CTA each, largest first.
template <typename T>
static int launch_qrcp_stream(DevMem& tmp, const std::vector<QrStreamTask<T>>& tasks, int* d_flags, T eps,
                              cudaStream_t st) {
  int dev = 0, nsm = 0;
  SPAND_CUDA_TRY(cudaGetDevice(&dev));
  SPAND_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int cap = std::min(nsm, QR_GMAX);
  const size_t nt = tasks.size();
  auto work = [&](int i) { return (double)tasks[i].n * std::min(tasks[i].n, tasks[i].c) * tasks[i].c; };
  double wsum = 0;
  for (size_t i = 0; i < nt; ++i) wsum += work((int)i);
  const double fair = wsum / cap;
  std::vector<int> order(nt);
  for (size_t i = 0; i < nt; ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  std::vector<int> big, solo;
  for (int i : order) {
    if (work(i) > 2.0 * fair && tasks[i].c >= 2 && (int)big.size() < cap / 2) big.push_back(i);
    else solo.push_back(i);
  }
  QrStreamTask<T>* dt = tmp.upload(tasks);
  if (tmp.err) return SPAND_ERR_NOMEM;
  if (!big.empty()) {
    // every SM over the large interfaces, in proportion to their work (>= 2 each)
    double wb = 0;
    for (int i : big) wb += work(i);
    std::vector<int> G(big.size(), 2);
    int left = cap - 2 * (int)big.size();
    for (size_t b = 0; b < big.size(); ++b) {
      const int extra = (int)std::floor((cap - 2.0 * big.size()) * work(big[b]) / wb);
      const int add = std::max(0, std::min({extra, left, QR_GMAX - 2, tasks[big[b]].c - 2}));
      G[b] += add;
      left -= add;
    }
    std::vector<QrGroupDesc> desc;
    for (size_t b = 0; b < big.size(); ++b)
      for (int g = 0; g < G[b]; ++g) desc.push_back({big[b], g, G[b], 0});
    SPAND_TRY(launch_stream_nv<T>(tmp, dt, nt, tasks, desc, std::vector<int>(), d_flags, eps, st));
  }
  if (!solo.empty()) SPAND_TRY(launch_stream_nv<T>(tmp, dt, nt, tasks, std::vector<QrGroupDesc>(), solo, d_flags, eps, st));
  return SPAND_OK;
}

// LU panel kernel choice: SPAND_LU_PANEL=smem never uses the cluster kernel,
// SPAND_LU_PANEL=cluster uses it for every panel taller than LU_CL_ROWS rows
// (a checking aid: the same factorization by the other code path)
static int lu_panel_mode() {   // 0: automatic, 1: smem, 2: cluster
  static const int m = [] {
    const char* v = std::getenv("SPAND_LU_PANEL");
    if (v && std::strcmp(v, "smem") == 0) return 1;
    if (v && std::strcmp(v, "cluster") == 0) return 2;
    return 0;
  }();
  return m;
}
constexpr int LU_CL_FEW = 48;    // fewer active matrices than this: clusters
constexpr int LU_CL_ROWS = 256;  // panel rows per cluster CTA aimed at

// blocked getrf of every matrix, in place; pivots + permutations
template <typename T>
static void batched_getrf(DevMem& tmp, std::vector<MatRef<T>>& mats, int* d_flags, cudaStream_t st) {
  if (mats.empty()) return;
  int nmax = 0;
  for (auto& m : mats) nmax = std::max(nmax, m.n);
  auto* dm = tmp.upload(mats);
  if (tmp.err) return;
  // a panel whose rows fit the shared-memory budget takes the staged kernel,
  // decided panel by panel (a tall matrix moves to it once its panels shrink);
  // the staged kernel's interchange records need one slot per matrix
  int* aff = tmp.alloc<int>(mats.size() * (1 + 4 * LU_NB));
  if (tmp.err) return;
  int* aff_cl = tmp.alloc<int>(mats.size() * (1 + 4 * LU_NB));
  if (tmp.err) return;
  static std::atomic<uint64_t> attr{0};
  once_per_device(attr, [] {
    set_dyn_smem((const void*)k_getrf_panel_smem<T>, LU_SMEM_BYTES);
    set_dyn_smem((const void*)k_getrf_panel_cl<T>, LU_SMEM_BYTES);
    set_dyn_smem((const void*)k_ipiv_to_perm<T>, 200 * 1024);
  });
  // the panel's row interchanges and U12 on the columns outside it, 32 columns
  // per CTA, for the matrices of one panel launch (their records in aff order)
  auto swap_trsm = [&](const std::vector<MatRef<T>>& list, const MatRef<T>* dlist, int k0, int tcol) {
    std::vector<LuColTile> tl;
    for (int b = 0; b < (int)list.size(); ++b) {
      const int nb = list[b].n;
      if (k0 >= nb) continue;
      const int outside = nb - std::min(LU_NB, nb - k0);
      for (int c0 = 0; c0 < outside; c0 += 32) tl.push_back({b, c0});
    }
    if (tl.empty()) return;
    auto* dtl = tmp.upload(tl);
    if (tmp.err) return;
    note_launch();
    k_getrf_swap_trsm<T><<<(unsigned)tl.size(), 256, 0, st>>>(dlist, dtl, k0, tcol);
  };
  // Two-level blocking (the arrangement of LAPACK's blocked getrf): panels of
  // LU_NB columns are grouped in blocks of LU_NB2.  Inside a block a panel's
  // row interchanges reach every column, but its TRSM and its rank-LU_NB
  // update touch only the block's own columns; the columns right of the block
  // stay un-updated (so interchanging their rows is consistent).  When the
  // block is done, their rows K0..Ke-1 become U12 (staged TRSM, one panel's
  // rows at a time) and the rest takes one rank-(Ke-K0) update.
  for (int k0 = 0; k0 < nmax; k0 += LU_NB) {
    const int K0 = k0 / LU_NB2 * LU_NB2;
    const int tcol = K0 + LU_NB2;            // TRSM / updates inside the block only
    // panel kernels: one CTA per matrix with the panel in shared memory when
    // there are enough matrices to fill the GPU and the panel fits; a cluster
    // of C CTAs per matrix (the panel's rows spread over their shared memory)
    // when the matrices are few or the panel is too tall for one CTA; the
    // global-memory kernel beyond the clusters' capacity
    int nact = 0;
    for (auto& m : mats) nact += k0 < m.n;
    std::vector<MatRef<T>> small, large;
    std::vector<std::vector<MatRef<T>>> clus(3);    // by cluster size 2 << q: 2, 4, 8
    int nsmall_max = 0;
    std::array<int, 3> ncl_max{0, 0, 0};
    for (auto m : mats) {
      if (k0 >= m.n) continue;
      const int rows = m.n - k0;
      const bool fits1 = (size_t)rows * LU_NB * sizeof(T) <= (size_t)LU_SMEM_BYTES;
      int q = -1;
      if (lu_panel_mode() != 1 && (!fits1 || nact < LU_CL_FEW || lu_panel_mode() == 2) && rows > LU_CL_ROWS) {
        for (q = 0; q < 3; ++q) {                    // smallest portable cluster with <= LU_CL_ROWS rows per CTA
          const int C = 2 << q;
          if ((rows + C - 1) / C <= LU_CL_ROWS) break;
        }
        if (q == 3) q = 2;                           // 8 CTAs, more rows each
        const int C = 2 << q;
        if (lu_cl_smem<T>((rows + C - 1) / C) > (size_t)LU_SMEM_BYTES) q = -1;
      }
      if (q >= 0) {
        m.aff = aff_cl;
        clus[q].push_back(m);
        ncl_max[q] = std::max(ncl_max[q], rows);
      } else if (fits1) {
        m.aff = aff;
        small.push_back(m);
        nsmall_max = std::max(nsmall_max, m.n);
      } else {
        large.push_back(m);
      }
    }
    auto* ds = small.empty() ? nullptr : tmp.upload(small);
    auto* dlg = large.empty() ? nullptr : tmp.upload(large);
    if (tmp.err) return;
    if (ds) {
      const size_t sm = (size_t)(nsmall_max - k0) * std::min(LU_NB, nsmall_max - k0) * sizeof(T);
      note_launch();
      k_getrf_panel_smem<T><<<(unsigned)small.size(), 512, sm, st>>>(ds, (int)small.size(), k0, d_flags);
      swap_trsm(small, ds, k0, tcol);
    }
    for (int q = 0; q < 3; ++q) {
      if (clus[q].empty()) continue;
      const int C = 2 << q;
      auto* dc = tmp.upload(clus[q]);
      if (tmp.err) return;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(clus[q].size() * C), 1, 1);
      cfg.blockDim = dim3(512, 1, 1);
      cfg.dynamicSmemBytes = lu_cl_smem<T>((ncl_max[q] + C - 1) / C);
      cfg.stream = st;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      note_launch();
      if (cudaLaunchKernelEx(&cfg, k_getrf_panel_cl<T>, (const MatRef<T>*)dc, (int)clus[q].size(), k0, d_flags) !=
          cudaSuccess) {
        tmp.err = 1;
        return;
      }
      swap_trsm(clus[q], dc, k0, tcol);
    }
    if (dlg) {
      note_launch();
      k_getrf_panel<T><<<(unsigned)large.size(), 256, 0, st>>>(dlg, (int)large.size(), k0, tcol, d_flags);
    }
    // rank-LU_NB update of the block's columns [r, Ke), every row below the panel
    std::vector<GemmTask<T>> tasks;
    std::vector<GemmTerm<T>> terms;
    bool block_end = false;
    for (auto& m : mats) {
      const int n = m.n;
      if (k0 + LU_NB >= n) continue;
      const int jb = LU_NB, r = k0 + jb, Ke = std::min(tcol, n);
      if (Ke > r) {
        terms.push_back({m.A + r + (size_t)k0 * n, m.A + k0 + (size_t)r * n, n, n, jb, 0, 0, 0});
        tasks.push_back({m.A + r + (size_t)r * n, n, n - r, Ke - r, (T)-1, (T)1, (int)terms.size() - 1,
                         (int)terms.size()});
      } else if (n > Ke) {
        block_end = true;
      }
    }
    launch_gemm(tmp, tasks, terms, st, "lu-trailing");
    if (!block_end) continue;
    // the block [K0, Ke) is done: rows K0..Ke-1 of the columns right of it,
    // one panel's rows at a time (TRSM, then the rank-LU_NB update of the
    // block rows below), then everything right of and below the block
    for (int p0 = K0; p0 < tcol; p0 += LU_NB) {
      std::vector<LuColTile> tl;
      std::vector<MatRef<T>> sub;
      std::vector<GemmTask<T>> rt;
      std::vector<GemmTerm<T>> rm;
      for (auto& m : mats) {
        const int n = m.n;
        if (n <= tcol || p0 >= n) continue;  // only matrices whose block ended here with columns right of it
        const int b = (int)sub.size();
        sub.push_back(m);
        for (int c0 = tcol; c0 < n; c0 += 32) tl.push_back({b, c0});
        const int r = p0 + LU_NB;
        if (r < tcol) {
          rm.push_back({m.A + r + (size_t)p0 * n, m.A + p0 + (size_t)tcol * n, n, n, LU_NB, 0, 0, 0});
          rt.push_back({m.A + r + (size_t)tcol * n, n, tcol - r, n - tcol, (T)-1, (T)1, (int)rm.size() - 1,
                        (int)rm.size()});
        }
      }
      if (tl.empty()) break;
      auto* dsub = tmp.upload(sub);
      auto* dtl = tmp.upload(tl);
      if (tmp.err) return;
      note_launch();
      k_lu_trsm_cols<T><<<(unsigned)tl.size(), 256, 0, st>>>(dsub, dtl, p0);
      launch_gemm(tmp, rt, rm, st, "lu-block-rows");
    }
    std::vector<GemmTask<T>> bt;
    std::vector<GemmTerm<T>> bm;
    for (auto& m : mats) {
      const int n = m.n;
      if (n <= tcol) continue;
      bm.push_back({m.A + tcol + (size_t)K0 * n, m.A + K0 + (size_t)tcol * n, n, n, tcol - K0, 0, 0, 0});
      bt.push_back({m.A + tcol + (size_t)tcol * n, n, n - tcol, n - tcol, (T)-1, (T)1, (int)bm.size() - 1,
                    (int)bm.size()});
    }
    launch_gemm(tmp, bt, bm, st, "lu-block");
  }
  note_launch();
  k_ipiv_to_perm<T><<<(unsigned)mats.size(), 128, (size_t)nmax * sizeof(int), st>>>(dm, (int)mats.size());
}

// L^-1 (optionally row-scaled by 1/d) and U^-1 (optionally column-scaled by d)
// by a bottom-up block recursion on the grouped GEMM: invert the 32 x 32
// diagonal blocks, then for block sizes 32, 64, 128, ... combine neighbouring
// blocks,  X21 = -X22 (L21 X11)  and  Y12 = -Y11 (U12 Y22).
template <typename T>
static void batched_inverses(DevMem& tmp, const std::vector<MatRef<T>>& mats, const std::vector<T*>& Linv,
                             const std::vector<T*>& Uinv, const std::vector<const T*>& dscale, cudaStream_t st) {
  if (mats.empty()) return;
  // zero both outputs (the opposite triangles must read as zeros)
  {
    std::vector<T*> ptr;
    std::vector<int> nn;
    for (size_t b = 0; b < mats.size(); ++b) {
      ptr.push_back(Linv[b]);
      nn.push_back(mats[b].n);
      ptr.push_back(Uinv[b]);
      nn.push_back(mats[b].n);
    }
    auto* dp = tmp.upload(ptr);
    auto* dn = tmp.upload(nn);
    if (tmp.err) return;
    for (size_t off = 0; off < ptr.size(); off += 65535) {
      const unsigned cnt = (unsigned)std::min<size_t>(65535, ptr.size() - off);
      note_launch();
      k_zero_mats<T><<<dim3(32, cnt), 256, 0, st>>>(dp + off, dn + off);
    }
  }
  std::vector<DiagInvTask<T>> dt;
  int nmax = 0;
  for (size_t b = 0; b < mats.size(); ++b) {
    const int n = mats[b].n;
    nmax = std::max(nmax, n);
    for (int p = 0; 32 * p < n; ++p) {
      dt.push_back({mats[b].A, Linv[b], n, p, 1});
      dt.push_back({mats[b].A, Uinv[b], n, p, 0});
    }
  }
  if (!dt.empty()) {
    auto* dd = tmp.upload(dt);
    if (tmp.err) return;
    note_launch();
    k_inv_diag<T><<<(unsigned)dt.size(), 32, 0, st>>>(dd);
  }
  for (int bs = 32; bs < nmax; bs *= 2) {
    // one scratch array per level for the products L21 X11 and U12 Y22
    size_t wtot = 0;
    for (size_t b = 0; b < mats.size(); ++b)
      for (int a0 = 0; a0 + bs < mats[b].n; a0 += 2 * bs) wtot += 2 * (size_t)bs * std::min(bs, mats[b].n - a0 - bs);
    if (wtot == 0) continue;
    T* W = tmp.alloc<T>(wtot);
    if (tmp.err) return;
    size_t woff = 0;
    std::vector<GemmTask<T>> t1, t2;
    std::vector<GemmTerm<T>> m1, m2;
    for (size_t b = 0; b < mats.size(); ++b) {
      const int n = mats[b].n;
      const T* LU = mats[b].A;
      for (int a0 = 0; a0 + bs < n; a0 += 2 * bs) {
        const int c0 = a0 + bs, na = bs, nc = std::min(bs, n - c0);
        // lower: X21 (nc x na) = -X22 (L21 X11)
        T* W1 = W + woff;
        woff += (size_t)nc * na;
        m1.push_back({LU + c0 + (size_t)a0 * n, Linv[b] + a0 + (size_t)a0 * n, n, n, na, 0, 0, 0});
        t1.push_back({W1, nc, nc, na, (T)1, (T)0, (int)m1.size() - 1, (int)m1.size()});
        m2.push_back({Linv[b] + c0 + (size_t)c0 * n, W1, n, nc, nc, 0, 0, 1});   // X22 lower
        t2.push_back({Linv[b] + c0 + (size_t)a0 * n, n, nc, na, (T)-1, (T)0, (int)m2.size() - 1, (int)m2.size()});
        // upper: Y12 (na x nc) = -Y11 (U12 Y22)
        T* W2 = W + woff;
        woff += (size_t)na * nc;
        m1.push_back({LU + a0 + (size_t)c0 * n, Uinv[b] + c0 + (size_t)c0 * n, n, n, nc, 0, 0, 2});   // Y22 upper
        t1.push_back({W2, na, na, nc, (T)1, (T)0, (int)m1.size() - 1, (int)m1.size()});
        m2.push_back({Uinv[b] + a0 + (size_t)a0 * n, W2, n, na, na, 0, 0, 0});
        t2.push_back({Uinv[b] + a0 + (size_t)c0 * n, n, na, nc, (T)-1, (T)0, (int)m2.size() - 1, (int)m2.size()});
      }
    }
    launch_gemm(tmp, t1, m1, st, "tri-inverse");
    launch_gemm(tmp, t2, m2, st, "tri-inverse");
  }
  // scalings of the interface form: SL = diag(1/d) L^-1, SU = U^-1 diag(d)
  std::vector<InvTask<T>> lt, ut;
  std::vector<InvTile> tiles;
  bool any = false;
  for (size_t b = 0; b < mats.size(); ++b) {
    lt.push_back({mats[b].A, Linv[b], nullptr, dscale[b], mats[b].n});
    ut.push_back({mats[b].A, Uinv[b], nullptr, dscale[b], mats[b].n});
    if (dscale[b]) any = true;
    for (int j0 = 0; j0 < mats[b].n; j0 += 32) tiles.push_back({(int)b, j0});
  }
  if (!any || tiles.empty()) return;
  auto* dlt = tmp.upload(lt);
  auto* dut = tmp.upload(ut);
  auto* dtl = tmp.upload(tiles);
  if (tmp.err) return;
  note_launch();
  k_scale_rows<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dlt, dtl);
  note_launch();
  k_scale_cols<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dut, dtl);
}

// U^-1 only (no permutation, no scaling)
template <typename T>
static void batched_upper_inverse(DevMem& tmp, const std::vector<MatRef<T>>& mats, const std::vector<T*>& Uinv,
                                  cudaStream_t st) {
  if (mats.empty()) return;
  std::vector<InvTask<T>> ut;
  std::vector<InvTile> tiles;
  for (size_t b = 0; b < mats.size(); ++b) {
    ut.push_back({mats[b].A, Uinv[b], nullptr, nullptr, mats[b].n});
    for (int j0 = 0; j0 < mats[b].n; j0 += 32) tiles.push_back({(int)b, j0});
  }
  auto* dut = tmp.upload(ut);
  auto* dtl = tmp.upload(tiles);
  if (tmp.err || tiles.empty()) return;
  note_launch();
  k_inv_upper<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dut, dtl);
}

// ------------------------------------------------------------------ factor object
template <typename T>
struct ApplyProg {
  struct Phase {
    GvTask<T>* tasks = nullptr;
    GvTerm<T>* terms = nullptr;
    GvTile* tiles = nullptr;
    int ntiles = 0;
    int kmax = 0;
  };
  std::vector<Phase> fwd, bwd;     // M^-1
  std::vector<Phase> tfwd, tbwd;   // M^-T
};

// apply of one system (or of every system) of a factorization: the unknowns
// [off, off + N) of the factor's slot space and the sweeps that touch them
template <typename T>
struct Program {
  ApplyProg<T> prog;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int off = 0, N = 0;
  int64_t bytes = 0;          // factor bytes one apply reads
  ~Program() {
    for (int t = 0; t < 2; ++t)
      if (graph[t]) cudaGraphExecDestroy(graph[t]);
  }
};

struct FactorBase {
  virtual ~FactorBase() {}
  int precision = 0;
  int N = 0, D = 0;
  spand_stats stats{};
  std::vector<spand_stats> sys_stats;   // per system of a batched factorization
  DevMem mem;               // persistent device memory
  virtual int apply(int prog, const double* r, double* z, int transpose, cudaStream_t st, bool direct) = 0;
  // sweeps only: the output stays in the factor's own vector (returned)
  virtual int apply_slot(int prog, const double* r, int transpose, cudaStream_t st, bool direct, const void** w,
                         int* w_is_float) = 0;
  virtual int prog_size(int prog) const = 0;
  virtual int64_t prog_bytes(int prog) const = 0;
};

template <typename T>
struct FactorT;
template <typename T>
int apply_impl(FactorT<T>* F, Program<T>& pg, const double* r, double* zout, int transpose, cudaStream_t st,
               bool direct);

template <typename T>
struct FactorT : FactorBase {
  T* w = nullptr;           // apply vectors (slot space)
  T* z = nullptr;
  T* park_b = nullptr;
  T* park_c = nullptr;
  // [0]: every system; [1 + q]: system q alone (batched factorizations)
  std::vector<std::unique_ptr<Program<T>>> progs;
  int apply(int prog, const double* r, double* zz, int transpose, cudaStream_t st, bool direct) override {
    return apply_impl<T>(this, *progs[prog], r, zz, transpose, st, direct);
  }
  int apply_slot(int prog, const double* r, int transpose, cudaStream_t st, bool direct, const void** wout,
                 int* w_is_float) override {
    *wout = w + progs[prog]->off;
    *w_is_float = std::is_same<T, float>::value ? 1 : 0;
    return apply_impl<T>(this, *progs[prog], r, nullptr, transpose, st, direct);
  }
  int prog_size(int prog) const override { return progs[prog]->N; }
  int64_t prog_bytes(int prog) const override { return progs[prog]->bytes; }
};

// host-side records of one level for building the apply program
template <typename T>
struct LevelRec {
  struct Interior {
    const T* Linv;
    const T* Uinv;
    const int* perm;       // device, n
    int c, n;
    std::vector<int> nbr;  // cluster ids
    std::vector<const T*> X, Y;
  };
  struct Iface {
    const T* SL;
    const T* SU;
    const T* Q;
    const int* perm;
    int c, n, r;
    bool sparsified;
    size_t park_b_off, park_c_off;
  };
  std::vector<Interior> in;
  std::vector<Iface> fa;
  std::vector<int*> d_slots;  // per cluster (device, current size at this level)
  std::vector<int*> d_pslots; // per interior: slots permuted by perm (device)
  std::vector<int> n;         // per cluster size
};

struct PermSlotTask {
  const int* slots;
  const int* perm;
  int* out;
  int n;
};

// out[i] = slots[perm[i]] for every task (one CTA per task)
__global__ void k_perm_slots(const PermSlotTask* tasks) {
  const PermSlotTask tk = tasks[blockIdx.x];
  for (int i = threadIdx.x; i < tk.n; i += blockDim.x) tk.out[i] = tk.slots[tk.perm[i]];
}

// Offsets of a level's cluster-pair blocks in its arena: keys a nc + b in
// ascending order, looked up by binary search (a sorted array is built and
// copied far faster than a node-based map of the same pairs).
struct BlockIndex {
  int nc = 0;
  std::vector<long long> keys;
  std::vector<unsigned long long> offs;
  size_t at(int a, int b) const {
    const long long k = (long long)a * nc + b;
    const auto it = std::lower_bound(keys.begin(), keys.end(), k);
    if (it == keys.end() || *it != k) throw std::out_of_range("cluster pair not in the level's block pattern");
    return (size_t)offs[it - keys.begin()];
  }
};

// The level-0 gather with the pattern checks on the device (no copy of the
// pattern to the host, no synchronisation): one CTA per BSR block k of one
// system; its row e by binary search of row_ptr, its target cluster pair by
// binary search of the arena's sorted pair keys (a nc + b).  A pattern the plan
// does not describe (row pointers out of range, a column outside the system,
// a pair absent from the level-0 pattern) sets flags[0] |= 32 and copies
// nothing for that block; the factorization then returns SPAND_ERR_ARG.
template <typename T>
__global__ void k_level0_gather_dev(const double* val, const int* rp, const int* col, int Kq, int nnzb, int e0,
                                    int B, const int* cl_of, const int* pos_in, const int* ncl,
                                    const long long* keys, const unsigned long long* offs, int npairs, int nc,
                                    T* arena, int* flags) {
  __shared__ unsigned long long s_off;
  __shared__ int s_ld, s_ok;
  const int k = blockIdx.x;
  if (k >= nnzb) return;
  if (threadIdx.x == 0) {
    int ok = rp[0] == 0 && rp[Kq] == nnzb;
    int lo = 0, hi = Kq;                      // the e with rp[e] <= k < rp[e + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (rp[mid] <= k) lo = mid;
      else hi = mid;
    }
    const int e = lo;
    ok = ok && rp[e] <= k && k < rp[e + 1];
    const int f = ok ? col[k] : 0;
    ok = ok && f >= 0 && f < Kq;
    unsigned long long off = 0;
    int ld = 0;
    if (ok) {
      const int a = cl_of[e0 + e], b = cl_of[e0 + f];
      const long long key = (long long)a * nc + b;
      int l2 = 0, h2 = npairs;
      while (l2 < h2) {
        const int m = (l2 + h2) >> 1;
        if (keys[m] < key) l2 = m + 1;
        else h2 = m;
      }
      ok = l2 < npairs && keys[l2] == key;
      if (ok) {
        ld = ncl[a];
        off = offs[l2] + (unsigned long long)pos_in[e0 + e] * B + (unsigned long long)pos_in[e0 + f] * B * ld;
      }
    }
    if (!ok) atomicOr(flags, 32);
    s_ok = ok;
    s_off = off;
    s_ld = ld;
  }
  __syncthreads();
  if (!s_ok) return;
  T* d = arena + s_off;
  const int ld = s_ld;
  const double* src = val + (size_t)k * B * B;
  for (int idx = threadIdx.x; idx < B * B; idx += blockDim.x) {
    const int r = idx % B, c = idx / B;
    d[r + (size_t)c * ld] = (T)src[idx];
  }
}

template <typename T>
static int factor_impl(const Plan& P, const bsr_matrix* const* As, double eps, int precision, FactorT<T>* F,
                       cudaStream_t st) {
  const int D = P.D;
  const int nsys = P.nsys;
  auto sysB = [&](int s) { return P.sys_B.empty() ? P.B : P.sys_B[s]; };
  auto sysE0 = [&](int s) { return P.sys_elem0.empty() ? 0 : P.sys_elem0[s]; };
  auto sysDof0 = [&](int s) -> int64_t { return P.sys_dof0.empty() ? 0 : P.sys_dof0[s]; };
  auto sysK = [&](int s) { return P.sys_K.empty() ? P.K : P.sys_K[s]; };
  const double t_begin = now_ms();
  double t_wait = 0;
  PinnedStage stage;
  struct StageGuard {
    DevMem* m;
    ~StageGuard() { m->stage = nullptr; }
  } stage_guard{&F->mem};
  F->mem.stage = &stage;
  double t_mark = t_begin;
  double ph_acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  auto mark = [&](int ph) {
    const double t = now_ms();
    ph_acc[ph] += t - t_mark;
    t_mark = t;
  };

  // SPAND_DEBUG=2: host time between named points of the level loop, summed
  // over levels and printed at the end (where the host, not the GPU, is busy)
  // (with the GPU time between the same points from events on the stream: a
  // segment whose GPU time is close to its host time kept the GPU waiting)
  std::map<std::string, double> host_ticks;
  std::vector<std::pair<const char*, cudaEvent_t>> tick_ev;
  std::vector<int> tick_lv;                 // level of each event (SPAND_DEBUG=3 prints per level)
  int tick_level = 0;
  double t_tick = t_begin;
  auto tick = [&](const char* what) {
    if (debug_level() < 2) return;
    const double t = now_ms();
    host_ticks[what] += t - t_tick;
    t_tick = t;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) == cudaSuccess && cudaEventRecord(e, st) == cudaSuccess) {
      tick_ev.push_back({what, e});
      tick_lv.push_back(tick_level);
    }
  };
  tick("start");
  auto sync_st = [&]() -> cudaError_t {
    const double t0 = now_ms();
    const cudaError_t e = cudaStreamSynchronize(st);
    t_wait += now_ms() - t0;
    if (e == cudaSuccess) stage.reset();    // every queued upload has been read
    return e;
  };
  F->N = (int)P.n_dof();
  F->D = D;
  F->precision = precision;
  F->mem.st = st;
  DevMem& pm = F->mem;
  spand_stats& S = F->stats;
  memset(&S, 0, sizeof(S));
  S.levels = D + 1;
  F->sys_stats.assign(nsys, spand_stats{});
  for (int q = 0; q < nsys; ++q) F->sys_stats[q].levels = (P.sys_D.empty() ? D : P.sys_D[q]) + 1;
  int* d_flags = pm.alloc<int>(4);
  if (pm.err) return SPAND_ERR_NOMEM;
  SPAND_CUDA_TRY(cudaMemsetAsync(d_flags, 0, 4 * sizeof(int), st));

  // ---- level-0 sizes, slots, blocks (a cluster never mixes systems)
  std::vector<int> cl_of, pos_in;
  level0_positions(P, cl_of, pos_in);
  std::vector<int> n(P.lv[0].cl.size());
  std::vector<std::vector<int>> slots(n.size());
  for (size_t c = 0; c < n.size(); ++c) {
    const int q = P.system_of(0, (int)c), Bq = sysB(q);
    n[c] = (int)P.lv[0].cl[c].elems.size() * Bq;
    for (int e : P.lv[0].cl[c].elems)
      for (int d = 0; d < Bq; ++d) slots[c].push_back((int)(sysDof0(q) + (int64_t)(e - sysE0(q)) * Bq + d));
  }
  tick("a0 level-0 positions and slots");
  // arena of the current level: blocks in pattern U after, in (a, b) order
  T* arena = nullptr;
  BlockIndex boff;
  auto layout = [&](const LevelInfo& L, const std::vector<int>& nn, DevMem& lm) -> int {
    const int nc = (int)nn.size();
    boff.nc = nc;
    boff.keys.clear();
    boff.keys.reserve(L.pattern.size() + L.after.size());
    for (auto& pr : L.pattern) boff.keys.push_back((long long)pr.first * nc + pr.second);
    for (auto& pr : L.after) boff.keys.push_back((long long)pr.first * nc + pr.second);
    std::sort(boff.keys.begin(), boff.keys.end());
    boff.keys.erase(std::unique(boff.keys.begin(), boff.keys.end()), boff.keys.end());
    boff.offs.resize(boff.keys.size());
    size_t tot = 0;
    for (size_t i = 0; i < boff.keys.size(); ++i) {
      boff.offs[i] = tot;
      tot += (size_t)nn[boff.keys[i] / nc] * nn[boff.keys[i] % nc];
    }
    arena = lm.alloc<T>(tot);
    if (lm.err) return SPAND_ERR_NOMEM;
    SPAND_CUDA_TRY(cudaMemsetAsync(arena, 0, std::max<size_t>(tot, 1) * sizeof(T), st));
    return SPAND_OK;
  };
  auto blk = [&](int a, int b) -> T* { return arena + boff.at(a, b); };

  DevMem lvmem;  // memory of the current level arena (freed after compression)
  lvmem.st = st;
  lvmem.stage = &stage;
  SPAND_TRY(layout(P.lv[0], n, lvmem));
  tick("a1 level-0 block layout");
  {
    // gather every system's BSR blocks into the level-0 cluster blocks (pattern
    // checked on the device, see k_level0_gather_dev)
    DevMem tmp;
    tmp.st = st;
    tmp.stage = &stage;
    const std::vector<long long>& keys = boff.keys;          // ascending a nc + b
    const int nc0 = (int)n.size();
    const long long* d_keys = tmp.upload(keys);
    const unsigned long long* d_offs = tmp.upload(boff.offs);
    const int* d_cl = tmp.upload(cl_of);
    const int* d_pos = tmp.upload(pos_in);
    const int* d_n = tmp.upload(n);
    if (tmp.err) return SPAND_ERR_NOMEM;
    for (int q = 0; q < nsys; ++q) {
      const bsr_matrix* A = As[q];
      if (A->nnzb == 0) continue;
      note_launch();
      k_level0_gather_dev<T><<<A->nnzb, 256, 0, st>>>(A->val, A->row_ptr, A->col, sysK(q), A->nnzb, sysE0(q),
                                                      sysB(q), d_cl, d_pos, d_n, d_keys, d_offs, (int)keys.size(),
                                                      nc0, arena, d_flags);
      SPAND_CUDA_TRY(cudaGetLastError());
    }
    tmp.free_all();
  }
  tick("a2 level-0 gather");

  // phase timers (events on the factorization stream): per level RRQR and
  // elimination-GEMM start/stop; read after each level's synchronisation
  struct Ev {
    cudaEvent_t a = nullptr, b = nullptr;
    bool used = false;
  };
  std::vector<Ev> ev_qr(D + 1), ev_gm(D + 1);
  auto ev_begin = [&](Ev& e) {
    if (!e.a) {
      cudaEventCreate(&e.a);
      cudaEventCreate(&e.b);
    }
    cudaEventRecord(e.a, st);
    e.used = true;
  };
  auto ev_end = [&](Ev& e) { cudaEventRecord(e.b, st); };
  auto ev_read = [&](Ev& e) -> double {
    float ms = 0.f;
    if (e.used && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) return ms;
    return 0.0;
  };
  struct EvGuard {
    std::vector<Ev>* v[2];
    ~EvGuard() {
      for (auto* p : v)
        for (auto& e : *p) {
          if (e.a) cudaEventDestroy(e.a);
          if (e.b) cudaEventDestroy(e.b);
        }
    }
  } ev_guard{{&ev_qr, &ev_gm}};
  // side streams for the RRQR launches of a level (one per cluster size), forked
  // from and joined back to the factorization's stream
  constexpr int kQrClasses = 5;                      // clusters of 1, 2, 4, 8, 16 CTAs
  struct SideGuard {
    cudaStream_t s[kQrClasses] = {};
    cudaEvent_t join[kQrClasses] = {};
    cudaEvent_t fork = nullptr;
    ~SideGuard() {
      for (int i = 0; i < kQrClasses; ++i) {
        if (s[i]) {
          cudaStreamSynchronize(s[i]);
          cudaStreamDestroy(s[i]);
        }
        if (join[i]) cudaEventDestroy(join[i]);
      }
      if (fork) cudaEventDestroy(fork);
    }
  } sides;
  for (int i = 0; i < kQrClasses; ++i) {
    SPAND_CUDA_TRY(cudaStreamCreateWithFlags(&sides.s[i], cudaStreamNonBlocking));
    SPAND_CUDA_TRY(cudaEventCreateWithFlags(&sides.join[i], cudaEventDisableTiming));
  }
  SPAND_CUDA_TRY(cudaEventCreateWithFlags(&sides.fork, cudaEventDisableTiming));
  std::vector<LevelRec<T>> recs(D + 1);
  size_t park_b_tot = 0, park_c_tot = 0;
  double flops = 0;

  for (int l = 0; l <= D; ++l) {
    const LevelInfo& L = P.lv[l];
    const int nc = (int)L.cl.size();
    LevelRec<T>& R = recs[l];
    R.n = n;
    R.d_slots.resize(nc);
    tick_level = l;
    tick("a3 level start");
    {
      // every cluster's slot list of the level in one upload
      std::vector<int> all;
      std::vector<size_t> off(nc + 1, 0);
      for (int c = 0; c < nc; ++c) off[c + 1] = off[c] + slots[c].size();
      all.reserve(off[nc]);
      for (int c = 0; c < nc; ++c) all.insert(all.end(), slots[c].begin(), slots[c].end());
      int* base = pm.upload(all);
      if (pm.err) return SPAND_ERR_NOMEM;
      for (int c = 0; c < nc; ++c) R.d_slots[c] = base + off[c];
    }
    tick("a4 slot upload");
    DevMem tmp;
    tmp.st = st;
    tmp.stage = &stage;
    // neighbour lists in the current pattern
    std::vector<std::vector<int>> nbr(nc);
    for (auto& pr : L.pattern)
      if (pr.first != pr.second) nbr[pr.first].push_back(pr.second);
    mark(0);
    tick_level = l;
    tick("a nbr lists (and level start)");
    // ================= 1. eliminate interiors (Eq. 10)
    std::vector<int> I;
    for (int c = 0; c < nc; ++c)
      if (L.cl[c].interior && n[c] > 0) I.push_back(c);
    if (!I.empty()) {
      std::vector<MatRef<T>> mats;
      std::vector<T*> Linv, Uinv;
      std::vector<const T*> nod;
      for (int c : I) {
        MatRef<T> m;
        m.A = blk(c, c);
        m.n = n[c];
        m.ipiv = tmp.alloc<int>(n[c]);
        m.perm = pm.alloc<int>(n[c]);
        mats.push_back(m);
        Linv.push_back(pm.alloc<T>((size_t)n[c] * n[c]));
        Uinv.push_back(pm.alloc<T>((size_t)n[c] * n[c]));
        nod.push_back(nullptr);
        flops += 2.0 / 3.0 * pow((double)n[c], 3);
      }
      if (tmp.err || pm.err) return SPAND_ERR_NOMEM;
      batched_getrf(tmp, mats, d_flags, st);
      batched_inverses(tmp, mats, Linv, Uinv, nod, st);
      // P^T A_sn (row permutation), then Y = L^-1 (P^T A_sn), X = A_ns U^-1
      std::vector<const T*> ps;
      std::vector<T*> pd;
      std::vector<const int*> pp;
      std::vector<int> pr_, pc_;
      std::vector<GemmTask<T>> tasks;
      std::vector<GemmTerm<T>> terms;
      std::map<std::pair<int, int>, T*> Xm, Ym;
      for (size_t q = 0; q < I.size(); ++q) {
        const int s = I[q];
        typename LevelRec<T>::Interior rec;
        rec.Linv = Linv[q];
        rec.Uinv = Uinv[q];
        rec.perm = mats[q].perm;
        rec.c = s;
        rec.n = n[s];
        for (int b : nbr[s]) {
          if (n[b] == 0) continue;
          T* Ap = tmp.alloc<T>((size_t)n[s] * n[b]);
          ps.push_back(blk(s, b));
          pd.push_back(Ap);
          pp.push_back(mats[q].perm);
          pr_.push_back(n[s]);
          pc_.push_back(n[b]);
          T* Y = pm.alloc<T>((size_t)n[s] * n[b]);
          T* X = pm.alloc<T>((size_t)n[b] * n[s]);
          Ym[{s, b}] = Y;
          Xm[{b, s}] = X;
          terms.push_back({Linv[q], Ap, n[s], n[s], n[s], 0, 0, 1});
          tasks.push_back({Y, n[s], n[s], n[b], (T)1, (T)0, (int)terms.size() - 1, (int)terms.size()});
          terms.push_back({blk(b, s), Uinv[q], n[b], n[s], n[s], 0, 0, 2});
          tasks.push_back({X, n[b], n[b], n[s], (T)1, (T)0, (int)terms.size() - 1, (int)terms.size()});
          rec.nbr.push_back(b);
          rec.X.push_back(X);
          rec.Y.push_back(Y);
          flops += 2.0 * n[s] * (double)n[s] * n[b];
        }
        R.in.push_back(rec);
      }
      if (tmp.err || pm.err) return SPAND_ERR_NOMEM;
      launch_row_perm(tmp, ps, pd, pp, pr_, pc_, st);
      // triangular-times-dense products: m n k useful flops each (half of a full product)
      double gflops = 0;
      for (size_t q = 0; q < tasks.size(); ++q) gflops += 1.0 * tasks[q].m * (double)tasks[q].n * terms[q].k;
      ev_begin(ev_gm[l]);
      launch_gemm(tmp, tasks, terms, st, "elim-YX");
      // Schur updates grouped by target block
      std::map<std::pair<int, int>, std::vector<int>> contrib;
      for (int s : I)
        for (int a : nbr[s])
          for (int b : nbr[s])
            if (n[a] > 0 && n[b] > 0) contrib[{a, b}].push_back(s);
      tasks.clear();
      terms.clear();
      for (auto& kv : contrib) {
        const int a = kv.first.first, b = kv.first.second;
        const int t0 = (int)terms.size();
        for (int s : kv.second) {
          terms.push_back({Xm.at({a, s}), Ym.at({s, b}), n[a], n[s], n[s], 0, 0, 0});
          flops += 2.0 * n[a] * (double)n[b] * n[s];
        }
        tasks.push_back({blk(a, b), n[a], n[a], n[b], (T)-1, (T)1, t0, (int)terms.size()});
        for (int q = t0; q < (int)terms.size(); ++q) gflops += 2.0 * n[a] * (double)n[b] * terms[q].k;
      }
      launch_gemm(tmp, tasks, terms, st, "elim-schur");
      ev_end(ev_gm[l]);
      S.elim_gemm_flops += gflops;
      S.elim_gemm_launches += 2;
      if (l == D)
        for (int s : I) S.top_size += n[s];
      for (int s : I) {
        const int q = P.system_of(l, s);
        if (l == (P.sys_D.empty() ? D : P.sys_D[q])) F->sys_stats[q].top_size += n[s];
      }
    }
    if (l == D) {
      tmp.free_all();
      break;
    }
    mark(1);
    tick("b eliminate interiors");
    // ================= 2. scale interfaces (Eq. 11)
    std::vector<int> Fc;
    for (int c = 0; c < nc; ++c)
      if (!L.cl[c].interior && n[c] > 0) Fc.push_back(c);
    std::vector<int> fidx(nc, -1);
    for (size_t q = 0; q < Fc.size(); ++q) fidx[Fc[q]] = (int)q;
    std::vector<std::vector<int>> nba(nc);
    for (auto& pr : L.after)
      if (pr.first != pr.second && n[pr.first] > 0 && n[pr.second] > 0) nba[pr.first].push_back(pr.second);
    std::vector<MatRef<T>> mats;
    std::vector<T*> SL, SU;
    std::vector<const T*> dsc;
    std::vector<T*> dsc_mut;
    for (int c : Fc) {
      MatRef<T> m;
      m.A = blk(c, c);
      m.n = n[c];
      m.ipiv = tmp.alloc<int>(n[c]);
      m.perm = pm.alloc<int>(n[c]);
      mats.push_back(m);
      SL.push_back(pm.alloc<T>((size_t)n[c] * n[c]));
      SU.push_back(pm.alloc<T>((size_t)n[c] * n[c]));
      T* d = tmp.alloc<T>(n[c]);
      dsc.push_back(d);
      dsc_mut.push_back(d);
      flops += 2.0 / 3.0 * pow((double)n[c], 3);
    }
    if (tmp.err || pm.err) return SPAND_ERR_NOMEM;
    batched_getrf(tmp, mats, d_flags, st);
    if (!mats.empty()) {
      auto* dm = tmp.upload(mats);
      auto* dd = tmp.upload(dsc_mut);
      note_launch();
      k_diag_sqrt<T><<<(unsigned)mats.size(), 128, 0, st>>>(dm, dd, (int)mats.size());
    }
    batched_inverses(tmp, mats, SL, SU, dsc, st);
    {
      // A_ab <- SL_a P_a^T A_ab SU_b for every off-diagonal block among interfaces
      std::vector<const T*> ps;
      std::vector<T*> pd;
      std::vector<const int*> pp;
      std::vector<int> pr_, pc_;
      std::vector<GemmTask<T>> t1, t2;
      std::vector<GemmTerm<T>> m1, m2;
      for (auto& pr : L.after) {
        const int a = pr.first, b = pr.second;
        if (a == b || n[a] == 0 || n[b] == 0) continue;
        T* Ap = tmp.alloc<T>((size_t)n[a] * n[b]);
        T* Tm = tmp.alloc<T>((size_t)n[a] * n[b]);
        ps.push_back(blk(a, b));
        pd.push_back(Ap);
        pp.push_back(mats[fidx[a]].perm);
        pr_.push_back(n[a]);
        pc_.push_back(n[b]);
        m1.push_back({SL[fidx[a]], Ap, n[a], n[a], n[a], 0, 0, 1});
        t1.push_back({Tm, n[a], n[a], n[b], (T)1, (T)0, (int)m1.size() - 1, (int)m1.size()});
        m2.push_back({Tm, SU[fidx[b]], n[a], n[b], n[b], 0, 0, 2});
        t2.push_back({blk(a, b), n[a], n[a], n[b], (T)1, (T)0, (int)m2.size() - 1, (int)m2.size()});
        flops += 2.0 * n[a] * (double)n[b] * (n[a] + n[b]);
      }
      if (tmp.err) return SPAND_ERR_NOMEM;
      launch_row_perm(tmp, ps, pd, pp, pr_, pc_, st);
      launch_gemm(tmp, t1, m1, st, "scale");
      launch_gemm(tmp, t2, m2, st, "scale");
    }
    mark(2);
    tick("c scale interfaces");
    // ================= 3. all Q first (Eq. 12): RRQR of [A_sn A_ns^T]
    std::vector<QrTask<T>> qt;
    std::vector<int> qcl;
    std::vector<CopyTask<T>> cps;
    std::map<const T*, int> w2q;                        // W buffer -> index in qt
    std::vector<std::pair<int, int>> cps_rng;           // per qt entry: its copy tasks [lo, hi)
    int* d_rank = tmp.alloc<int>(std::max<size_t>(Fc.size(), 1));
    int nmax_qr = 0;
    // the reflector arrays of all interfaces in one zeroed allocation (zero
    // above the diagonal for the WY products)
    size_t vtot = 0;
    for (size_t q = 0; q < Fc.size(); ++q) {
      const int s = Fc[q];
      if (nba[s].empty()) continue;
      int cs = 0;
      for (int b : nba[s]) cs += 2 * n[b];
      vtot += (((size_t)n[s] * std::min(n[s], cs)) + 63) & ~size_t(63);
    }
    T* vall = tmp.alloc<T>(std::max<size_t>(vtot, 1));
    if (tmp.err) return SPAND_ERR_NOMEM;
    SPAND_CUDA_TRY(cudaMemsetAsync(vall, 0, sizeof(T) * std::max<size_t>(vtot, 1), st));
    size_t voff = 0;
    for (size_t q = 0; q < Fc.size(); ++q) {
      const int s = Fc[q];
      if (nba[s].empty()) continue;
      int cs = 0;
      for (int b : nba[s]) cs += 2 * n[b];
      QrTask<T> t;
      t.n = n[s];
      t.c = cs;
      // row-major n x c; room for the column-major n x c layout with its
      // leading dimension padded to 16 bytes (the streaming kernel's form)
      t.W = tmp.alloc<T>((size_t)qrs_ldw<T>(n[s]) * cs);
      t.V = vall + voff;
      voff += (((size_t)n[s] * std::min(n[s], cs)) + 63) & ~size_t(63);
      t.tau = tmp.alloc<T>(std::min(n[s], cs));
      t.norm2 = tmp.alloc<T>(cs);
      t.Q = nullptr;
      t.rank = d_rank + qt.size();
      // W = [A_sn A_ns^T]; as a column-major c x n array (ld c) it holds W^T
      int off = 0;
      cps_rng.push_back({(int)cps.size(), (int)cps.size() + 2 * (int)nba[s].size()});
      for (int b : nba[s]) {
        cps.push_back({blk(s, b), t.W + off, n[s], cs, n[b], n[s], 1});
        off += n[b];
      }
      for (int b : nba[s]) {
        cps.push_back({blk(b, s), t.W + off, n[b], cs, n[b], n[s], 0});
        off += n[b];
      }
      w2q[t.W] = (int)qt.size();
      qt.push_back(t);
      qcl.push_back(s);
      nmax_qr = std::max(nmax_qr, n[s]);
      if (cs >= n[s]) flops += 2.0 * cs * (double)n[s] * n[s] - 2.0 / 3.0 * pow((double)n[s], 3);
    }
    if (tmp.err) return SPAND_ERR_NOMEM;
    std::vector<int> rank(qt.size());
    std::vector<std::array<int, 3>> strm_dbg;     // (n, c, index in qt) of the streamed interfaces (debug)
    std::vector<unsigned long long> strm_work;   // elements each streamed interface's passes moved
    int qf[4] = {0, 0, 0, 0};
    if (!qt.empty()) {
      // 16-CTA clusters (non-portable size) where the device schedules them
      // (per device: an on-chip probe of the two 16-CTA kernels)
      static std::atomic<uint64_t> probed{0}, can16{0};
      once_per_device(probed, [&] {
        auto probe16 = [](auto kp, int nt) -> int {
          if (cudaFuncSetAttribute(kp, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
            return 0;
          }
          const long long lim = set_dyn_smem((const void*)kp, kQrSmemMax);
          if (lim < 0) return 0;
          cudaLaunchConfig_t probe = {};
          cudaLaunchAttribute pa[1];
          pa[0].id = cudaLaunchAttributeClusterDimension;
          pa[0].val.clusterDim.x = 16;
          pa[0].val.clusterDim.y = 1;
          pa[0].val.clusterDim.z = 1;
          probe.gridDim = dim3(16, 1, 1);
          probe.blockDim = dim3(nt, 1, 1);
          probe.dynamicSmemBytes = (size_t)lim;
          probe.attrs = pa;
          probe.numAttrs = 1;
          int ncl = 0;
          if (cudaOccupancyMaxActiveClusters(&ncl, kp, &probe) != cudaSuccess) ncl = 0;
          cudaGetLastError();
          return ncl;
        };
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && probe16(k_qrcp_cluster<T, false, 16, 1024>, 1024) > 0 &&
            probe16(k_qrcp_cluster<T, true, 16, QR_THREADS>, QR_THREADS) > 0)
          can16.fetch_or(uint64_t(1) << dev);
      });
      int cur_dev = 0;
      cudaGetDevice(&cur_dev);
      const int cl16 = (cur_dev >= 0 && cur_dev < 64 && ((can16.load() >> cur_dev) & 1)) ? 1 : 0;
      // on-chip variants: chunk resident in shared memory with 8 or 16 CTAs;
      // the rest streams W from L2 / HBM
      // on-chip cluster forms: W's column chunks in shared memory on 1, 2, 4, 8
      // or 16 CTAs.  Each interface starts at the smallest cluster that holds it;
      // while the level's clusters leave SMs idle, the interface with the most
      // W per CTA doubles its cluster (fewer CTAs per interface cost less
      // barrier time per unit of work when the GPU is full; more CTAs shorten
      // the critical path when it is not).
      std::vector<QrTask<T>> q_gl, q_big;
      size_t gl_max = 0;
      const int csz[kQrClasses] = {1, 2, 4, 8, 16};
      long long limc[kQrClasses];
      limc[0] = set_dyn_smem((const void*)k_qrcp_cluster<T, true, 1, QR_THREADS>, kQrSmemMax);
      limc[1] = set_dyn_smem((const void*)k_qrcp_cluster<T, true, 2, QR_THREADS>, kQrSmemMax);
      limc[2] = set_dyn_smem((const void*)k_qrcp_cluster<T, true, 4, QR_THREADS>, kQrSmemMax);
      limc[3] = set_dyn_smem((const void*)k_qrcp_cluster<T, true, QR_CS, QR_THREADS>, kQrSmemMax);
      limc[4] = cl16 ? set_dyn_smem((const void*)k_qrcp_cluster<T, true, 16, QR_THREADS>, kQrSmemMax) : -1;
      const int top_cls = cl16 ? 4 : 3;
      // Every interface goes to the streaming kernel when the device runs
      // cooperative launches: its dropping of dead columns, its balanced column
      // split and its persistent launches beat the on-chip forms at every level
      // (same ranks and Q).  The on-chip forms below remain for devices without
      // cooperative launches and for comparison (SPAND_QR_STREAM=0).
      const bool all_stream = stream_forced() >= 0 && qrs_capacity<T>() > 0;
      std::vector<int> cls_of(qt.size(), -1);
      long long ctas = 0;
      for (size_t k = 0; k < qt.size(); ++k) {
        for (int ci = 0; ci <= top_cls && !all_stream; ++ci)
          if ((long long)qrcp_smem_bytes<T>(qt[k].n, qt[k].c, csz[ci]) <= limc[ci]) {
            cls_of[k] = ci;
            break;
          }
        if (cls_of[k] < 0) q_big.push_back(qt[k]);
        else ctas += csz[cls_of[k]];
      }
      {
        int nsm_dev = 0, devq = 0;
        cudaGetDevice(&devq);
        cudaDeviceGetAttribute(&nsm_dev, cudaDevAttrMultiProcessorCount, devq);
        while (ctas < nsm_dev) {
          int best = -1;
          double bw = -1;
          for (size_t k = 0; k < qt.size(); ++k)
            if (cls_of[k] >= 0 && cls_of[k] < top_cls) {
              const double w = (double)qt[k].n * qt[k].c / csz[cls_of[k]];
              if (w > bw) {
                bw = w;
                best = (int)k;
              }
            }
          if (best < 0) break;
          ctas += csz[cls_of[best]];
          ++cls_of[best];
        }
      }
      std::vector<QrTask<T>> q_cls[kQrClasses];
      size_t cls_bytes[kQrClasses] = {0, 0, 0, 0, 0};
      for (size_t k = 0; k < qt.size(); ++k)
        if (cls_of[k] >= 0) {
          q_cls[cls_of[k]].push_back(qt[k]);
          cls_bytes[cls_of[k]] = std::max(cls_bytes[cls_of[k]], qrcp_smem_bytes<T>(qt[k].n, qt[k].c, csz[cls_of[k]]));
        }
      // too large for one cluster: CTA groups of cooperative launches, as many
      // groups per launch as fit on the GPU at once.  A group keeps W in
      // shared memory when its chunks fit (G <= the resident-CTA capacity);
      // otherwise W streams from L2 / HBM through a group sized to the problem.
      struct CoopLaunch {
        std::vector<QrGroupDesc> desc;
        size_t bytes = 0;
        bool smem = true;
      };
      std::vector<CoopLaunch> coop;
      std::vector<QrTask<T>> q_coop;
      std::vector<int> q_strm;                     // indices in qt of the interfaces W streams for
      int n_group_smem = 0, n_group_stream = 0;
      if (!q_big.empty()) {
        auto kg = k_qrcp_group<T, true, QR_THREADS>;
        auto ks = k_qrcp_group<T, false, 1024>;
        const long long limg = set_dyn_smem((const void*)kg, kQrSmemMax);
        const long long lims = set_dyn_smem((const void*)ks, kQrSmemMax);
        int dev = 0, nsm = 0, coop_ok = 0, per_sm = 0, per_sm_s = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, dev);
        if (limg > 0 && coop_ok &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kg, QR_THREADS, (size_t)limg) != cudaSuccess)
          per_sm = 0;
        if (lims > 0 && coop_ok &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, ks, 1024, (size_t)lims) != cudaSuccess)
          per_sm_s = 0;
        cudaGetLastError();
        const int cap = std::min(QR_GMAX, coop_ok ? per_sm * nsm : 0);
        const int cap_s = std::min(QR_GMAX, coop_ok ? per_sm_s * nsm : 0);
        std::vector<std::pair<int, int>> in_smem, streamed;   // (task index in q_coop, G)
        // the streaming kernel: one 512-thread CTA per SM in a cooperative launch
        const bool strm_ok = coop_ok && stream_forced() >= 0 && qrs_capacity<T>() > 0;
        for (auto& t : q_big) {
          int G = 2;
          while (G <= cap && (long long)qrcp_smem_bytes<T>(t.n, t.c, G) > limg) ++G;
          if (strm_ok && all_stream) {
            q_strm.push_back(w2q.at(t.W));
          } else if (G <= cap && limg > 0) {
            in_smem.push_back({(int)q_coop.size(), G});
            q_coop.push_back(t);
          } else if (strm_ok) {
            q_strm.push_back(w2q.at(t.W));     // W streams from L2 / HBM (k_qrcp_stream)
          } else if (cap_s >= 16) {
            // about 1 MB of W per CTA, at least 16 CTAs, at most the resident capacity
            const double mb = (double)t.n * t.c * sizeof(T) / (1 << 20);
            const int Gs = std::max(16, std::min(cap_s, (int)std::ceil(mb)));
            streamed.push_back({(int)q_coop.size(), Gs});
            q_coop.push_back(t);
          } else {
            q_gl.push_back(t);
            gl_max = std::max(gl_max, ((size_t)t.n + 31) * sizeof(T));
          }
        }
        auto pack = [&](const std::vector<std::pair<int, int>>& v, bool smem, int capk) {
          CoopLaunch cur;
          cur.smem = smem;
          int used = 0;
          for (auto& pr : v) {
            const QrTask<T>& t = q_coop[pr.first];
            const int G = pr.second;
            if (used + G > capk && !cur.desc.empty()) {
              coop.push_back(cur);
              cur = CoopLaunch();
              cur.smem = smem;
              used = 0;
            }
            for (int g = 0; g < G; ++g) cur.desc.push_back({pr.first, g, G, 0});
            cur.bytes = std::max(cur.bytes, smem ? qrcp_smem_bytes<T>(t.n, t.c, G) : ((size_t)t.n + 31) * sizeof(T));
            used += G;
          }
          if (!cur.desc.empty()) coop.push_back(cur);
        };
        pack(in_smem, true, cap);
        pack(streamed, false, cap_s);
        n_group_smem = (int)in_smem.size();
        n_group_stream = (int)streamed.size();
      }
      T* d_prop_v = nullptr;
      int* d_prop_i = nullptr;
      T* d_slots = nullptr;
      int slot_ns = 32;
      GroupSync* d_gs = nullptr;
      QrTask<T>* d_coop = nullptr;
      std::vector<QrGroupDesc*> d_desc;
      if (!q_coop.empty()) {
        d_coop = tmp.upload(q_coop);
        d_prop_v = tmp.alloc<T>(q_coop.size() * 2 * QR_GMAX);
        d_prop_i = tmp.alloc<int>(q_coop.size() * 2 * QR_GMAX);
        // candidate-column slots, reused launch after launch (stream order)
        int ncta = 0;
        for (auto& cl : coop) ncta = std::max(ncta, (int)cl.desc.size());
        for (auto& t : q_coop) slot_ns = std::max(slot_ns, (t.n + 31) & ~31);
        d_slots = tmp.alloc<T>((size_t)ncta * 2 * slot_ns);
        d_gs = tmp.alloc<GroupSync>(q_coop.size());
        for (auto& cl : coop) d_desc.push_back(tmp.upload(cl.desc));
        if (tmp.err) return SPAND_ERR_NOMEM;
        SPAND_CUDA_TRY(cudaMemsetAsync(d_gs, 0, sizeof(GroupSync) * q_coop.size(), st));
      }
      if (debug_level() >= 2) {
        // shapes of the level's RRQR problems and how they were placed
        double sn = 0, sc = 0;
        int mn = 0, mc = 0;
        for (auto& t : qt) {
          sn += t.n;
          sc += t.c;
          mn = std::max(mn, t.n);
          mc = std::max(mc, t.c);
        }
        std::fprintf(stderr, "spand: level %d RRQR: %zu interfaces, n mean %.0f max %d, c mean %.0f max %d; "
                             "clusters 1/2/4/8/16: %zu/%zu/%zu/%zu/%zu, groups in smem %d, streamed %d, "
                             "cooperative launches %zu\n",
                     l, qt.size(), sn / std::max<size_t>(1, qt.size()), mn, sc / std::max<size_t>(1, qt.size()), mc,
                     q_cls[0].size(), q_cls[1].size(), q_cls[2].size(), q_cls[3].size(), q_cls[4].size(),
                     n_group_smem, n_group_stream + (int)q_gl.size(), coop.size());
        for (size_t li = 0; li < coop.size() && li < 8; ++li) {
          std::map<int, int> gsz;
          for (auto& d : coop[li].desc) gsz[d.G] += (d.q == 0);
          std::fprintf(stderr, "spand:   cooperative launch %zu: %zu CTAs, %s, groups (G x count):", li,
                       coop[li].desc.size(), coop[li].smem ? "W in smem" : "W streamed");
          for (auto& kv : gsz) std::fprintf(stderr, " %dx%d", kv.first, kv.second);
          std::fprintf(stderr, "\n");
        }
      }
      qf[0] = (int)(q_cls[0].size() + q_cls[1].size() + q_cls[2].size() + q_cls[3].size());
      qf[1] = (int)q_cls[4].size();
      qf[2] = n_group_smem;
      qf[3] = n_group_stream + (int)q_gl.size() + (int)q_strm.size();
      // task arrays are uploaded on st before the fork, so the side stream
      // never reads them ahead of their copies
      QrTask<T>* d_gl = q_gl.empty() ? nullptr : tmp.upload(q_gl);
      QrTask<T>* d_cls[kQrClasses];
      for (int ci = 0; ci < kQrClasses; ++ci) d_cls[ci] = q_cls[ci].empty() ? nullptr : tmp.upload(q_cls[ci]);
      if (tmp.err) return SPAND_ERR_NOMEM;
      auto launch_qr = [&](const QrTask<T>* dq, size_t count, cudaStream_t s2, int cs, int nt, size_t bytes,
                           auto kern) -> int {
        if (count == 0) return SPAND_OK;
        if (cs > 8) SPAND_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        if (set_dyn_smem((const void*)kern, bytes) < (long long)bytes) return SPAND_ERR_UNSUPPORTED;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(count * cs), 1, 1);
        cfg.blockDim = dim3(nt, 1, 1);
        cfg.dynamicSmemBytes = bytes;
        cfg.stream = s2;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        note_launch();
        SPAND_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, dq, (T)eps));
        return SPAND_OK;
      };
      // W of every interface: row-major for the on-chip forms, column-major
      // (leading dimension padded to 16 bytes, padding rows zero) for the
      // streaming kernel
      std::vector<QrStreamTask<T>> strm;
      std::vector<int> strm_qi;                    // index in qt of each streamed interface
      unsigned long long* d_work = nullptr;
      {
        std::vector<char> is_strm(qt.size(), 0);
        for (int qi : q_strm) is_strm[qi] = 1;
        if (!q_strm.empty()) {
          d_work = tmp.alloc<unsigned long long>(q_strm.size());
          if (tmp.err) return SPAND_ERR_NOMEM;
          SPAND_CUDA_TRY(cudaMemsetAsync(d_work, 0, sizeof(unsigned long long) * q_strm.size(), st));
        }
        std::vector<CopyTask<T>> cps2;
        cps2.reserve(cps.size());
        for (size_t qi = 0; qi < qt.size(); ++qi) {
          const auto rg = cps_rng[qi];
          if (!is_strm[qi]) {
            for (int e = rg.first; e < rg.second; ++e) cps2.push_back(cps[e]);
            continue;
          }
          const QrTask<T>& t = qt[qi];
          const int ldw = qrs_ldw<T>(t.n);
          if (ldw > t.n) SPAND_CUDA_TRY(cudaMemsetAsync(t.W, 0, sizeof(T) * (size_t)ldw * t.c, st));
          for (int e = rg.first; e < rg.second; ++e) {
            const CopyTask<T>& o = cps[e];
            const size_t off = (size_t)(o.dst - t.W);          // first column of the block in W
            cps2.push_back({o.src, t.W + off * ldw, o.lds, ldw, o.cols, o.rows, 1 - o.trans});
          }
          QrStreamTask<T> u;
          u.W = t.W;
          u.V = t.V;
          u.tau = t.tau;
          u.Q = nullptr;
          u.n = t.n;
          u.c = t.c;
          u.ldw = ldw;
          u.rank = t.rank;
          u.work = d_work + strm.size();
          strm.push_back(u);
          strm_qi.push_back((int)qi);
        }
        launch_copy(tmp, cps2, st);
        for (size_t i = 0; i < strm.size(); ++i) strm_dbg.push_back({strm[i].n, strm[i].c, strm_qi[i]});
      }
      ev_begin(ev_qr[l]);
      // the streaming launch and the on-chip launches (one stream per cluster size) overlap
      SPAND_CUDA_TRY(cudaEventRecord(sides.fork, st));
      for (int ci = 0; ci < kQrClasses; ++ci) SPAND_CUDA_TRY(cudaStreamWaitEvent(sides.s[ci], sides.fork, 0));
      if (cl16)
        SPAND_TRY(launch_qr(d_gl, q_gl.size(), st, 16, 1024, gl_max, k_qrcp_cluster<T, false, 16, 1024>));
      else
        SPAND_TRY(launch_qr(d_gl, q_gl.size(), st, QR_CS, 1024, gl_max, k_qrcp_cluster<T, false, QR_CS, 1024>));
      SPAND_TRY(launch_qr(d_cls[4], q_cls[4].size(), sides.s[4], 16, QR_THREADS, cls_bytes[4],
                          k_qrcp_cluster<T, true, 16, QR_THREADS>));
      SPAND_TRY(launch_qr(d_cls[3], q_cls[3].size(), sides.s[3], QR_CS, QR_THREADS, cls_bytes[3],
                          k_qrcp_cluster<T, true, QR_CS, QR_THREADS>));
      SPAND_TRY(launch_qr(d_cls[2], q_cls[2].size(), sides.s[2], 4, QR_THREADS, cls_bytes[2],
                          k_qrcp_cluster<T, true, 4, QR_THREADS>));
      SPAND_TRY(launch_qr(d_cls[1], q_cls[1].size(), sides.s[1], 2, QR_THREADS, cls_bytes[1],
                          k_qrcp_cluster<T, true, 2, QR_THREADS>));
      SPAND_TRY(launch_qr(d_cls[0], q_cls[0].size(), sides.s[0], 1, QR_THREADS, cls_bytes[0],
                          k_qrcp_cluster<T, true, 1, QR_THREADS>));
      for (int ci = 0; ci < kQrClasses; ++ci) {
        SPAND_CUDA_TRY(cudaEventRecord(sides.join[ci], sides.s[ci]));
        SPAND_CUDA_TRY(cudaStreamWaitEvent(st, sides.join[ci], 0));
      }
      // cooperative CTA groups after the join, so that nothing else holds SMs
      // while a launch that needs all of its CTAs resident at once starts
      {
        for (size_t li = 0; li < coop.size(); ++li) {
          const void* kfn = coop[li].smem ? (const void*)k_qrcp_group<T, true, QR_THREADS>
                                          : (const void*)k_qrcp_group<T, false, 1024>;
          if (set_dyn_smem(kfn, coop[li].bytes) < (long long)coop[li].bytes) return SPAND_ERR_UNSUPPORTED;
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3((unsigned)coop[li].desc.size(), 1, 1);
          cfg.blockDim = dim3(coop[li].smem ? QR_THREADS : 1024, 1, 1);
          cfg.dynamicSmemBytes = coop[li].bytes;
          cfg.stream = st;
          cudaLaunchAttribute attr[1];
          attr[0].id = cudaLaunchAttributeCooperative;
          attr[0].val.cooperative = 1;
          cfg.attrs = attr;
          cfg.numAttrs = 1;
          note_launch();
          const QrTask<T>* a0 = d_coop;
          const QrGroupDesc* a1 = d_desc[li];
          if (coop[li].smem)
            SPAND_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qrcp_group<T, true, QR_THREADS>, a0, a1, d_prop_v, d_prop_i,
                                              d_gs, d_flags, d_slots, slot_ns, (T)eps));
          else
            SPAND_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qrcp_group<T, false, 1024>, a0, a1, d_prop_v, d_prop_i, d_gs,
                                              d_flags, d_slots, slot_ns, (T)eps));
        }
      }
      if (!strm.empty()) SPAND_TRY(launch_qrcp_stream<T>(tmp, strm, d_flags, (T)eps, st));
      ev_end(ev_qr[l]);
      S.rrqr_launches += 1;
      SPAND_CUDA_TRY(cudaMemcpyAsync(rank.data(), d_rank, sizeof(int) * qt.size(), cudaMemcpyDeviceToHost, st));
      if (!strm.empty()) {
        strm_work.assign(strm.size(), 0ull);
        SPAND_CUDA_TRY(cudaMemcpyAsync(strm_work.data(), d_work, sizeof(unsigned long long) * strm.size(),
                                       cudaMemcpyDeviceToHost, st));
      }
    }
    mark(3);
    tick("d RRQR setup, launch, D2H of streamed work");
    int hflags[4];
    SPAND_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    SPAND_CUDA_TRY(sync_st());
    mark(4);
    tick("e sync after RRQR");
    if (hflags[0] & 32) return SPAND_ERR_ARG;          // a matrix pattern the plan does not describe
    if (hflags[0] & 1) return SPAND_ERR_ZERO_PIVOT;   // the root cause when both are set
    if (hflags[0] & 2) return SPAND_ERR_NONFINITE;
    if (hflags[0] & 16) {
      report_cuda_error(cudaErrorLaunchTimeout, "RRQR group barrier", __FILE__, __LINE__);
      return SPAND_ERR_CUDA;                          // a group barrier ran out of time
    }
    S.t_rrqr_level_ms[l] = ev_read(ev_qr[l]);
    for (unsigned long long w : strm_work) S.rrqr_stream_bytes_level[l] += 2.0 * (double)w * sizeof(T);
    S.rrqr_stream_bytes += S.rrqr_stream_bytes_level[l];
    if (debug_level() >= 2 && !strm_dbg.empty() && strm_work.size() == strm_dbg.size()) {
      const std::vector<unsigned long long>& wk = strm_work;
      {
        std::vector<int> ord(wk.size());
        double tot = 0;
        for (size_t i = 0; i < wk.size(); ++i) {
          ord[i] = (int)i;
          tot += (double)wk[i];
        }
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return wk[a] > wk[b]; });
        std::fprintf(stderr, "spand: level %d streamed %zu interfaces, %.3g elements streamed (%.2f GB read+written)\n",
                     l, wk.size(), tot, tot * 2 * sizeof(T) / 1e9);
        for (size_t i = 0; i < std::min<size_t>(6, ord.size()); ++i) {
          const auto& d = strm_dbg[ord[i]];
          std::fprintf(stderr, "spand:   n %d c %d rank %d: %.3g elements (%.1f%% of the level)\n", d[0], d[1],
                       rank[d[2]], (double)wk[ord[i]], 100.0 * wk[ord[i]] / std::max(1.0, tot));
        }
      }
    }
    if (debug_level() >= 2 && !qt.empty()) {
      long long sr = 0;
      int mr = 0;
      for (size_t q = 0; q < qt.size(); ++q) {
        sr += rank[q];
        mr = std::max(mr, rank[q]);
      }
      std::fprintf(stderr, "spand: level %d RRQR %.3f ms, ranks sum %lld mean %.1f max %d\n", l,
                   S.t_rrqr_level_ms[l], sr, (double)sr / qt.size(), mr);
    }
    S.t_rrqr_ms += S.t_rrqr_level_ms[l];
    S.t_elim_gemm_ms += ev_read(ev_gm[l]);
    for (size_t q = 0; q < qt.size(); ++q)
      for (int k = 0; k < rank[q]; ++k)
        S.rrqr_bytes_level[l] += 2.0 * (double)(qt[q].n - k) * (double)(qt[q].c - k) * sizeof(T);
    S.rrqr_bytes += S.rrqr_bytes_level[l];
    S.rrqr_form_count[l][0] = qf[0];
    S.rrqr_form_count[l][1] = qf[1];
    S.rrqr_form_count[l][2] = qf[2];
    S.rrqr_form_count[l][3] = qf[3];
    std::vector<int> r(nc, 0);
    std::vector<char> spars(nc, 0);
    std::vector<T*> Qc(nc, nullptr);
    for (int c : Fc) r[c] = n[c];
    for (size_t q = 0; q < qt.size(); ++q) {
      const int s = qcl[q];
      r[s] = rank[q];
      spars[s] = 1;
      Qc[s] = pm.alloc<T>((size_t)n[s] * std::max(rank[q], 1));
      qt[q].Q = Qc[s];
      S.n_sparsified[l] += 1;
      S.sum_n[l] += n[s];
      S.sum_r[l] += rank[q];
      S.max_r[l] = std::max<int64_t>(S.max_r[l], rank[q]);
      spand_stats& Sq = F->sys_stats[P.system_of(l, s)];
      Sq.n_sparsified[l] += 1;
      Sq.sum_n[l] += n[s];
      Sq.sum_r[l] += rank[q];
      Sq.max_r[l] = std::max<int64_t>(Sq.max_r[l], rank[q]);
    }
    if (pm.err) return SPAND_ERR_NOMEM;
    tick("f ranks, stats, Q_c allocation");
    if (!qt.empty()) {
      // Q_c = [I_r; 0] - V M with M = T V_top^T (compact WY); G = V^T V first
      std::vector<GemmTask<T>> gt, mt, qtk;
      std::vector<GemmTerm<T>> gm, mm, qm;
      std::vector<WyTask<T>> wy;
      std::vector<MatRef<T>> tri;
      std::vector<T*> Tinv;
      std::vector<const T*> nod;
      std::vector<EyeTask<T>> eye_q;
      for (size_t q = 0; q < qt.size(); ++q) {
        const int r = rank[q], nn = qt[q].n;
        if (r <= 0) continue;
        T* G = tmp.alloc<T>((size_t)r * r);
        T* Tm = tmp.alloc<T>((size_t)r * r);
        T* M = tmp.alloc<T>((size_t)r * r);
        gm.push_back({qt[q].V, qt[q].V, nn, nn, nn, 1, 0, 0});
        gt.push_back({G, r, r, r, (T)1, (T)0, (int)gm.size() - 1, (int)gm.size()});
        wy.push_back({G, qt[q].tau, r});
        MatRef<T> mr;
        mr.A = G;
        mr.n = r;
        mr.ipiv = nullptr;
        mr.perm = nullptr;
        tri.push_back(mr);
        Tinv.push_back(Tm);
        nod.push_back(nullptr);
        mm.push_back({Tm, qt[q].V, r, nn, r, 0, 1, 0});
        mt.push_back({M, r, r, r, (T)1, (T)0, (int)mm.size() - 1, (int)mm.size()});
        eye_q.push_back({qt[q].Q, nn, r, nn});     // Q_c = [I_r; 0] before the update below
        qm.push_back({qt[q].V, M, nn, r, r, 0, 0, 0});
        qtk.push_back({qt[q].Q, nn, nn, r, (T)-1, (T)1, (int)qm.size() - 1, (int)qm.size()});
      }
      if (tmp.err) return SPAND_ERR_NOMEM;
      tick("g WY task lists");
      launch_gemm(tmp, gt, gm, st, "wy");
      if (!wy.empty()) {
        auto* dw = tmp.upload(wy);
        note_launch();
        k_wy_tinv<T><<<(unsigned)wy.size(), 256, 0, st>>>(dw);
        // T = (T^-1)^-1 with the batched upper-triangular inverse
        batched_upper_inverse(tmp, tri, Tinv, st);
        auto* de = tmp.upload(eye_q);
        note_launch();
        k_eye<T><<<std::min<unsigned>((unsigned)eye_q.size(), 4096), 256, 0, st>>>(de, (int)eye_q.size());
      }
      launch_gemm(tmp, mt, mm, st, "wy");
      launch_gemm(tmp, qtk, qm, st, "wy");
    }
    // records for the apply
    for (size_t q = 0; q < Fc.size(); ++q) {
      const int s = Fc[q];
      typename LevelRec<T>::Iface f;
      f.SL = SL[q];
      f.SU = SU[q];
      f.Q = Qc[s];
      f.perm = mats[q].perm;
      f.c = s;
      f.n = n[s];
      f.r = r[s];
      f.sparsified = spars[s] != 0;
      f.park_b_off = park_b_tot;
      f.park_c_off = park_c_tot;
      if (f.sparsified) {
        park_b_tot += n[s];
        park_c_tot += r[s];
      }
      R.fa.push_back(f);
    }
    mark(5);
    tick("h WY launches, apply records");
    // ================= 4. next level: sizes, slots, merged blocks
    const LevelInfo& L2 = P.lv[l + 1];
    const int nc2 = (int)L2.cl.size();
    std::vector<int> n2(nc2, 0), off(nc, 0);
    std::vector<std::vector<int>> slots2(nc2);
    for (int p2 = 0; p2 < nc2; ++p2)
      for (int ch : L2.cl[p2].children) {
        const int c = L.surv[ch];
        off[c] = n2[p2];
        n2[p2] += r[c];
        slots2[p2].insert(slots2[p2].end(), slots[c].begin(), slots[c].begin() + r[c]);
      }
    std::vector<int> parent(nc, -1);
    for (size_t k = 0; k < L.surv.size(); ++k) parent[L.surv[k]] = L.parent[k];
    // new arena
    DevMem lvmem2;
    lvmem2.st = st;
    lvmem2.stage = &stage;
    T* old_arena = arena;
    const BlockIndex old_off = boff;
    SPAND_TRY(layout(L2, n2, lvmem2));
    auto oblk = [&](int a, int b) -> T* { return old_arena + old_off.at(a, b); };
    tick("i next-level sizes, slots, layout");
    std::vector<EyeTask<T>> eyes;
    std::vector<GemmTask<T>> t1, t2;
    std::vector<GemmTerm<T>> m1, m2;
    for (auto& pr : L.after) {
      const int a = pr.first, b = pr.second;
      if (n[a] == 0 || n[b] == 0 || r[a] == 0 || r[b] == 0) continue;
      const int pa = parent[a], pb = parent[b];
      T* dst = blk(pa, pb) + off[a] + (size_t)off[b] * n2[pa];
      if (a == b) {
        eyes.push_back({dst, n2[pa], r[a], 0});
        continue;
      }
      // both are sparsified (they have neighbours).  First (Q_ac^T A_ab)^T =
      // A_ab^T Q_ac (n_b x r_a: the long side along the tiles' 128 rows, both
      // operands read along k), then Q_ac^T A_ab Q_bc from it
      T* Tm = tmp.alloc<T>((size_t)n[b] * r[a]);
      m1.push_back({oblk(a, b), Qc[a], n[a], n[a], n[a], 1, 0, 0});
      t1.push_back({Tm, n[b], n[b], r[a], (T)1, (T)0, (int)m1.size() - 1, (int)m1.size()});
      m2.push_back({Tm, Qc[b], n[b], n[b], n[b], 1, 0, 0});
      t2.push_back({dst, n2[pa], r[a], r[b], (T)1, (T)0, (int)m2.size() - 1, (int)m2.size()});
      flops += 2.0 * n[a] * (double)n[b] * (r[a] + r[b]);
    }
    if (tmp.err) return SPAND_ERR_NOMEM;
    tick("j compress task lists");
    launch_gemm(tmp, t1, m1, st, "compress");
    launch_gemm(tmp, t2, m2, st, "compress");
    if (!eyes.empty()) {
      auto* de = tmp.upload(eyes);
      note_launch();
      k_eye<T><<<std::min<unsigned>((unsigned)eyes.size(), 1024), 128, 0, st>>>(de, (int)eyes.size());
    }
    SPAND_CUDA_TRY(cudaGetLastError());
    tmp.free_all();
    lvmem.free_all();
    lvmem = lvmem2;
    lvmem2.ptrs.clear();
    n = n2;
    slots = slots2;
    tick("k compress launches, frees");
  }
  lvmem.free_all();
  {
    int hflags[4];
    SPAND_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    SPAND_CUDA_TRY(sync_st());
    S.t_elim_gemm_ms += ev_read(ev_gm[D]);
    if (hflags[0] & 32) return SPAND_ERR_ARG;
    if (hflags[0] & 1) return SPAND_ERR_ZERO_PIVOT;   // the root cause when both are set
    if (hflags[0] & 2) return SPAND_ERR_NONFINITE;
    if (std::is_same<T, float>::value && gemm_mode() != 2) {
      int uf = 0;
      SPAND_CUDA_TRY(cudaMemcpyFromSymbol(&uf, g_umma_fail, sizeof(int)));
      if (uf) {
        report_cuda_error(cudaErrorLaunchTimeout, "tcgen05 GEMM completion wait", __FILE__, __LINE__);
        return SPAND_ERR_CUDA;
      }
    }
  }
  S.factor_flops = flops;
  if (debug_level() >= 3) GemmLog::get().print_and_clear();
  tick("l final sync");
  if (!tick_ev.empty()) {
    std::map<std::string, double> gpu_ticks;
    cudaEventSynchronize(tick_ev.back().second);
    for (size_t i = 1; i < tick_ev.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, tick_ev[i - 1].second, tick_ev[i].second) == cudaSuccess) {
        gpu_ticks[tick_ev[i].first] += ms;
        if (debug_level() >= 3)
          std::fprintf(stderr, "spand: level %d GPU %-46s %9.2f ms\n", tick_lv[i], tick_ev[i].first, ms);
      } else {
        cudaGetLastError();
      }
    }
    for (auto& te : tick_ev) cudaEventDestroy(te.second);
    for (auto& kv : host_ticks)
      std::fprintf(stderr, "spand: host %-46s %9.2f ms   GPU %9.2f ms\n", kv.first.c_str(), kv.second,
                   gpu_ticks[kv.first]);
  }

  mark(6);
  // ================= apply program
  F->w = pm.alloc<T>(F->N);
  F->z = pm.alloc<T>(F->N);
  F->park_b = pm.alloc<T>(std::max<size_t>(park_b_tot, 1));
  F->park_c = pm.alloc<T>(std::max<size_t>(park_c_tot, 1));
  if (pm.err) return SPAND_ERR_NOMEM;
  // permuted slot lists (P^T folded into the gather) for interiors and interfaces
  std::vector<std::vector<int*>> fa_ps(D + 1);
  {
    std::vector<PermSlotTask> pt;
    for (int l = 0; l <= D; ++l) {
      LevelRec<T>& R = recs[l];
      for (auto& in : R.in) {
        int* ps = pm.alloc<int>(in.n);
        pt.push_back({R.d_slots[in.c], in.perm, ps, in.n});
        R.d_pslots.push_back(ps);
      }
      for (auto& f : R.fa) {
        int* ps = pm.alloc<int>(f.n);
        pt.push_back({R.d_slots[f.c], f.perm, ps, f.n});
        fa_ps[l].push_back(ps);
      }
    }
    if (pm.err) return SPAND_ERR_NOMEM;
    if (!pt.empty()) {
      DevMem tmpp;
      tmpp.st = st;
      tmpp.stage = &stage;
      auto* dpt = tmpp.upload(pt);
      if (tmpp.err) return SPAND_ERR_NOMEM;
      note_launch();
      k_perm_slots<<<(unsigned)pt.size(), 256, 0, st>>>(dpt);
      tmpp.free_all();
    }
  }
  typedef typename ApplyProg<T>::Phase Phase;
  auto build = [&](std::vector<GvTask<T>>& tasks, std::vector<GvTerm<T>>& terms) -> Phase {
    Phase ph;
    std::vector<GvTile> tiles;
    for (int t = 0; t < (int)tasks.size(); ++t)
      for (int r0 = 0; r0 < tasks[t].m; r0 += GV_ROWS) tiles.push_back({t, r0});
    for (auto& tm : terms) ph.kmax = std::max(ph.kmax, tm.k);
    if (tiles.empty()) return ph;
    upload3(pm, tasks, terms, tiles, ph.tasks, ph.terms, ph.tiles);
    ph.ntiles = (int)tiles.size();
    return ph;
  };
  T* w = F->w;
  T* z = F->z;
  const size_t es = sizeof(T);
  // sweeps of the clusters keep(l, c) selects (one system, or all of them)
  auto build_prog = [&](Program<T>& pg, auto keep) {
  int64_t& apply_bytes = pg.bytes;
  for (int tr = 0; tr < 2; ++tr) {
    std::vector<Phase>& fwd = tr ? pg.prog.tfwd : pg.prog.fwd;
    std::vector<Phase>& bwd = tr ? pg.prog.tbwd : pg.prog.bwd;
    for (int l = 0; l <= D; ++l) {
      LevelRec<T>& R = recs[l];
      std::vector<GvTask<T>> tk;
      std::vector<GvTerm<T>> tm;
      auto task = [&](T* y, const int* yidx, const T* base, const int* bidx, T* y2, T alpha, int m) {
        tk.push_back({y, yidx, base, bidx, y2, alpha, m, (int)tm.size(), (int)tm.size()});
      };
      auto term = [&](const T* M, const T* x, const int* xidx, const T* xsub, int ld, int k, int trans, int tri) {
        tm.push_back({M, x, xidx, xsub, ld, k, trans, tri});
        tk.back().t1 = (int)tm.size();
      };
      auto flush = [&](std::vector<Phase>& dst) {
        Phase ph = build(tk, tm);
        if (ph.ntiles) dst.push_back(ph);
        tk.clear();
        tm.clear();
      };
      // neighbour -> interiors map for grouped coupling updates
      std::map<int, std::vector<std::pair<int, int>>> by_nb;   // b -> (interior index, nbr index)
      for (int q = 0; q < (int)R.in.size(); ++q)
        if (keep(l, R.in[q].c))
          for (int t = 0; t < (int)R.in[q].nbr.size(); ++t) by_nb[R.in[q].nbr[t]].push_back({q, t});
      if (!tr) {
        // E1: z[s] = L^-1 P^T w[s]
        for (int q = 0; q < (int)R.in.size(); ++q) {
          auto& in = R.in[q];
          if (!keep(l, in.c)) continue;
          task(z, R.d_slots[in.c], nullptr, nullptr, nullptr, (T)1, in.n);
          term(in.Linv, w, R.d_pslots[q], nullptr, in.n, in.n, 0, 1);
          apply_bytes += (int64_t)in.n * (in.n + 1) / 2 * es;
        }
        flush(fwd);
        // E2: w[b] -= sum_s X_bs z[s]
        for (auto& kv : by_nb) {
          const int b = kv.first;
          task(w, R.d_slots[b], w, R.d_slots[b], nullptr, (T)-1, R.n[b]);
          for (auto& pr : kv.second) {
            auto& in = R.in[pr.first];
            term(in.X[pr.second], z, R.d_slots[in.c], nullptr, R.n[b], in.n, 0, 0);
            apply_bytes += (int64_t)R.n[b] * in.n * es;
          }
        }
        flush(fwd);
      } else {
        // E3^T: z[s] = U^-T w[s];  w[b] -= Y_sb^T z[s]
        for (int q = 0; q < (int)R.in.size(); ++q) {
          auto& in = R.in[q];
          if (!keep(l, in.c)) continue;
          task(z, R.d_slots[in.c], nullptr, nullptr, nullptr, (T)1, in.n);
          term(in.Uinv, w, R.d_slots[in.c], nullptr, in.n, in.n, 1, 2);
        }
        flush(fwd);
        for (auto& kv : by_nb) {
          const int b = kv.first;
          task(w, R.d_slots[b], w, R.d_slots[b], nullptr, (T)-1, R.n[b]);
          for (auto& pr : kv.second) {
            auto& in = R.in[pr.first];
            term(in.Y[pr.second], z, R.d_slots[in.c], nullptr, in.n, in.n, 1, 0);
          }
        }
        flush(fwd);
      }
      if (l < D) {
        // S1: z[s] = SL P^T w[s]   (transpose: z[s] = SU^T w[s])
        for (size_t q = 0; q < R.fa.size(); ++q) {
          auto& f = R.fa[q];
          if (!keep(l, f.c)) continue;
          task(z, R.d_slots[f.c], nullptr, nullptr, nullptr, (T)1, f.n);
          if (!tr) term(f.SL, w, fa_ps[l][q], nullptr, f.n, f.n, 0, 1);
          else term(f.SU, w, R.d_slots[f.c], nullptr, f.n, f.n, 1, 2);
          if (!tr) apply_bytes += (int64_t)f.n * (f.n + 1) / 2 * es;
        }
        flush(fwd);
        // Q1: park z[s]; w[s][:r] = Q_c^T z[s]  (identity copy when unsparsified)
        for (auto& f : R.fa) {
          if (!keep(l, f.c)) continue;
          if (f.sparsified) {
            task(F->park_b + f.park_b_off, nullptr, nullptr, nullptr, nullptr, (T)1, f.n);
            term(nullptr, z, R.d_slots[f.c], nullptr, f.n, f.n, 0, 0);
            if (f.r > 0) {
              task(w, R.d_slots[f.c], nullptr, nullptr, F->park_c + f.park_c_off, (T)1, f.r);
              term(f.Q, z, R.d_slots[f.c], nullptr, f.n, f.n, 1, 0);
              if (!tr) apply_bytes += (int64_t)f.n * f.r * es;
            }
          } else {
            task(w, R.d_slots[f.c], nullptr, nullptr, nullptr, (T)1, f.n);
            term(nullptr, z, R.d_slots[f.c], nullptr, f.n, f.n, 0, 0);
          }
        }
        flush(fwd);
      }
    }
    for (int l = D; l >= 0; --l) {
      LevelRec<T>& R = recs[l];
      std::vector<GvTask<T>> tk;
      std::vector<GvTerm<T>> tm;
      auto task = [&](T* y, const int* yidx, const T* base, const int* bidx, T* y2, T alpha, int m) {
        tk.push_back({y, yidx, base, bidx, y2, alpha, m, (int)tm.size(), (int)tm.size()});
      };
      auto term = [&](const T* M, const T* x, const int* xidx, const T* xsub, int ld, int k, int trans, int tri) {
        tm.push_back({M, x, xidx, xsub, ld, k, trans, tri});
        tk.back().t1 = (int)tm.size();
      };
      auto flush = [&](std::vector<Phase>& dst) {
        Phase ph = build(tk, tm);
        if (ph.ntiles) dst.push_back(ph);
        tk.clear();
        tm.clear();
      };
      if (l < D) {
        // Q2: z[s] = park_b + Q_c (w[s][:r] - park_c)
        for (auto& f : R.fa) {
          if (!keep(l, f.c)) continue;
          task(z, R.d_slots[f.c], f.sparsified ? F->park_b + f.park_b_off : nullptr, nullptr, nullptr, (T)1, f.n);
          if (f.sparsified) {
            if (f.r > 0) {
              term(f.Q, w, R.d_slots[f.c], F->park_c + f.park_c_off, f.n, f.r, 0, 0);
              if (!tr) apply_bytes += (int64_t)f.n * f.r * es;
            }
          } else {
            term(nullptr, w, R.d_slots[f.c], nullptr, f.n, f.n, 0, 0);
          }
        }
        flush(bwd);
        // S2: w[s] = SU z[s]   (transpose: w[P s] = SL^T z[s])
        for (size_t q = 0; q < R.fa.size(); ++q) {
          auto& f = R.fa[q];
          if (!keep(l, f.c)) continue;
          if (!tr) {
            task(w, R.d_slots[f.c], nullptr, nullptr, nullptr, (T)1, f.n);
            term(f.SU, z, R.d_slots[f.c], nullptr, f.n, f.n, 0, 2);
            apply_bytes += (int64_t)f.n * (f.n + 1) / 2 * es;
          } else {
            task(w, fa_ps[l][q], nullptr, nullptr, nullptr, (T)1, f.n);
            term(f.SL, z, R.d_slots[f.c], nullptr, f.n, f.n, 1, 1);
          }
        }
        flush(bwd);
      }
      // neighbour map
      if (!tr) {
        // E3a: z[s] -= sum_b Y_sb w[b];  E3b: w[s] = U^-1 z[s]
        for (auto& in : R.in) {
          if (in.nbr.empty() || !keep(l, in.c)) continue;
          task(z, R.d_slots[in.c], z, R.d_slots[in.c], nullptr, (T)-1, in.n);
          for (size_t t = 0; t < in.nbr.size(); ++t) {
            term(in.Y[t], w, R.d_slots[in.nbr[t]], nullptr, in.n, R.n[in.nbr[t]], 0, 0);
            apply_bytes += (int64_t)in.n * R.n[in.nbr[t]] * es;
          }
        }
        flush(bwd);
        for (auto& in : R.in) {
          if (!keep(l, in.c)) continue;
          task(w, R.d_slots[in.c], nullptr, nullptr, nullptr, (T)1, in.n);
          term(in.Uinv, z, R.d_slots[in.c], nullptr, in.n, in.n, 0, 2);
          apply_bytes += (int64_t)in.n * (in.n + 1) / 2 * es;
        }
        flush(bwd);
      } else {
        // E2^T: z[s] -= sum_b X_bs^T w[b];  E1^T: w[P s] = L^-T z[s]
        for (auto& in : R.in) {
          if (in.nbr.empty() || !keep(l, in.c)) continue;
          task(z, R.d_slots[in.c], z, R.d_slots[in.c], nullptr, (T)-1, in.n);
          for (size_t t = 0; t < in.nbr.size(); ++t)
            term(in.X[t], w, R.d_slots[in.nbr[t]], nullptr, R.n[in.nbr[t]], R.n[in.nbr[t]], 1, 0);
        }
        flush(bwd);
        for (size_t q = 0; q < R.in.size(); ++q) {
          auto& in = R.in[q];
          if (!keep(l, in.c)) continue;
          task(w, R.d_pslots[q], nullptr, nullptr, nullptr, (T)1, in.n);
          term(in.Linv, z, R.d_slots[in.c], nullptr, in.n, in.n, 1, 1);
        }
        flush(bwd);
      }
    }
  }
  };
  F->progs.clear();
  {
    auto pg = std::make_unique<Program<T>>();
    pg->off = 0;
    pg->N = F->N;
    build_prog(*pg, [](int, int) { return true; });
    F->progs.push_back(std::move(pg));
  }
  if (nsys > 1)
    for (int q = 0; q < nsys; ++q) {
      auto pg = std::make_unique<Program<T>>();
      pg->off = (int)sysDof0(q);
      pg->N = sysK(q) * sysB(q);
      build_prog(*pg, [&P, q](int l, int c) { return P.system_of(l, c) == q; });
      F->sys_stats[q].factor_bytes = pg->bytes;
      F->progs.push_back(std::move(pg));
    }

  S.factor_bytes = F->progs[0]->bytes;
  mark(7);
  S.t_host_ms = now_ms() - t_begin;
  S.t_wait_ms = t_wait;
  for (int i = 0; i < 8; ++i) S.t_host_phase_ms[i] = ph_acc[i];
  if (pm.err) return SPAND_ERR_NOMEM;
  SPAND_CUDA_TRY(cudaGetLastError());
  SPAND_CUDA_TRY(sync_st());
  return SPAND_OK;
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* a, Tout* b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (Tout)a[i];
}

template <typename T>
static void gemv_attr() {
  static std::atomic<uint64_t> attr{0};
  once_per_device(attr, [] {
    set_dyn_smem((const void*)k_gemv<T>, kGemvSmemMax);
  });
}

template <typename T>
static int run_phases(const std::vector<typename ApplyProg<T>::Phase>& ph, cudaStream_t st, bool capturing = false) {
  gemv_attr<T>();
  if (!capturing) note_launch(ph.size());
  for (auto& p : ph) {
    const size_t sm = (size_t)std::max(p.kmax, 1) * sizeof(T);
    k_gemv<T><<<p.ntiles, 256, sm, st>>>(p.tasks, p.terms, p.tiles);
  }
  return SPAND_OK;
}

// The phase launches of one sweep pair never change for a factor, so they are
// captured once per direction into a CUDA graph and replayed; the conversions
// of the caller's r and z stay outside the graph.  When the caller's stream is
// itself being captured, or when `direct` is set (the caller may not allocate,
// and building a graph does), the phases are launched directly.
template <typename T>
int apply_impl(FactorT<T>* F, Program<T>& pg, const double* r, double* zout, int transpose, cudaStream_t st,
               bool direct) {
  const int N = pg.N;
  T* w = F->w + pg.off;
  const unsigned g = (unsigned)std::max(1, std::min(4096, (N + 255) / 256));
  note_launch();
  k_convert<double, T><<<g, 256, 0, st>>>(r, w, N);
  const int d = transpose ? 1 : 0;
  const auto& fwd = transpose ? pg.prog.tfwd : pg.prog.fwd;
  const auto& bwd = transpose ? pg.prog.tbwd : pg.prog.bwd;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SPAND_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone || direct) {
    run_phases<T>(fwd, st);
    run_phases<T>(bwd, st);
  } else {
    if (!pg.graph[d]) {
      // a private stream for the capture keeps the caller's stream untouched
      cudaStream_t cap;
      SPAND_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      gemv_attr<T>();            // function attributes are not captured: set them first
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        run_phases<T>(fwd, cap, true);
        run_phases<T>(bwd, cap, true);
        ok = cudaStreamEndCapture(cap, &graph) == cudaSuccess && graph;
      }
      if (ok) ok = cudaGraphInstantiate(&pg.graph[d], graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      cudaGetLastError();
      if (!ok) pg.graph[d] = nullptr;
    }
    if (pg.graph[d]) {
      note_launch(fwd.size() + bwd.size());
      SPAND_CUDA_TRY(cudaGraphLaunch(pg.graph[d], st));
    } else {
      run_phases<T>(fwd, st);
      run_phases<T>(bwd, st);
    }
  }
  if (zout) {                   // zout == nullptr: the caller reads the factor's vector itself
    note_launch();
    k_convert<T, double><<<g, 256, 0, st>>>(w, zout, N);
  }
  SPAND_CUDA_TRY(cudaGetLastError());
  return SPAND_OK;
}

template <typename T>
static int max_kmax(FactorT<T>* F) {
  int k = 1;
  for (auto& pg : F->progs)
    for (auto* v : {&pg->prog.fwd, &pg->prog.bwd, &pg->prog.tfwd, &pg->prog.tbwd})
      for (auto& p : *v) k = std::max(k, p.kmax);
  return k;
}

// factorization of the union plan U (one system or several) into F
static int factor_any(const Plan& U, const bsr_matrix* const* As, double eps, int precision, cudaStream_t stream,
                      std::shared_ptr<FactorBase>& out) {
  int st;
  if (precision == SPAND_FP64) {
    auto F = std::make_shared<FactorT<double>>();
    out = F;
    st = factor_impl<double>(U, As, eps, precision, F.get(), stream);
    if (st == SPAND_OK && (size_t)max_kmax(F.get()) * sizeof(double) > kGemvSmemMax) st = SPAND_ERR_UNSUPPORTED;
  } else {
    auto F = std::make_shared<FactorT<float>>();
    out = F;
    st = factor_impl<float>(U, As, eps, precision, F.get(), stream);
    if (st == SPAND_OK && (size_t)max_kmax(F.get()) * sizeof(float) > kGemvSmemMax) st = SPAND_ERR_UNSUPPORTED;
  }
  if (st != SPAND_OK) {
    cudaStreamSynchronize(stream);
    out->mem.free_all();
    cudaStreamSynchronize(stream);
    out.reset();
  }
  return st;
}

}  // namespace spand

struct spand_factor_s {
  std::shared_ptr<spand::FactorBase> impl;   // shared by the handles of one batched factorization
  int prog = 0;                              // 0: every system; 1 + q: system q
};

namespace spand {
int factor_apply(spand_factor_t F, const double* r, double* z, int transpose, cudaStream_t st, bool direct) {
  return F->impl->apply(F->prog, r, z, transpose, st, direct);
}
int factor_size(spand_factor_t F) { return F->impl->prog_size(F->prog); }
int factor_apply_slot(spand_factor_t F, const double* r, int transpose, cudaStream_t st, bool direct, const void** w,
                      int* w_is_float) {
  return F->impl->apply_slot(F->prog, r, transpose, st, direct, w, w_is_float);
}
}  // namespace spand

extern "C" {

int spand_factor(spand_plan_t plan, const bsr_matrix* A, double eps, int precision, spand_factor_t* out,
                 cudaStream_t stream) {
  if (!plan || !A || !out || !A->row_ptr || !A->col || !A->val) return SPAND_ERR_ARG;
  *out = nullptr;
  if (A->K != plan->P.K || A->B != plan->P.B || !(eps >= 0.0)) return SPAND_ERR_ARG;
  if (precision != SPAND_FP64 && precision != SPAND_MIXED) return SPAND_ERR_ARG;
  spand_factor_s* f = new (std::nothrow) spand_factor_s();
  if (!f) return SPAND_ERR_NOMEM;
  const int st = spand::factor_any(plan->P, &A, eps, precision, stream, f->impl);
  if (st != SPAND_OK) {
    delete f;
    return st;
  }
  *out = f;
  return SPAND_OK;
}

int spand_factor_batched(int nsys, const spand_plan_t* plans, const bsr_matrix* A, double eps, int precision,
                         spand_factor_t* out, cudaStream_t stream) {
  if (nsys <= 0 || !plans || !A || !out || !(eps >= 0.0)) return SPAND_ERR_ARG;
  if (precision != SPAND_FP64 && precision != SPAND_MIXED) return SPAND_ERR_ARG;
  for (int q = 0; q < nsys; ++q) out[q] = nullptr;
  std::vector<const spand::Plan*> ps(nsys);
  std::vector<const bsr_matrix*> as(nsys);
  for (int q = 0; q < nsys; ++q) {
    if (!plans[q] || !A[q].row_ptr || !A[q].col || !A[q].val) return SPAND_ERR_ARG;
    if (A[q].K != plans[q]->P.K || A[q].B != plans[q]->P.B) return SPAND_ERR_ARG;
    ps[q] = &plans[q]->P;
    as[q] = &A[q];
  }
  spand::Plan U;
  int st = spand::build_union_plan(ps, U);
  if (st != SPAND_OK) return st;
  std::shared_ptr<spand::FactorBase> impl;
  st = spand::factor_any(U, as.data(), eps, precision, stream, impl);
  if (st != SPAND_OK) return st;
  for (int q = 0; q < nsys; ++q) {
    spand_factor_s* f = new (std::nothrow) spand_factor_s();
    if (!f) {
      for (int k = 0; k < q; ++k) {
        delete out[k];
        out[k] = nullptr;
      }
      cudaStreamSynchronize(stream);
      impl->mem.free_all();
      cudaStreamSynchronize(stream);
      return SPAND_ERR_NOMEM;
    }
    f->impl = impl;
    f->prog = nsys > 1 ? 1 + q : 0;
    out[q] = f;
  }
  return SPAND_OK;
}

int spand_factor_destroy(spand_factor_t F) {
  if (!F) return SPAND_OK;
  if (F->impl && F->impl.use_count() == 1) {
    // the last handle of the factorization releases its device memory
    cudaDeviceSynchronize();
    F->impl->mem.free_all();
    cudaDeviceSynchronize();
  }
  delete F;
  return SPAND_OK;
}

int spand_factor_stats(spand_factor_t F, spand_stats* st) {
  if (!F || !st) return SPAND_ERR_ARG;
  const spand::FactorBase& B = *F->impl;
  if (F->prog == 0) {
    *st = B.stats;
  } else {
    // the system's own ranks and bytes; phase times and flops are those of the
    // whole batched factorization
    *st = B.sys_stats[F->prog - 1];
    st->factor_flops = B.stats.factor_flops;
    st->t_rrqr_ms = B.stats.t_rrqr_ms;
    st->rrqr_bytes = B.stats.rrqr_bytes;
    st->rrqr_launches = B.stats.rrqr_launches;
    st->t_elim_gemm_ms = B.stats.t_elim_gemm_ms;
    st->elim_gemm_flops = B.stats.elim_gemm_flops;
    st->elim_gemm_launches = B.stats.elim_gemm_launches;
    memcpy(st->t_rrqr_level_ms, B.stats.t_rrqr_level_ms, sizeof(st->t_rrqr_level_ms));
    memcpy(st->rrqr_bytes_level, B.stats.rrqr_bytes_level, sizeof(st->rrqr_bytes_level));
    memcpy(st->rrqr_form_count, B.stats.rrqr_form_count, sizeof(st->rrqr_form_count));
    st->rrqr_stream_bytes = B.stats.rrqr_stream_bytes;
    memcpy(st->rrqr_stream_bytes_level, B.stats.rrqr_stream_bytes_level, sizeof(st->rrqr_stream_bytes_level));
  }
  return SPAND_OK;
}

uint64_t spand_kernel_launches(void) { return spand::g_kernel_launches.load(); }

int spand_apply(spand_factor_t F, const double* r, double* z, int transpose, cudaStream_t stream) {
  if (!F || !r || !z || r == z) return SPAND_ERR_ARG;
  return spand::factor_apply(F, r, z, transpose, stream, false);
}

}  // extern "C"
