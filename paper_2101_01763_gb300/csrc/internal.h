// Internal declarations shared by the library's translation units.
#pragma once
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/spand_gb300.h"

namespace spand {

// With SPAND_DEBUG=1 in the environment, a failing CUDA call is reported on
// stderr with its source location and the runtime's error string.
void report_cuda_error(cudaError_t e, const char* expr, const char* file, int line);
// SPAND_DEBUG level from the environment (0 when unset); 2 also prints the
// shapes, placements, times and ranks of every level's RRQR problems.
int debug_level();

#define SPAND_CUDA_TRY(call)                                   \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) {                                  \
      spand::report_cuda_error(e__, #call, __FILE__, __LINE__); \
      return SPAND_ERR_CUDA;                                   \
    }                                                          \
  } while (0)

#define SPAND_TRY(call)              \
  do {                               \
    int s__ = (call);                \
    if (s__ != SPAND_OK) return s__; \
  } while (0)

// Runs f() once per device of the calling thread (kernel attributes are
// per-device settings); setting them twice from two threads is harmless.
template <typename F>
inline void once_per_device(std::atomic<uint64_t>& done, F f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    f();
    return;
  }
  const uint64_t bit = uint64_t(1) << dev;
  if (done.load(std::memory_order_acquire) & bit) return;
  f();
  done.fetch_or(bit, std::memory_order_release);
}

// Kernel launches issued by the library since it was loaded (a CUDA-graph
// replay adds the kernels of the graph); read by spand_kernel_launches().
extern std::atomic<uint64_t> g_kernel_launches;
// The library's stream-ordered memory pool (factorizations, solver scratch),
// one per device, separate from the device's default pool: its release threshold is unbounded, so the
// memory a factorization frees stays mapped in the pool and the next
// factorization (and the next level of this one) reuses it instead of mapping
// gigabytes again after every synchronisation (the default pool returns freed
// memory to the system at each one).  The pool keeps the largest working set
// it has served until the process ends.
inline cudaMemPool_t factor_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    pool = nullptr;                      // the device's default pool then
  } else {
    uint64_t keep = ~uint64_t(0);
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
  }
  pools[dev] = pool;
  return pool;
}

inline cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = factor_pool();
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

inline void note_launch(uint64_t n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// Sets the kernel's dynamic shared-memory limit to min(want, opt-in limit of
// the device - the kernel's static shared memory) and returns the value set,
// or -1 when a query fails.  A failing runtime call here is cleared, so it
// cannot surface later as the error of an unrelated launch.
inline long long set_dyn_smem(const void* func, size_t want) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  long long v = (long long)optin - (long long)fa.sharedSizeBytes;
  if ((long long)want < v) v = (long long)want;
  if (v < 0) return -1;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return v;
}

// ----------------------------------------------------------------- analysis
struct Cluster {
  int node = -1;
  std::vector<int> key;
  std::vector<int> elems;     // sorted element ids (union over children)
  std::vector<int> children;  // indices into the surviving clusters of level l-1
  bool interior = false;
};

struct LevelInfo {
  std::vector<Cluster> cl;
  std::vector<int> surv;                      // indices of non-interior clusters
  std::vector<std::pair<int, int>> pattern;   // blocks present before elimination
  std::vector<std::pair<int, int>> after;     // blocks after elimination + fill (interfaces only)
  std::vector<int> parent;                    // surviving cluster -> index in level l+1
};

struct Plan {
  int n_theta = 0, n_r = 0, K = 0, B = 0, D = 0;
  std::vector<int> depth, parent, is_leaf, level;
  std::vector<std::vector<int>> node_elems;
  std::vector<int> owner;
  std::vector<LevelInfo> lv;  // D + 1 levels
  // Disjoint union of several systems (batched factorization).  Levels are
  // aligned from the bottom (level l of every system with D_s >= l forms
  // union level l); a system whose top level D_s < D has no clusters above
  // it.  For one system: nsys = 1, sys_of empty, sys_* hold that system.
  int nsys = 1;
  std::vector<std::vector<int>> sys_of;   // per level: cluster -> system
  std::vector<int> sys_elem0, sys_K, sys_B, sys_D;
  std::vector<int64_t> sys_dof0;          // first unknown of each system
  int64_t n_dof() const { return sys_dof0.empty() ? (int64_t)K * B : sys_dof0.back() + (int64_t)sys_K.back() * sys_B.back(); }
  int system_of(int l, int c) const { return sys_of.empty() ? 0 : sys_of[l][c]; }
};

int build_plan(int n_theta, int n_r, int B, int D, Plan& P);
// union of the given plans (each keeps its own block size)
int build_union_plan(const std::vector<const Plan*>& ps, Plan& U);

// position of element e inside its level-0 cluster and that cluster's index
void level0_positions(const Plan& P, std::vector<int>& cl_of, std::vector<int>& pos_in);

}  // namespace spand

struct spand_plan_s {
  spand::Plan P;
};
