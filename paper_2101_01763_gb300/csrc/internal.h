// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/spand_gb300.h"

namespace spand {

#define SPAND_CUDA_TRY(call)                                   \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) return SPAND_ERR_CUDA;             \
  } while (0)

#define SPAND_TRY(call)              \
  do {                               \
    int s__ = (call);                \
    if (s__ != SPAND_OK) return s__; \
  } while (0)

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
};

int build_plan(int n_theta, int n_r, int B, int D, Plan& P);

// position of element e inside its level-0 cluster and that cluster's index
void level0_positions(const Plan& P, std::vector<int>& cl_of, std::vector<int>& pos_in);

}  // namespace spand

struct spand_plan_s {
  spand::Plan P;
};
