// Nested-dissection analysis of the structured O-grid (host, integer only).
//
// Sec. 2.2.1 (interiors, separators and interfaces per level; merge) and
// Sec. 3.3 (elements mapped to integer (i, j) and split by recursive
// bisection).  The partition rules fixed here:
//   - root: the periodic ring, separated by the radial lines j = 0 and
//     j = n_theta/2; its children are the two j-ranges between them;
//   - below the root a box is split across its longer extent (ties split j)
//     at lo + (n-1)/2; a box is a leaf at depth D or when its longer extent < 3;
//   - leaves are eliminated at level 0, the separator of a depth-d box at D-d;
//   - level-0 interfaces group separator elements by (separator, set of
//     depth-D boxes touched by their face neighbours); the clusters surviving
//     level l are merged by (separator, union of the depth-(D-l-1) boxes their
//     elements touch), children kept in order;
//   - clusters are ordered by (node preorder id, key); elements ascend.
#include <algorithm>
#include <cmath>
#include <new>
#include <set>

#include "internal.h"

namespace spand {

namespace {

struct Builder {
  Plan& P;
  explicit Builder(Plan& p) : P(p) {}

  int new_node(int depth, int parent, bool leaf) {
    P.depth.push_back(depth);
    P.parent.push_back(parent);
    P.is_leaf.push_back(leaf ? 1 : 0);
    P.node_elems.emplace_back();
    return (int)P.depth.size() - 1;
  }

  void own(int v, std::vector<int> el) {
    std::sort(el.begin(), el.end());
    for (int e : el) P.owner[e] = v;
    P.node_elems[v] = std::move(el);
  }

  void rec(int i0, int i1, int j0, int j1, int depth, int parent) {
    const int ni = i1 - i0, nj = j1 - j0, nt = P.n_theta;
    if (depth == P.D || std::max(ni, nj) < 3) {
      int v = new_node(depth, parent, true);
      std::vector<int> el;
      for (int i = i0; i < i1; ++i)
        for (int j = j0; j < j1; ++j) el.push_back(i * nt + j);
      own(v, el);
      return;
    }
    int v = new_node(depth, parent, false);
    std::vector<int> el;
    if (nj >= ni) {
      int js = j0 + (nj - 1) / 2;
      for (int i = i0; i < i1; ++i) el.push_back(i * nt + js);
      own(v, el);
      rec(i0, i1, j0, js, depth + 1, v);
      rec(i0, i1, js + 1, j1, depth + 1, v);
    } else {
      int is = i0 + (ni - 1) / 2;
      for (int j = j0; j < j1; ++j) el.push_back(is * nt + j);
      own(v, el);
      rec(i0, is, j0, j1, depth + 1, v);
      rec(is + 1, i1, j0, j1, depth + 1, v);
    }
  }
};

void neighbours(const Plan& P, int e, int out[4], int& n) {
  const int nt = P.n_theta, nr = P.n_r;
  const int i = e / nt, j = e % nt;
  n = 0;
  out[n++] = i * nt + (j + 1) % nt;
  out[n++] = i * nt + (j + nt - 1) % nt;
  if (i > 0) out[n++] = e - nt;
  if (i < nr - 1) out[n++] = e + nt;
}

// depth-k box holding element e, or -1
int box_of(const Plan& P, int e, int k) {
  int v = P.owner[e];
  if (P.depth[v] >= k) {
    while (P.depth[v] > k) v = P.parent[v];
    return v;
  }
  return P.is_leaf[v] ? v : -1;
}

std::vector<int> adj_boxes(const Plan& P, const std::vector<int>& elems, int k) {
  std::set<int> s;
  int nb[4], n;
  for (int e : elems) {
    neighbours(P, e, nb, n);
    for (int t = 0; t < n; ++t) {
      int b = box_of(P, nb[t], k);
      if (b >= 0) s.insert(b);
    }
  }
  return std::vector<int>(s.begin(), s.end());
}

}  // namespace

int build_plan(int n_theta, int n_r, int B, int D, Plan& P) {
  if (n_theta < 4 || n_r < 1 || B <= 0 || D < 1 || D > 30) return SPAND_ERR_ARG;
  P = Plan();
  P.n_theta = n_theta;
  P.n_r = n_r;
  P.K = n_theta * n_r;
  P.B = B;
  P.D = D;
  P.owner.assign(P.K, -1);
  Builder b(P);
  const int J2 = n_theta / 2;
  int root = b.new_node(0, -1, false);
  std::vector<int> sep;
  for (int i = 0; i < n_r; ++i) {
    sep.push_back(i * n_theta);
    sep.push_back(i * n_theta + J2);
  }
  b.own(root, sep);
  b.rec(0, n_r, 1, J2, 1, root);
  b.rec(0, n_r, J2 + 1, n_theta, 1, root);
  for (int e = 0; e < P.K; ++e)
    if (P.owner[e] < 0) return SPAND_ERR_ARG;
  const int nn = (int)P.depth.size();
  P.level.resize(nn);
  for (int v = 0; v < nn; ++v) P.level[v] = P.is_leaf[v] ? 0 : D - P.depth[v];

  // ---- level-0 clusters
  std::map<std::pair<int, std::vector<int>>, std::vector<int>> groups;
  for (int v = 0; v < nn; ++v)
    if (P.is_leaf[v]) groups[{v, {}}] = P.node_elems[v];
  for (int e = 0; e < P.K; ++e) {
    int v = P.owner[e];
    if (P.is_leaf[v]) continue;
    groups[{v, adj_boxes(P, {e}, D)}].push_back(e);
  }
  P.lv.resize(D + 1);
  for (auto& g : groups) {
    Cluster c;
    c.node = g.first.first;
    c.key = g.first.second;
    c.elems = g.second;
    std::sort(c.elems.begin(), c.elems.end());
    c.interior = (P.level[c.node] == 0);
    P.lv[0].cl.push_back(std::move(c));
  }
  // ---- levels 1..D by merging the survivors
  for (int l = 0; l < D; ++l) {
    LevelInfo& L = P.lv[l];
    L.surv.clear();
    for (int i = 0; i < (int)L.cl.size(); ++i)
      if (!L.cl[i].interior) L.surv.push_back(i);
    std::map<std::pair<int, std::vector<int>>, std::vector<int>> g2;
    for (int ci = 0; ci < (int)L.surv.size(); ++ci) {
      const Cluster& c = L.cl[L.surv[ci]];
      g2[{c.node, adj_boxes(P, c.elems, D - l - 1)}].push_back(ci);
    }
    L.parent.assign(L.surv.size(), -1);
    for (auto& g : g2) {
      Cluster c;
      c.node = g.first.first;
      c.key = g.first.second;
      c.children = g.second;
      for (int ci : c.children) {
        const auto& el = L.cl[L.surv[ci]].elems;
        c.elems.insert(c.elems.end(), el.begin(), el.end());
        L.parent[ci] = (int)P.lv[l + 1].cl.size();
      }
      std::sort(c.elems.begin(), c.elems.end());
      c.interior = (P.level[c.node] == l + 1);
      P.lv[l + 1].cl.push_back(std::move(c));
    }
  }
  for (const Cluster& c : P.lv[D].cl)
    if (!c.interior) return SPAND_ERR_ARG;

  // ---- symbolic block pattern with fill-in
  std::vector<int> cl_of, pos;
  level0_positions(P, cl_of, pos);
  std::set<std::pair<int, int>> pat;
  int nb[4], n;
  for (int e = 0; e < P.K; ++e) {
    int a = cl_of[e];
    pat.insert({a, a});
    neighbours(P, e, nb, n);
    for (int t = 0; t < n; ++t) pat.insert({a, cl_of[nb[t]]});
  }
  for (int l = 0; l <= D; ++l) {
    LevelInfo& L = P.lv[l];
    L.pattern.assign(pat.begin(), pat.end());
    const int nc = (int)L.cl.size();
    std::vector<std::vector<int>> nbr(nc);
    for (auto& pr : pat)
      if (pr.first != pr.second) nbr[pr.first].push_back(pr.second);
    std::set<std::pair<int, int>> after;
    for (auto& pr : pat)
      if (!L.cl[pr.first].interior && !L.cl[pr.second].interior) after.insert(pr);
    for (int s = 0; s < nc; ++s) {
      if (!L.cl[s].interior) continue;
      for (int a : nbr[s])
        for (int c : nbr[s]) after.insert({a, c});
    }
    L.after.assign(after.begin(), after.end());
    if (l == D) break;
    if (L.surv.empty()) {
      for (int i = 0; i < nc; ++i)
        if (!L.cl[i].interior) L.surv.push_back(i);
    }
    std::vector<int> to_surv(nc, -1);
    for (int k = 0; k < (int)L.surv.size(); ++k) to_surv[L.surv[k]] = k;
    pat.clear();
    for (auto& pr : after) pat.insert({L.parent[to_surv[pr.first]], L.parent[to_surv[pr.second]]});
  }
  return SPAND_OK;
}

int build_union_plan(const std::vector<const Plan*>& ps, Plan& U) {
  if (ps.empty()) return SPAND_ERR_ARG;
  U = Plan();
  U.nsys = (int)ps.size();
  int64_t dof = 0;
  int64_t K = 0;
  for (const Plan* p : ps) {
    if (!p || p->lv.size() != (size_t)p->D + 1) return SPAND_ERR_ARG;
    U.sys_elem0.push_back((int)K);
    U.sys_dof0.push_back(dof);
    U.sys_K.push_back(p->K);
    U.sys_B.push_back(p->B);
    U.sys_D.push_back(p->D);
    K += p->K;
    dof += (int64_t)p->K * p->B;
    U.D = std::max(U.D, p->D);
  }
  if (K > INT32_MAX || dof > INT32_MAX) return SPAND_ERR_UNSUPPORTED;
  U.K = (int)K;
  U.B = ps[0]->B;
  for (const Plan* p : ps)
    if (p->B != U.B) U.B = 0;   // mixed block sizes: per-system sys_B
  U.lv.resize(U.D + 1);
  U.sys_of.resize(U.D + 1);
  // per level: offset of each system's clusters and surviving clusters
  std::vector<std::vector<int>> c_off(U.D + 2, std::vector<int>(ps.size(), 0));
  std::vector<std::vector<int>> s_off(U.D + 2, std::vector<int>(ps.size(), 0));
  for (int l = 0; l <= U.D; ++l) {
    int cc = 0, sc = 0;
    for (size_t s = 0; s < ps.size(); ++s) {
      c_off[l][s] = cc;
      s_off[l][s] = sc;
      if (l <= ps[s]->D) {
        cc += (int)ps[s]->lv[l].cl.size();
        sc += (int)ps[s]->lv[l].surv.size();
      }
    }
  }
  int node0 = 0;
  std::vector<int> node_off(ps.size());
  for (size_t s = 0; s < ps.size(); ++s) {
    node_off[s] = node0;
    node0 += (int)ps[s]->depth.size();
  }
  for (int l = 0; l <= U.D; ++l) {
    LevelInfo& L = U.lv[l];
    for (size_t s = 0; s < ps.size(); ++s) {
      if (l > ps[s]->D) continue;
      const LevelInfo& Ls = ps[s]->lv[l];
      const int co = c_off[l][s];
      for (const Cluster& c : Ls.cl) {
        Cluster u = c;
        u.node = c.node + node_off[s];
        for (int& e : u.elems) e += U.sys_elem0[s];
        for (int& ch : u.children) ch += s_off[l > 0 ? l - 1 : 0][s];
        L.cl.push_back(std::move(u));
        U.sys_of[l].push_back((int)s);
      }
      for (int v : Ls.surv) L.surv.push_back(v + co);
      for (auto& pr : Ls.pattern) L.pattern.push_back({pr.first + co, pr.second + co});
      for (auto& pr : Ls.after) L.after.push_back({pr.first + co, pr.second + co});
      for (int v : Ls.parent) {
        if (l + 1 > ps[s]->D) return SPAND_ERR_ARG;
        L.parent.push_back(v + c_off[l + 1][s]);
      }
    }
  }
  return SPAND_OK;
}

void level0_positions(const Plan& P, std::vector<int>& cl_of, std::vector<int>& pos_in) {
  cl_of.assign(P.K, -1);
  pos_in.assign(P.K, -1);
  const auto& cl = P.lv[0].cl;
  for (int c = 0; c < (int)cl.size(); ++c)
    for (int k = 0; k < (int)cl[c].elems.size(); ++k) {
      cl_of[cl[c].elems[k]] = c;
      pos_in[cl[c].elems[k]] = k;
    }
}

}  // namespace spand

extern "C" {

int spand_analyze(int n_theta, int n_r, int B, int depth_D, spand_plan_t* out) {
  if (!out) return SPAND_ERR_ARG;
  *out = nullptr;
  if (n_theta < 4 || n_r < 1 || B <= 0) return SPAND_ERR_ARG;
  int D = depth_D;
  if (D <= 0) {
    double K = (double)n_theta * n_r;
    D = std::max(1, (int)std::ceil(std::log2(K / 32.0)));
  }
  spand_plan_s* p = new (std::nothrow) spand_plan_s();
  if (!p) return SPAND_ERR_NOMEM;
  int st = spand::build_plan(n_theta, n_r, B, D, p->P);
  if (st != SPAND_OK) {
    delete p;
    return st;
  }
  *out = p;
  return SPAND_OK;
}

int spand_plan_destroy(spand_plan_t plan) {
  delete plan;
  return SPAND_OK;
}

static int64_t table_length(const spand::Plan& P) {
  int64_t n = 0;
  for (const auto& L : P.lv) {
    n += 1;
    for (const auto& c : L.cl) n += 5 + (int64_t)c.key.size() + (int64_t)c.elems.size() + (int64_t)c.children.size();
  }
  return n;
}

int spand_plan_sizes(spand_plan_t plan, int* K, int* D, int* n_nodes, int64_t* table_len) {
  if (!plan) return SPAND_ERR_ARG;
  if (K) *K = plan->P.K;
  if (D) *D = plan->P.D;
  if (n_nodes) *n_nodes = (int)plan->P.depth.size();
  if (table_len) *table_len = table_length(plan->P);
  return SPAND_OK;
}

int spand_plan_export(spand_plan_t plan, int* owner, int* node_level, int* table) {
  if (!plan) return SPAND_ERR_ARG;
  const spand::Plan& P = plan->P;
  if (owner)
    for (int e = 0; e < P.K; ++e) owner[e] = P.owner[e];
  if (node_level)
    for (size_t v = 0; v < P.level.size(); ++v) node_level[v] = P.level[v];
  if (table) {
    int64_t k = 0;
    for (const auto& L : P.lv) {
      table[k++] = (int)L.cl.size();
      for (const auto& c : L.cl) {
        table[k++] = c.node;
        table[k++] = c.interior ? 1 : 0;
        table[k++] = (int)c.key.size();
        for (int x : c.key) table[k++] = x;
        table[k++] = (int)c.elems.size();
        for (int x : c.elems) table[k++] = x;
        table[k++] = (int)c.children.size();
        for (int x : c.children) table[k++] = x;
      }
    }
  }
  return SPAND_OK;
}

const char* spand_status_string(int status) {
  switch (status) {
    case SPAND_OK: return "ok";
    case SPAND_ERR_ARG: return "invalid argument";
    case SPAND_ERR_NOMEM: return "out of memory";
    case SPAND_ERR_ZERO_PIVOT: return "zero pivot in block LU";
    case SPAND_ERR_CHOLQR: return "CholQR breakdown (Gram matrix not positive definite)";
    case SPAND_ERR_NONFINITE: return "non-finite value";
    case SPAND_ERR_NOT_CONVERGED: return "GMRES did not converge";
    case SPAND_ERR_CUDA: return "CUDA error";
    case SPAND_ERR_UNSUPPORTED: return "unsupported configuration";
    case SPAND_ERR_SCRATCH: return "problem larger than the fixed scratch of the no-allocation entry point";
  }
  return "unknown status";
}

}  // extern "C"
