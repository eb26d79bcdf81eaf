// spaND factorization and apply on the GPU (Sec. 2.2.1, Eqs. 9-11).
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
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "dense.cuh"
#include "gemv.cuh"
#include "internal.h"

namespace spand {

// largest dynamic shared memory any kernel here asks for (x vectors, reflectors)
constexpr size_t kGemvSmemMax = 200 * 1024;

// ------------------------------------------------------------------ device memory
struct DevMem {
  std::vector<void*> ptrs;
  cudaStream_t st = nullptr;
  int err = 0;
  template <typename X>
  X* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    if (cudaMallocAsync(&p, n * sizeof(X), st) != cudaSuccess) {
      err = 1;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<X*>(p);
  }
  template <typename X>
  X* upload(const std::vector<X>& h) {
    X* d = alloc<X>(h.size());
    if (d && !h.empty() && cudaMemcpyAsync(d, h.data(), h.size() * sizeof(X), cudaMemcpyHostToDevice, st) != cudaSuccess)
      err = 1;
    return d;
  }
  void free_all() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
  }
};

// ------------------------------------------------------------------ launch helpers
template <typename T>
static void launch_gemm(DevMem& tmp, const std::vector<GemmTask<T>>& tasks, const std::vector<GemmTerm<T>>& terms,
                        cudaStream_t st) {
  std::vector<TileItem> tiles;
  for (int t = 0; t < (int)tasks.size(); ++t) {
    if (tasks[t].m <= 0 || tasks[t].n <= 0) continue;
    for (int a = 0; a < (tasks[t].m + 63) / 64; ++a)
      for (int b = 0; b < (tasks[t].n + 63) / 64; ++b) tiles.push_back({t, a, b});
  }
  if (tiles.empty()) return;
  auto* dt = tmp.upload(tasks);
  auto* dm = tmp.upload(terms);
  auto* dl = tmp.upload(tiles);
  if (tmp.err) return;
  k_gemm<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dt, dm, dl);
}

template <typename T>
static void launch_copy(DevMem& tmp, const std::vector<CopyTask<T>>& tasks, cudaStream_t st) {
  std::vector<CopyTile> tiles;
  for (int t = 0; t < (int)tasks.size(); ++t)
    for (int a = 0; a < (tasks[t].rows + 31) / 32; ++a)
      for (int b = 0; b < (tasks[t].cols + 31) / 32; ++b) tiles.push_back({t, a, b});
  if (tiles.empty()) return;
  auto* dt = tmp.upload(tasks);
  auto* dl = tmp.upload(tiles);
  if (tmp.err) return;
  k_copy_tiles<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dt, dl);
}

// row-permuted copy: dst[r, c] = src[perm[r], c]; one CTA per task
template <typename T>
__global__ void k_row_perm(const T* const* src, T* const* dst, const int* const* perm, const int* rows,
                           const int* cols) {
  const int t = blockIdx.x;
  const int n = rows[t], m = cols[t];
  const size_t tot = (size_t)n * m;
  const T* s = src[t];
  T* d = dst[t];
  const int* p = perm[t];
  for (size_t idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int r = (int)(idx % n);
    const size_t c = idx / n;
    d[r + c * n] = s[p[r] + c * n];
  }
}

template <typename T>
static void launch_row_perm(DevMem& tmp, const std::vector<const T*>& src, const std::vector<T*>& dst,
                            const std::vector<const int*>& perm, const std::vector<int>& rows,
                            const std::vector<int>& cols, cudaStream_t st) {
  if (src.empty()) return;
  auto* a = tmp.upload(src);
  auto* b = tmp.upload(dst);
  auto* c = tmp.upload(perm);
  auto* d = tmp.upload(rows);
  auto* e = tmp.upload(cols);
  if (tmp.err) return;
  k_row_perm<T><<<(unsigned)src.size(), 256, 0, st>>>(a, b, c, d, e);
}

// blocked getrf of every matrix, in place; pivots + permutations
template <typename T>
static void batched_getrf(DevMem& tmp, std::vector<MatRef<T>>& mats, int* d_flags, cudaStream_t st) {
  if (mats.empty()) return;
  int nmax = 0;
  for (auto& m : mats) nmax = std::max(nmax, m.n);
  auto* dm = tmp.upload(mats);
  if (tmp.err) return;
  for (int k0 = 0; k0 < nmax; k0 += LU_NB) {
    k_getrf_panel<T><<<(unsigned)mats.size(), 256, 0, st>>>(dm, (int)mats.size(), k0, d_flags);
    std::vector<GemmTask<T>> tasks;
    std::vector<GemmTerm<T>> terms;
    for (auto& m : mats) {
      const int n = m.n;
      if (k0 + LU_NB >= n) continue;
      const int jb = LU_NB, r = k0 + jb, rem = n - r;
      GemmTerm<T> tm{m.A + r + (size_t)k0 * n, m.A + k0 + (size_t)r * n, n, n, jb, 0, 0};
      GemmTask<T> tk{m.A + r + (size_t)r * n, n, rem, rem, (T)-1, (T)1, (int)terms.size(), (int)terms.size() + 1};
      terms.push_back(tm);
      tasks.push_back(tk);
    }
    launch_gemm(tmp, tasks, terms, st);
  }
  k_ipiv_to_perm<T><<<((unsigned)mats.size() + 127) / 128, 128, 0, st>>>(dm, (int)mats.size());
}

// L^-1 (optionally row-scaled by 1/d) and U^-1 (optionally column-scaled by d)
template <typename T>
static void batched_inverses(DevMem& tmp, const std::vector<MatRef<T>>& mats, const std::vector<T*>& Linv,
                             const std::vector<T*>& Uinv, const std::vector<const T*>& dscale, cudaStream_t st) {
  if (mats.empty()) return;
  std::vector<InvTask<T>> lt, ut;
  std::vector<int> ident_max;
  std::vector<InvTile> tiles;
  for (size_t b = 0; b < mats.size(); ++b) {
    // L^-1 unpermuted: pass the identity placement
    lt.push_back({mats[b].A, Linv[b], nullptr, dscale[b], mats[b].n});
    ut.push_back({mats[b].A, Uinv[b], nullptr, dscale[b], mats[b].n});
    for (int j0 = 0; j0 < mats[b].n; j0 += 32) tiles.push_back({(int)b, j0});
  }
  int nmax = 0;
  for (auto& m : mats) nmax = std::max(nmax, m.n);
  std::vector<int> iota(nmax);
  for (int i = 0; i < nmax; ++i) iota[i] = i;
  const int* d_iota = tmp.upload(iota);
  for (auto& t : lt) t.perm = d_iota;
  auto* dlt = tmp.upload(lt);
  auto* dut = tmp.upload(ut);
  auto* dtl = tmp.upload(tiles);
  if (tmp.err || tiles.empty()) return;
  k_inv_lower<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dlt, dtl);
  k_inv_upper<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dut, dtl);
  k_scale_rows<T><<<(unsigned)tiles.size(), 256, 0, st>>>(dlt, dtl);
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

struct FactorBase {
  virtual ~FactorBase() {}
  int precision = 0;
  int N = 0, D = 0;
  spand_stats stats{};
  DevMem mem;               // persistent device memory
};

template <typename T>
struct FactorT : FactorBase {
  T* w = nullptr;           // apply vectors (slot space)
  T* z = nullptr;
  T* park_b = nullptr;
  T* park_c = nullptr;
  ApplyProg<T> prog;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t graph_stream[2] = {nullptr, nullptr};
  ~FactorT() override {
    for (int t = 0; t < 2; ++t)
      if (graph[t]) cudaGraphExecDestroy(graph[t]);
  }
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

template <typename T>
__global__ void k_perm_slots(const int* slots, const int* perm, int* out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = slots[perm[i]];
}

template <typename T>
__global__ void k_level0_gather(const double* val, const int* row_of, const int* col, const int* cl_of,
                                const int* pos_in, const int* loc_row_ld, T* const* dst, int nnzb, int B) {
  // one CTA per BSR block; dst[k] = block origin, ld from the row cluster
  const int k = blockIdx.x;
  if (k >= nnzb) return;
  T* d = dst[k];
  const int ld = loc_row_ld[k];
  const double* s = val + (size_t)k * B * B;
  for (int idx = threadIdx.x; idx < B * B; idx += blockDim.x) {
    const int r = idx % B, c = idx / B;
    d[r + (size_t)c * ld] = (T)s[idx];
  }
}

template <typename T>
static int factor_impl(const Plan& P, const bsr_matrix* A, double eps, int precision, FactorT<T>* F,
                       cudaStream_t st) {
  const int D = P.D, B = P.B, K = P.K;
  F->N = K * B;
  F->D = D;
  F->precision = precision;
  F->mem.st = st;
  DevMem& pm = F->mem;
  spand_stats& S = F->stats;
  memset(&S, 0, sizeof(S));
  S.levels = D + 1;
  int* d_flags = pm.alloc<int>(4);
  if (pm.err) return SPAND_ERR_NOMEM;
  SPAND_CUDA_TRY(cudaMemsetAsync(d_flags, 0, 4 * sizeof(int), st));

  // ---- level-0 sizes, slots, blocks
  std::vector<int> cl_of, pos_in;
  level0_positions(P, cl_of, pos_in);
  std::vector<int> n(P.lv[0].cl.size());
  std::vector<std::vector<int>> slots(n.size());
  for (size_t c = 0; c < n.size(); ++c) {
    n[c] = (int)P.lv[0].cl[c].elems.size() * B;
    for (int e : P.lv[0].cl[c].elems)
      for (int d = 0; d < B; ++d) slots[c].push_back(e * B + d);
  }
  // arena of the current level: blocks in pattern U after
  T* arena = nullptr;
  std::map<std::pair<int, int>, size_t> boff;
  auto layout = [&](const LevelInfo& L, const std::vector<int>& nn, DevMem& lm) -> int {
    boff.clear();
    size_t tot = 0;
    std::vector<std::pair<int, int>> all(L.pattern);
    all.insert(all.end(), L.after.begin(), L.after.end());
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    for (auto& pr : all) {
      boff[pr] = tot;
      tot += (size_t)nn[pr.first] * nn[pr.second];
    }
    arena = lm.alloc<T>(tot);
    if (lm.err) return SPAND_ERR_NOMEM;
    SPAND_CUDA_TRY(cudaMemsetAsync(arena, 0, std::max<size_t>(tot, 1) * sizeof(T), st));
    return SPAND_OK;
  };
  auto blk = [&](int a, int b) -> T* { return arena + boff.at({a, b}); };

  DevMem lvmem;  // memory of the current level arena (freed after compression)
  lvmem.st = st;
  SPAND_TRY(layout(P.lv[0], n, lvmem));
  {
    // gather the BSR blocks into the level-0 cluster blocks
    DevMem tmp;
    tmp.st = st;
    std::vector<int> rp(K + 1), col(A->nnzb);
    SPAND_CUDA_TRY(cudaMemcpyAsync(rp.data(), A->row_ptr, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, st));
    SPAND_CUDA_TRY(cudaMemcpyAsync(col.data(), A->col, sizeof(int) * A->nnzb, cudaMemcpyDeviceToHost, st));
    SPAND_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<T*> dst(A->nnzb);
    std::vector<int> ldv(A->nnzb);
    for (int e = 0; e < K; ++e)
      for (int k = rp[e]; k < rp[e + 1]; ++k) {
        const int f = col[k];
        const int a = cl_of[e], b = cl_of[f];
        auto it = boff.find({a, b});
        if (it == boff.end()) return SPAND_ERR_ARG;
        dst[k] = arena + it->second + (size_t)pos_in[e] * B + (size_t)pos_in[f] * B * n[a];
        ldv[k] = n[a];
      }
    T* const* d_dst = tmp.upload(dst);
    const int* d_ld = tmp.upload(ldv);
    if (tmp.err) return SPAND_ERR_NOMEM;
    k_level0_gather<T><<<A->nnzb, 256, 0, st>>>(A->val, nullptr, nullptr, nullptr, nullptr, d_ld, d_dst, A->nnzb, B);
    SPAND_CUDA_TRY(cudaGetLastError());
    tmp.free_all();
  }

  std::vector<LevelRec<T>> recs(D + 1);
  size_t park_b_tot = 0, park_c_tot = 0;
  int64_t apply_bytes = 0;
  double flops = 0;

  for (int l = 0; l <= D; ++l) {
    const LevelInfo& L = P.lv[l];
    const int nc = (int)L.cl.size();
    LevelRec<T>& R = recs[l];
    R.n = n;
    R.d_slots.resize(nc);
    for (int c = 0; c < nc; ++c) R.d_slots[c] = pm.upload(slots[c]);
    DevMem tmp;
    tmp.st = st;
    // neighbour lists in the current pattern
    std::vector<std::vector<int>> nbr(nc);
    for (auto& pr : L.pattern)
      if (pr.first != pr.second) nbr[pr.first].push_back(pr.second);
    // ================= 1. eliminate interiors (Eq. 9)
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
          terms.push_back({Linv[q], Ap, n[s], n[s], n[s], 0, 0});
          tasks.push_back({Y, n[s], n[s], n[b], (T)1, (T)0, (int)terms.size() - 1, (int)terms.size()});
          terms.push_back({blk(b, s), Uinv[q], n[b], n[s], n[s], 0, 0});
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
      launch_gemm(tmp, tasks, terms, st);
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
          terms.push_back({Xm.at({a, s}), Ym.at({s, b}), n[a], n[s], n[s], 0, 0});
          flops += 2.0 * n[a] * (double)n[b] * n[s];
        }
        tasks.push_back({blk(a, b), n[a], n[a], n[b], (T)-1, (T)1, t0, (int)terms.size()});
      }
      launch_gemm(tmp, tasks, terms, st);
      if (l == D)
        for (int s : I) S.top_size += n[s];
    }
    if (l == D) {
      tmp.free_all();
      break;
    }
    // ================= 2. scale interfaces (Eq. 10)
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
        m1.push_back({SL[fidx[a]], Ap, n[a], n[a], n[a], 0, 0});
        t1.push_back({Tm, n[a], n[a], n[b], (T)1, (T)0, (int)m1.size() - 1, (int)m1.size()});
        m2.push_back({Tm, SU[fidx[b]], n[a], n[b], n[b], 0, 0});
        t2.push_back({blk(a, b), n[a], n[a], n[b], (T)1, (T)0, (int)m2.size() - 1, (int)m2.size()});
        flops += 2.0 * n[a] * (double)n[b] * (n[a] + n[b]);
      }
      if (tmp.err) return SPAND_ERR_NOMEM;
      launch_row_perm(tmp, ps, pd, pp, pr_, pc_, st);
      launch_gemm(tmp, t1, m1, st);
      launch_gemm(tmp, t2, m2, st);
    }
    // ================= 3. all Q first (Eq. 11): RRQR of [A_sn A_ns^T]
    std::vector<QrTask<T>> qt;
    std::vector<int> qcl;
    std::vector<CopyTask<T>> cps;
    int* d_rank = tmp.alloc<int>(std::max<size_t>(Fc.size(), 1));
    int nmax_qr = 0;
    for (size_t q = 0; q < Fc.size(); ++q) {
      const int s = Fc[q];
      if (nba[s].empty()) continue;
      int cs = 0;
      for (int b : nba[s]) cs += 2 * n[b];
      QrTask<T> t;
      t.n = n[s];
      t.c = cs;
      t.W = tmp.alloc<T>((size_t)n[s] * cs);             // row-major n x c
      t.V = tmp.alloc<T>((size_t)n[s] * std::min(n[s], cs));
      t.tau = tmp.alloc<T>(std::min(n[s], cs));
      t.norm2 = tmp.alloc<T>(cs);
      t.Q = nullptr;
      t.rank = d_rank + qt.size();
      // W = [A_sn A_ns^T]; as a column-major c x n array (ld c) it holds W^T
      int off = 0;
      for (int b : nba[s]) {
        cps.push_back({blk(s, b), t.W + off, n[s], cs, n[b], n[s], 1});
        off += n[b];
      }
      for (int b : nba[s]) {
        cps.push_back({blk(b, s), t.W + off, n[b], cs, n[b], n[s], 0});
        off += n[b];
      }
      qt.push_back(t);
      qcl.push_back(s);
      nmax_qr = std::max(nmax_qr, n[s]);
      if (cs >= n[s]) flops += 2.0 * cs * (double)n[s] * n[s] - 2.0 / 3.0 * pow((double)n[s], 3);
    }
    if (tmp.err) return SPAND_ERR_NOMEM;
    launch_copy(tmp, cps, st);
    std::vector<int> rank(qt.size());
    if (!qt.empty()) {
      auto* dq = tmp.upload(qt);
      const size_t sm = (size_t)nmax_qr * sizeof(T);
      if (sm > kGemvSmemMax) return SPAND_ERR_UNSUPPORTED;
      cudaFuncSetAttribute(k_qrcp_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemvSmemMax);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(qt.size() * QR_CS), 1, 1);
      cfg.blockDim = dim3(QR_THREADS, 1, 1);
      cfg.dynamicSmemBytes = sm;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = QR_CS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      SPAND_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_qrcp_cluster<T>, (const QrTask<T>*)dq, (T)eps));
      SPAND_CUDA_TRY(cudaMemcpyAsync(rank.data(), d_rank, sizeof(int) * qt.size(), cudaMemcpyDeviceToHost, st));
    }
    int hflags[4];
    SPAND_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    SPAND_CUDA_TRY(cudaStreamSynchronize(st));
    if (hflags[0] & 1) return SPAND_ERR_ZERO_PIVOT;   // the root cause when both are set
    if (hflags[0] & 2) return SPAND_ERR_NONFINITE;
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
    }
    if (pm.err) return SPAND_ERR_NOMEM;
    if (!qt.empty()) {
      auto* dq = tmp.upload(qt);
      k_form_q_v<T><<<(unsigned)qt.size(), 512, 0, st>>>(dq);
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
    T* old_arena = arena;
    std::map<std::pair<int, int>, size_t> old_off = boff;
    SPAND_TRY(layout(L2, n2, lvmem2));
    auto oblk = [&](int a, int b) -> T* { return old_arena + old_off.at({a, b}); };
    std::vector<EyeTask<T>> eyes;
    std::vector<GemmTask<T>> t1, t2;
    std::vector<GemmTerm<T>> m1, m2;
    for (auto& pr : L.after) {
      const int a = pr.first, b = pr.second;
      if (n[a] == 0 || n[b] == 0 || r[a] == 0 || r[b] == 0) continue;
      const int pa = parent[a], pb = parent[b];
      T* dst = blk(pa, pb) + off[a] + (size_t)off[b] * n2[pa];
      if (a == b) {
        eyes.push_back({dst, n2[pa], r[a]});
        continue;
      }
      // both are sparsified (they have neighbours)
      T* Tm = tmp.alloc<T>((size_t)r[a] * n[b]);
      m1.push_back({Qc[a], oblk(a, b), n[a], n[a], n[a], 1, 0});
      t1.push_back({Tm, r[a], r[a], n[b], (T)1, (T)0, (int)m1.size() - 1, (int)m1.size()});
      m2.push_back({Tm, Qc[b], r[a], n[b], n[b], 0, 0});
      t2.push_back({dst, n2[pa], r[a], r[b], (T)1, (T)0, (int)m2.size() - 1, (int)m2.size()});
      flops += 2.0 * n[a] * (double)n[b] * (r[a] + r[b]);
    }
    if (tmp.err) return SPAND_ERR_NOMEM;
    launch_gemm(tmp, t1, m1, st);
    launch_gemm(tmp, t2, m2, st);
    if (!eyes.empty()) {
      auto* de = tmp.upload(eyes);
      k_eye<T><<<std::min<unsigned>((unsigned)eyes.size(), 1024), 128, 0, st>>>(de, (int)eyes.size());
    }
    SPAND_CUDA_TRY(cudaGetLastError());
    tmp.free_all();
    lvmem.free_all();
    lvmem = lvmem2;
    lvmem2.ptrs.clear();
    n = n2;
    slots = slots2;
  }
  lvmem.free_all();
  {
    int hflags[4];
    SPAND_CUDA_TRY(cudaMemcpyAsync(hflags, d_flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    SPAND_CUDA_TRY(cudaStreamSynchronize(st));
    if (hflags[0] & 1) return SPAND_ERR_ZERO_PIVOT;   // the root cause when both are set
    if (hflags[0] & 2) return SPAND_ERR_NONFINITE;
  }
  S.factor_flops = flops;

  // ================= apply program
  F->w = pm.alloc<T>(F->N);
  F->z = pm.alloc<T>(F->N);
  F->park_b = pm.alloc<T>(std::max<size_t>(park_b_tot, 1));
  F->park_c = pm.alloc<T>(std::max<size_t>(park_c_tot, 1));
  if (pm.err) return SPAND_ERR_NOMEM;
  // permuted slot lists (P^T folded into the gather) for interiors and interfaces
  for (int l = 0; l <= D; ++l) {
    LevelRec<T>& R = recs[l];
    for (auto& in : R.in) {
      int* ps = pm.alloc<int>(in.n);
      k_perm_slots<T><<<(in.n + 255) / 256, 256, 0, st>>>(R.d_slots[in.c], in.perm, ps, in.n);
      R.d_pslots.push_back(ps);
    }
  }
  std::vector<int*> fa_pslots;
  std::vector<std::vector<int*>> fa_ps(D + 1);
  for (int l = 0; l <= D; ++l)
    for (auto& f : recs[l].fa) {
      int* ps = pm.alloc<int>(f.n);
      k_perm_slots<T><<<(f.n + 255) / 256, 256, 0, st>>>(recs[l].d_slots[f.c], f.perm, ps, f.n);
      fa_ps[l].push_back(ps);
    }
  if (pm.err) return SPAND_ERR_NOMEM;
  typedef typename ApplyProg<T>::Phase Phase;
  auto build = [&](std::vector<GvTask<T>>& tasks, std::vector<GvTerm<T>>& terms) -> Phase {
    Phase ph;
    std::vector<GvTile> tiles;
    for (int t = 0; t < (int)tasks.size(); ++t)
      for (int r0 = 0; r0 < tasks[t].m; r0 += GV_ROWS) tiles.push_back({t, r0});
    for (auto& tm : terms) ph.kmax = std::max(ph.kmax, tm.k);
    if (tiles.empty()) return ph;
    ph.tasks = pm.upload(tasks);
    ph.terms = pm.upload(terms);
    ph.tiles = pm.upload(tiles);
    ph.ntiles = (int)tiles.size();
    return ph;
  };
  T* w = F->w;
  T* z = F->z;
  const size_t es = sizeof(T);
  for (int tr = 0; tr < 2; ++tr) {
    std::vector<Phase>& fwd = tr ? F->prog.tfwd : F->prog.fwd;
    std::vector<Phase>& bwd = tr ? F->prog.tbwd : F->prog.bwd;
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
        for (int t = 0; t < (int)R.in[q].nbr.size(); ++t) by_nb[R.in[q].nbr[t]].push_back({q, t});
      if (!tr) {
        // E1: z[s] = L^-1 P^T w[s]
        for (int q = 0; q < (int)R.in.size(); ++q) {
          auto& in = R.in[q];
          task(z, R.d_slots[in.c], nullptr, nullptr, nullptr, (T)1, in.n);
          term(in.Linv, w, R.d_pslots[q], nullptr, in.n, in.n, 0, 1);
          if (l == 0 || true) apply_bytes += (int64_t)in.n * (in.n + 1) / 2 * es;
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
          task(z, R.d_slots[f.c], nullptr, nullptr, nullptr, (T)1, f.n);
          if (!tr) term(f.SL, w, fa_ps[l][q], nullptr, f.n, f.n, 0, 1);
          else term(f.SU, w, R.d_slots[f.c], nullptr, f.n, f.n, 1, 2);
          if (!tr) apply_bytes += (int64_t)f.n * (f.n + 1) / 2 * es;
        }
        flush(fwd);
        // Q1: park z[s]; w[s][:r] = Q_c^T z[s]  (identity copy when unsparsified)
        for (auto& f : R.fa) {
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
          if (in.nbr.empty()) continue;
          task(z, R.d_slots[in.c], z, R.d_slots[in.c], nullptr, (T)-1, in.n);
          for (size_t t = 0; t < in.nbr.size(); ++t) {
            term(in.Y[t], w, R.d_slots[in.nbr[t]], nullptr, in.n, R.n[in.nbr[t]], 0, 0);
            apply_bytes += (int64_t)in.n * R.n[in.nbr[t]] * es;
          }
        }
        flush(bwd);
        for (auto& in : R.in) {
          task(w, R.d_slots[in.c], nullptr, nullptr, nullptr, (T)1, in.n);
          term(in.Uinv, z, R.d_slots[in.c], nullptr, in.n, in.n, 0, 2);
          apply_bytes += (int64_t)in.n * (in.n + 1) / 2 * es;
        }
        flush(bwd);
      } else {
        // E2^T: z[s] -= sum_b X_bs^T w[b];  E1^T: w[P s] = L^-T z[s]
        for (auto& in : R.in) {
          if (in.nbr.empty()) continue;
          task(z, R.d_slots[in.c], z, R.d_slots[in.c], nullptr, (T)-1, in.n);
          for (size_t t = 0; t < in.nbr.size(); ++t)
            term(in.X[t], w, R.d_slots[in.nbr[t]], nullptr, R.n[in.nbr[t]], R.n[in.nbr[t]], 1, 0);
        }
        flush(bwd);
        for (size_t q = 0; q < R.in.size(); ++q) {
          auto& in = R.in[q];
          task(w, R.d_pslots[q], nullptr, nullptr, nullptr, (T)1, in.n);
          term(in.Linv, z, R.d_slots[in.c], nullptr, in.n, in.n, 1, 1);
        }
        flush(bwd);
      }
    }
  }
  S.factor_bytes = apply_bytes;
  if (pm.err) return SPAND_ERR_NOMEM;
  SPAND_CUDA_TRY(cudaGetLastError());
  SPAND_CUDA_TRY(cudaStreamSynchronize(st));
  return SPAND_OK;
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* a, Tout* b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (Tout)a[i];
}

template <typename T>
static int run_phases(const std::vector<typename ApplyProg<T>::Phase>& ph, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemvSmemMax);
    attr = true;
  }
  for (auto& p : ph) {
    const size_t sm = (size_t)std::max(p.kmax, 1) * sizeof(T);
    k_gemv<T><<<p.ntiles, 256, sm, st>>>(p.tasks, p.terms, p.tiles);
  }
  return SPAND_OK;
}

template <typename T>
static int apply_impl(FactorT<T>* F, const double* r, double* zout, int transpose, cudaStream_t st) {
  const int N = F->N;
  const unsigned g = (unsigned)std::min(4096, (N + 255) / 256);
  k_convert<double, T><<<g, 256, 0, st>>>(r, F->w, N);
  if (!transpose) {
    run_phases<T>(F->prog.fwd, st);
    run_phases<T>(F->prog.bwd, st);
  } else {
    run_phases<T>(F->prog.tfwd, st);
    run_phases<T>(F->prog.tbwd, st);
  }
  k_convert<T, double><<<g, 256, 0, st>>>(F->w, zout, N);
  SPAND_CUDA_TRY(cudaGetLastError());
  return SPAND_OK;
}

template <typename T>
static int max_kmax(FactorT<T>* F) {
  int k = 1;
  for (auto* v : {&F->prog.fwd, &F->prog.bwd, &F->prog.tfwd, &F->prog.tbwd})
    for (auto& p : *v) k = std::max(k, p.kmax);
  return k;
}

}  // namespace spand

struct spand_factor_s {
  std::unique_ptr<spand::FactorBase> impl;
};

namespace spand {
int factor_apply(spand_factor_t F, const double* r, double* z, int transpose, cudaStream_t st) {
  if (F->impl->precision == SPAND_FP64)
    return apply_impl(static_cast<FactorT<double>*>(F->impl.get()), r, z, transpose, st);
  return apply_impl(static_cast<FactorT<float>*>(F->impl.get()), r, z, transpose, st);
}
int factor_size(spand_factor_t F) { return F->impl->N; }
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
  int st;
  if (precision == SPAND_FP64) {
    auto* F = new (std::nothrow) spand::FactorT<double>();
    f->impl.reset(F);
    st = F ? spand::factor_impl<double>(plan->P, A, eps, precision, F, stream) : SPAND_ERR_NOMEM;
    if (st == SPAND_OK && (size_t)spand::max_kmax(F) * sizeof(double) > spand::kGemvSmemMax)
      st = SPAND_ERR_UNSUPPORTED;
  } else {
    auto* F = new (std::nothrow) spand::FactorT<float>();
    f->impl.reset(F);
    st = F ? spand::factor_impl<float>(plan->P, A, eps, precision, F, stream) : SPAND_ERR_NOMEM;
    if (st == SPAND_OK && (size_t)spand::max_kmax(F) * sizeof(float) > spand::kGemvSmemMax)
      st = SPAND_ERR_UNSUPPORTED;
  }
  if (st != SPAND_OK) {
    if (f->impl) {
      cudaStreamSynchronize(stream);
      f->impl->mem.free_all();
      cudaStreamSynchronize(stream);
    }
    delete f;
    return st;
  }
  *out = f;
  return SPAND_OK;
}

int spand_factor_destroy(spand_factor_t F) {
  if (!F) return SPAND_OK;
  if (F->impl) {
    cudaDeviceSynchronize();
    F->impl->mem.free_all();
    cudaDeviceSynchronize();
  }
  delete F;
  return SPAND_OK;
}

int spand_factor_stats(spand_factor_t F, spand_stats* st) {
  if (!F || !st) return SPAND_ERR_ARG;
  *st = F->impl->stats;
  return SPAND_OK;
}

int spand_apply(spand_factor_t F, const double* r, double* z, int transpose, cudaStream_t stream) {
  if (!F || !r || !z || r == z) return SPAND_ERR_ARG;
  return spand::factor_apply(F, r, z, transpose, stream);
}

}  // extern "C"
