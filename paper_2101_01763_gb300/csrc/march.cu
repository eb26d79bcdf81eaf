// Pseudo-time continuation around the Newton-step solve (Sec. 2.1.2, Eqs. 5, 8, 9).
//
// One step: dg_assemble_jacobian at CFL^n, ||R^n|| by a two-pass FP64 reduction (fixed order, so the CFL
// sequence does not depend on scheduling), spand_factor on the plan made once for the grid, s-step GMRES
// from du = 0, and u += du.  The host reads ||R^n|| once per step: it sets CFL^{n+1} (Eq. 9) and the stop.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace {

constexpr int kNormBlocks = 152 * 4;

__global__ void __launch_bounds__(256) k_sumsq_partial(int64_t N, const double* __restrict__ x,
                                                       double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += w[k];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_sumsq_final(int nblk, const double* __restrict__ part,
                                                     double* __restrict__ out) {
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) s += part[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += w[k];
    out[0] = t;
  }
}

__global__ void k_state_update(int64_t N, const double* __restrict__ du, double* __restrict__ u) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    u[i] += du[i];
}

// Device scratch of one march, released on the stream on every exit.
struct MarchScratch {
  cudaStream_t st = nullptr;
  double* rhs = nullptr;
  double* du = nullptr;
  double* val = nullptr;
  double* red = nullptr;   // kNormBlocks partial sums + the total
  int* row_ptr = nullptr;
  int* col = nullptr;
  ~MarchScratch() {
    void* ps[] = {rhs, du, val, red, row_ptr, col};
    for (void* p : ps)
      if (p) cudaFreeAsync(p, st);
  }
};

int norm2(int64_t N, const double* x, double* red, double* out, cudaStream_t st) {
  const int nblk = (int)std::min<int64_t>(kNormBlocks, (N + 255) / 256);
  spand::note_launch(2);
  k_sumsq_partial<<<nblk, 256, 0, st>>>(N, x, red);
  k_sumsq_final<<<1, 256, 0, st>>>(nblk, red, red + kNormBlocks);
  SPAND_CUDA_TRY(cudaGetLastError());
  double s = 0.0;
  SPAND_CUDA_TRY(cudaMemcpyAsync(&s, red + kNormBlocks, sizeof(double), cudaMemcpyDeviceToHost, st));
  SPAND_CUDA_TRY(cudaStreamSynchronize(st));
  *out = std::sqrt(s);
  return SPAND_OK;
}

}  // namespace

extern "C" double dg_cfl_ramp(double cfl0, double cfl_inf, double r0, double r_prev) {
  if (!(r_prev > 0.0)) return cfl_inf;
  const double c = cfl0 * r0 / r_prev;
  return c < cfl_inf ? c : cfl_inf;
}

extern "C" int dg_pseudo_time_march(const dg_mesh* mesh, int p, double* u_hat, const dg_flow_params* flow,
                                    spand_plan_t plan, const dg_march_opts* opts, dg_march_history* hist,
                                    cudaStream_t stream) {
  if (!mesh || !flow || !opts || !u_hat || !plan || !mesh->nodes) return SPAND_ERR_ARG;
  if (p < 1 || p > 3) return SPAND_ERR_UNSUPPORTED;
  const spand::Plan& P = plan->P;
  const int nt = mesh->n_theta, nr = mesh->n_r, K = nt * nr, B = 4 * (p + 1) * (p + 1);
  if (P.nsys != 1 || P.n_theta != nt || P.n_r != nr || P.B != B) return SPAND_ERR_ARG;
  if (!(flow->cfl > 0.0) || !(opts->cfl_inf >= flow->cfl) || opts->max_steps < 0 || !(opts->rtol >= 0.0))
    return SPAND_ERR_ARG;
  if (hist) hist->steps = 0;
  const int64_t N = (int64_t)K * B;
  const int nnzb_max = 5 * K;   // 5K - 2 n_theta when n_r > 1; the assembler reports the exact count
  MarchScratch S;
  S.st = stream;
  SPAND_CUDA_TRY(cudaMallocAsync(&S.rhs, N * sizeof(double), stream));
  SPAND_CUDA_TRY(cudaMallocAsync(&S.du, N * sizeof(double), stream));
  SPAND_CUDA_TRY(cudaMallocAsync(&S.val, (size_t)nnzb_max * B * B * sizeof(double), stream));
  SPAND_CUDA_TRY(cudaMallocAsync(&S.red, (kNormBlocks + 1) * sizeof(double), stream));
  SPAND_CUDA_TRY(cudaMallocAsync(&S.row_ptr, (size_t)(K + 1) * sizeof(int), stream));
  SPAND_CUDA_TRY(cudaMallocAsync(&S.col, (size_t)nnzb_max * sizeof(int), stream));
  bsr_matrix A{K, B, 0, S.row_ptr, S.col, S.val};
  gmres_opts go = opts->gmres;
  go.transpose = 0;
  const unsigned ug = (unsigned)std::min<int64_t>(152 * 8, (N + 255) / 256);
  double cfl = flow->cfl, r0 = 0.0;
  for (int n = 0;; ++n) {
    dg_flow_params fl = *flow;
    fl.cfl = cfl;
    double dtau = 0.0, r = 0.0;
    SPAND_TRY(dg_assemble_jacobian(mesh, p, u_hat, &fl, S.rhs, &A, &dtau, stream));
    SPAND_TRY(norm2(N, S.rhs, S.red, &r, stream));
    if (!std::isfinite(r)) return SPAND_ERR_NONFINITE;
    if (n == 0) r0 = r;
    if (hist) {
      if (hist->res_norm) hist->res_norm[n] = r;
      if (hist->cfl) hist->cfl[n] = cfl;
      if (hist->dtau) hist->dtau[n] = dtau;
    }
    if (n == opts->max_steps || r <= opts->rtol * r0) break;
    spand_factor_t F = nullptr;
    SPAND_TRY(spand_factor(plan, &A, opts->eps, opts->precision, &F, stream));
    gmres_stats gs;
    int st = cudaMemsetAsync(S.du, 0, N * sizeof(double), stream) == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
    if (st == SPAND_OK) st = sstep_gmres_solve(&A, F, S.rhs, S.du, &go, &gs, stream);
    spand_factor_destroy(F);
    if (st != SPAND_OK) return st;
    if (hist && hist->gmres_iters) hist->gmres_iters[n] = gs.iters;
    spand::note_launch();
    k_state_update<<<ug, 256, 0, stream>>>(N, S.du, u_hat);
    SPAND_CUDA_TRY(cudaGetLastError());
    if (hist) hist->steps = n + 1;
    cfl = dg_cfl_ramp(flow->cfl, opts->cfl_inf, r0, r);
  }
  SPAND_CUDA_TRY(cudaStreamSynchronize(stream));
  return SPAND_OK;
}
