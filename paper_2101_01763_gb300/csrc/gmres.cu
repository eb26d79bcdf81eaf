// s-step GMRES with single-reduce lagged re-orthogonalization (Algorithm 2).
//
// Right preconditioning, A M^-1 u = b, x = x0 + M^-1 Q y.  Per s-block:
//   matrix powers  v_{k+1} = A M^-1 v_k - theta_k v_k (conjugate pairs as real
//                  two-steps), s x (spaND apply + fused SpMV);
//   one reduction  G = [Q_f, P, V]^T [P, V]  (the single Gram product);
//   small FP64 work on the device (one CTA): second CGS + CholQR pass of the
//                  pending block P from G (Pythagorean Gram correction), the
//                  Hessenberg columns H_new = (T B - H_old T_top) T_cc^-1,
//                  Givens rotations, first pass coefficients of V;
//   block updates  Q_P = P S2^-1 - Q_f (X_P S2^-1),  P' = V S1^-1 - Q_f (R1 S1^-1).
// The host reads one residual estimate per block (the convergence check) and
// confirms convergence with the true FP64 residual at each restart.  Newton
// shifts are the Ritz values of s classical GMRES (MGS) steps in the first
// cycle, computed from the s x s Hessenberg on the host, in real Leja order.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "vec.cuh"

namespace spand {
namespace {

struct Small {
  double *H, *R, *cs, *sn, *g, *B, *G, *R1P, *S1P, *t0P, *CP, *S2inv, *CV, *S1inv, *T, *Hn, *y, *scal, *M1;
  int* status;
  int m, s, ldh, ldg, ldt;
};

enum { MODE_INIT = 0, MODE_ARNOLDI = 1, MODE_FIRST = 2, MODE_PENDING = 3, MODE_FLUSH = 4, MODE_SOLVE = 5, MODE_ORTH = 6 };

// in-place upper Cholesky of an s x s column-major matrix (A = U^T U); false on breakdown
__device__ bool chol_upper(double* A, int s) {
  for (int j = 0; j < s; ++j) {
    double d = A[j + j * s];
    for (int k = 0; k < j; ++k) d -= A[k + j * s] * A[k + j * s];
    if (!(d > 0.0) || !isfinite(d)) return false;
    d = sqrt(d);
    A[j + j * s] = d;
    for (int i = j + 1; i < s; ++i) {
      double v = A[j + i * s];
      for (int k = 0; k < j; ++k) v -= A[k + j * s] * A[k + i * s];
      A[j + i * s] = v / d;
    }
    for (int i = j + 1; i < s; ++i) A[i + j * s] = 0.0;
  }
  return true;
}

__device__ void givens_col(Small& S, int j) {
  // rotate column j of H into R with the stored rotations, then a new rotation
  const int ld = S.ldh;
  double h[512];
  for (int i = 0; i <= j + 1; ++i) h[i] = S.H[i + j * ld];
  for (int i = 0; i < j; ++i) {
    const double t = S.cs[i] * h[i] + S.sn[i] * h[i + 1];
    h[i + 1] = -S.sn[i] * h[i] + S.cs[i] * h[i + 1];
    h[i] = t;
  }
  double c = 1.0, sn = 0.0;
  if (h[j + 1] != 0.0) {
    const double r = hypot(h[j], h[j + 1]);
    c = h[j] / r;
    sn = h[j + 1] / r;
  }
  S.cs[j] = c;
  S.sn[j] = sn;
  h[j] = c * h[j] + sn * h[j + 1];
  h[j + 1] = 0.0;
  for (int i = 0; i <= j; ++i) S.R[i + j * ld] = h[i];
  S.g[j + 1] = -sn * S.g[j];
  S.g[j] = c * S.g[j];
  S.scal[0] = fabs(S.g[j + 1]);
}

// finalize the pending block: second pass (S2), T, Hessenberg columns, Givens
// nf = final columns before, cs = start column of the pending block (== nf-1)
__device__ bool finalize(Small& S, int nf, const double* XP, int ldxp, const double* GPP, int ldgpp) {
  const int s = S.s, tid = threadIdx.x;
  double* S2 = S.M1;  // s x s
  for (int t = tid; t < s * s; t += blockDim.x) {
    const int i = t % s, j = t / s;
    double v = GPP[i + j * ldgpp];
    for (int a = 0; a < nf; ++a) v -= XP[a + i * ldxp] * XP[a + j * ldxp];
    S2[i + j * s] = v;
  }
  __syncthreads();
  __shared__ int ok;
  if (tid == 0) ok = chol_upper(S2, s) ? 1 : 0;
  __syncthreads();
  if (!ok) return false;
  const int cs = nf - 1, rows = nf + s, ldt = S.ldt;
  // T: (rows) x (s+1)
  for (int t = tid; t < rows * (s + 1); t += blockDim.x) {
    const int i = t % rows, j = t / rows;
    double v = 0.0;
    if (j == 0) v = (i <= cs) ? S.t0P[i] : 0.0;
    else if (i < nf) {
      v = S.R1P[i + (j - 1) * S.ldh];
      for (int b = 0; b < s; ++b) v += XP[i + b * ldxp] * S.S1P[b + (j - 1) * s];
    } else {
      const int ii = i - nf;
      for (int b = 0; b < s; ++b) v += S2[ii + b * s] * S.S1P[b + (j - 1) * s];
    }
    S.T[i + j * ldt] = v;
  }
  __syncthreads();
  // Hn = T B - H[:, 0:cs] T[0:cs, 0:s]
  for (int t = tid; t < rows * s; t += blockDim.x) {
    const int i = t % rows, j = t / rows;
    double v = 0.0;
    for (int b = 0; b <= s; ++b) v += S.T[i + b * ldt] * S.B[b + j * (s + 1)];
    for (int a = 0; a < cs; ++a) v -= S.H[i + a * S.ldh] * S.T[a + j * ldt];
    S.Hn[i + j * ldt] = v;
  }
  __syncthreads();
  // Hn <- Hn Tcc^-1, Tcc = T[cs:cs+s, 0:s] upper triangular; then into H
  for (int i = tid; i < rows; i += blockDim.x) {
    double x[16];
    for (int j = 0; j < s; ++j) {
      double v = S.Hn[i + j * ldt];
      for (int a = 0; a < j; ++a) v -= x[a] * S.T[(cs + a) + j * ldt];
      x[j] = v / S.T[(cs + j) + j * ldt];
    }
    for (int j = 0; j < s; ++j) S.H[i + (cs + j) * S.ldh] = x[j];
  }
  __syncthreads();
  if (tid == 0)
    for (int j = cs; j < cs + s; ++j) givens_col(S, j);
  __syncthreads();
  return true;
}

// CP = XP S2^-1 (nf x s), S2inv
__device__ void second_pass_coeffs(Small& S, int nf, const double* XP, int ldxp) {
  const int s = S.s, tid = threadIdx.x;
  const double* S2 = S.M1;
  for (int i = tid; i < nf; i += blockDim.x) {
    double x[16];
    for (int j = 0; j < s; ++j) {
      double v = XP[i + j * ldxp];
      for (int a = 0; a < j; ++a) v -= x[a] * S2[a + j * s];
      x[j] = v / S2[j + j * s];
    }
    for (int j = 0; j < s; ++j) S.CP[i + j * S.ldh] = x[j];
  }
  for (int i = tid; i < s; i += blockDim.x) {
    // row i of S2^-1: solve x S2 = e_i
    double x[16];
    for (int j = 0; j < s; ++j) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int a = 0; a < j; ++a) v -= x[a] * S2[a + j * s];
      x[j] = v / S2[j + j * s];
    }
    for (int j = 0; j < s; ++j) S.S2inv[i + j * s] = x[j];
  }
  __syncthreads();
}

// first pass of V: R1 (nr x s) given, GVV; S1, CV = R1 S1^-1, S1inv, and the pending state
__device__ bool first_pass(Small& S, int nr, const double* R1, int ldr, const double* GVV, int ldgvv) {
  const int s = S.s, tid = threadIdx.x;
  __shared__ double S1[256];
  for (int t = tid; t < s * s; t += blockDim.x) {
    const int i = t % s, j = t / s;
    double v = GVV[i + j * ldgvv];
    for (int a = 0; a < nr; ++a) v -= R1[a + i * ldr] * R1[a + j * ldr];
    S1[i + j * s] = v;
  }
  __syncthreads();
  __shared__ int ok;
  if (tid == 0) ok = chol_upper(S1, s) ? 1 : 0;
  __syncthreads();
  if (!ok) return false;
  for (int i = tid; i < nr; i += blockDim.x) {
    double x[16];
    for (int j = 0; j < s; ++j) {
      double v = R1[i + j * ldr];
      for (int a = 0; a < j; ++a) v -= x[a] * S1[a + j * s];
      x[j] = v / S1[j + j * s];
    }
    for (int j = 0; j < s; ++j) {
      S.CV[i + j * S.ldh] = x[j];
      S.R1P[i + j * S.ldh] = R1[i + j * ldr];
    }
  }
  for (int i = tid; i < s; i += blockDim.x) {
    double x[16];
    for (int j = 0; j < s; ++j) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int a = 0; a < j; ++a) v -= x[a] * S1[a + j * s];
      x[j] = v / S1[j + j * s];
    }
    for (int j = 0; j < s; ++j) S.S1inv[i + j * s] = x[j];
  }
  for (int t = tid; t < s * s; t += blockDim.x) S.S1P[t] = S1[t];
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(256) k_small(Small S, int mode, int a0, int a1) {
  const int tid = threadIdx.x, s = S.s;
  if (mode == MODE_INIT) {
    // a0 unused; scal[2] holds ||r||^2
    for (int t = tid; t < S.ldh * S.m; t += blockDim.x) {
      S.H[t] = 0.0;
      S.R[t] = 0.0;
    }
    for (int t = tid; t < S.ldh; t += blockDim.x) S.g[t] = 0.0;
    __syncthreads();
    if (tid == 0) {
      const double beta = sqrt(S.scal[2]);
      S.g[0] = beta;
      S.scal[1] = beta;
      S.scal[0] = beta;
      S.scal[7] = 1.0;
      S.status[0] = 0;
    }
    return;
  }
  if (mode == MODE_ARNOLDI) {
    // column j = a0: H[0..j, j] already written by the MGS dots; scal[2] = ||v||^2
    if (tid == 0) {
      const double h = sqrt(S.scal[2]);
      S.H[(a0 + 1) + a0 * S.ldh] = h;
      S.scal[4] = h;
      givens_col(S, a0);
    }
    return;
  }
  if (mode == MODE_FIRST) {
    // no pending block; final columns 0..c (c = a0); G rows [Q 0..c, V] x cols V
    const int nf = a0 + 1;
    if (!first_pass(S, nf, S.G, S.ldg, S.G + nf, S.ldg)) {
      if (tid == 0) S.status[0] = 1;
      return;
    }
    for (int i = tid; i < nf; i += blockDim.x) S.t0P[i] = (i == a0) ? 1.0 : 0.0;
    return;
  }
  if (mode == MODE_PENDING) {
    // pending block starts at column c (= a0); final columns 0..c; G rows
    // [Q 0..c, P, V] x cols [P, V]
    const int nf = a0 + 1, ldg = S.ldg;
    const double* XP = S.G;
    const double* GPP = S.G + nf;
    const double* XV = S.G + (size_t)s * ldg;
    const double* GPV = S.G + nf + (size_t)s * ldg;
    const double* GVV = S.G + nf + s + (size_t)s * ldg;
    if (!finalize(S, nf, XP, ldg, GPP, ldg)) {
      if (tid == 0) S.status[0] = 1;
      return;
    }
    second_pass_coeffs(S, nf, XP, ldg);
    // R1 = [XV; S2^-T (GPV - XP^T XV)]  ((nf+s) x s) in the T workspace
    double* R1 = S.Hn;  // reuse: ldt rows
    const int ldr = S.ldt;
    const double* S2 = S.M1;
    for (int t = tid; t < nf * s; t += blockDim.x) {
      const int i = t % nf, j = t / nf;
      R1[i + j * ldr] = XV[i + j * ldg];
    }
    for (int j = tid; j < s; j += blockDim.x) {
      double m2[16], x[16];
      for (int i = 0; i < s; ++i) {
        double v = GPV[i + j * ldg];
        for (int a = 0; a < nf; ++a) v -= XP[a + i * ldg] * XV[a + j * ldg];
        m2[i] = v;
      }
      for (int i = 0; i < s; ++i) {  // S2^T x = m2 (S2^T lower)
        double v = m2[i];
        for (int a = 0; a < i; ++a) v -= S2[a + i * s] * x[a];
        x[i] = v / S2[i + i * s];
      }
      for (int i = 0; i < s; ++i) R1[nf + i + j * ldr] = x[i];
    }
    // new start coefficients t0 = [XP[:, s-1]; S2[:, s-1]]
    __syncthreads();
    double* t0 = S.y;  // temporary
    for (int i = tid; i < nf + s; i += blockDim.x) t0[i] = (i < nf) ? XP[i + (s - 1) * ldg] : S2[(i - nf) + (s - 1) * s];
    __syncthreads();
    if (!first_pass(S, nf + s, R1, ldr, GVV, ldg)) {
      if (tid == 0) S.status[0] = 1;
      return;
    }
    for (int i = tid; i < nf + s; i += blockDim.x) S.t0P[i] = t0[i];
    return;
  }
  if (mode == MODE_FLUSH) {
    const int nf = a0 + 1, ldg = S.ldg;
    if (!finalize(S, nf, S.G, ldg, S.G + nf, ldg)) {
      if (tid == 0) S.status[0] = 1;
      return;
    }
    second_pass_coeffs(S, nf, S.G, ldg);
    return;
  }
  if (mode == MODE_SOLVE) {
    const int k = a0;
    if (tid == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double v = S.g[i];
        for (int j = i + 1; j < k; ++j) v -= S.R[i + j * S.ldh] * S.y[j];
        S.y[i] = v / S.R[i + i * S.ldh];
      }
    }
    return;
  }
  if (mode == MODE_ORTH) {
    // G holds Q^T Q (a0 x a0, ld ldg); scal[3] = max(scal[3], ||G - I||_F)
    __shared__ double red[256];
    double v = 0.0;
    for (int t = tid; t < a0 * a0; t += blockDim.x) {
      const int i = t % a0, j = t / a0;
      const double d = S.G[i + j * S.ldg] - (i == j ? 1.0 : 0.0);
      v += d * d;
    }
    red[tid] = v;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < (int)blockDim.x; ++i) tot += red[i];
      S.scal[3] = fmax(S.scal[3], sqrt(tot));
    }
    return;
  }
  (void)a1;
}

// ------------------------------------------------------------------ host: Ritz values + Leja order
std::vector<std::complex<double>> hessenberg_eigs(std::vector<double> Hr, int n) {
  typedef std::complex<double> C;
  std::vector<C> A(n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) A[i + j * n] = Hr[i + j * n];
  std::vector<C> ev;
  int hi = n - 1, it = 0;
  auto a = [&](int i, int j) -> C& { return A[i + j * n]; };
  while (hi >= 0) {
    if (hi == 0) {
      ev.push_back(a(0, 0));
      break;
    }
    int lo = hi;
    while (lo > 0) {
      const double sc = std::abs(a(lo, lo)) + std::abs(a(lo - 1, lo - 1));
      if (std::abs(a(lo, lo - 1)) <= 1e-15 * (sc > 0 ? sc : 1.0)) {
        a(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      ev.push_back(a(hi, hi));
      --hi;
      it = 0;
      continue;
    }
    if (++it > 500) break;
    // Wilkinson shift from the trailing 2 x 2
    const C p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), d = a(hi, hi);
    const C tr = p + d, det = p * d - q * r;
    const C disc = std::sqrt(tr * tr * 0.25 - det);
    C m1 = tr * 0.5 + disc, m2 = tr * 0.5 - disc;
    C mu = (std::abs(m1 - d) < std::abs(m2 - d)) ? m1 : m2;
    if (it % 11 == 10) mu += std::abs(a(hi, hi - 1));     // exceptional shift
    for (int i = lo; i <= hi; ++i) a(i, i) -= mu;
    std::vector<C> cs(hi - lo), sn(hi - lo);
    for (int k = lo; k < hi; ++k) {
      const C x = a(k, k), y = a(k + 1, k);
      const double rr = std::sqrt(std::norm(x) + std::norm(y));
      C c = 1.0, s = 0.0;
      if (rr > 0) {
        c = x / rr;
        s = y / rr;
      }
      cs[k - lo] = c;
      sn[k - lo] = s;
      for (int j = k; j <= hi; ++j) {
        const C u = a(k, j), v = a(k + 1, j);
        a(k, j) = std::conj(c) * u + std::conj(s) * v;
        a(k + 1, j) = -s * u + c * v;
      }
    }
    for (int k = lo; k < hi; ++k) {
      const C c = cs[k - lo], s = sn[k - lo];
      for (int i = lo; i <= std::min(k + 2, hi); ++i) {
        const C u = a(i, k), v = a(i, k + 1);
        a(i, k) = u * c + v * s;
        a(i, k + 1) = -u * std::conj(s) + v * std::conj(c);
      }
    }
    for (int i = lo; i <= hi; ++i) a(i, i) += mu;
  }
  return ev;
}

std::vector<std::complex<double>> leja(std::vector<std::complex<double>> th) {
  typedef std::complex<double> C;
  // snap near-real values and make conjugate pairs exact
  for (auto& t : th)
    if (std::abs(t.imag()) <= 1e-10 * std::max(1.0, std::abs(t))) t = C(t.real(), 0.0);
  std::vector<int> rem(th.size());
  for (size_t i = 0; i < th.size(); ++i) rem[i] = (int)i;
  std::vector<C> out;
  auto take = [&](int i) {
    const C t = th[i];
    rem.erase(std::find(rem.begin(), rem.end(), i));
    if (t.imag() != 0.0) {
      out.push_back(C(t.real(), std::abs(t.imag())));
      int best = -1;
      double bd = 1e300;
      for (int q : rem)
        if (std::abs(th[q] - std::conj(t)) < bd) {
          bd = std::abs(th[q] - std::conj(t));
          best = q;
        }
      if (best >= 0) rem.erase(std::find(rem.begin(), rem.end(), best));
      out.push_back(C(t.real(), -std::abs(t.imag())));
    } else {
      out.push_back(C(t.real(), 0.0));
    }
  };
  int i0 = rem[0];
  for (int q : rem) {
    const double a = std::abs(th[q]), b = std::abs(th[i0]);
    if (a > b || (a == b && th[q].imag() > th[i0].imag())) i0 = q;
  }
  take(i0);
  while (!rem.empty()) {
    int best = rem[0];
    double bs = -1e300;
    for (int q : rem) {
      double sc = 0;
      for (auto& o : out) sc += std::log(std::abs(th[q] - o) + 1e-300);
      if (sc > bs || (sc == bs && th[q].imag() > th[best].imag())) {
        bs = sc;
        best = q;
      }
    }
    take(best);
  }
  return out;
}

}  // namespace
}  // namespace spand

namespace spand {
namespace {

// Device buffers of one solve: small dense work, basis vectors, Gram partial
// sums, status words and the Gram column-pointer tables.
struct GmresScratch {
  double* small;
  double* vec;
  double* part;
  int* stat;
  const double** dZ;
  const double** dY;
  bool timed = false;   // phase times by CUDA events (not in the no-allocation entry point)
  bool direct_apply = false;   // preconditioner launches issued one by one, never through a CUDA graph
};

// The solve's stream timeline split into phases: mark(p) records an event, and
// the time from one mark to the next is charged to the earlier mark's phase
// (so a host round trip is charged to the phase that ends in it).  Read once,
// after the stream has been synchronized.
enum { PH_SPMV = 0, PH_APPLY = 1, PH_ORTH = 2, PH_SMALL = 3 };
struct PhaseClock {
  cudaStream_t st = nullptr;
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ph;
  void mark(int p) {
    if (!on) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      on = false;
      return;
    }
    if (cudaEventRecord(e, st) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(e);
      on = false;
      return;
    }
    ev.push_back(e);
    ph.push_back(p);
  }
  // kernel timers of the block Gram reductions (kind 0) and block updates
  // (kind 1): an event pair around each launch and the bytes it reads/writes
  struct Kt {
    cudaEvent_t a, b;
    int kind;
    double bytes;
  };
  std::vector<Kt> kt;
  bool kbegin(cudaEvent_t& a) {
    if (!on) return false;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventRecord(a, st) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  }
  void kend(cudaEvent_t a, int kind, double bytes) {
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(b, st) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      return;
    }
    kt.push_back({a, b, kind, bytes});
  }
  void finish(gmres_stats& s) {
    if (on && !kt.empty() && cudaStreamSynchronize(st) == cudaSuccess) {
      for (auto& k : kt) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, k.a, k.b) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        if (k.kind == 0) {
          s.t_gram_ms += ms;
          s.gram_bytes += k.bytes;
          s.gram_calls += 1;
        } else {
          s.t_bupd_ms += ms;
          s.bupd_bytes += k.bytes;
          s.bupd_calls += 1;
        }
      }
    }
    if (on && ev.size() >= 2 && cudaStreamSynchronize(st) == cudaSuccess) {
      double t[4] = {0.0, 0.0, 0.0, 0.0};
      for (size_t i = 0; i + 1 < ev.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) t[ph[i]] += ms;
        else cudaGetLastError();
      }
      s.t_spmv_ms = t[PH_SPMV];
      s.t_apply_ms = t[PH_APPLY];
      s.t_orth_ms = t[PH_ORTH];
      s.t_small_ms = t[PH_SMALL];
    }
    release();
  }
  void release() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    ph.clear();
    for (auto& k : kt) {
      cudaEventDestroy(k.a);
      cudaEventDestroy(k.b);
    }
    kt.clear();
  }
  ~PhaseClock() { release(); }
};

// <x, y> of two device vectors into *out (device): per-CTA partial sums in a
// fixed order, then one CTA adds them (the inner products of the MGS Arnoldi).
__global__ void __launch_bounds__(256) k_dot_partial(int64_t N, const double* __restrict__ x,
                                                     const double* __restrict__ y, double* __restrict__ part) {
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    v += x[i] * y[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += w[k];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_dot_final(int nblk, const double* __restrict__ part,
                                                   double* __restrict__ out) {
  double v = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) v += part[k];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += w[k];
    out[0] = t;
  }
}

struct GmresSizes {
  std::vector<size_t> small;  // doubles per small-matrix piece
  size_t small_tot, nvec, part, maxptr;
};

constexpr int kGramBlocks = 2 * 152;

GmresSizes gmres_sizes(int m, int s) {
  GmresSizes z;
  const int ldh = m + 1, ldg = m + 2 * s + 2, ldt = m + s + 2;
  z.small = {(size_t)ldh * m, (size_t)ldh * m, (size_t)m + 1, (size_t)m + 1, (size_t)ldh,
             (size_t)(s + 1) * s, (size_t)ldg * (ldg), (size_t)ldh * s, (size_t)s * s, (size_t)ldh + s,
             (size_t)ldh * s, (size_t)s * s, (size_t)ldh * s, (size_t)s * s, (size_t)ldt * (s + 1),
             (size_t)ldt * s, (size_t)ldh + s, 16, (size_t)s * s};
  z.small_tot = 0;
  for (auto v : z.small) z.small_tot += v;
  z.nvec = (size_t)(m + 1) + 2 * s + 3;
  z.part = (size_t)kGramBlocks * ldg * 32;
  z.maxptr = (size_t)ldg + 64;
  return z;
}

int gmres_validate(const bsr_matrix* A, spand_factor_t M, const double* b, double* x, const gmres_opts* opts) {
  if (!A || !b || !x || !opts || !A->row_ptr || !A->col || !A->val) return SPAND_ERR_ARG;
  const int s = opts->s, m = opts->restart;
  if (s < 1 || s > 16 || m < s || m % s != 0 || m > 480 || opts->max_iters < 1 || !(opts->tol >= 0))
    return SPAND_ERR_ARG;
  const int64_t N = (int64_t)A->K * A->B;
  if (M && factor_size(M) != N) return SPAND_ERR_ARG;
  return SPAND_OK;
}

// The solve itself; every device buffer comes from `sc` (the caller owns them).
int sstep_core(const bsr_matrix* A, spand_factor_t M, const double* b, double* x, const gmres_opts* opts,
               gmres_stats* stats, cudaStream_t st, const GmresScratch& sc) {
  const int s = opts->s, m = opts->restart;
  const int64_t N = (int64_t)A->K * A->B;
  const int tr = opts->transpose ? 1 : 0;
  const bool newton = opts->basis == SPAND_BASIS_NEWTON;
  gmres_stats stl;
  memset(&stl, 0, sizeof(stl));
  const int ldh = m + 1, ldg = m + 2 * s + 2, ldt = m + s + 2;
  const int nblk = kGramBlocks;
  const GmresSizes zs = gmres_sizes(m, s);
  const std::vector<size_t>& sz = zs.small;
  const size_t tot = zs.small_tot;
  double* dsmall = sc.small;
  double* dvec = sc.vec;
  double* dpart = sc.part;
  int* dstat = sc.stat;
  const double** dZ = sc.dZ;
  const double** dY = sc.dY;
  cudaMemsetAsync(dsmall, 0, tot * sizeof(double), st);
  cudaMemsetAsync(dstat, 0, 4 * sizeof(int), st);
  Small S;
  {
    double* p = dsmall;
    double** f[] = {&S.H, &S.R, &S.cs, &S.sn, &S.g, &S.B, &S.G, &S.R1P, &S.S1P, &S.t0P, &S.CP, &S.S2inv, &S.CV,
                    &S.S1inv, &S.T, &S.Hn, &S.y, &S.scal, &S.M1};
    for (size_t k = 0; k < sz.size(); ++k) {
      *f[k] = p;
      p += sz[k];
    }
  }
  S.status = dstat;
  S.m = m;
  S.s = s;
  S.ldh = ldh;
  S.ldg = ldg;
  S.ldt = ldt;
  double* Q = dvec;                       // N x (m+1)
  double* PV = dvec + (size_t)(m + 1) * N;  // N x 2s: P then V
  double* r = PV + (size_t)2 * s * N;
  double* u = r + N;
  double* wv = u + N;
  auto Qc = [&](int j) { return Q + (size_t)j * N; };
  auto Pc = [&](int j) { return PV + (size_t)j * N; };
  auto Vc = [&](int j) { return PV + (size_t)(s + j) * N; };
  int status = SPAND_OK;
  PhaseClock clk;
  clk.st = st;
  clk.on = sc.timed;
  auto applyM = [&](const double* in, double* out) -> int {
    if (!M) return cudaMemcpyAsync(out, in, N * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess
                       ? SPAND_OK : SPAND_ERR_CUDA;
    return factor_apply(M, in, out, tr, st, sc.direct_apply);
  };
  // G = Z^T Y with column pointer lists
  std::vector<const double*> hz, hy;
  auto gram_run = [&](double* G, int ldG) -> int {
    if (cudaMemcpyAsync(dZ, hz.data(), hz.size() * sizeof(double*), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dY, hy.data(), hy.size() * sizeof(double*), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return SPAND_ERR_CUDA;
    cudaEvent_t e0 = nullptr;
    const bool tk = hy.size() >= 2 && clk.kbegin(e0);     // the block Gram reductions of Algorithm 2
    const int r = gram(N, (int)hz.size(), dZ, (int)hy.size(), dY, dpart, nblk, G, ldG, st);
    if (tk) clk.kend(e0, 0, (double)(hz.size() + hy.size()) * (double)N * sizeof(double));
    return r;
  };
  // X = Y Sinv + Z C (the block updates of CGS2 + CholQR2), timed like the Gram
  auto bupd = [&](int ny, const double* Y, const double* Sinv, int nz, const double* Z, const double* Cm, int ldc,
                  double* X) -> int {
    cudaEvent_t e0 = nullptr;
    const bool tk = clk.kbegin(e0);
    const int r = block_update(N, s, ny, Y, N, Sinv, nz, Z, N, Cm, ldc, X, N, 0, st);
    if (tk) clk.kend(e0, 1, (double)(ny + nz + s) * (double)N * sizeof(double));
    return r;
  };
  auto read_scal = [&](int idx, double& v) -> int {
    if (cudaMemcpyAsync(&v, S.scal + idx, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SPAND_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SPAND_ERR_CUDA;
    return SPAND_OK;
  };
  auto check_status = [&]() -> int {
    int hs[4];
    if (cudaMemcpyAsync(hs, dstat, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SPAND_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SPAND_ERR_CUDA;
    return hs[0] ? SPAND_ERR_CHOLQR : SPAND_OK;
  };
  // ||b||
  double bn2 = 0;
  hz = {b};
  hy = {b};
  status = gram_run(S.scal + 5, 1);
  if (status == SPAND_OK) status = read_scal(5, bn2);
  const double bn = sqrt(bn2);
  std::vector<std::complex<double>> shifts;
  std::vector<double> Bh((s + 1) * s, 0.0);
  int iters = 0;
  double est_rel = INFINITY;
  while (status == SPAND_OK) {
    // ---- true residual r = b - A x
    clk.mark(PH_SPMV);
    status = spmv_fused(A, x, r, tr, -1.0, 1.0, b, 0.0, nullptr, st);
    if (status) break;
    hz = {r};
    hy = {r};
    clk.mark(PH_ORTH);
    status = gram_run(S.scal + 2, 1);
    if (status) break;
    double rr;
    clk.mark(PH_SMALL);
    status = read_scal(2, rr);
    if (status) break;
    const double beta = sqrt(rr);
    stl.true_relres = bn > 0 ? beta / bn : beta;
    if (!std::isfinite(beta)) {
      status = SPAND_ERR_NONFINITE;
      break;
    }
    if (stl.true_relres <= opts->tol) break;
    if (iters >= opts->max_iters) {
      status = SPAND_ERR_NOT_CONVERGED;
      break;
    }
    int mc = std::min(m, opts->max_iters - iters);
    mc -= mc % s;
    if (mc == 0) {
      status = SPAND_ERR_NOT_CONVERGED;
      break;
    }
    note_launch();
    k_small<<<1, 256, 0, st>>>(S, MODE_INIT, 0, 0);
    // q0 = r / beta  (scal[1] = beta after INIT)
    clk.mark(PH_ORTH);
    status = scale_copy(N, r, Qc(0), S.scal + 1, 1, st);
    if (status) break;
    int c = 0;        // last final column
    bool pend = false;
    int csP = 0;
    bool done = false;
    int k_cols = 0;   // Hessenberg columns in this cycle
    if (newton && shifts.empty()) {
      for (int j = 0; j < s && !done; ++j) {
        clk.mark(PH_APPLY);
        status = applyM(Qc(j), u);
        if (status) break;
        clk.mark(PH_SPMV);
        status = spmv_fused(A, u, wv, tr, 1.0, 0.0, nullptr, 0.0, nullptr, st);
        if (status) break;
        clk.mark(PH_ORTH);
        for (int i = 0; i <= j; ++i) {
          hz = {Qc(i)};
          hy = {wv};
          status = gram_run(S.H + i + (size_t)j * ldh, 1);
          if (status) break;
          status = axpy_dev(N, S.H + i + (size_t)j * ldh, -1.0, Qc(i), wv, st);
          if (status) break;
        }
        if (status) break;
        hz = {wv};
        hy = {wv};
        status = gram_run(S.scal + 2, 1);
        if (status) break;
        clk.mark(PH_SMALL);
        note_launch();
        k_small<<<1, 256, 0, st>>>(S, MODE_ARNOLDI, j, 0);
        clk.mark(PH_ORTH);
        status = scale_copy(N, wv, Qc(j + 1), S.scal + 4, 1, st);
        if (status) break;
        double est;
        clk.mark(PH_SMALL);
        status = read_scal(0, est);
        if (status) break;
        ++iters;
        ++k_cols;
        c = j + 1;
        est_rel = est / bn;
        if (est_rel <= opts->tol) done = true;
        double h;
        status = read_scal(4, h);
        if (status) break;
        if (h == 0.0) done = true;
      }
      if (status) break;
      if (!done) {
        std::vector<double> Hs(s * s), Hf((size_t)ldh * m);
        if (cudaMemcpyAsync(Hf.data(), S.H, Hf.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          status = SPAND_ERR_CUDA;
          break;
        }
        for (int j = 0; j < s; ++j)
          for (int i = 0; i < s; ++i) Hs[i + j * s] = Hf[i + (size_t)j * ldh];
        shifts = leja(hessenberg_eigs(Hs, s));
        if ((int)shifts.size() != s) shifts.assign(s, 0.0);
      }
    }
    if (shifts.empty() && !done) shifts.assign(s, 0.0);
    if (!done) {
      std::fill(Bh.begin(), Bh.end(), 0.0);
      for (int k = 0; k < s; ++k) {
        Bh[k + k * (s + 1)] = shifts[k].real();
        Bh[(k + 1) + k * (s + 1)] = 1.0;
        if (shifts[k].imag() < 0) Bh[(k - 1) + k * (s + 1)] = -shifts[k].imag() * shifts[k].imag();
        stl.shifts_re[k] = shifts[k].real();
        stl.shifts_im[k] = shifts[k].imag();
      }
      if (cudaMemcpyAsync(S.B, Bh.data(), Bh.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        status = SPAND_ERR_CUDA;
        break;
      }
    }
    while (!done && status == SPAND_OK) {
      if (pend && csP + 2 * s > mc) break;
      if (!pend && c + s > mc) break;
      // ---- matrix powers from the last column
      const double* w0 = pend ? Pc(s - 1) : Qc(c);
      for (int k = 0; k < s && !status; ++k) {
        const double* vk = (k == 0) ? w0 : Vc(k - 1);
        const double* vkm = (k == 0) ? nullptr : ((k == 1) ? w0 : Vc(k - 2));
        const std::complex<double> t = shifts[k];
        const double a2 = t.imag() < 0 ? t.imag() * t.imag() : 0.0;
        if (!M) {
          clk.mark(PH_SPMV);
          status = spmv_fused(A, vk, Vc(k), tr, 1.0, -t.real(), vk, a2, t.imag() < 0 ? vkm : nullptr, st);
          continue;
        }
        // the preconditioner's sweeps leave M^-1 v_k in the factor's own vector
        // (FP32 in the mixed form), which the shifted SpMV reads in place
        clk.mark(PH_APPLY);
        const void* w = nullptr;
        int wf = 0;
        status = factor_apply_slot(M, vk, tr, st, sc.direct_apply, &w, &wf);
        if (status) break;
        clk.mark(PH_SPMV);
        status = spmv_fused_x(A, w, wf, Vc(k), tr, 1.0, -t.real(), vk, a2, t.imag() < 0 ? vkm : nullptr, st);
      }
      if (status) break;
      // ---- the single reduction
      hz.clear();
      for (int j = 0; j <= c; ++j) hz.push_back(Qc(j));
      hy.clear();
      if (pend)
        for (int j = 0; j < s; ++j) {
          hz.push_back(Pc(j));
          hy.push_back(Pc(j));
        }
      for (int j = 0; j < s; ++j) {
        hz.push_back(Vc(j));
        hy.push_back(Vc(j));
      }
      clk.mark(PH_ORTH);
      status = gram_run(S.G, ldg);
      if (status) break;
      stl.reductions++;
      if (pend) {
        clk.mark(PH_SMALL);
        note_launch();
        k_small<<<1, 256, 0, st>>>(S, MODE_PENDING, c, 0);
        status = check_status();
        if (status) break;
        // Q_P = P S2^-1 - Q_f CP  -> columns c+1..c+s
        clk.mark(PH_ORTH);
        status = bupd(s, Pc(0), S.S2inv, c + 1, Qc(0), S.CP, ldh, Qc(c + 1));
        if (status) break;
        const int c_old = c;
        c += s;
        iters += s;
        k_cols += s;
        double est;
        clk.mark(PH_SMALL);
        status = read_scal(0, est);
        if (status) break;
        est_rel = est / bn;
        (void)c_old;
        if (est_rel <= opts->tol) {
          done = true;
          break;
        }
        // P' = V S1^-1 - Q_{0..c} CV  (into the P slot)
        clk.mark(PH_ORTH);
        status = bupd(s, Vc(0), S.S1inv, c + 1, Qc(0), S.CV, ldh, Pc(0));
        csP = c;
      } else {
        clk.mark(PH_SMALL);
        note_launch();
        k_small<<<1, 256, 0, st>>>(S, MODE_FIRST, c, 0);
        status = check_status();
        if (status) break;
        clk.mark(PH_ORTH);
        status = bupd(s, Vc(0), S.S1inv, c + 1, Qc(0), S.CV, ldh, Pc(0));
        csP = c;
        pend = true;
      }
    }
    if (status) break;
    if (!done && pend) {
      // ---- flush: second pass of the last block
      hz.clear();
      for (int j = 0; j <= c; ++j) hz.push_back(Qc(j));
      hy.clear();
      for (int j = 0; j < s; ++j) {
        hz.push_back(Pc(j));
        hy.push_back(Pc(j));
      }
      clk.mark(PH_ORTH);
      status = gram_run(S.G, ldg);
      if (status) break;
      stl.reductions++;
      clk.mark(PH_SMALL);
      note_launch();
      k_small<<<1, 256, 0, st>>>(S, MODE_FLUSH, c, 0);
      status = check_status();
      if (status) break;
      clk.mark(PH_ORTH);
      status = bupd(s, Pc(0), S.S2inv, c + 1, Qc(0), S.CP, ldh, Qc(c + 1));
      if (status) break;
      c += s;
      iters += s;
      k_cols += s;
      double est;
      clk.mark(PH_SMALL);
      status = read_scal(0, est);
      if (status) break;
      est_rel = est / bn;
    }
    // ---- orthogonality diagnostic ||Q^T Q - I||_F over the k+1 final columns
    clk.mark(PH_SMALL);
    {
      const int kq = k_cols + 1;
      if (kq <= 32) {
        hz.clear();
        hy.clear();
        for (int j = 0; j < kq; ++j) {
          hz.push_back(Qc(j));
          hy.push_back(Qc(j));
        }
        status = gram_run(S.G, ldg);
        if (status) break;
        note_launch();
        k_small<<<1, 256, 0, st>>>(S, MODE_ORTH, kq, 0);
      }
    }
    // ---- x += M^-1 (Q_{0:k} y)
    note_launch();
    k_small<<<1, 256, 0, st>>>(S, MODE_SOLVE, k_cols, 0);
    {
      // wv = Q[:, 0:k] y  via block update with no Y part: X = -Z C, C = -y
      status = block_update(N, 1, 0, nullptr, N, nullptr, k_cols, Qc(0), N, S.y, k_cols, wv, N, 0, st);
      if (status) break;
      // block_update computes -Z y; negate through the M^-1 + axpy sign
      clk.mark(PH_APPLY);
      status = applyM(wv, u);
      if (status) break;
      clk.mark(PH_SMALL);
      status = axpy_dev(N, S.scal + 7, -1.0, u, x, st);   // scal[7] = 1
      if (status) break;
    }
    stl.restarts++;
    if (cudaGetLastError() != cudaSuccess) status = SPAND_ERR_CUDA;
  }
  clk.mark(PH_SMALL);
  stl.iters = iters;
  stl.est_relres = est_rel;
  {
    double o = 0;
    if (status == SPAND_OK || status == SPAND_ERR_NOT_CONVERGED) {
      if (cudaMemcpyAsync(&o, S.scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess)
        cudaStreamSynchronize(st);
    }
    stl.orth_err = o;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && status == SPAND_OK) status = SPAND_ERR_CUDA;
  clk.finish(stl);
  if (stats) *stats = stl;
  return status;
}

// Algorithm 1: restarted GMRES, modified Gram-Schmidt Arnoldi, Givens
// rotations, right preconditioning.  Per column j: one preconditioner apply,
// one SpMV, j+1 inner products each followed by its axpy (MGS), one norm, the
// Givens update (k_small) and a host read of the residual estimate.  Every
// inner product is a separate reduction; that is the cost s-step GMRES
// removes.  Same scratch layout as the s-step solve with s = 1.
int mgs_core(const bsr_matrix* A, spand_factor_t M, const double* b, double* x, const gmres_opts* opts,
             gmres_stats* stats, cudaStream_t st, const GmresScratch& sc) {
  const int m = opts->restart;
  const int64_t N = (int64_t)A->K * A->B;
  const int tr = opts->transpose ? 1 : 0;
  gmres_stats stl;
  memset(&stl, 0, sizeof(stl));
  const int ldh = m + 1;
  const GmresSizes zs = gmres_sizes(m, 1);
  cudaMemsetAsync(sc.small, 0, zs.small_tot * sizeof(double), st);
  cudaMemsetAsync(sc.stat, 0, 4 * sizeof(int), st);
  Small S;
  {
    double* p = sc.small;
    double** f[] = {&S.H, &S.R, &S.cs, &S.sn, &S.g, &S.B, &S.G, &S.R1P, &S.S1P, &S.t0P, &S.CP, &S.S2inv, &S.CV,
                    &S.S1inv, &S.T, &S.Hn, &S.y, &S.scal, &S.M1};
    for (size_t k = 0; k < zs.small.size(); ++k) {
      *f[k] = p;
      p += zs.small[k];
    }
  }
  S.status = sc.stat;
  S.m = m;
  S.s = 1;
  S.ldh = ldh;
  S.ldg = m + 4;
  S.ldt = m + 3;
  double* Q = sc.vec;                          // N x (m+1), then 2 unused columns
  double* r = sc.vec + (size_t)(m + 3) * N;
  double* u = r + N;
  double* wv = u + N;
  auto Qc = [&](int j) { return Q + (size_t)j * N; };
  const int nblk = (int)std::min<int64_t>(kGramBlocks, (N + 255) / 256);
  PhaseClock clk;
  clk.st = st;
  clk.on = sc.timed;
  auto dot = [&](const double* a, const double* c, double* out) -> int {
    note_launch(2);
    k_dot_partial<<<nblk, 256, 0, st>>>(N, a, c, sc.part);
    k_dot_final<<<1, 256, 0, st>>>(nblk, sc.part, out);
    return cudaGetLastError() == cudaSuccess ? SPAND_OK : SPAND_ERR_CUDA;
  };
  auto applyM = [&](const double* in, double* out) -> int {
    if (!M) return cudaMemcpyAsync(out, in, N * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess
                       ? SPAND_OK : SPAND_ERR_CUDA;
    return factor_apply(M, in, out, tr, st);
  };
  double hs[8];
  auto read_scal = [&]() -> int {   // scal[0..4] in one read
    if (cudaMemcpyAsync(hs, S.scal, 5 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SPAND_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SPAND_ERR_CUDA;
    return SPAND_OK;
  };
  int status = dot(b, b, S.scal + 2);
  if (status == SPAND_OK) status = read_scal();
  const double bn = sqrt(hs[2]);
  int iters = 0;
  double est_rel = INFINITY;
  while (status == SPAND_OK) {
    // ---- true residual r = b - A x
    clk.mark(PH_SPMV);
    status = spmv_fused(A, x, r, tr, -1.0, 1.0, b, 0.0, nullptr, st);
    if (status) break;
    clk.mark(PH_ORTH);
    status = dot(r, r, S.scal + 2);
    if (status) break;
    stl.reductions++;
    clk.mark(PH_SMALL);
    status = read_scal();
    if (status) break;
    const double beta = sqrt(hs[2]);
    stl.true_relres = bn > 0 ? beta / bn : beta;
    if (!std::isfinite(beta)) {
      status = SPAND_ERR_NONFINITE;
      break;
    }
    if (stl.true_relres <= opts->tol) break;
    if (iters >= opts->max_iters) {
      status = SPAND_ERR_NOT_CONVERGED;
      break;
    }
    const int mc = std::min(m, opts->max_iters - iters);
    note_launch();
    k_small<<<1, 256, 0, st>>>(S, MODE_INIT, 0, 0);
    clk.mark(PH_ORTH);
    status = scale_copy(N, r, Qc(0), S.scal + 1, 1, st);   // q0 = r / beta
    if (status) break;
    int k_cols = 0;
    for (int j = 0; j < mc; ++j) {
      clk.mark(PH_APPLY);
      status = applyM(Qc(j), u);
      if (status) break;
      clk.mark(PH_SPMV);
      status = spmv_fused(A, u, wv, tr, 1.0, 0.0, nullptr, 0.0, nullptr, st);
      if (status) break;
      clk.mark(PH_ORTH);
      for (int i = 0; i <= j && !status; ++i) {
        double* hij = S.H + i + (size_t)j * ldh;
        status = dot(Qc(i), wv, hij);
        if (status == SPAND_OK) status = axpy_dev(N, hij, -1.0, Qc(i), wv, st);
      }
      if (status) break;
      status = dot(wv, wv, S.scal + 2);
      if (status) break;
      stl.reductions += j + 2;
      clk.mark(PH_SMALL);
      note_launch();
      k_small<<<1, 256, 0, st>>>(S, MODE_ARNOLDI, j, 0);
      clk.mark(PH_ORTH);
      status = scale_copy(N, wv, Qc(j + 1), S.scal + 4, 1, st);
      if (status) break;
      clk.mark(PH_SMALL);
      status = read_scal();
      if (status) break;
      ++iters;
      ++k_cols;
      est_rel = hs[0] / bn;
      if (!std::isfinite(est_rel)) {
        status = SPAND_ERR_NONFINITE;
        break;
      }
      if (est_rel <= opts->tol || hs[4] == 0.0) break;
    }
    if (status) break;
    // ---- x += M^-1 (Q_{0:k} y)
    clk.mark(PH_SMALL);
    note_launch();
    k_small<<<1, 256, 0, st>>>(S, MODE_SOLVE, k_cols, 0);
    status = block_update(N, 1, 0, nullptr, N, nullptr, k_cols, Qc(0), N, S.y, k_cols, wv, N, 0, st);
    if (status) break;
    clk.mark(PH_APPLY);
    status = applyM(wv, u);     // wv = -Q y
    if (status) break;
    clk.mark(PH_SMALL);
    status = axpy_dev(N, S.scal + 7, -1.0, u, x, st);   // scal[7] = 1
    if (status) break;
    stl.restarts++;
    if (cudaGetLastError() != cudaSuccess) status = SPAND_ERR_CUDA;
  }
  clk.mark(PH_SMALL);
  stl.iters = iters;
  stl.est_relres = est_rel;
  if (cudaStreamSynchronize(st) != cudaSuccess && status == SPAND_OK) status = SPAND_ERR_CUDA;
  clk.finish(stl);
  if (stats) *stats = stl;
  return status;
}

// Device scratch of one solve (released on the stream).
struct OwnedScratch {
  GmresScratch sc{};
  cudaStream_t st = nullptr;
  int alloc(const GmresSizes& zs, int64_t N, cudaStream_t s) {
    st = s;
    sc.timed = true;
    if (pool_alloc((void**)&sc.small, zs.small_tot * sizeof(double), st) != cudaSuccess ||
        pool_alloc((void**)&sc.vec, zs.nvec * N * sizeof(double), st) != cudaSuccess ||
        pool_alloc((void**)&sc.part, zs.part * sizeof(double), st) != cudaSuccess ||
        pool_alloc((void**)&sc.stat, 4 * sizeof(int), st) != cudaSuccess ||
        pool_alloc((void**)&sc.dZ, zs.maxptr * sizeof(double*), st) != cudaSuccess ||
        pool_alloc((void**)&sc.dY, 64 * sizeof(double*), st) != cudaSuccess) {
      cudaGetLastError();
      return SPAND_ERR_NOMEM;
    }
    return SPAND_OK;
  }
  ~OwnedScratch() {
    for (void* p : {(void*)sc.small, (void*)sc.vec, (void*)sc.part, (void*)sc.stat, (void*)sc.dZ, (void*)sc.dY})
      if (p) cudaFreeAsync(p, st);
  }
};

}  // namespace
}  // namespace spand

extern "C" int sstep_gmres_solve(const bsr_matrix* A, spand_factor_t M, const double* b, double* x,
                                 const gmres_opts* opts, gmres_stats* stats, cudaStream_t st) {
  using namespace spand;
  const int v = gmres_validate(A, M, b, x, opts);
  if (v != SPAND_OK) return v;
  const int64_t N = (int64_t)A->K * A->B;
  int status;
  {
    OwnedScratch os;
    status = os.alloc(gmres_sizes(opts->restart, opts->s), N, st);
    if (status == SPAND_OK) status = sstep_core(A, M, b, x, opts, stats, st, os.sc);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && status == SPAND_OK) status = SPAND_ERR_CUDA;
  return status;
}

extern "C" int gmres_solve(const bsr_matrix* A, spand_factor_t M, const double* b, double* x,
                           const gmres_opts* opts, gmres_stats* stats, cudaStream_t st) {
  using namespace spand;
  if (!opts) return SPAND_ERR_ARG;
  gmres_opts o1 = *opts;
  o1.s = 1;                       // Algorithm 1 has no block size
  const int v = gmres_validate(A, M, b, x, &o1);
  if (v != SPAND_OK) return v;
  const int64_t N = (int64_t)A->K * A->B;
  int status;
  {
    OwnedScratch os;
    status = os.alloc(gmres_sizes(o1.restart, 1), N, st);
    if (status == SPAND_OK) status = mgs_core(A, M, b, x, &o1, stats, st, os.sc);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && status == SPAND_OK) status = SPAND_ERR_CUDA;
  return status;
}


// ------------------------------------------------------------------ batched solve
// Independent systems solved concurrently: each on its own stream (ordered
// after the caller's stream by an event, and the caller's stream after all of
// them), driven by a small pool of host threads, so that one system's host
// round trips overlap the others' kernels.
extern "C" int sstep_gmres_solve_batched(int nsys, const bsr_matrix* A, const spand_factor_t* M,
                                         const double* const* b, double* const* x, const gmres_opts* opts,
                                         gmres_stats* stats, int* status, cudaStream_t st) {
  using namespace spand;
  if (nsys <= 0 || !A || !b || !x || !opts || !stats || !status) return SPAND_ERR_ARG;
  for (int q = 0; q < nsys; ++q) {
    status[q] = SPAND_ERR_ARG;
    const int v = gmres_validate(&A[q], M ? M[q] : nullptr, b[q], x[q], &opts[q]);
    if (v != SPAND_OK) return v;
  }
  int dev = 0;
  SPAND_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<cudaStream_t> ss(nsys, nullptr);
  std::vector<cudaEvent_t> done(nsys, nullptr);
  cudaEvent_t start = nullptr;
  auto cleanup = [&] {
    for (int q = 0; q < nsys; ++q) {
      if (done[q]) cudaEventDestroy(done[q]);
      if (ss[q]) cudaStreamDestroy(ss[q]);
    }
    if (start) cudaEventDestroy(start);
  };
  int rc = SPAND_OK;
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) rc = SPAND_ERR_CUDA;
  for (int q = 0; q < nsys && rc == SPAND_OK; ++q)
    if (cudaStreamCreateWithFlags(&ss[q], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done[q], cudaEventDisableTiming) != cudaSuccess)
      rc = SPAND_ERR_CUDA;
  if (rc == SPAND_OK && cudaEventRecord(start, st) != cudaSuccess) rc = SPAND_ERR_CUDA;
  for (int q = 0; q < nsys && rc == SPAND_OK; ++q)
    if (cudaStreamWaitEvent(ss[q], start, 0) != cudaSuccess) rc = SPAND_ERR_CUDA;
  if (rc != SPAND_OK) {
    cudaGetLastError();
    cleanup();
    return rc;
  }
  std::atomic<int> next{0};
  auto worker = [&] {
    cudaSetDevice(dev);
    for (int q = next++; q < nsys; q = next++)
      status[q] = sstep_gmres_solve(&A[q], M ? M[q] : nullptr, b[q], x[q], &opts[q], &stats[q], ss[q]);
  };
  const int nthr = std::max(1, std::min(nsys, 16));
  std::vector<std::thread> pool;
  for (int t = 1; t < nthr; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  for (int q = 0; q < nsys; ++q) {
    if (cudaEventRecord(done[q], ss[q]) != cudaSuccess || cudaStreamWaitEvent(st, done[q], 0) != cudaSuccess)
      rc = SPAND_ERR_CUDA;
  }
  cleanup();
  if (rc != SPAND_OK) return rc;
  for (int q = 0; q < nsys; ++q)
    if (status[q] != SPAND_OK) return status[q];
  return SPAND_OK;
}

// ------------------------------------------------------------------ no-allocation variant
// Same solve as sstep_gmres_solve, for callers that must not allocate device
// memory while they run: for example a host program that hands all device
// memory to its own pool allocator at start-up, or one that runs under a fixed
// device-memory budget and cannot afford an allocation failing in mid-solve.
// Its scratch (basis vectors, Gram partial sums, small dense work, pointer
// tables) lives in one fixed file-scope device array instead.
namespace spand {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB on every GPU that loads the library
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device.  Host code may
// not use g_noalloc_scratch directly: its name there is a host-side stand-in.
int noalloc_base(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPAND_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SPAND_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPAND_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return SPAND_OK;
}

}  // namespace
}  // namespace spand

extern "C" int sstep_gmres_solve_noalloc(const bsr_matrix* A, spand_factor_t M, const double* b, double* x,
                                         const gmres_opts* opts, gmres_stats* stats, cudaStream_t st) {
  using namespace spand;
  const int v = gmres_validate(A, M, b, x, opts);
  if (v != SPAND_OK) return v;
  const int64_t N = (int64_t)A->K * A->B;
  const GmresSizes zs = gmres_sizes(opts->restart, opts->s);
  const size_t b_small = align256(zs.small_tot * sizeof(double));
  const size_t b_vec = align256(zs.nvec * (size_t)N * sizeof(double));
  const size_t b_part = align256(zs.part * sizeof(double));
  const size_t b_stat = align256(4 * sizeof(int));
  const size_t b_z = align256(zs.maxptr * sizeof(double*));
  const size_t b_y = align256(64 * sizeof(double*));
  if (b_small + b_vec + b_part + b_stat + b_z + b_y > kNoAllocScratchBytes) return SPAND_ERR_SCRATCH;
  unsigned char* base = nullptr;
  const int sb = noalloc_base(&base);
  if (sb != SPAND_OK) return sb;
  GmresScratch sc;
  unsigned char* p = base;
  sc.small = reinterpret_cast<double*>(p);
  p += b_small;
  sc.vec = reinterpret_cast<double*>(p);
  p += b_vec;
  sc.part = reinterpret_cast<double*>(p);
  p += b_part;
  sc.stat = reinterpret_cast<int*>(p);
  p += b_stat;
  sc.dZ = reinterpret_cast<const double**>(p);
  p += b_z;
  sc.dY = reinterpret_cast<const double**>(p);
  // the factor's apply graph is built on its first use, and building it
  // allocates: here the apply's launches go on the stream one by one
  sc.direct_apply = true;
  // sstep_core clears the small-matrix and status words it needs zeroed; the
  // vectors and partial sums are always written before they are read.
  return sstep_core(A, M, b, x, opts, stats, st, sc);
}

extern "C" size_t sstep_gmres_noalloc_capacity(void) { return spand::kNoAllocScratchBytes; }

// ------------------------------------------------------------------ matrix powers
// The Newton-basis matrix-powers step of Algorithm 2 on its own: with M the
// preconditioner, V[:, k] = A M^-1 V[:, k-1] - Re(t_k) V[:, k-1]
// (+ Im(t_k)^2 V[:, k-2] for the second shift of a conjugate pair), V[:, -1] = v0.
// Each step is the preconditioner's sweeps followed by one shifted block SpMV
// that reads the preconditioner's output vector in place (FP32 in the mixed
// form): no conversion pass and no FP64 copy of M^-1 v_k.
extern "C" int sstep_matrix_powers(const bsr_matrix* A, spand_factor_t M, const double* v0, int s,
                                   const double* shifts_re, const double* shifts_im, double* V, int transpose,
                                   cudaStream_t st) {
  using namespace spand;
  if (!A || !v0 || !V || !shifts_re || !shifts_im || !A->row_ptr || !A->col || !A->val || s < 1 || s > 64)
    return SPAND_ERR_ARG;
  const int64_t N = (int64_t)A->K * A->B;
  if (M && factor_size(M) != N) return SPAND_ERR_ARG;
  if (v0 >= V && v0 < V + (size_t)s * N) return SPAND_ERR_ARG;     // v0 may not lie in V
  for (int k = 0; k < s; ++k)
    if (shifts_im[k] < 0 && (k == 0 || shifts_im[k - 1] != -shifts_im[k] || shifts_re[k - 1] != shifts_re[k]))
      return SPAND_ERR_ARG;                                          // a pair's second shift follows its first
  const int tr = transpose ? 1 : 0;
  for (int k = 0; k < s; ++k) {
    const double* vk = (k == 0) ? v0 : V + (size_t)(k - 1) * N;
    const double* vkm = (k == 0) ? nullptr : ((k == 1) ? v0 : V + (size_t)(k - 2) * N);
    const double a2 = shifts_im[k] < 0 ? shifts_im[k] * shifts_im[k] : 0.0;
    double* out = V + (size_t)k * N;
    int status;
    if (!M) {
      status = spmv_fused(A, vk, out, tr, 1.0, -shifts_re[k], vk, a2, shifts_im[k] < 0 ? vkm : nullptr, st);
    } else {
      const void* w = nullptr;
      int wf = 0;
      status = factor_apply_slot(M, vk, tr, st, false, &w, &wf);
      if (status == SPAND_OK)
        status = spmv_fused_x(A, w, wf, out, tr, 1.0, -shifts_re[k], vk, a2, shifts_im[k] < 0 ? vkm : nullptr, st);
    }
    if (status != SPAND_OK) return status;
  }
  return SPAND_OK;
}
