// DG residual and Jacobian assembly for 2D Euler (Sec. 2.1.2, Eqs. 3-8).
//
// One CTA per element computes its whole block row: the volume term of Eq. 7
// and its exact derivative, the surface terms of its four faces (Rusanov flux
// evaluated in the face's global L->R orientation, so both neighbours see the
// same flux and the same branch of the max), the mass term M/dtau (Eq. 6) and
// the residual entries.  Each face is evaluated by both adjacent elements;
// no scratch, no atomics, deterministic.  A first pass computes the CFL time
// step of Eq. 8.  Gauss-Legendre nodes (Newton iteration on P_q) and the
// orthonormal Legendre basis (three-term recurrence) are tabulated once on the
// host for the reference element and passed to the kernels by value.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

constexpr int PMAX = 3;
constexpr int QMAX = PMAX + 2;            // points per direction
constexpr int NPMAX = (PMAX + 1) * (PMAX + 1);
constexpr int VQMAX = QMAX * QMAX;

struct Flow {
  double gamma, uinf[4], cfl;
  int bc_wall;
};

// Reference-element tables, built once on the host and passed by value:
// Gauss-Legendre rule, basis values / derivatives at the q x q volume points
// (xi fastest) and basis values on the four local faces.
struct Tables {
  int q, np, Q;
  double tq[QMAX], wq[QMAX];
  double psi[VQMAX][NPMAX], pxi[VQMAX][NPMAX], peta[VQMAX][NPMAX];
  double fpsi[4][QMAX][NPMAX];
};

// orthonormal Legendre values / derivatives of degree 0..p at t
__host__ __device__ void legendre(int p, double t, double* V, double* D) {
  double P0 = 1.0, P1 = t, dP0 = 0.0, dP1 = 1.0;
  double P[PMAX + 1], dP[PMAX + 1];
  P[0] = P0;
  dP[0] = dP0;
  if (p >= 1) {
    P[1] = P1;
    dP[1] = dP1;
  }
  for (int a = 1; a < p; ++a) {
    P[a + 1] = ((2 * a + 1) * t * P[a] - a * P[a - 1]) / (a + 1);
    dP[a + 1] = (a + 1) * P[a] + t * dP[a];
  }
  for (int a = 0; a <= p; ++a) {
    double s = sqrt((2 * a + 1) * 0.5);
    V[a] = s * P[a];
    D[a] = s * dP[a];
  }
}

// Gauss-Legendre rule with q points on [-1, 1], ascending nodes
__host__ __device__ void gauss_rule(int q, double* t, double* w) {
  for (int i = 0; i < q; ++i) {
    double x = cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < q; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = q * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < q; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = q * (x * p1 - p0) / (x * x - 1.0);
    }
    t[q - 1 - i] = x;
    w[q - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

__host__ __device__ void basis_at(int p, double xi, double eta, double* psi, double* pxi, double* peta) {
  double Vx[PMAX + 1], Dx[PMAX + 1], Ve[PMAX + 1], De[PMAX + 1];
  legendre(p, xi, Vx, Dx);
  legendre(p, eta, Ve, De);
  for (int b = 0; b <= p; ++b)
    for (int a = 0; a <= p; ++a) {
      int m = b * (p + 1) + a;
      psi[m] = Vx[a] * Ve[b];
      if (pxi) pxi[m] = Dx[a] * Ve[b];
      if (peta) peta[m] = Vx[a] * De[b];
    }
}

// local face f of the reference square at parameter t: 0 east (1,t), 1 west (-1,t),
// 2 north (t,1), 3 south (t,-1)
__host__ __device__ void face_point(int f, double t, double& xi, double& eta) {
  if (f == 0) { xi = 1.0; eta = t; }
  else if (f == 1) { xi = -1.0; eta = t; }
  else if (f == 2) { xi = t; eta = 1.0; }
  else { xi = t; eta = -1.0; }
}

__host__ __device__ bool primitive(const double* U, double g, double& rho, double& ux, double& uy, double& p) {
  rho = U[0];
  ux = U[1] / rho;
  uy = U[2] / rho;
  p = (g - 1.0) * (U[3] - 0.5 * rho * (ux * ux + uy * uy));
  return rho > 0.0 && p > 0.0 && isfinite(p);
}

// F.n and d(F.n)/dU (row-major 4x4)
__host__ __device__ void flux_n(const double* U, double nx, double ny, double g, double* F, double* A) {
  double rho, ux, uy, p;
  primitive(U, g, rho, ux, uy, p);
  const double E = U[3], g1 = g - 1.0;
  const double vn = ux * nx + uy * ny;
  F[0] = rho * vn;
  F[1] = U[1] * vn + p * nx;
  F[2] = U[2] * vn + p * ny;
  F[3] = (E + p) * vn;
  if (!A) return;
  const double phi = 0.5 * g1 * (ux * ux + uy * uy), H = (E + p) / rho;
  A[0] = 0.0; A[1] = nx; A[2] = ny; A[3] = 0.0;
  A[4] = phi * nx - ux * vn; A[5] = vn + ux * nx - g1 * ux * nx; A[6] = ux * ny - g1 * uy * nx; A[7] = g1 * nx;
  A[8] = phi * ny - uy * vn; A[9] = uy * nx - g1 * ux * ny; A[10] = vn + uy * ny - g1 * uy * ny; A[11] = g1 * ny;
  A[12] = vn * (phi - H); A[13] = H * nx - g1 * ux * vn; A[14] = H * ny - g1 * uy * vn; A[15] = g * vn;
}

// a = |v.n| + c and da/dU
__host__ __device__ double wave(const double* U, double nx, double ny, double g, double* da) {
  double rho, ux, uy, p;
  primitive(U, g, rho, ux, uy, p);
  const double c = sqrt(g * p / rho), vn = ux * nx + uy * ny, g1 = g - 1.0;
  const double sg = vn >= 0.0 ? 1.0 : -1.0;
  const double k = g / (2.0 * c * rho);
  da[0] = sg * (-vn / rho) + k * 0.5 * g1 * (ux * ux + uy * uy) - c / (2.0 * rho);
  da[1] = sg * (nx / rho) - k * g1 * ux;
  da[2] = sg * (ny / rho) - k * g1 * uy;
  da[3] = k * g1;
  return fabs(vn) + c;
}

// Rusanov F*.n with dF/dUL, dF/dUR (row-major 4x4); L branch of the max on ties
__host__ __device__ void rusanov(const double* UL, const double* UR, double nx, double ny, double g,
                        double* F, double* dL, double* dR) {
  double FL[4], FR[4], AL[16], AR[16], daL[4], daR[4];
  flux_n(UL, nx, ny, g, FL, AL);
  flux_n(UR, nx, ny, g, FR, AR);
  double aL = wave(UL, nx, ny, g, daL), aR = wave(UR, nx, ny, g, daR);
  const bool takeL = aL >= aR;
  const double lam = takeL ? aL : aR;
  double dU[4];
  for (int v = 0; v < 4; ++v) {
    dU[v] = UR[v] - UL[v];
    F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * dU[v];
  }
  for (int v = 0; v < 4; ++v)
    for (int w = 0; w < 4; ++w) {
      double id = (v == w) ? 1.0 : 0.0;
      dL[v * 4 + w] = 0.5 * AL[v * 4 + w] + 0.5 * lam * id - 0.5 * dU[v] * (takeL ? daL[w] : 0.0);
      dR[v * 4 + w] = 0.5 * AR[v * 4 + w] - 0.5 * lam * id - 0.5 * dU[v] * (takeL ? 0.0 : daR[w]);
    }
}

__host__ __device__ void corners(const double* X, int n_theta, int i, int j, double C[4][2]) {
  const int jp = (j + 1) % n_theta;
  const int idx[4] = {i * n_theta + j, i * n_theta + jp, (i + 1) * n_theta + jp, (i + 1) * n_theta + j};
  for (int c = 0; c < 4; ++c) {
    C[c][0] = X[2 * idx[c]];
    C[c][1] = X[2 * idx[c] + 1];
  }
}

__host__ __device__ void jac_map(const double C[4][2], double xi, double eta, double* dxi, double* deta) {
  for (int d = 0; d < 2; ++d) {
    dxi[d] = 0.25 * (-(1 - eta) * C[0][d] + (1 - eta) * C[1][d] + (1 + eta) * C[2][d] - (1 + eta) * C[3][d]);
    deta[d] = 0.25 * (-(1 - xi) * C[0][d] - (1 + xi) * C[1][d] + (1 + xi) * C[2][d] + (1 - xi) * C[3][d]);
  }
}

__device__ inline void atomic_min_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// ------------------------------------------------------------------ time step
__global__ void k_time_step(const double* X, int n_theta, int n_r, int p, const double* uh, Flow fl,
                            double* dtau, int* bad, const __grid_constant__ Tables T) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_theta * n_r) return;
  const int q = T.q, np = T.np;
  const int i = e / n_theta, j = e % n_theta;
  double C[4][2];
  corners(X, n_theta, i, j, C);
  double area = 0.0, smax = 0.0;
  for (int b = 0; b < q; ++b)
    for (int a = 0; a < q; ++a) {
      double dxi[2], deta[2];
      jac_map(C, T.tq[a], T.tq[b], dxi, deta);
      area += T.wq[a] * T.wq[b] * (dxi[0] * deta[1] - deta[0] * dxi[1]);
      const int pt = b * q + a;
      double U[4] = {0, 0, 0, 0};
      for (int m = 0; m < np; ++m)
        for (int v = 0; v < 4; ++v) U[v] += T.psi[pt][m] * uh[(size_t)e * np * 4 + m * 4 + v];
      double rho, ux, uy, pr;
      if (!primitive(U, fl.gamma, rho, ux, uy, pr)) atomicExch(bad, 1);
      smax = fmax(smax, sqrt(ux * ux + uy * uy) + sqrt(fl.gamma * pr / rho));
    }
  double perim = 0.0;
  for (int c = 0; c < 4; ++c) {
    double dx = C[(c + 1) % 4][0] - C[c][0], dy = C[(c + 1) % 4][1] - C[c][1];
    perim += sqrt(dx * dx + dy * dy);
  }
  const double lam = smax * (2 * p + 1) * perim / area;
  double v = fl.cfl / lam;
  if (!(v > 0.0) || !isfinite(v)) {
    atomicExch(bad, 1);
    return;
  }
  atomic_min_pos(dtau, v);
}

// ------------------------------------------------------------------ assembly
struct Smem {
  double tq[QMAX], wq[QMAX];
  double uh[5][NPMAX][4];                   // self + 4 neighbours
  double psi[VQMAX][NPMAX], gx[VQMAX][NPMAX], gy[VQMAX][NPMAX];
  double wdet[VQMAX];
  double Fx[VQMAX][4], Fy[VQMAX][4], Ax[VQMAX][16], Ay[VQMAX][16];
  double fpsi_s[4][QMAX][NPMAX], fpsi_n[4][QMAX][NPMAX];
  double hws[4][QMAX];                      // signed half-length x weight
  double Fs[4][QMAX][4], dFs[4][QMAX][16], dFn[4][QMAX][16];
  int nb[4];                                // neighbour element per local face or -1
  int col_rank[5];                          // BSR position of self / faces
};

__global__ void __launch_bounds__(256) k_assemble(const double* X, int n_theta, int n_r, int p,
                                                  const double* uh, Flow fl, const double* dtau_p,
                                                  const int* row_ptr, double* rhs, double* val, int* bad,
                                                  const __grid_constant__ Tables T) {
  extern __shared__ double smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int e = blockIdx.x;
  const int i = e / n_theta, j = e % n_theta;
  const int q = p + 2, np = (p + 1) * (p + 1), Q = q * q, B = 4 * np;
  const int tid = threadIdx.x;
  const double g = fl.gamma;
  if (tid < QMAX) {
    S.tq[tid] = T.tq[tid];
    S.wq[tid] = T.wq[tid];
  }
  if (tid == 0) {
    const int jp = (j + 1) % n_theta, jm = (j + n_theta - 1) % n_theta;
    S.nb[0] = i * n_theta + jp;                          // east: self is L
    S.nb[1] = i * n_theta + jm;                          // west: self is R
    S.nb[2] = (i < n_r - 1) ? e + n_theta : -1;          // north: self is L (outer boundary if -1)
    S.nb[3] = (i > 0) ? e - n_theta : -1;                // south: self is R (airfoil if -1)
    // BSR order of the row: columns ascending
    int cols[5] = {e, S.nb[0], S.nb[1], S.nb[2], S.nb[3]};
    for (int a = 0; a < 5; ++a) {
      int r = 0;
      if (cols[a] < 0) { S.col_rank[a] = -1; continue; }
      for (int b = 0; b < 5; ++b)
        if (cols[b] >= 0 && cols[b] < cols[a]) ++r;
      S.col_rank[a] = r;
    }
  }
  __syncthreads();
  for (int t = tid; t < 5 * np * 4; t += blockDim.x) {
    int s = t / (np * 4), r = t % (np * 4);
    int el = (s == 0) ? e : S.nb[s - 1];
    S.uh[s][r / 4][r % 4] = (el >= 0) ? uh[(size_t)el * np * 4 + r] : 0.0;
  }
  __syncthreads();
  double C[4][2];
  corners(X, n_theta, i, j, C);
  if (tid < Q) {
    // ---- volume point
    const int a = tid % q, b = tid / q;
    const double xi = S.tq[a], eta = S.tq[b], w = S.wq[a] * S.wq[b];
    double dxi[2], deta[2];
    jac_map(C, xi, eta, dxi, deta);
    const double det = dxi[0] * deta[1] - deta[0] * dxi[1];
    const double* ps = T.psi[tid];
    const double* px = T.pxi[tid];
    const double* pe = T.peta[tid];
    double U[4] = {0, 0, 0, 0};
    for (int m = 0; m < np; ++m) {
      S.psi[tid][m] = ps[m];
      S.gx[tid][m] = w * (deta[1] * px[m] - dxi[1] * pe[m]);
      S.gy[tid][m] = w * (-deta[0] * px[m] + dxi[0] * pe[m]);
      for (int v = 0; v < 4; ++v) U[v] += ps[m] * S.uh[0][m][v];
    }
    S.wdet[tid] = w * det;
    double rho, ux, uy, pr;
    if (!primitive(U, g, rho, ux, uy, pr)) atomicExch(bad, 1);
    flux_n(U, 1.0, 0.0, g, S.Fx[tid], S.Ax[tid]);
    flux_n(U, 0.0, 1.0, g, S.Fy[tid], S.Ay[tid]);
  } else if (tid >= 32 && tid < 32 + 4 * q) {
    // ---- face point: local face f, point k
    const int f = (tid - 32) / q, k = (tid - 32) % q;
    const double t = S.tq[k];
    int node_a, node_b;                                   // edge end points (node ids)
    const int jp = (j + 1) % n_theta;
    bool self_is_L;
    int nf;                                               // neighbour's local face
    double nx, ny;
    if (f == 0) { node_a = i * n_theta + jp; node_b = (i + 1) * n_theta + jp; self_is_L = true; nf = 1; }
    else if (f == 1) { node_a = i * n_theta + j; node_b = (i + 1) * n_theta + j; self_is_L = false; nf = 0; }
    else if (f == 2) { node_a = (i + 1) * n_theta + j; node_b = (i + 1) * n_theta + jp; self_is_L = true; nf = 3; }
    else { node_a = i * n_theta + j; node_b = i * n_theta + jp; self_is_L = false; nf = 2; }
    const double tx = X[2 * node_b] - X[2 * node_a], ty = X[2 * node_b + 1] - X[2 * node_a + 1];
    const double len = sqrt(tx * tx + ty * ty);
    // global L->R normal: east/west faces use the L element's east edge, north/south its north edge
    if (f <= 1) { nx = ty / len; ny = -tx / len; }
    else { nx = -ty / len; ny = tx / len; }
    const int nbe = S.nb[f];
    const bool boundary = nbe < 0;
    if (boundary && f == 3) {            // airfoil: the element is L with outward normal
      nx = -nx; ny = -ny; self_is_L = true;
    }
    (void)t;
    const double* ps = T.fpsi[f][k];
    const double* pn = T.fpsi[nf][k];
    double Us[4] = {0, 0, 0, 0}, Un[4] = {0, 0, 0, 0};
    for (int m = 0; m < np; ++m)
      for (int v = 0; v < 4; ++v) {
        Us[v] += ps[m] * S.uh[0][m][v];
        if (!boundary) Un[v] += pn[m] * S.uh[f + 1][m][v];
      }
    double W[16];
    bool wall = false;
    if (boundary) {
      wall = (f == 3) && fl.bc_wall;
      if (wall) {
        for (int a = 0; a < 16; ++a) W[a] = 0.0;
        W[0] = 1.0; W[15] = 1.0;
        W[5] = 1.0 - 2.0 * nx * nx; W[6] = -2.0 * nx * ny;
        W[9] = -2.0 * nx * ny; W[10] = 1.0 - 2.0 * ny * ny;
        for (int v = 0; v < 4; ++v) {
          Un[v] = 0.0;
          for (int w2 = 0; w2 < 4; ++w2) Un[v] += W[v * 4 + w2] * Us[w2];
        }
      } else {
        for (int v = 0; v < 4; ++v) Un[v] = fl.uinf[v];
      }
    }
    double F[4], dL[16], dR[16];
    const double* UL = self_is_L ? Us : Un;
    const double* UR = self_is_L ? Un : Us;
    {
      double r0, a0, b0, c0;
      if (!primitive(Us, g, r0, a0, b0, c0) || !primitive(Un, g, r0, a0, b0, c0)) atomicExch(bad, 1);
    }
    rusanov(UL, UR, nx, ny, g, F, dL, dR);
    const double sgn = self_is_L ? 1.0 : -1.0;
    const double hw = sgn * 0.5 * len * S.wq[k];
    S.hws[f][k] = hw;
    for (int m = 0; m < np; ++m) {
      S.fpsi_s[f][k][m] = ps[m];
      S.fpsi_n[f][k][m] = boundary ? 0.0 : pn[m];
    }
    for (int v = 0; v < 4; ++v) S.Fs[f][k][v] = F[v];
    const double* dSelf = self_is_L ? dL : dR;
    const double* dNb = self_is_L ? dR : dL;
    for (int a = 0; a < 16; ++a) {
      double ds = dSelf[a];
      if (wall) {                                          // chain rule through the ghost state
        const int v = a / 4, w2 = a % 4;
        for (int u = 0; u < 4; ++u) ds += dR[v * 4 + u] * W[u * 4 + w2];
      }
      S.dFs[f][k][a] = ds;
      S.dFn[f][k][a] = boundary ? 0.0 : dNb[a];
    }
  }
  __syncthreads();
  const double inv_dt = 1.0 / *dtau_p;
  // ---- residual
  for (int t = tid; t < np * 4; t += blockDim.x) {
    const int m = t / 4, v = t % 4;
    double r = 0.0;
    for (int a = 0; a < Q; ++a) r -= S.gx[a][m] * S.Fx[a][v] + S.gy[a][m] * S.Fy[a][v];
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < q; ++k) r += S.hws[f][k] * S.fpsi_s[f][k][m] * S.Fs[f][k][v];
    rhs[(size_t)e * B + t] = -r;
  }
  // ---- Jacobian blocks: thread per (row mode mi, column mode mj)
  const size_t bb = (size_t)B * B;
  const int rp = row_ptr[e];
  for (int t = tid; t < np * np; t += blockDim.x) {
    const int mi = t / np, mj = t % np;
    double Jd[16], Jo[4][16];
    for (int a = 0; a < 16; ++a) {
      Jd[a] = 0.0;
      for (int f = 0; f < 4; ++f) Jo[f][a] = 0.0;
    }
    double mass = 0.0;
    for (int a = 0; a < Q; ++a) {
      const double cx = S.gx[a][mi] * S.psi[a][mj], cy = S.gy[a][mi] * S.psi[a][mj];
      for (int vw = 0; vw < 16; ++vw) Jd[vw] -= cx * S.Ax[a][vw] + cy * S.Ay[a][vw];
      mass += S.wdet[a] * S.psi[a][mi] * S.psi[a][mj];
    }
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < q; ++k) {
        const double cs = S.hws[f][k] * S.fpsi_s[f][k][mi];
        const double c1 = cs * S.fpsi_s[f][k][mj], c2 = cs * S.fpsi_n[f][k][mj];
        for (int vw = 0; vw < 16; ++vw) {
          Jd[vw] += c1 * S.dFs[f][k][vw];
          Jo[f][vw] += c2 * S.dFn[f][k][vw];
        }
      }
    for (int v = 0; v < 4; ++v) Jd[v * 4 + v] += mass * inv_dt;
    for (int v = 0; v < 4; ++v)
      for (int w = 0; w < 4; ++w) {
        const int r = mi * 4 + v, c = mj * 4 + w;
        val[(size_t)(rp + S.col_rank[0]) * bb + (size_t)c * B + r] = Jd[v * 4 + w];
        for (int f = 0; f < 4; ++f)
          if (S.nb[f] >= 0)
            val[(size_t)(rp + S.col_rank[f + 1]) * bb + (size_t)c * B + r] = Jo[f][v * 4 + w];
      }
  }
}

}  // namespace

extern "C" int dg_assemble_jacobian(const dg_mesh* mesh, int p, const double* u_hat,
                                    const dg_flow_params* flow, double* rhs, bsr_matrix* A,
                                    double* dtau_out, cudaStream_t stream) {
  if (!mesh || !flow || !A || !u_hat || !rhs || !mesh->nodes || !A->row_ptr || !A->col || !A->val)
    return SPAND_ERR_ARG;
  if (p < 1 || p > PMAX || mesh->n_theta < 4 || mesh->n_r < 1) return SPAND_ERR_UNSUPPORTED;
  const int nt = mesh->n_theta, nr = mesh->n_r, K = nt * nr, B = 4 * (p + 1) * (p + 1);
  // block pattern: each element with its face neighbours, ascending columns
  std::vector<int> rp(K + 1, 0), col;
  col.reserve((size_t)5 * K);
  for (int e = 0; e < K; ++e) {
    const int i = e / nt, j = e % nt;
    int c[5], n = 0;
    c[n++] = e;
    c[n++] = i * nt + (j + 1) % nt;
    c[n++] = i * nt + (j + nt - 1) % nt;
    if (i > 0) c[n++] = e - nt;
    if (i < nr - 1) c[n++] = e + nt;
    for (int a = 1; a < n; ++a)
      for (int b = a; b > 0 && c[b] < c[b - 1]; --b) std::swap(c[b], c[b - 1]);
    for (int a = 0; a < n; ++a) col.push_back(c[a]);
    rp[e + 1] = (int)col.size();
  }
  A->K = K;
  A->B = B;
  A->nnzb = (int)col.size();
  SPAND_CUDA_TRY(cudaMemcpyAsync(A->row_ptr, rp.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, stream));
  SPAND_CUDA_TRY(cudaMemcpyAsync(A->col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, stream));
  Flow fl;
  fl.gamma = flow->gamma;
  fl.cfl = flow->cfl;
  fl.bc_wall = flow->bc_mode == SPAND_BC_WALL;
  {
    const double a = flow->alpha_deg * M_PI / 180.0, g = flow->gamma;
    const double u = flow->mach * cos(a), v = flow->mach * sin(a), pr = 1.0 / g;
    fl.uinf[0] = 1.0;
    fl.uinf[1] = u;
    fl.uinf[2] = v;
    fl.uinf[3] = pr / (g - 1.0) + 0.5 * (u * u + v * v);
  }
  Tables T;
  memset(&T, 0, sizeof(T));
  T.q = p + 2;
  T.np = (p + 1) * (p + 1);
  T.Q = T.q * T.q;
  gauss_rule(T.q, T.tq, T.wq);
  for (int b = 0; b < T.q; ++b)
    for (int a = 0; a < T.q; ++a) basis_at(p, T.tq[a], T.tq[b], T.psi[b * T.q + a], T.pxi[b * T.q + a],
                                           T.peta[b * T.q + a]);
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k < T.q; ++k) {
      double xi, eta;
      face_point(f, T.tq[k], xi, eta);
      basis_at(p, xi, eta, T.fpsi[f][k], nullptr, nullptr);
    }
  if (spand::set_dyn_smem((const void*)k_assemble, sizeof(Smem)) < (long long)sizeof(Smem)) return SPAND_ERR_UNSUPPORTED;
  double* d_scr = nullptr;  // [0] = dtau, [1] = bad flag (as int)
  SPAND_CUDA_TRY(cudaMallocAsync(&d_scr, 2 * sizeof(double), stream));
  const double big = 1e300;
  SPAND_CUDA_TRY(cudaMemcpyAsync(d_scr, &big, sizeof(double), cudaMemcpyHostToDevice, stream));
  SPAND_CUDA_TRY(cudaMemsetAsync(d_scr + 1, 0, sizeof(double), stream));
  int* d_bad = reinterpret_cast<int*>(d_scr + 1);
  spand::note_launch();
  k_time_step<<<(K + 127) / 128, 128, 0, stream>>>(mesh->nodes, nt, nr, p, u_hat, fl, d_scr, d_bad, T);
  const size_t smem = sizeof(Smem);
  spand::note_launch();
  k_assemble<<<K, 256, smem, stream>>>(mesh->nodes, nt, nr, p, u_hat, fl, d_scr, A->row_ptr, rhs,
                                       A->val, d_bad, T);
  SPAND_CUDA_TRY(cudaGetLastError());
  double h[2];
  SPAND_CUDA_TRY(cudaMemcpyAsync(h, d_scr, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
  SPAND_CUDA_TRY(cudaFreeAsync(d_scr, stream));
  SPAND_CUDA_TRY(cudaStreamSynchronize(stream));
  int badv;
  memcpy(&badv, &h[1], sizeof(int));
  if (dtau_out) *dtau_out = h[0];
  if (badv) return SPAND_ERR_NONFINITE;
  return SPAND_OK;
}
