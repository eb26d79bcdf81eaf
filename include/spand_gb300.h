/*
 * spand_gb300.h - C ABI of the GB300 (sm_103a) spaND + s-step GMRES library.
 *
 * Hot path of the implicit DG solver of arXiv 2101.01763: the linear solve of
 * one pseudo-time Newton step (Sec. 2.1.2, Eq. 5)
 *        (M/dtau + dR/du) du = -R,
 * by sparsified nested dissection (spaND, Sec. 2.2.1) used as a preconditioner
 * for s-step GMRES (Sec. 2.3, Algorithm 2).
 *
 * Conventions shared by every entry point
 *  - Return value: int status; 0 = SPAND_OK, negative = error (codes below).
 *    On error no output is guaranteed; handles stay valid and must still be
 *    destroyed.  No entry point keeps results in host globals.  The only
 *    host-side state that outlives a call is set once and then read: kernel
 *    attributes (dynamic shared-memory limits), whether the device schedules
 *    16-CTA clusters, and the per-device address cache of
 *    sstep_gmres_solve_noalloc (below).
 *  - Pointers documented as "device" must point to device memory owned by the
 *    caller (any allocator); "host" pointers are caller-owned host memory.
 *    Handles (spand_plan_t, spand_factor_t) are owned by the library and are
 *    released by the matching *_destroy.
 *  - Block-CSR (BSR) matrices: K block rows of size B = 4 (p+1)^2, 0-based
 *    int32 row_ptr[K+1] / col[nnzb] with ascending columns in a row, values
 *    val[nnzb * B * B] with block k stored column-major:
 *    element (r, c) of block k at val[k*B*B + c*B + r].
 *  - DOF numbering: element e (e = i*n_theta + j, i radial, j angular), mode
 *    m = b*(p+1) + a (degree a in xi, b in eta), variable v in
 *    (rho, rho u, rho v, E): global index e*B + m*4 + v.
 *  - Work is enqueued on the given stream; entry points that must read a
 *    device result (ranks in spand_factor, residual estimates in the GMRES
 *    loop, dtau) synchronize that stream before returning.
 */
#ifndef SPAND_GB300_H
#define SPAND_GB300_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SPAND_OK = 0,
  SPAND_ERR_ARG = -1,            /* invalid argument (null pointer, bad size)        */
  SPAND_ERR_NOMEM = -2,          /* device or host allocation failed                 */
  SPAND_ERR_ZERO_PIVOT = -3,     /* exact zero pivot in a block LU                    */
  SPAND_ERR_CHOLQR = -4,         /* CholQR Gram matrix not positive definite          */
  SPAND_ERR_NONFINITE = -5,      /* NaN/Inf met in a residual or a factor             */
  SPAND_ERR_NOT_CONVERGED = -6,  /* GMRES reached max_iters above tolerance           */
  SPAND_ERR_CUDA = -7,           /* a CUDA runtime call failed                        */
  SPAND_ERR_UNSUPPORTED = -8,    /* configuration outside the supported range         */
  SPAND_ERR_SCRATCH = -9         /* problem needs more than the fixed scratch of
                                    sstep_gmres_solve_noalloc                          */
};

enum { SPAND_BC_WALL = 0, SPAND_BC_FARFIELD = 1 };
enum { SPAND_FP64 = 0, SPAND_MIXED = 1 };
enum { SPAND_BASIS_NEWTON = 0, SPAND_BASIS_MONOMIAL = 1 };

/* Structured O-grid: nodes[(i*n_theta + j)*2 + {0,1}] = (x, y) of node (i, j),
 * i = 0..n_r (0 = airfoil), j = 0..n_theta-1 (periodic, clockwise).  Device. */
typedef struct {
  int n_theta;
  int n_r;
  const double* nodes;
} dg_mesh;

typedef struct {
  double gamma;      /* ratio of specific heats                                   */
  double mach;       /* free-stream Mach number (rho_inf = 1, p_inf = 1/gamma)     */
  double alpha_deg;  /* angle of attack in degrees                                 */
  double cfl;        /* CFL number of Eq. 8                                        */
  int bc_mode;       /* SPAND_BC_WALL (slip wall on the airfoil) or SPAND_BC_FARFIELD */
} dg_flow_params;

/* Device BSR matrix (see conventions above).  For dg_assemble_jacobian the
 * caller allocates row_ptr (K+1), col (nnzb = 5K - 2 n_theta) and val
 * (nnzb*B*B) and the library fills all three. */
typedef struct {
  int K;
  int B;
  int nnzb;
  int* row_ptr;
  int* col;
  double* val;
} bsr_matrix;

/* ---------------------------------------------------------------- assembly
 * dg_assemble_jacobian - Sec. 2.1.2 (Eqs. 3-8): modal DG discretisation of 2D
 * Euler (tensor orthonormal Legendre basis of degree p in 1..3, Gauss-Legendre
 * quadrature with p+2 points per direction, Rusanov flux), returning
 *     rhs = -R(u_hat)                       (device, N = K*B doubles)
 *     A   = M/dtau + dR/du (exact derivative; block-CSR, device)
 *     *dtau_out = min_k CFL/lambda_k        (host double)
 * with lambda_k = max over the element's quadrature points of (|v| + c)
 * times (2p+1) |dD_k| / |D_k|.  u_hat is device [K, (p+1)^2, 4] doubles.
 * Errors: SPAND_ERR_ARG, SPAND_ERR_UNSUPPORTED (p outside 1..3, n_theta < 4),
 * SPAND_ERR_NONFINITE (non-physical state), SPAND_ERR_CUDA.               */
int dg_assemble_jacobian(const dg_mesh* mesh, int p, const double* u_hat,
                         const dg_flow_params* flow, double* rhs, bsr_matrix* A,
                         double* dtau_out, cudaStream_t stream);

/* y = A x (transpose = 0) or y = A^T x (transpose = 1); FP64, device vectors
 * of length K*B.  The block-SpMV of Algorithm 2's matrix-powers step. */
int bsr_spmv(const bsr_matrix* A, const double* x, double* y, int transpose,
             cudaStream_t stream);

/* out = alpha * u v^T restricted to the block pattern of A: block k of row e
 * and column col[k] becomes alpha * u[e*B : e*B+B] v[col[k]*B : col[k]*B+B]^T
 * (column-major, like val).  With u = lambda = A^-T dL/dx and v = x,
 * alpha = -1 this is dL/dA of the adjoint of x = A^-1 b on A's pattern.
 * u, v: device FP64 vectors of length K*B; out: device nnzb*B*B doubles. */
int bsr_pattern_outer(const bsr_matrix* A, const double* u, const double* v, double alpha, double* out,
                      cudaStream_t stream);

/* ---------------------------------------------------------------- analysis
 * spand_analyze - Sec. 2.2.1 and Sec. 3.3: nested dissection of the
 * n_theta x n_r element grid (root separator = radial lines j = 0 and
 * j = n_theta/2; then recursive bisection across the longer extent, ties
 * along j, at lo + (n-1)/2; leaves at depth D or extent < 3), the interiors,
 * interfaces and merges of every level 0..D, and the block pattern with
 * fill-in.  Pattern-only (integer) work on the host; reusable for every
 * factorization of matrices on the same grid.  depth_D <= 0 selects
 * D = max(1, ceil(log2(K/32))).  Errors: SPAND_ERR_ARG, SPAND_ERR_NOMEM. */
typedef struct spand_plan_s* spand_plan_t;
int spand_analyze(int n_theta, int n_r, int B, int depth_D, spand_plan_t* out);
int spand_plan_destroy(spand_plan_t plan);

/* Plan tables, for checking against an independent implementation.  Host
 * buffers.  spand_plan_sizes: K, D, number of tree nodes and the length of
 * the serialized cluster table.  spand_plan_export writes owner[K] (tree node
 * owning each element, nodes in preorder), node_level[n_nodes] and the
 * cluster table: for each level l = 0..D: n_clusters, then per cluster
 * node, interior, n_key, key[n_key], n_elems, elems[n_elems], n_children,
 * children[n_children] (n_children = 0 at level 0). */
int spand_plan_sizes(spand_plan_t plan, int* K, int* D, int* n_nodes, int64_t* table_len);
int spand_plan_export(spand_plan_t plan, int* owner, int* node_level, int* table);

/* ---------------------------------------------------------------- factor
 * spand_factor - Sec. 2.2.1 (Eqs. 10-12), level by level: eliminate interiors
 * by row-pivoted block LU with Schur updates; scale every interface by its
 * own PLU with diag(U) split evenly (L~ = L|D|^1/2, U~ = |D|^-1/2 U); compute
 * every interface's column-pivoted Householder QR of [A_sn A_ns^T], keep the
 * rank r = #{k : |R_kk| > eps |R_00|}, compress every block to
 * Q_ic^T A_ij Q_jc and merge.  eps = 0 gives an exact direct factorization.
 * precision: SPAND_FP64 (all factor arithmetic in FP64) or SPAND_MIXED
 * (factors computed and stored in FP32 with FP32 accumulation; the outer
 * GMRES stays FP64 and acts as iterative refinement).  A is read only; the factor owns its device memory.
 * Device memory (the factor's and the factorization's working memory, and
 * the solvers' scratch) comes from a stream-ordered pool of the library, one
 * per device, that keeps freed memory mapped for the next factorization or
 * solve: after the first call the pool holds the largest working set served
 * so far until the process ends (the device's default pool is not used).
 * A's pattern is checked on the device against the plan (no copy to the
 * host): a pattern the plan does not describe gives SPAND_ERR_ARG.
 * Errors: SPAND_ERR_ARG, SPAND_ERR_NOMEM, SPAND_ERR_ZERO_PIVOT,
 * SPAND_ERR_NONFINITE, SPAND_ERR_CUDA. */
typedef struct spand_factor_s* spand_factor_t;
int spand_factor(spand_plan_t plan, const bsr_matrix* A, double eps, int precision,
                 spand_factor_t* out, cudaStream_t stream);
int spand_factor_destroy(spand_factor_t F);

/* spand_factor_batched - the factorization of spand_factor for nsys
 * independent systems at once (the paper factors one system; batching is an
 * execution choice of this library).  plans[q] and A[q] (host array of nsys
 * matrices, each with its own block size) describe system q.  The systems'
 * levels are aligned from the bottom (level l of every system with D_q >= l
 * is processed together) and every phase of a level (batched LU, inverses,
 * elimination and Schur products, scaling, RRQR, compression, merge) is one
 * launch over the clusters of all systems, so small systems fill the GPU
 * together.  out[q] receives a handle for system q: spand_apply,
 * spand_factor_stats and sstep_gmres_solve on it act on system q alone (its
 * own apply program, captured in its own CUDA graph).  The handles share one
 * factorization; its device memory is released when the last of them is
 * destroyed.  Handles of different systems may be applied concurrently
 * (their sweeps touch disjoint memory).  Stats of a handle hold the system's
 * ranks, root size and apply bytes; phase times and flops are those of the
 * whole batch.  Errors: as spand_factor (no handle is returned on error). */
int spand_factor_batched(int nsys, const spand_plan_t* plans, const bsr_matrix* A, double eps,
                         int precision, spand_factor_t* out, cudaStream_t stream);

typedef struct {
  int levels;               /* D + 1                                          */
  int64_t n_sparsified[32]; /* interfaces sparsified at level l               */
  int64_t sum_n[32];        /* sum of their sizes before sparsification      */
  int64_t sum_r[32];        /* sum of kept ranks                              */
  int64_t max_r[32];        /* largest kept rank                              */
  int64_t top_size;         /* size of the last (root) interior               */
  int64_t factor_bytes;     /* device bytes one spand_apply streams (both sweeps) */
  double factor_flops;      /* algorithmic flops of the factorization         */
  /* Live CUDA-event timings of the factorization on its stream (ms), with
   * the algorithmic work of the timed kernels: the rank-revealing QRs
   * (bytes: the trailing block of W read and written once per pivot step)
   * and the elimination products Y, X and Schur updates (flops 2mnk).      */
  double t_rrqr_ms;
  double rrqr_bytes;
  int rrqr_launches;
  double t_elim_gemm_ms;
  double elim_gemm_flops;
  int elim_gemm_launches;
  /* per level: RRQR time (ms) and algorithmic bytes, and how many interfaces
   * ran in each RRQR form: [0] cluster of 1 to 8 CTAs, [1] 16-CTA cluster
   * (both with W in shared memory), [2] cooperative CTA group (W in shared
   * memory),
   * [3] W streamed from L2 / HBM (cooperative CTA group or 16-CTA cluster) */
  double t_rrqr_level_ms[32];
  double rrqr_bytes_level[32];
  int rrqr_form_count[32][4];
  /* host side of spand_factor: wall time of the call and the part of it spent
   * waiting for the GPU (one wait per level for the ranks, one at the end);
   * the difference is host work (planning, task tables, allocations).      */
  double t_host_ms;
  double t_wait_ms;
  /* the host wall time split by phase (summed over levels): [0] level setup
   * and last-level tail, [1] elimination, [2] scaling, [3] RRQR set-up and
   * launch, ending in the read-back of the level's ranks into pageable host
   * memory, which returns only once the level's queued kernels have run (so
   * [3] holds most of the time the host waits for the GPU), [4] the stream
   * synchronization after it, [5] Q_c formation, [6] merge into the next
   * level (and the root elimination with the final check), [7] apply
   * programs                                                                */
  double t_host_phase_ms[8];
  /* the streaming RRQR kernel's memory traffic: bytes its column passes moved
   * (each live column read and written once per pivot step; dead columns are
   * skipped), in total and per level                                       */
  double rrqr_stream_bytes;
  double rrqr_stream_bytes_level[32];
} spand_stats;
int spand_factor_stats(spand_factor_t F, spand_stats* st);

/* ---------------------------------------------------------------- apply
 * spand_apply - z = M^-1 r (transpose = 0) or z = M^-T r (transpose = 1) for
 * the preconditioner M = prod F_i of Sec. 2.2.1: the forward sweep applies the
 * elimination, scaling and orthogonal operators level by level, the backward
 * sweep their counterparts in reverse; the transpose runs the transposed
 * operators in the opposite order.  r, z: device FP64 vectors of length N
 * (may not alias).  In SPAND_MIXED the sweep runs in FP32.  Not reentrant on
 * one factor: calls on one factor must be ordered (same stream). */
int spand_apply(spand_factor_t F, const double* r, double* z, int transpose,
                cudaStream_t stream);

/* ---------------------------------------------------------------- GMRES
 * sstep_gmres_solve - Algorithm 2: s-step GMRES with right preconditioning
 * (A M^-1 u = b, x = x0 + M^-1 Q y), Newton basis (shifts = Ritz values of s
 * classical GMRES steps of the first cycle, real Leja order) or monomial
 * basis, one Gram reduction per s-block with the lagged second CGS + CholQR
 * pass, Givens least squares, restart after `restart` basis vectors.
 * Converged when the true FP64 residual ||b - A x|| / ||b|| <= tol at a
 * restart.  M may be NULL (no preconditioner).  x: device, in = x0,
 * out = solution.  transpose = 1 solves A^T x = b with M^-T.
 * Errors: SPAND_ERR_ARG, SPAND_ERR_CHOLQR, SPAND_ERR_NONFINITE,
 * SPAND_ERR_NOT_CONVERGED (x holds the last iterate), SPAND_ERR_CUDA. */
typedef struct {
  int s;            /* block size (1..16)                          */
  int restart;      /* basis vectors per cycle, multiple of s      */
  double tol;       /* relative residual target                    */
  int max_iters;    /* cap on Hessenberg columns over all cycles   */
  int basis;        /* SPAND_BASIS_NEWTON / SPAND_BASIS_MONOMIAL   */
  int transpose;    /* 0: A x = b; 1: A^T x = b                    */
} gmres_opts;

typedef struct {
  int iters;            /* Hessenberg columns used                        */
  int restarts;         /* completed cycles                               */
  int reductions;       /* Gram reductions                                */
  double true_relres;   /* final ||b - A x|| / ||b|| (FP64)               */
  double est_relres;    /* last Givens estimate                           */
  double orth_err;      /* max over cycles of ||Q^T Q - I||_F             */
  double shifts_re[16]; /* Newton shifts in Leja order                    */
  double shifts_im[16];
  /* Phase times (ms) of the solve's stream, from CUDA events at every phase
   * boundary (the time from one boundary to the next is charged to the
   * phase it opens, host round trips included): block SpMV; preconditioner
   * apply; orthogonalization (inner products / Gram reductions, CGS or MGS
   * updates, normalization); the rest (small dense work on the device:
   * Hessenberg, Cholesky, Givens, least squares; host reads of residual
   * estimates; solution update).  Zero in sstep_gmres_solve_noalloc.     */
  double t_spmv_ms, t_apply_ms, t_orth_ms, t_small_ms;
  /* Kernel times of the block Gram reductions of Algorithm 2 (G = Z^T Y,
   * Z = [Q_f, P, V], Y = [P, V]) and of the CGS2 / CholQR2 block updates
   * (X = Y S^-1 - Z C), each with the bytes its launches read and write
   * (Gram: (nz + ny) N 8 per reduction; update: (ny + nz + s) N 8), CUDA events
   * around each launch.  Zero in gmres_solve and in
   * sstep_gmres_solve_noalloc.                                              */
  double t_gram_ms, gram_bytes;
  int gram_calls;
  double t_bupd_ms, bupd_bytes;
  int bupd_calls;
} gmres_stats;

int sstep_gmres_solve(const bsr_matrix* A, spand_factor_t M, const double* b, double* x,
                      const gmres_opts* opts, gmres_stats* stats, cudaStream_t stream);

/* sstep_matrix_powers - the matrix-powers step of Algorithm 2 (line 4, Sec.
 * 2.3) on its own, with the preconditioner fused into the SpMV chain (the
 * paper applies the s SpMVs with the preconditioner one by one and leaves a
 * communication-avoiding form to future work).  With V[:, -1] = v0:
 *   V[:, k] = A M^-1 V[:, k-1] - Re(t_k) V[:, k-1] + [Im(t_k) < 0] Im(t_k)^2 V[:, k-2],
 * k = 0..s-1 (transpose = 1: A^T M^-T), the Newton basis with conjugate
 * pairs as real two-steps (the second shift of a pair, Im < 0, follows its
 * conjugate).  Each step runs the preconditioner's sweeps and then one
 * shifted block SpMV that reads the preconditioner's own output vector in
 * place (FP32 in SPAND_MIXED), so M^-1 v is never converted or stored in FP64.
 * sstep_gmres_solve generates its basis the same way.
 *  - A, M: as sstep_gmres_solve (M may be NULL: no preconditioner).
 *  - v0: device FP64 vector of length N = K*B; V: device N x s column-major
 *    (column k at V + k*N), written; v0 may not lie inside V.
 *  - shifts_re, shifts_im: host arrays of s doubles (zeros: monomial basis).
 *  - Not reentrant on one factor (it uses the factor's own vectors).
 * Errors: SPAND_ERR_ARG (null pointer, s outside 1..64, size mismatch, v0 in
 * V, a negative-imaginary shift without its conjugate just before it),
 * SPAND_ERR_CUDA. */
int sstep_matrix_powers(const bsr_matrix* A, spand_factor_t M, const double* v0, int s,
                        const double* shifts_re, const double* shifts_im, double* V, int transpose,
                        cudaStream_t stream);

/* gmres_solve - Algorithm 1: restarted GMRES with modified Gram-Schmidt
 * Arnoldi and Givens rotations, right preconditioning (A M^-1 u = b,
 * x = x0 + M^-1 Q y), the baseline of the s-step solver (Sec. 3.4).  Each
 * column takes one apply, one SpMV and j+2 inner products (j+1 for MGS, one
 * norm), each its own reduction; stats->reductions counts them.  Same
 * arguments, convergence test (Givens estimate per column, true FP64
 * residual at restarts) and errors as sstep_gmres_solve; opts->s and
 * opts->basis are ignored; stats->shifts_* and orth_err are 0. */
int gmres_solve(const bsr_matrix* A, spand_factor_t M, const double* b, double* x,
                const gmres_opts* opts, gmres_stats* stats, cudaStream_t stream);

/* sstep_gmres_solve_batched - nsys independent solves of sstep_gmres_solve
 * (host arrays of nsys: A, M (NULL or per-system handles, e.g. from
 * spand_factor_batched), b, x (device vectors), opts, stats, status).  Each
 * system runs on its own stream, ordered after `stream`; `stream` is ordered
 * after all of them on return, and the host has waited for every solve.  A
 * pool of up to 16 host threads drives the systems so their host round trips
 * (one per s-block) overlap other systems' kernels.  status[q] is system q's
 * own status; the return value is SPAND_OK or the first failing status in
 * system order (argument errors are checked for all systems before any work
 * is queued).  Not part of the paper: an execution choice of this library. */
int sstep_gmres_solve_batched(int nsys, const bsr_matrix* A, const spand_factor_t* M,
                              const double* const* b, double* const* x, const gmres_opts* opts,
                              gmres_stats* stats, int* status, cudaStream_t stream);

/* sstep_gmres_solve_noalloc - the same solve as sstep_gmres_solve (same
 * arguments, same results), for callers that must not allocate device memory
 * during a solve: for example a program that gives all device memory to its own
 * pool allocator at start-up, or one that runs under a fixed device-memory
 * budget and cannot let an allocation fail half-way through a solve.  This
 * entry point calls no cudaMalloc / cudaFree or any allocating routine; its
 * scratch (Krylov basis, Gram partial sums, small dense work) is carved from
 * one fixed device array of sstep_gmres_noalloc_capacity() bytes (8 MiB) that
 * every GPU which loads this library holds until the process exits.  The
 * paper has no counterpart; it is an interface choice of this library.
 *  - Size limit: the scratch needs about (restart + 2s + 4) * N doubles plus
 *    (restart + 2s + 2) * 304 * 32 doubles of Gram partial sums; larger
 *    problems are rejected with SPAND_ERR_SCRATCH before any work is queued.
 *  - The first call on each device looks up the array's device address (with
 *    that device current) and caches it; make that first call before any
 *    stream capture.  The array and the library's kernels are loaded into
 *    device memory when first used (the CUDA runtime loads modules lazily), so
 *    a caller that then hands all remaining device memory to its own pool
 *    should make one call (or one regular solve) on each device first.
 *  - The preconditioner's launches go on the stream one by one: its CUDA graph
 *    (built on first use by spand_apply and sstep_gmres_solve, and building
 *    it allocates) is neither built nor used here, so a factor that was never
 *    applied takes no memory either.  Like sstep_gmres_solve, the call
 *    synchronizes its stream to read residual estimates during the solve.
 *  - Every call on a device shares the one array and it keeps the previous
 *    call's contents (the solver clears what it needs zeroed).  Calls whose
 *    work overlaps on the GPU (other streams, other host threads) race on the
 *    array: order them, e.g. on one stream.
 *  - The preconditioner M is applied through its own factor-owned buffers
 *    (allocated by spand_factor, not by this call). */
int sstep_gmres_solve_noalloc(const bsr_matrix* A, spand_factor_t M, const double* b, double* x,
                              const gmres_opts* opts, gmres_stats* stats, cudaStream_t stream);
size_t sstep_gmres_noalloc_capacity(void);

/* ---------------------------------------------------------------- pseudo-time march
 * dg_pseudo_time_march - the continuation of Sec. 2.1.2 around the solve:
 * for n = 0, 1, ... assemble rhs = -R^n and A^n = M/dtau^n + dR/du|^n at
 * CFL^n (dg_assemble_jacobian, Eqs. 5-8), factor A^n with spaND on the
 * plan made once for the grid (the ordering is computed in preprocessing and
 * the factorization redone at every nonlinear step, Sec. 3.3), solve
 * A^n du = rhs by s-step GMRES from du = 0, and set u^{n+1} = u^n + du, with
 * the CFL number ramped by the residual ratio (Eq. 9):
 *     CFL^0 = flow->cfl,
 *     CFL^n = min(CFL^0 ||R^0|| / ||R^{n-1}||, CFL^inf)   (n >= 1),
 * ||.|| the 2-norm of all N residual coefficients (CFL^inf when ||R^{n-1}||
 * is 0).  The march stops, before solving, at the first n with
 * ||R^n|| <= rtol ||R^0|| or at n = max_steps; the state reached is
 * assembled once more so that its residual norm is reported.
 *  - mesh, p, flow: as dg_assemble_jacobian; u_hat: device [K, (p+1)^2, 4]
 *    doubles, in = u^0, out = the last state (also on error: the last
 *    state whose update completed).
 *  - plan: from spand_analyze(n_theta, n_r, 4 (p+1)^2, ...) of this grid.
 *  - opts->gmres.transpose is ignored (forward solves only).
 *  - hist (may be NULL; each array may be NULL): host arrays written for
 *    n = 0..steps: res_norm[n] = ||R^n||, cfl[n] = CFL^n, dtau[n]; and
 *    gmres_iters[n] for the steps < steps that were solved.  Arrays of
 *    res_norm, cfl, dtau need max_steps + 1 entries, gmres_iters max_steps.
 *    hist->steps = number of completed solves (updates).
 * Device scratch (A, rhs, du: about nnzb B^2 + 3 N doubles) is allocated on
 * the stream and released before return.  Synchronizes the stream at every
 * step (the residual norm decides CFL^{n+1} and the stop).
 * Errors: those of dg_assemble_jacobian, spand_factor and sstep_gmres_solve
 * (SPAND_ERR_NOT_CONVERGED when a linear solve misses its tolerance; u_hat
 * then holds the state before that step), SPAND_ERR_ARG (plan of another
 * grid, cfl <= 0, cfl_inf < cfl, max_steps < 0), SPAND_ERR_NONFINITE. */
typedef struct {
  int max_steps;      /* pseudo-time steps (linear solves) at most            */
  double cfl_inf;     /* CFL^inf of Eq. 9 (CFL^0 is flow->cfl)                */
  double rtol;        /* stop once ||R^n|| <= rtol ||R^0||                    */
  double eps;         /* spaND tolerance                                      */
  int precision;      /* SPAND_FP64 or SPAND_MIXED                            */
  gmres_opts gmres;   /* linear solver (tolerance relative to ||R^n||)        */
} dg_march_opts;

typedef struct {
  int steps;          /* completed solves                                     */
  double* res_norm;   /* host [max_steps + 1]                                 */
  double* cfl;        /* host [max_steps + 1]                                 */
  double* dtau;       /* host [max_steps + 1]                                 */
  int* gmres_iters;   /* host [max_steps]                                     */
} dg_march_history;

int dg_pseudo_time_march(const dg_mesh* mesh, int p, double* u_hat, const dg_flow_params* flow,
                         spand_plan_t plan, const dg_march_opts* opts, dg_march_history* hist,
                         cudaStream_t stream);

/* CFL^n of Eq. 9 from CFL^0, CFL^inf, ||R^0|| and ||R^{n-1}|| (the rule
 * dg_pseudo_time_march applies; host only).  Returns CFL^inf when
 * r_prev <= 0. */
double dg_cfl_ramp(double cfl0, double cfl_inf, double r0, double r_prev);

const char* spand_status_string(int status);

/* Number of kernel launches this library has issued in the process so far
 * (a replay of a captured apply graph adds the kernels in the graph; kernels
 * queued while the caller's stream is being captured count when queued).
 * For accounting, e.g. launches per solve; not part of the paper. */
uint64_t spand_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* SPAND_GB300_H */
