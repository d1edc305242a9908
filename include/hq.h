/*
 * hq.h -- C ABI of the GB300 (sm_103a) quasi-orthogonal inverse-operator
 * eigensolver: the discrete scheme Eq. (4.1) of Wang & Zhou, "A
 * quasi-orthogonal method based on the inverse operator for Schroedinger
 * eigenvalue problems" (arXiv 2605.25149), driven by Algorithm 1, for the N
 * lowest eigenpairs of H = -Delta/2 + V on a 7-point finite-difference grid.
 *
 * Problem (Section 2.2): find U (n x N) and Lambda with <U,V>_a = <U Lambda,V>
 * for all V, <U,U> = I.  Discretisation used by this library:
 *   grid     m^3 interior nodes of [lo,hi]^3, h = (hi-lo)/(m+1), Dirichlet 0;
 *            node (i,j,k) -> p = i + m*(j + m*k), x fastest, n = m^3;
 *   blocks   n x N, point-major (U[p*N + c]); V is n values, same order;
 *   product  <A,B> = h^3 A^T B (Section 2.1);
 *   inverse  G = (H + sigma)^{-1} (Section 3.1) with a Garding shift sigma
 *            (Section 2.2; automatic rule: sigma = 0 when
 *            lambda_min(-Delta_h/2) + min V > 0, else 1 - that bound).
 *
 * Ownership: the caller allocates one device workspace of
 * hq_workspace_bytes() bytes and passes a CUDA stream; the library never
 * allocates device memory after hq_init and every kernel runs on that
 * stream, or on a private stream forked from it and joined back to it within
 * the same call (the warm start's N x N solve of a step, beside the
 * predictor system), so the work of each call stays ordered on the caller's
 * stream.  Pointers passed to a call are borrowed for the duration of the
 * call only.  Arrays flagged on_device are device pointers, otherwise host
 * pointers.  All arrays are FP64 unless stated.
 *
 * Errors: every function returns hq_status; hq_last_error() gives detail.
 * After any status other than HQ_ERR_CUDA the context stays usable.  No C++
 * exception crosses this boundary.  Device-side failures (CG breakdown, a
 * singular small system) are reported through a status word read at the
 * next synchronisation point; no kernel traps.  Waits inside the tensor-core
 * kernels are bounded (2 s of %globaltimer); a wait that gives up reports
 * HQ_ERR_TIMEOUT ("tensor-core wait expired"), and then only that status is
 * meaningful: the blocks and matrices the call was writing are undefined.
 *
 * Determinism: reductions run in a fixed order; identical inputs give
 * bit-identical outputs.
 */
#ifndef HQ_H
#define HQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hq_ctx hq_ctx;

typedef enum {
    HQ_OK = 0,
    HQ_ERR_ARG = 1,            /* invalid argument (size, pointer, value)        */
    HQ_ERR_STATE = 2,          /* call out of order (e.g. step before potential) */
    HQ_ERR_CUDA = 3,           /* CUDA runtime error; the context is lost        */
    HQ_ERR_NOMEM = 4,          /* workspace too small / host allocation failed   */
    HQ_ERR_BREAKDOWN = 5,      /* inner CG: p^T A p <= 0 or not finite           */
    HQ_ERR_SINGULAR = 6,       /* zero pivot in the predictor system             */
    HQ_ERR_NOT_CONVERGED = 7,  /* inner CG or Algorithm 1 hit its iteration cap  */
    HQ_ERR_TIMEOUT = 8,        /* wall-clock limit of hq_solve reached           */
    HQ_ERR_NONFINITE = 9       /* NaN/Inf in an input or in the gradient norm    */
} hq_status;

typedef enum {
    HQ_FP64 = 0,   /* every operation in IEEE FP64                               */
    HQ_MIXED = 1   /* FP32 blocks, FP32 stencil / CG / multigrid, Gram products   */
                   /* on tcgen05 tensor cores (3xTF32, FP32 accumulation),        */
                   /* FP64 small solve, FP64 Rayleigh-Ritz refinement             */
} hq_precision;

typedef struct {
    int m;               /* interior nodes per side (>= 3)                         */
    double lo, hi;       /* box [lo,hi]^3                                          */
    int nev;             /* N, number of eigenpairs (1 <= N <= min(n, 512))        */
    double tau;          /* fixed time step tau_n of Algorithm 1 (> 0)             */
    double shift;        /* sigma; NaN selects the automatic rule                  */
    int precision;       /* hq_precision                                           */
    double cg_rtol;      /* inner PCG: stop column j when ||r_j|| <= rtol ||b_j||  */
    int cg_maxit;        /* inner PCG iteration cap                                */
    int mg_nu1, mg_nu2;  /* damped-Jacobi pre/post sweeps per V-cycle level (>=1) */
    int mg_coarsest;     /* coarsen m -> m/2 while m > mg_coarsest (1..4)          */
    double mg_omega;     /* Jacobi damping                                         */
    double timeout_s;    /* hq_solve wall-clock limit (<= 0: none)                 */
    int z_warm_start;    /* 1: start the corrector solve G Uh from W (C1 + S^-1 Puw C2), */
                         /* exact when span(U) is G-invariant; 0: from zero          */
    int adaptive_tau;    /* 0: tau_n = tau.  1: tau_n = min(tau_max, c lam / s_max,    */
                         /* 1.05 tau_{n-1}) with lam = 1/(largest Ritz value of G on  */
                         /* span(U)), s_max = max_i sum_j |<U,U>_ij| (a bound on its  */
                         /* largest eigenvalue); the first step starts from the       */
                         /* closed-form lower bound of lambda_1(H + sigma)            */
    double tau_max;      /* delta_T of Algorithm 1 for adaptive_tau (<= 0: no cap)    */
    int grid_block;      /* threads per CTA of the grid kernels: 0 (= 256), 64, 128, 256 */
    int grid_ctas;       /* target CTAs per SM of the grid kernels: 0 (= 16) .. 64;     */
                         /* both set the launch shape only (hq_tune picks them)      */
    int fp64_tc;         /* HQ_FP64 only: 2 = the Gram of [U W] and the n x N block   */
                         /* products (Uh, U_{n+1}, the gradient residual, the warm   */
                         /* start) on tensor cores by exact integer slicing of the   */
                         /* FP64 values (error below 2^-53 |row max| |column max|    */
                         /* per term, FP64 results; for 2N <= 128); 1 (default) =    */
                         /* the same for products of at least 2^25 multiply-adds,    */
                         /* FP64 SIMT below; 0 = FP64 SIMT                          */
    int mg_fp32;         /* HQ_FP64 only: 1 = the multigrid preconditioner of the     */
                         /* FP64 block PCG runs in FP32 (r rounded to FP32, z widened */
                         /* back, r.z in FP64); the PCG residuals, updates, stopping  */
                         /* test and every other step stay FP64, so W = G U is still  */
                         /* solved to cg_rtol in FP64.  0 (default) = FP64 V-cycle   */
    double tau_safety;   /* c of the adaptive time step (adaptive_tau = 1): tau_n    */
                         /* <= c lam / s_max; 0 < c <= 1, default 0.8.  Near          */
                         /* convergence tau < lambda_1(H + sigma) keeps the           */
                         /* orthogonality error contracting, and lam overestimates    */
                         /* lambda_1 until the Ritz value has converged               */
} hq_config;

/* Defaults: box [-6,6]^3, tau 0.4, automatic shift, FP64, cg_rtol 1e-10,
 * cg_maxit 200, nu1 = nu2 = 2, coarsest 4, omega 0.8, no timeout, warm start
 * of the corrector solve on, fp64_tc 1, tau_safety 0.8.  m and nev are left 0
 * and must be set.                                                          */
void hq_default_config(hq_config *cfg);

/* Bytes of device workspace hq_init needs for cfg (0 if cfg is invalid). */
size_t hq_workspace_bytes(const hq_config *cfg);

/* Creates a context on the current CUDA device.  d_workspace: device buffer
 * of at least hq_workspace_bytes(cfg) bytes, 256-byte aligned, owned by the
 * caller and kept alive until hq_destroy.  cuda_stream: a cudaStream_t (NULL
 * = default stream).  Two environment switches are read here, for tests and
 * profiling: HQ_NO_GRAPHS=1 runs hq_step / hq_solve host-driven instead of
 * replaying captured graphs (same kernels in the same order, bit-identical
 * results); HQ_ZMARCH=1 / 0 forces the z-marching finest-level sweeps on / off
 * (by default they run for finest-level blocks of 100 MB or more; same
 * element values, PCG dot products summed in another order);
 * HQ_FUSED_COARSE=0 runs every level of the FP32 V-cycles (HQ_MIXED, mg_fp32)
 * as separate kernels (by default the levels from the first one whose
 * vectors fit one CTA's shared memory, about 16^3 points, down to the
 * coarsest run as one launch, one CTA per column).  HQ_LOG=<path> appends
 * one JSON line per hq_step call to <path> (context, step counter, steps
 * taken, g, inner PCG solves and iterations, wall ms, status); it makes
 * every hq_step call synchronise.  Every public call is an NVTX range named
 * after the call.                                                          */
hq_status hq_init(const hq_config *cfg, void *d_workspace, size_t bytes,
                  void *cuda_stream, hq_ctx **out);

/* Sets V (n values, unshifted) and rebuilds the multigrid hierarchy and the
 * shift (setup of G, Section 3.1).  Resets the step counter and invalidates
 * the iterate.  HQ_ERR_NONFINITE on NaN/Inf in V; HQ_ERR_ARG if a given shift
 * leaves the coarsest operator indefinite.                                  */
hq_status hq_set_potential(hq_ctx *ctx, const double *V, int on_device);

/* Sets U0 (n x N, point-major) and rescales it by 1/sqrt(lambda_min(<U0,U0>))
 * so that <U0,U0> >= I with equality in one direction: U0 enters the
 * quasi-Stiefel set of Theorem 3.2 without being orthogonalised.            */
hq_status hq_set_initial(hq_ctx *ctx, const double *U0, int on_device);

/* Advances Eq. (4.1) nsteps times (predictor, corrector; two inner solves
 * per step).  resid_out (nullable, host): the gradient norm
 * ||G U - U <G U,U>|| (Remark 3.1) of the state at the start of the last
 * step taken.                                                              */
hq_status hq_step(hq_ctx *ctx, int nsteps, double *resid_out);

/* Algorithm 1: steps until ||grad_G E_G(U_n)|| < eps (discrete L2 norm) or
 * max_steps steps.  steps_out / resid_out (nullable, host) receive the steps
 * taken in this call and the final gradient norm.  HQ_ERR_NOT_CONVERGED if
 * max_steps was reached, HQ_ERR_TIMEOUT on the wall-clock limit.            */
hq_status hq_solve(hq_ctx *ctx, double eps, long max_steps, long *steps_out,
                   double *resid_out);

/* Eigenpairs of the current iterate.  evals_paper (N, host, nullable): the
 * eigenvalues of <G U,U>^{-1} shifted back by sigma (Section 5's
 * definition), ascending.  evals_rr (N, host, nullable): FP64 Rayleigh-Ritz
 * values of H on span(U), ascending.  evecs (n x N, point-major, nullable):
 * Ritz vectors, <u_i,u_j> = delta_ij, largest-magnitude entry positive;
 * device pointer if evecs_on_device else host.  resid (N, host, nullable):
 * ||H u_i - lambda_i u_i|| in the discrete L2 norm.                        */
hq_status hq_eigenpairs(hq_ctx *ctx, double *evals_paper, double *evals_rr,
                        double *evecs, int evecs_on_device, double *resid);

/* Monitoring of the current iterate (all host outputs, nullable), in FP64:
 * energy = E(U) = (1/2)(U,U)_a = (1/2) h^3 tr(U^T H U) with the unshifted H
 * (Section 2.2; decays along the scheme, Theorem 4.5), onorm = ||<U,U> - I||_F
 * (the orthogonality error of Theorem 4.6), smin / smax = extreme
 * eigenvalues of <U,U> (quasi-Stiefel membership, Theorem 4.3).            */
hq_status hq_monitor(hq_ctx *ctx, double *energy, double *onorm, double *smin, double *smax);

/* ---- differentiation (HQ_FP64 contexts; the iterate should be converged) ----
 * The Ritz vectors u_i and values lambda_i of hq_eigenpairs define
 * rho = sum_i u_i^2 (the density, n values).                               */
/* rho_out (n, FP64): the density of the current Ritz vectors.               */
hq_status hq_density(hq_ctx *ctx, double *rho_out, int on_device);
/* dV = sum_i w_i d lambda_i / dV = h^3 sum_i w_i u_i^2 (Hellmann-Feynman for
 * the discrete operator; w: N host weights, NULL = all ones, giving
 * d(sum lambda_i)/dV).  dV: n values.                                      */
hq_status hq_grad_eigs(hq_ctx *ctx, const double *w, double *dV, int on_device);
/* Adjoint of the density: for a loss L(rho) with G = dL/drho (n values),
 *   dL/dV = -2 sum_i u_i o xi_i,  (H - lambda_i) xi_i = P (G o u_i),  xi_i in range(P),
 * P = I - u (h^3 u^T) the projector onto the complement of span(u_1..u_N)
 * (first-order perturbation of the eigenvectors; components inside the span
 * leave rho unchanged).  The N systems are solved together by block PCG on
 * the projected, column-shifted operator with the multigrid V-cycle of
 * H + sigma as preconditioner (symmetric positive definite on range(P) when
 * lambda_N < lambda_{N+1}), each to ||r_i|| <= rtol ||P(G o u_i)||.
 * If rho_target is non-null, G is ignored and the loss
 * L = (1/2) h^3 sum (rho - rho_target)^2 is used (G = h^3 (rho - rho_target));
 * *loss (host, nullable) receives L.  iters (host, nullable): PCG
 * iterations taken.                                                        */
hq_status hq_grad_density(hq_ctx *ctx, const double *G, const double *rho_target, int on_device,
                          double rtol, int maxit, double *dV, double *loss, int *iters);

/* ---- FP64 residual refinement (not in the paper; HQ_FP64 contexts) ----
 * Refines span(U) of the current iterate in FP64, e.g. after the state of an
 * HQ_MIXED context was handed over with hq_set_state.  Each of `rounds`
 * rounds: Rayleigh-Ritz pairs (theta_i, u_i) of H on span(U); residuals
 * r_i = H u_i - theta_i u_i; corrections t_i in the complement of span(u)
 * from P (H - theta_i) P t_i = -r_i with P = I - u (h^3 u^T) (Newton's
 * equation for an invariant subspace, one equation per Ritz vector), solved
 * together by block PCG with the multigrid V-cycle of H + sigma as
 * preconditioner, each to ||res_i|| <= rtol ||r_i|| within maxit
 * iterations; U <- u + t.  P (H - theta_i) P is positive definite on the
 * complement when every theta_i lies below the spectrum of H there (U close
 * enough to the N lowest eigenvectors, lambda_N < lambda_{N+1}).  A last
 * Rayleigh-Ritz leaves U = the Ritz vectors (<u_i,u_j> = delta_ij).  The
 * step counter is kept; the inner solver's warm start is dropped.
 * resid (N, host, nullable): ||H u_i - theta_i u_i|| of the final Ritz
 * pairs; iters (host, nullable): PCG iterations over all rounds.  Errors:
 * HQ_ERR_STATE (HQ_MIXED context, or no iterate), HQ_ERR_ARG (rounds < 0,
 * maxit < 1, rtol <= 0), HQ_ERR_NOT_CONVERGED (a correction reached maxit;
 * U keeps the last completed round), HQ_ERR_BREAKDOWN.                     */
hq_status hq_refine(hq_ctx *ctx, int rounds, double rtol, int maxit, double *resid, int *iters);

/* Checkpoint: copy U_n (n x N, FP64) and the step counter out / in.  Zwarm
 * (nullable, n x N) is the inner solver's warm start, G Uh of the last step;
 * restoring U together with Zwarm continues bit-identically to the
 * uninterrupted run, restoring U alone within the inner-solve tolerance.
 * hq_get_state with Zwarm before any step returns HQ_ERR_STATE.             */
hq_status hq_get_state(hq_ctx *ctx, double *U, double *Zwarm, int on_device, long *step);
hq_status hq_set_state(hq_ctx *ctx, const double *U, const double *Zwarm, int on_device,
                       long step);

/* Time step tau_n used by the last step taken (host output). */
hq_status hq_time_step(hq_ctx *ctx, double *tau);

/* Scalars of the configured problem (host outputs, nullable). */
hq_status hq_problem_info(hq_ctx *ctx, double *h, double *sigma, int *levels,
                          int *level_m /* up to 24 entries */);

/* ---- operations of one step, on caller device buffers (point-major,
 * ncol columns, FP64 in HQ_FP64 contexts, FP32 in HQ_MIXED contexts). ---- */

/* y = (H + sigma) x on the finest grid (the operator G inverts).  With
 * ncol == N this is the block PCG's own operator launch (same kernel and
 * launch shape, its per-column x.y partial sums formed into the context's
 * scratch). */
hq_status hq_apply_operator(hq_ctx *ctx, const void *x, void *y, int ncol);

/* z = M r: one multigrid V-cycle for (H + sigma) (symmetric when nu1 == nu2),
 * the preconditioner of the inner solve.  ncol must equal N.                */
hq_status hq_mg_vcycle(hq_ctx *ctx, const void *r, void *z);

/* X = G B by block PCG, all N columns at once, column j stopped when
 * ||r_j|| <= rtol ||b_j||; rtol = 0 runs exactly maxit iterations.  X holds
 * the initial guess on entry.  iters (N ints, host, nullable).             */
hq_status hq_block_pcg(hq_ctx *ctx, const void *B, void *X, double rtol, int maxit,
                       int *iters);

/* O'Leary's block PCG (not in the paper; an alternative to hq_block_pcg's
 * per-column recurrences): X = G B with all N columns in one block Krylov
 * space and N x N step matrices, alpha = (P^T A P)^{-1} (Z^T R),
 * beta = (Z^T R)^{-1} (Z'^T R') (Z = M R, the multigrid V-cycle), the inner
 * products plain sums over the grid points.  X holds the initial guess on
 * entry; stops when every column has ||r_j|| <= rtol ||b_j|| (rtol = 0: after
 * exactly maxit iterations).  iters (host, nullable): iterations run.
 * Errors: HQ_ERR_NOT_CONVERGED at maxit, HQ_ERR_SINGULAR when P^T A P or
 * Z^T R lost positive definiteness (the block lost rank: a column converged
 * far ahead of the others).  Uses the context's PCG blocks as scratch.    */
hq_status hq_block_pcg_coupled(hq_ctx *ctx, const void *B, void *X, double rtol, int maxit,
                               int *iters);

/* out = w A^T B (Na x Nb, row-major, FP64, device) for point-major blocks
 * A (n x Na) and B (n x Nb) on the finest grid: the inner-product matrices
 * <A,B> of Section 2.1 with w = h^3.  Na, Nb <= 2N.                        */
hq_status hq_gram(hq_ctx *ctx, const void *A, int Na, const void *B, int Nb, double w,
                  double *out);

/* Out = A1 M1 + A2 M2 (+ Cin): the block x small-matrix products of the
 * updates of Eq. (4.1) (Uh = U C1 + W C2, U+ = Uh - tau Z (<Uh,Uh> - I)).
 * A1 (n x k1), A2 (n x k2; nullable with k2 = 0), Cin (nullable) and Out are
 * point-major device blocks of the context's element type with N columns
 * (Out, Cin) and 1 <= k1, 0 <= k2 <= N; M1 (k1 x N), M2 (k2 x N) are FP64
 * row-major device matrices.  FP64 SIMT in HQ_FP64 contexts, tcgen05 3xTF32
 * (FP32 accumulation) in HQ_MIXED contexts.                                */
hq_status hq_block_gemm(hq_ctx *ctx, const void *A1, int k1, const double *M1, const void *A2,
                        int k2, const double *M2, const void *Cin, void *Out);

/* One step of Eq. (4.1) from the current iterate, exporting its
 * intermediates to device buffers (each nullable): W = G U_n (n x N),
 * gram = Gram of [U W] (2N x 2N, FP64), g (1 value, FP64), XY = [X; Y]
 * (2N x N, FP64) with X = <U,Ut>, Y = <G U,Ut>, Uh (n x N), Shat = <Uh,Uh>
 * (N x N, FP64), Z = G Uh (n x N), Unew = U_{n+1} (n x N).  Block outputs
 * have the context's element type.  The iterate advances as in hq_step.    */
hq_status hq_step_trace(hq_ctx *ctx, void *W, double *gram, double *g, double *XY,
                        void *Uh, double *Shat, void *Z, void *Unew);

/* Multigrid pieces on level l (0 = finest) for parity tests: one damped
 * Jacobi sweep z_out = z_in + omega D^{-1}(r - A_l z_in); restriction
 * rc = ((m_c+1)/(m_f+1))^3 P^T rf from level l to l+1; prolongation
 * ef_out = ef_in + P ec from level l+1 to l; exact solve on the coarsest
 * level.  ncol must equal N.                                               */
hq_status hq_mg_smooth(hq_ctx *ctx, int level, const void *r, const void *z_in, void *z_out);
/* The same sweep as the FP64 V-cycle forms it, from the pre-scaled right-hand
 * side rt = omega D^{-1} r (device, n_l x N, FP64):
 * z_out = omega c D^{-1} nbrsum(z_in) + ((1 - omega) z_in + rt), with
 * c = 1/(2 h_l^2).  FP64 contexts without mg_fp32 only (HQ_ERR_STATE
 * otherwise) and levels above the coarsest (HQ_ERR_ARG).                   */
hq_status hq_mg_smooth_prescaled(hq_ctx *ctx, int level, const void *rt, const void *z_in,
                                 void *z_out);
hq_status hq_mg_restrict(hq_ctx *ctx, int level, const void *rf, void *rc);
hq_status hq_mg_prolong(hq_ctx *ctx, int level, const void *ec, const void *ef_in,
                        void *ef_out);
hq_status hq_mg_coarse_solve(hq_ctx *ctx, const void *r, void *z);
/* Level-l potential (n_l values, FP64, device). */
hq_status hq_mg_level_potential(hq_ctx *ctx, int level, double *V_out);

/* ---- allocation-free variant ----
 * hq_gram_static: out = w A^T B (Na x Nb, row-major, FP64, device) for
 * point-major FP64 device blocks A (n x Na) and B (n x Nb), with no context
 * and no workspace.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- code that runs inside a
 * stream capture whose allocation policy forbids cudaMalloc, plugin hosts
 * that only hand out pre-registered buffers, and real-time loops that must
 * not allocate after start-up.  Its split-K partial sums live in one fixed
 * file-scope device array of 2^19 doubles (4 MiB) that every GPU which loads
 * this library keeps until the process exits; it calls no cudaMalloc,
 * cudaFree or allocating library routine.
 * Limits: 1 <= Na, Nb <= 512, n >= 1; anything else returns HQ_ERR_ARG.
 * The first call on each device (with that device current) looks up the
 * array's device address; make that first call before any stream capture.
 * All calls share the one array, which keeps the previous call's contents
 * (every partial is written before it is read, so nothing needs clearing):
 * calls that can overlap on the GPU -- on different streams, or from
 * different host threads -- race and must be serialised by the caller.
 * The cached address belongs to the device's context at the first call: after
 * cudaDeviceReset of that device this entry point must not be called again in
 * the same process.
 * cuda_stream: a cudaStream_t (NULL = default stream); the call is
 * asynchronous on it.  Returns HQ_ERR_CUDA on a runtime error: a launch error
 * already pending on the calling thread (left by earlier work) is reported
 * before anything is launched and left in place for the caller; an error of
 * this call's own launches is reported and cleared.                        */
hq_status hq_gram_static(const double *A, int Na, const double *B, int Nb, long n, double w,
                         double *out, void *cuda_stream);

/* ---- instrumentation ---- */
/* Kernel classes counted by the launch counters. */
typedef enum {
    HQ_K_STENCIL = 0,   /* 7-point operator y = (H + sigma) x              */
    HQ_K_RESIDUAL,      /* residual r - (H + sigma) z                      */
    HQ_K_SMOOTH,        /* damped-Jacobi sweeps                            */
    HQ_K_TRANSFER,      /* restriction / prolongation                      */
    HQ_K_COARSE,        /* coarsest-level solve, or the coarse levels of an */
                        /* FP32 V-cycle in one launch                      */
    HQ_K_VECTOR,        /* PCG vector updates, dots, conversions           */
    HQ_K_REDUCE,        /* per-column / global finalising reductions       */
    HQ_K_GRAM,          /* inner-product matrices <A,B>                    */
    HQ_K_BLOCKGEMM,     /* block x small-matrix products (updates)         */
    HQ_K_SMALL,         /* N x N / 2N x 2N FP64 algebra                    */
    HQ_K_SETUP,         /* once-per-potential setup                        */
    HQ_K_COARSE_GRIDS,  /* grid kernels on multigrid levels >= 1 (the      */
                        /* classes above count the finest level only)      */
    HQ_K_NCLASS
} hq_kernel_class;

/* Resets the per-class launch counters of this context; with timing != 0
 * also brackets every kernel launch with CUDA events on the context's
 * stream (adds host overhead; for measurement runs only).                  */
hq_status hq_profile(hq_ctx *ctx, int timing);
/* launches (HQ_K_NCLASS longs, host, nullable): kernels launched per class
 * since the last hq_profile; ms (HQ_K_NCLASS doubles, host, nullable): summed
 * event time per class (0 unless timing was on); elements (HQ_K_NCLASS
 * doubles, host, nullable): grid point-columns written by the grid kernels
 * of each class (0 for the dense classes).  Synchronises the stream.        */
hq_status hq_profile_read(hq_ctx *ctx, long *launches, double *ms, double *elements);
/* Inner-solve statistics since the last hq_profile: block-PCG solves run and
 * PCG iterations summed over them (host outputs, nullable).                 */
hq_status hq_pcg_stats(hq_ctx *ctx, long *solves, long *iterations);

const char *hq_last_error(hq_ctx *ctx);
const char *hq_status_string(hq_status s);
void hq_destroy(hq_ctx *ctx);

/* ------------------------------------------------------------------------
 * Launch-shape autotuner (no counterpart in the paper).  For cfg's m, nev and
 * precision it times a 10-iteration multigrid-preconditioned block PCG (the
 * inner solve of Eq. (4.1); harmonic potential, pseudo-random right-hand
 * side) under each candidate grid_block in {64, 128, 256} x grid_ctas in
 * {4, 8, 16, 32} and writes cfg with the fastest pair into *tuned.  The launch
 * shape changes only the order of the per-column reductions, so results agree
 * with the default shape to rounding.  workspace: device buffer of at least
 * hq_tune_workspace_bytes(cfg) bytes (256-byte aligned), scratch for the call
 * only.  ms_out: the fastest time per PCG iteration in ms (nullable).
 * Synchronises cuda_stream.  Errors: HQ_ERR_ARG (invalid cfg or null
 * pointer), HQ_ERR_NOMEM (workspace too small), HQ_ERR_CUDA.
 * ------------------------------------------------------------------------ */
size_t hq_tune_workspace_bytes(const hq_config *cfg);
hq_status hq_tune(const hq_config *cfg, void *d_workspace, size_t bytes, void *cuda_stream,
                  hq_config *tuned, double *ms_out);

/* ------------------------------------------------------------------------
 * Batched form: many independent problems (contexts of any m, N and
 * precision, each with its own potential and U0) advanced by Algorithm 1
 * (Section 5) in ONE CUDA-graph launch per call.  The graph holds the time
 * loop as a conditional WHILE node; inside it every problem is an IF node
 * (skipped once that problem has stopped) holding its two phases of
 * Eq. (4.1), each with its inner block PCG as nested WHILE / IF nodes.  The
 * problems' kernels run concurrently; nothing returns to the host until all
 * problems have stopped.  Each problem follows the trajectory that
 * hq_solve / hq_step of its context would produce, bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct hq_batch hq_batch;

/* ctxs: count (1..64) distinct contexts on the current device, borrowed: they
 * must outlive the batch and must not be used by another thread during a
 * batch call.  cuda_stream: the stream the batch graph is launched on (NULL:
 * legacy default stream).  The graph is captured at the first hq_batch_solve
 * / hq_batch_step and again after any member's hq_set_potential.  *out is
 * freed with hq_batch_destroy.  Errors: HQ_ERR_ARG (count, null or repeated
 * context).                                                                */
hq_status hq_batch_create(hq_ctx *const *ctxs, int count, void *cuda_stream, hq_batch **out);
/* Algorithm 1 for every member: problem k stops when its g < eps[k] (eps:
 * count host doubles, > 0) or after max_steps steps; timeout_s > 0 bounds the
 * wall-clock time of the whole batch on the device (0: none).  Outputs (host,
 * count entries each, nullable): steps taken, last g, per-problem status
 * (HQ_OK, HQ_ERR_NOT_CONVERGED, HQ_ERR_TIMEOUT, or the error a member hit;
 * its message is in hq_last_error of that context).  Returns HQ_OK when every
 * problem converged, else the first non-OK per-problem status (message in
 * hq_batch_last_error).  Synchronises the batch stream.                    */
hq_status hq_batch_solve(hq_batch *b, const double *eps, long max_steps, double timeout_s,
                         long *steps_out, double *resid_out, int *status_out);
/* nsteps steps of Eq. (4.1) for every member, as hq_step(ctx, nsteps).
 * resid_out / status_out: as in hq_batch_solve (nullable).                 */
hq_status hq_batch_step(hq_batch *b, long nsteps, double *resid_out, int *status_out);
/* batch-level kernels launched (loop control; the members' kernels are
 * counted in their contexts, see hq_profile_read) and time-loop iterations
 * run, since creation (host outputs, nullable).                            */
hq_status hq_batch_launches(const hq_batch *b, long *batch_kernels, long *loop_iterations);
const char *hq_batch_last_error(const hq_batch *b);
void hq_batch_destroy(hq_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* HQ_H */
