// Internal declarations shared by the CUDA translation units of libhq.
// Layout conventions: an n x N block is point-major (element (p, c) at
// p*N + c); grid node (i, j, k) of an m^3 grid is p = i + m*(j + m*k).
#pragma once
#include <cuda_runtime.h>

#include "../../include/hq.h"
#include <stdint.h>
#include <stddef.h>

namespace hq {

// launch instrumentation: every kernel launch is bracketed by these hooks,
// which count launches per class and optionally record CUDA events.
void hook_before(int cls);
void hook_after(int cls, double work);
#define HQ_LAUNCH_W(cls, work, ...)                 \
    do {                                            \
        ::hq::hook_before(cls);                     \
        __VA_ARGS__;                                \
        ::hq::hook_after(cls, (double)(work));      \
    } while (0)
#define HQ_LAUNCH(cls, ...) HQ_LAUNCH_W(cls, 0, __VA_ARGS__)

// ----------------------------------------------------------------------------
// launch geometry of the point-major grid kernels
// ----------------------------------------------------------------------------
struct GridGeom {
    int m;          // nodes per side
    long n;         // m^3
    int N;          // columns (= leading dimension)
    int vec;        // columns per thread (vector width)
    int tx, ty;     // block shape: tx column-vectors x ty points
    int gx, gy;     // grid shape
    int ppt;        // points per thread (consecutive slabs of ty points)
    int zch;        // > 0: smoothing sweeps without partial sums march in z
                    // (zch chunks of planes per x-segment / y-row), see k_jacobi_zm
};
// switches the operator, residual and smoothing sweeps of a level to
// z-marching CTAs (blocks larger than L2)
void enable_zmarch(GridGeom &g);
// rows of per-column partial sums written by the operator, residual and
// smoothing kernels of geometry g (one row per CTA along y); the vector
// kernels (launch_pcg_xr, launch_dot, launch_widen_dot) always write g.gy
int part_rows(const GridGeom &g);
// block: threads per CTA (0: 256); ctas_per_sm: target CTAs per SM of the
// grid (0: 16) -- the two launch-shape parameters the autotuner searches
GridGeom make_geom(int m, int N, int elem_bytes, int block = 0, int ctas_per_sm = 0);

// sum_{c < count} (double) p[c * stride] in index order (deterministic), the
// loads issued in groups of eight ahead of the additions: an add after each
// load would serialise the load latencies
template <typename P>
__device__ __forceinline__ double ordered_sum(const P *p, long count, size_t stride) {
    double s = 0.0;
    for (long c0 = 0; c0 < count; c0 += 8) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; u++) a[u] = c0 + u < count ? (double)p[(size_t)(c0 + u) * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (c0 + u < count) s += a[u];
    }
    return s;
}
// the elements i = t, t + step, ... < np of p, in that order
__device__ __forceinline__ double strided_sum(const double *p, int np, int t, int step,
                                              size_t stride = 1) {
    const long cnt = t < np ? (np - 1 - t) / step + 1 : 0;
    return ordered_sum(p + (size_t)t * stride, cnt, (size_t)step * stride);
}

// per-column PCG scalars, all device arrays of length N (FP64)
struct PcgScalars {
    double *rz, *alpha, *beta, *bnorm, *rnorm;
    int *active, *iters;
    int *num_active;   // 1 int
    int *status;       // 1 int, sticky error flags (bit 0: breakdown)
    double *fpart;     // 2 x ceil(gy / 128) x N: row-chunk sums of the finalisation
    unsigned *fcount;  // ceil(N / 32) arrival counters of the finalisation (start at 0)
};

enum { ST_BREAKDOWN = 1, ST_SINGULAR = 2, ST_NONFINITE = 4, ST_GJ_FAIL = 8, ST_TC_TIMEOUT = 16,
       ST_PCG_MAXIT = 32 };

// ----------------------------------------------------------------------------
// grid kernels (k_grid.cu); T = double or float
// ----------------------------------------------------------------------------
// y = A x with A = (H + sigma) on a level: A x = D x - c * (sum of 6 nbrs).
// Optional per-column partial of x.y (part_xy, gy x N) .
template <typename T>
void launch_apply(const GridGeom &g, const T *D, T c, const T *x, T *y, double *part_xy,
                  cudaStream_t s);
// y = b - A x, partials of y.y and b.b (nullable)
template <typename T>
void launch_resid(const GridGeom &g, const T *D, T c, const T *x, const T *b, T *y,
                  double *part_yy, double *part_bb, cudaStream_t s);
// x += alpha p, r -= alpha q (per-column alpha), partial r.r; if zf != null also
// zf = wD * r (first damped-Jacobi sweep from zero).
template <typename T>
void launch_pcg_xr(const GridGeom &g, const double *alpha, const T *p, const T *q, T *x, T *r,
                   double *part_rr, const T *wD, T *zf, cudaStream_t s);
// p = z + beta p
template <typename T>
void launch_pcg_p(const GridGeom &g, const double *beta, const T *z, T *p, cudaStream_t s);
// z_out = z_in + wD (r - A z_in); partial r.z_out (nullable)
template <typename T>
void launch_jacobi(const GridGeom &g, const T *D, const T *wD, T c, T one_minus_omega,
                   const T *r, const T *zin, T *zout, double *part_rz, cudaStream_t s);
// z = wD * r
template <typename T>
void launch_jacobi_first(const GridGeom &g, const T *wD, const T *r, T *z, cudaStream_t s);
// the damped-Jacobi sweep from the pre-scaled right-hand side rt = wD r and
// wc = wD c: z_out = wc nbrsum(z_in) + ((1 - omega) z_in + rt); r is read
// only for the partial r.z_out (part_rz non-null)
template <typename T>
void launch_jacobi_rt(const GridGeom &g, const T *wc, T one_minus_omega, const T *r,
                      const T *rt, const T *zin, T *zout, double *part_rz, cudaStream_t s);
// 1-D transfer tables between grids of mf and mc nodes per side:
// restriction taps (fine node, weight) per coarse node, XFER_RTAPS each;
// prolongation taps (coarse node, weight) per fine node, 2 each; index -1 =
// no tap.  Built once per potential by launch_xfer_tables.
constexpr int XFER_RTAPS = 6;
struct XferTab {
    int *ridx;
    double *rw;
    float *rwf;
    int *pidx;
    double *pw;
    float *pwf;
};
void launch_xfer_tables(int mf, int mc, const XferTab &t, cudaStream_t s);
// rc = ((mc+1)/(mf+1))^3 P^T rf, three 1-D passes through tmp1 (mf*mf*mc*N)
// and tmp2 (mf*mc*mc*N)
template <typename T>
void launch_restrict(int mf, int mc, int N, const XferTab &t, const T *rf, T *tmp1, T *tmp2,
                     T *rc, cudaStream_t s);
// ef_out = ef_in + P ec, three 1-D passes through tmp2 and tmp1
template <typename T>
void launch_prolong(int mf, int mc, int N, const XferTab &t, const T *ec, T *tmp1, T *tmp2,
                    const T *efin, T *efout, cudaStream_t s);
// z = Ainv r on the coarsest level (Ainv nc x nc, FP64)
template <typename T>
void launch_coarse_solve(const GridGeom &g, const double *Ainv, const T *r, T *z,
                         cudaStream_t s);
// partial of x.y per column
template <typename T>
void launch_dot(const GridGeom &g, const T *x, const T *y, double *part, cudaStream_t s);

// The coarse levels l0 .. L-1 of an FP32 V-cycle in one launch (k_vcoarse.cu):
// one CTA per column, every level's vectors in shared memory.  Arrays are
// indexed from l0 (entry 0 = level l0); the last entry is the coarsest level.
constexpr int VC_MAXLEV = 8;
constexpr int VC_MAX_SMEM = 200 * 1024;
struct VCoarse {
    int levels;                       // levels in the launch (>= 2)
    int m[VC_MAXLEV];                 // nodes per side
    float c[VC_MAXLEV];               // 1 / (2 h_l^2)
    const float *D[VC_MAXLEV], *wD[VC_MAXLEV];
    const int *ridx[VC_MAXLEV];       // transfer tables of level l to l + 1
    const float *rw[VC_MAXLEV];
    const int *pidx[VC_MAXLEV];
    const float *pw[VC_MAXLEV];
    float rscale[VC_MAXLEV];          // ((m_{l+1} + 1) / (m_l + 1))^3
    const double *Ainv;               // dense inverse of the coarsest operator
    int nc;
    float omw;                        // 1 - omega
    int nu1, nu2;
};
size_t vcoarse_smem_bytes(const VCoarse &v);
// sets the dynamic shared-memory limit (call once, outside any stream capture)
void vcoarse_prepare();
// z = V-cycle(r) from level l0 for all N columns (point-major n_l0 x N FP32 blocks)
void launch_vcoarse(const VCoarse &v, int N, const float *r, float *z, cudaStream_t s);
// the whole FP32 V-cycle (l0 = 0) between FP64 blocks: r32 = (float) r64,
// z64 = (double) V-cycle(r32) and (part non-null) the partials of r64 . z64
// in the rows of the FP64 geometry g64, as launch_convert_d2f +
// launch_vcoarse + launch_widen_dot give them, bit for bit
size_t vcoarse64_smem_bytes(const VCoarse &v, const GridGeom &g64);
void launch_vcoarse64(const VCoarse &v, const GridGeom &g64, const double *r64, double *z64,
                      double *part, cudaStream_t s);

// per-column reduction of gy partials + PCG scalar logic
enum FinMode { FIN_BNORM_RNORM = 0, FIN_ALPHA = 1, FIN_RR = 2, FIN_BETA = 3, FIN_RZ = 4 };
// row chunks of the finalisation for gy partial rows (sizes PcgScalars::fpart)
int finalize_chunks(int gy);
void launch_finalize(int mode, int N, int gy, const double *part, const double *part2,
                     PcgScalars sc, double rtol, cudaStream_t s);

// sets the WHILE condition of a captured PCG loop (num_active[0] > 0 and
// ++iter[0] < maxit)
void launch_pcg_cond(const int *num_active, int *iter, int maxit, cudaGraphConditionalHandle h,
                     cudaStream_t s);
// whole-step graphs: hw = (num_active[0] > 0 && maxit > 0) before the loop;
// in the loop body: ++iter[0], more = active && iter < maxit, counters[0] += 1,
// counters[1] += more, hif = hw = more, and ST_PCG_MAXIT in status when
// columns are still active at the cap (check_maxit)
void launch_pcg_cond_init(const int *num_active, int maxit, cudaGraphConditionalHandle hw,
                          cudaStream_t s);
void launch_pcg_cond2(const int *num_active, int *iter, int maxit, cudaGraphConditionalHandle hw,
                      cudaGraphConditionalHandle hif, long long *counters, int *status,
                      int check_maxit, cudaStream_t s);
// out[i] = pseudo-random value in [-1, 1) from a hash of (seed, i)
template <typename T>
void launch_fill_hash(long count, unsigned long long seed, T *out, cudaStream_t s);
// FP64 block products on tensor cores by exact integer slicing (k_tall_oz.cu):
// Out = A1 M1 (+ A2 M2) (+ Cin), FP64, for K = k1 + k2 <= 128; image: scratch
// of tall_oz_image_bytes(n, K, ncol); part_sq: tall_oz_partials(n, ncol) sums of
// squares of Out (nullable)
bool tall_oz_supported(int k1, int k2);
size_t tall_oz_image_bytes(long n, int K, int ncol);
int tall_oz_partials(long n, int ncol);
void oz_prepare();
// FP64 Gram w [X1 X2]^T [X1 X2] (n x na, na <= 128) by the same slicing;
// scratch: gram_oz_scratch_bytes(n, na); out: na x na row-major.  col0 > 0:
// only the output columns from the 64-column tile that holds col0 on are
// formed and written (a cross block X1^T X2 with n1 a multiple of 64)
bool gram_oz_supported(int na);
size_t gram_oz_scratch_bytes(long n, int na);
void launch_gram_oz(long n, const double *X1, int n1, const double *X2, int n2, double w,
                    double *scratch, double *out, int *status, cudaStream_t s, int col0 = 0);
void launch_tall_oz(long n, const double *A1, int k1, const double *M1, const double *A2, int k2,
                    const double *M2, int ncol, const double *Cin, double *Out, double *part_sq,
                    unsigned char *image, int *status, cudaStream_t s);
// sets the dynamic shared-memory limits of the tensor-core kernels (call once,
// outside any stream capture)
void tc_prepare();

// ----------------------------------------------------------------------------
// batched form (k_batch.cu): device state of the time loop of one problem in
// a batch graph, nine 64-bit words in the problem's workspace (T0, TIMEOUT
// and ITERS are used in the first problem's words only)
// ----------------------------------------------------------------------------
enum { BS_STEPS = 0, BS_DONE = 1, BS_AEXEC = 2, BS_MODE = 3, BS_MAXSTEPS = 4, BS_EPS = 5,
       BS_T0 = 6, BS_TIMEOUT = 7, BS_ITERS = 8 };
// BS_DONE codes
enum { BD_RUNNING = 0, BD_CONVERGED = 1, BD_MAXSTEPS = 2, BD_ERROR = 3, BD_TIMEOUT = 4 };
constexpr int BATCH_MAX = 64;
struct BatchArgs {
    int count;
    long long *slot[BATCH_MAX];
    cudaGraphConditionalHandle h[BATCH_MAX];   // per-problem IF handles (arm)
};
// before the time loop: steps, done and A-executions cleared, start time
// stamped in slot[0], hT = (count > 0)
void launch_batch_init(const BatchArgs &a, cudaGraphConditionalHandle hT, cudaStream_t s);
// start of each time-loop iteration: a problem in step mode that has taken
// its steps is done; h[k] = !done
void launch_batch_arm(const BatchArgs &a, cudaStream_t s);
// after phase A of one problem: stop on error, nonfinite g, g < eps (solve
// mode) or the step cap; hB = still running
void launch_batch_check(long long *slot, const double *g, const int *st1, const int *st2,
                        cudaGraphConditionalHandle hB, cudaStream_t s);
// after phase B of one problem: ++steps
void launch_batch_count(long long *slot, cudaStream_t s);
// end of each time-loop iteration: ++ITERS, wall-clock limit (slot[0] T0 /
// TIMEOUT), hT = any problem still running
void launch_batch_cond(const BatchArgs &a, cudaGraphConditionalHandle hT, cudaStream_t s);

// adjoint row kernels (FP64): mode 0 out[p] = scale sum_c w_c u_pc^2,
// mode 1 out[p] = scale sum_c u_pc v_pc
void launch_rowreduce(int mode, long n, int N, const double *u, const double *v, const double *w,
                      double scale, double *out, cudaStream_t s);
void launch_scale_rows(long n, int N, const double *g, const double *u, double *y, cudaStream_t s);
void launch_shift_cols(long n, int N, const double *sft, const double *x, double *y,
                       cudaStream_t s);
// An FP32 preconditioner inside an FP64 block PCG, its interface fused into
// the PCG passes (g: the FP64 geometry of the finest level for the PCG
// kernels, the FP32 one for the sweep):
// x += alpha p, r -= alpha q, partial r.r, r32 = (float) r, z32 = wD32 r32
void launch_pcg_xr_mg(const GridGeom &g, const double *alpha, const double *p, const double *q,
                      double *x, double *r, double *part_rr, const float *wD32, float *r32,
                      float *z32, cudaStream_t s);
// the damped-Jacobi sweep of launch_jacobi<float> with the partial
// r64 . (double) z_out per column (FP64), in g's partial rows (g.gy)
void launch_jacobi_dot64(const GridGeom &g, const float *wD, float c, float omw, const float *r,
                         const double *r64, const float *zin, float *zout, double *part,
                         cudaStream_t s);
// p = (double) z32 + beta p
void launch_pcg_p_mg(const GridGeom &g, const double *beta, const float *z32, double *p,
                     cudaStream_t s);
// out = a x + b y over count FP64 values (out may alias x or y)
void launch_axpby(size_t count, double a, const double *x, double b, const double *y, double *out,
                  cudaStream_t s);
// d = a - b, returns the number of partial sums of d^2 written to part
int launch_diff_sq(long n, const double *a, const double *b, double *d, double *part,
                   cudaStream_t s);

// setup
void launch_coarse_potential(int mf, const double *Vf, int mc, double *Vc, cudaStream_t s);
// D = 6c + V + sigma, wD = omega / D and (nullable) wcD = wD c per point
void launch_level_diag(long n, const double *V, double sigma, double c, double omega,
                       double *D, double *wD, double *wcD, cudaStream_t s);
void launch_assemble_dense(int mc, double c, const double *V, double sigma, double *A,
                           cudaStream_t s);
void launch_gauss_jordan(int nc, double *A, double *Ainv, int *status, cudaStream_t s);
void launch_minmax(long n, const double *V, double *out2 /* [min, max-abs-nonfinite flag] */,
                   cudaStream_t s);
void launch_convert_d2f(size_t count, const double *in, float *out, cudaStream_t s);
// z = (double) z32, partials of r.z per column (nullable) in g's layout (FP64 geometry)
void launch_widen_dot(const GridGeom &g, const float *z32, const double *r, double *z,
                      double *part, cudaStream_t s);
void launch_convert_f2d(size_t count, const float *in, double *out, cudaStream_t s);
template <typename T>
void launch_scale(size_t count, const double *factor, T *x, cudaStream_t s);

// ----------------------------------------------------------------------------
// dense kernels (k_dense.cu)
// ----------------------------------------------------------------------------
// Gram of logical blocks A = [A1 A2] (n x (na1+na2)) and B = [B1 B2]:
// out = w A^T B  (FP64, row-major).  If sym, A == B and only the upper tiles
// are computed (mirrored).  partials: workspace of gram_partial_bytes().
struct GramPlan {
    long n;
    int na, nb, tiles_a, tiles_b, ntiles, chunks;
    long chunk_rows;
    bool sym;
};
GramPlan make_gram_plan(long n, int na, int nb, bool sym);
size_t gram_partial_bytes(const GramPlan &p);
template <typename T>
void launch_gram(const GramPlan &p, const T *A1, int na1, const T *A2, int na2, const T *B1,
                 int nb1, const T *B2, int nb2, double w, double *partials, double *out,
                 cudaStream_t s);

// Symmetric Gram out = w [X1 X2]^T [X1 X2] of FP32 blocks on tcgen05 tensor
// cores (kind::tf32, 3xTF32 split, FP32 accumulation in TMEM, FP64 chunk
// reduction).  partials: gram_tc_partial_bytes(n, n1 + n2) bytes.
size_t gram_tc_partial_bytes(long n, int na);
size_t gram_tc_smem_bytes();
void launch_gram_tc(long n, const float *X1, int n1, const float *X2, int n2, double w,
                    float *partials, double *out, int *status, cudaStream_t s);

// FP32 block x small-matrix product on tcgen05 (3xTF32):
// Out (n x ncol) = A1 (n x k1) M1 (k1 x ncol) + A2 M2 (+ Cin); M1, M2 FP64
// row-major, split into the swizzled tf32 hi/lo image (tall_tc_image_bytes);
// part_sq (nullable): tall_tc_partials(n, ncol) partial sums of squares of Out.
size_t tall_tc_image_bytes(int k1, int k2, int ncol);
int tall_tc_partials(long n, int ncol);
void launch_tall_tc(long n, const float *A1, int k1, const double *M1, const float *A2, int k2,
                    const double *M2, int ncol, const float *Cin, float *Out, double *part_sq,
                    unsigned char *image, int *status, cudaStream_t s);

// Out = A1 M1 (+ A2 M2) (+ Cin), M's are FP64 K x Ncol row-major; optional
// partial sum of squares of Out (one double per CTA, npart entries).
struct TallPlan {
    long n;
    int ncol, k1, k2;
    int gx, gy;
};
TallPlan make_tall_plan(long n, int ncol, int k1, int k2);
template <typename T>
void launch_tall_gemm(const TallPlan &p, const T *A1, const double *M1, const T *A2,
                      const double *M2, const T *Cin, T *Out, double *part_sq,
                      cudaStream_t s);
// same with per-column partial sums of squares (gy x ncol)
template <typename T>
void launch_tall_gemm_colsq(const TallPlan &p, const T *A1, const double *M1, const T *A2,
                            const double *M2, const T *Cin, T *Out, double *part_sq,
                            cudaStream_t s);
// dst (rows x cols, ld ldd) = alpha * src (ld lds)
void launch_extract(int rows, int cols, double alpha, const double *src, int lds, double *dst,
                    int ldd, cudaStream_t s);
// out[i][j] = -Cv[i][j] * (lam[j] + add)   (N x N)
void launch_scale_cols(int N, const double *Cv, const double *lam, double add, double *out,
                       cudaStream_t s);
// out[0] = w * sum(part[0..np)); out[1] = ||A - I||_F for N x N A (nullable)
void launch_monitor_finish(int np, const double *part, double w, int N, const double *A,
                           double *out, cudaStream_t s);
// out[0] = sqrt(w * sum(part[0..np)))
void launch_sum_sqrt(int np, const double *part, double w, double *out, cudaStream_t s);
// per-column version: part is np x ncol, out[c] = sqrt(w * sum_i part[i*ncol+c])
void launch_colsum_sqrt(int np, int ncol, const double *part, double w, double *out,
                        cudaStream_t s);

// C = alpha op(A) op(B) + beta C (FP64, row-major, small)
void launch_small_gemm(int M, int Ncol, int K, double alpha, const double *A, int lda, bool ta,
                       const double *B, int ldb, bool tb, double beta, double *C, int ldc,
                       cudaStream_t s);
// predictor system of Eq. (4.1): from the 2N x 2N Gram of [U W] build
//   [I - tau/2 Puw, tau/2 S; -tau/2 Q, I + tau/2 Pwu] [X;Y] = [S; Pwu]
// and solve by LU with partial pivoting.  Mwork: 4N^2, XY: 2N x N.  Then
// C = [I - tau Y; tau X] (2N x N).
// ipiv: 2N ints of scratch for the blocked elimination used when 2N > 64
// (nullptr: always the one-CTA kernel)
// lu32 (4N^2 floats), pB, pR (2N x N doubles): scratch of the mixed-precision
// variant (FP32 elimination + FP64 iterative refinement), used when all are
// non-null and the system fits one CTA's shared memory
// true when the FP32 elimination of an nn x nn system with nr right-hand
// sides fits one CTA's shared memory
bool lu32_fits(int nn, int nr);
// X = A^-1 B (nn x nn, nn x nr, FP64) by FP32 elimination with partial
// pivoting and `refine` FP64 residual-correction steps; LU (nn^2 floats),
// ipiv (nn) and R (nn x nr doubles) are scratch; requires lu32_fits(nn, nr)
void launch_solve32_refined(int nn, int nr, const double *A, int lda, const double *B, int ldb,
                            double *X, float *LU, int *ipiv, double *R, int refine, int *status,
                            cudaStream_t s);
void launch_predictor_solve(int N, double tau, const double *G2, double *Mwork, double *XY,
                            double *C, int *status, cudaStream_t s,
                            const double *tau_dev = nullptr, int *ipiv = nullptr,
                            float *lu32 = nullptr, double *pB = nullptr, double *pR = nullptr);
// sets the shared-memory limits of the FP32 elimination kernels (call once,
// outside any stream capture)
void lu32_prepare();
// largest eigenvalue of sym(A) (N x N, leading dimension lda) -> out[0];
// vec (N): warm-start vector, updated (all zero: fixed start)
void launch_top_eig(int N, const double *A, int lda, double *vec, double *out, cudaStream_t s);
// the same estimate of the pencil (sym(K), S) in FP32 in one launch (mixed
// contexts): out[0] = largest eigenvalue to ~1e-6, vec the warm vector
bool lam_hat32_fits(int N);
void launch_lam_hat32(int N, const double *K, const double *S, double *vec, double *out,
                      int *status, cudaStream_t s);
// out[0] = max_i sum_j |A_ij|
void launch_gersh(int N, const double *A, int lda, double *out, cudaStream_t s);
// adaptive time step (see hq_config.adaptive_tau): st[0] = tau_n, st[1] = tau_{n-1},
// st[2] = first-step flag
void launch_adapt_tau(const double *mm, const double *sm, double tau_max, double c, double gamma,
                      double lb, double *st, cudaStream_t s);
// Om = -tau (Shat - I), tau from tau_dev when non-null
void launch_corrector_matrix(int N, const double *Shat, const double *tau_dev, double tau,
                             double *Om, cudaStream_t s);
// A += v I (N x N) in place
void launch_add_diag(int N, double *A, double v, cudaStream_t s);
// out = alpha * in  (count values)
void launch_dscale(int count, double alpha, const double *in, double *out, cudaStream_t s);
// symmetric eigen (cyclic Jacobi, one CTA): ascending evals, evecs columns (N x N)
void launch_sym_eig(int N, const double *A, double *work, double *evals, double *evecs,
                    cudaStream_t s);
// Rayleigh-Ritz reduction: given K (N x N, symmetrised inside) and S (SPD),
// Cm = L^{-1} K L^{-T} with S = L L^T; Linv kept in L (lower).  One CTA.
void launch_rr_reduce(int N, const double *K, const double *S, double *L, double *Cm,
                      int *status, cudaStream_t s);
// X = A^{-1} B for SPD A by Cholesky (one CTA); L: N x N work
// sets the shared-memory limit of the blocked elimination's panel kernel
// (call once, outside any stream capture)
void lu_prepare();
// in place: XY (nn x nrhs) <- Mw^-1 XY, Mw (nn x nn) overwritten; blocked
// elimination with partial pivoting (ipiv: nn ints of scratch)
void launch_lu_solve(int nn, int nrhs, double *Mw, double *XY, int *ipiv, int *status,
                     cudaStream_t s);
// X = A^-1 B, A N x N symmetric positive definite (lda), B N x N (ldb): with
// lu32 (N^2 floats) an FP32 elimination in one CTA (no refinement: used for a
// warm start), else the one-CTA Cholesky kernel (factor into L) for N <= 32
// or ipiv == nullptr, else the blocked elimination in the N x N scratch Mw
void launch_spd_solve(int N, const double *A, int lda, const double *B, int ldb, double *Mw,
                      double *L, double *X, int *ipiv, int *status, cudaStream_t s,
                      float *lu32 = nullptr);
void launch_chol_solve(int N, const double *A, int lda, const double *B, int ldb, double *L,
                       double *X, int *status, cudaStream_t s);
// c = L^{-T} y  (columns of Y), Cv output N x N
void launch_rr_back(int N, const double *L, const double *Y, double *Cv, cudaStream_t s);
// scale factor 1/sqrt(evals[0]) -> out
void launch_inv_sqrt_first(const double *evals, double *out, cudaStream_t s);
// lam_paper[i] = 1/mu[N-1-i] - sigma
void launch_paper_evals(int N, const double *mu, double sigma, double *lam, cudaStream_t s);
// subtract sigma from each of N values
void launch_add_scalar(int N, const double *in, double add, double *out, cudaStream_t s);
// K -= sigma * S (elementwise N x N)
void launch_axpy_small(int count, double a, const double *x, double *y, cudaStream_t s);
// Ritz-vector sign: flip column c if its largest-magnitude entry is negative
template <typename T>
void launch_fix_signs(long n, int N, T *U, double *work /* gx*N*2 */, cudaStream_t s);
// M3 = C1 + Msmall C2 etc. are done with small_gemm.

}  // namespace hq
