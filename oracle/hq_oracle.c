/*
 * hq_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle of the
 * quasi-orthogonal inverse-operator scheme of Wang & Zhou, "A quasi-orthogonal
 * method based on the inverse operator for Schroedinger eigenvalue problems"
 * (arXiv 2605.25149).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path under
 * paper_2605_25149_gb300/csrc, and neither side includes the other.
 *
 * Conventions (the discrete problem the scheme is run on):
 *   grid      m^3 interior nodes of the cube [lo,hi]^3, h = (hi-lo)/(m+1),
 *             node (i,j,k), 0 <= i,j,k < m, sits at lo + (i+1)h (etc.),
 *             Dirichlet zero on the boundary nodes;
 *   index     p = i + m*(j + m*k)   (x fastest), n = m^3;
 *   blocks    an n x N block U is stored point-major: U[p*N + c];
 *   operator  (H u)_p = (1/(2h^2)) (6 u_p - sum of the 6 neighbours) + V_p u_p,
 *             i.e. -Delta/2 + V (the operator of the paper's examples,
 *             Example 5.1 / 5.2), and G = (H + sigma I)^{-1} is the inverse
 *             operator of Section 3.1 with a Garding shift sigma (Section 2.2);
 *   products  <A,B> = h^3 A^T B, the discrete L2 inner-product matrix of
 *             Section 2.1.
 *
 * Parity status: every exported function is pinned by tests/test_oracle_*.py
 * against closed forms, brute-force dense eigensolves or exact identities of
 * the scheme; the exact step counts of the paper's Table 1 are NOT pinned
 * (different discretisation, see the design notes).
 *
 * Build: cc -O2 -std=c99 -fopenmp -ffp-contract=off -shared -fPIC
 * (-ffp-contract=off keeps x86_64 and aarch64 results bit-identical).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_BREAKDOWN 1
#define ORC_ERR_NOT_CONVERGED 2
#define ORC_ERR_SINGULAR 3
#define ORC_ERR_ARG 4
#define ORC_ERR_NOMEM 5

static const double ORC_PI = 3.14159265358979323846;

static long cube(long m) { return m * m * m; }

double orc_grid_h(int m, double lo, double hi) { return (hi - lo) / (double)(m + 1); }

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) accumulation, used for every inner product that   */
/* ends up in a Gram matrix or a reported norm.                             */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else                       k->c += (x - t) + k->s;
    k->s = t;
}
static double kval(const ksum *k) { return k->s + k->c; }

/* ------------------------------------------------------------------------ */
/* The 7-point finite-difference operator H + sigma on one contiguous       */
/* column (Section 2.2 with the -Delta/2 + V scaling of Example 5.1).        */
/* ------------------------------------------------------------------------ */
static void apply_col(int m, double h, const double *V, double sigma,
                      const double *x, double *y)
{
    double c = 0.5 / (h * h);
    for (int k = 0; k < m; k++)
        for (int j = 0; j < m; j++)
            for (int i = 0; i < m; i++) {
                long p = i + (long)m * (j + (long)m * k);
                double s = 0.0;
                if (i > 0) s += x[p - 1];
                if (i < m - 1) s += x[p + 1];
                if (j > 0) s += x[p - m];
                if (j < m - 1) s += x[p + m];
                if (k > 0) s += x[p - (long)m * m];
                if (k < m - 1) s += x[p + (long)m * m];
                y[p] = c * (6.0 * x[p] - s) + (V[p] + sigma) * x[p];
            }
}

/* y = (H + sigma) x for every column of a point-major n x N block. */
void orc_apply_h(int m, double h, const double *V, double sigma, int N,
                 const double *x, double *y)
{
    long n = cube(m);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; c++) {
        double *xc = malloc(sizeof(double) * n), *yc = malloc(sizeof(double) * n);
        for (long p = 0; p < n; p++) xc[p] = x[p * N + c];
        apply_col(m, h, V, sigma, xc, yc);
        for (long p = 0; p < n; p++) y[p * N + c] = yc[p];
        free(xc); free(yc);
    }
}

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long p = 0; p < n; p++) s += a[p] * b[p];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients on one column: (H + sigma) x = b.  Textbook CG,      */
/* stops when ||r||_2 <= rtol ||b||_2 (or after maxit iterations).          */
/* ------------------------------------------------------------------------ */
static int cg_col(int m, double h, const double *V, double sigma,
                  const double *b, double *x, double rtol, int maxit, int *iters)
{
    long n = cube(m);
    double *r = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n),
           *q = malloc(sizeof(double) * n);
    int st = ORC_ERR_NOT_CONVERGED, it = 0;
    double bn = sqrt(dot(n, b, b));
    apply_col(m, h, V, sigma, x, q);
    for (long i = 0; i < n; i++) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rr = dot(n, r, r);
    if (sqrt(rr) <= rtol * bn) st = ORC_OK;
    while (st != ORC_OK && it < maxit) {
        apply_col(m, h, V, sigma, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { st = ORC_ERR_BREAKDOWN; break; }
        double alpha = rr / pq;
        for (long i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rr1 = dot(n, r, r);
        it++;
        if (sqrt(rr1) <= rtol * bn) { st = ORC_OK; break; }
        double beta = rr1 / rr;
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rr = rr1;
    }
    free(r); free(p); free(q);
    *iters = it;
    return st;
}

/* Block of independent CG solves, x (point-major) holds the initial guess on
 * entry and the solution on exit.  iters[c] receives per-column counts.     */
int orc_cg(int m, double h, const double *V, double sigma, int N,
           const double *b, double *x, double rtol, int maxit, int *iters)
{
    long n = cube(m);
    int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < N; c++) {
        double *bc = malloc(sizeof(double) * n), *xc = malloc(sizeof(double) * n);
        for (long p = 0; p < n; p++) { bc[p] = b[p * N + c]; xc[p] = x[p * N + c]; }
        int it = 0;
        int st = cg_col(m, h, V, sigma, bc, xc, rtol, maxit, &it);
        for (long p = 0; p < n; p++) x[p * N + c] = xc[p];
        if (iters) iters[c] = it;
        if (st != ORC_OK) {
#pragma omp critical
            { if (status == ORC_OK) status = st; }
        }
        free(bc); free(xc);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Geometric multigrid (preconditioner of the inner solve; the paper leaves */
/* the solver open).  Level l has m_l interior nodes per side on the same   */
/* box, m_{l+1} = floor(m_l / 2), until m_l <= coarsest.  Grids of even m   */
/* are not nested; the transfer operators are defined for any pair:        */
/*   P : coarse -> fine is trilinear interpolation of the coarse nodal      */
/*       values (zero on the boundary) at the fine node positions;          */
/*   R : fine -> coarse is ((m_c+1)/(m_f+1))^3 P^T  (= (h_f/h_c)^3 P^T,     */
/*       the L2 adjoint of P);                                              */
/*   V_c = V_f interpolated trilinearly at the coarse nodes;                */
/*   A_c = -Delta_hc/2 + V_c + sigma (rediscretised).                       */
/* Smoother: damped Jacobi  z <- z + omega D^{-1}(r - A z),                 */
/*   D = 3/h^2 + V + sigma.  Coarsest level: exact dense Cholesky solve.    */
/* The cycle (nu1 pre-sweeps from z = 0, residual, restrict, recurse,       */
/* prolong-add, nu2 post-sweeps) is symmetric when nu1 == nu2.              */
/* ------------------------------------------------------------------------ */
#define ORC_MAXLEV 24

typedef struct {
    int L, nu1, nu2;
    double lo, hi, sigma, omega;
    int m[ORC_MAXLEV];
    double h[ORC_MAXLEV];
    double *V[ORC_MAXLEV];
    double *chol;   /* lower Cholesky factor of the coarsest matrix, nc x nc */
    long nc;
} orc_mg;

int orc_mg_levels(int m, int coarsest, int *ms)
{
    int L = 0;
    ms[L++] = m;
    while (ms[L - 1] > coarsest && ms[L - 1] >= 2 && L < ORC_MAXLEV) {
        ms[L] = ms[L - 1] / 2;
        L++;
    }
    return L;
}

/* 1-D interpolation stencil: node t (1-based, 1..mt) of a grid with mt nodes
 * lies between nodes s0 and s0+1 (0-based including the boundary node 0) of a
 * grid with ms nodes, with weights w0 (node s0) and w1 (node s0+1).  The
 * position ratio t*(ms+1)/(mt+1) is formed in integers so that it is exact. */
static void interp1(int t, int mt, int ms, int *s0, double *w0, double *w1)
{
    long num = (long)t * (ms + 1);
    long den = mt + 1;
    *s0 = (int)(num / den);
    long rem = num % den;
    *w1 = (double)rem / (double)den;
    *w0 = (double)(den - rem) / (double)den;
}

/* V_c = trilinear interpolation of V_f at the coarse nodes.  Every coarse
 * interior node lies inside the hull of the fine interior nodes, so no
 * boundary value is needed.                                                */
void orc_coarse_potential(int mf, const double *Vf, int mc, double *Vc)
{
    for (int k = 0; k < mc; k++)
        for (int j = 0; j < mc; j++)
            for (int i = 0; i < mc; i++) {
                int s[3]; double w[3][2];
                int t[3] = {i + 1, j + 1, k + 1};
                for (int d = 0; d < 3; d++) interp1(t[d], mc, mf, &s[d], &w[d][0], &w[d][1]);
                double v = 0.0;
                for (int c = 0; c < 8; c++) {
                    int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
                    int fi = s[0] + a, fj = s[1] + b, fk = s[2] + e;  /* 1-based */
                    double wt = w[0][a] * w[1][b] * w[2][e];
                    if (wt == 0.0) continue;
                    v += wt * Vf[(fi - 1) + (long)mf * ((fj - 1) + (long)mf * (fk - 1))];
                }
                Vc[i + (long)mc * (j + (long)mc * k)] = v;
            }
}

/* ef += P ec on one column. */
static void prolong_add_col(int mc, int mf, const double *ec, double *ef)
{
    for (int k = 0; k < mf; k++)
        for (int j = 0; j < mf; j++)
            for (int i = 0; i < mf; i++) {
                int s[3]; double w[3][2];
                int t[3] = {i + 1, j + 1, k + 1};
                for (int d = 0; d < 3; d++) interp1(t[d], mf, mc, &s[d], &w[d][0], &w[d][1]);
                double v = 0.0;
                for (int c = 0; c < 8; c++) {
                    int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
                    int ci = s[0] + a, cj = s[1] + b, ck = s[2] + e;  /* 1-based */
                    if (ci < 1 || ci > mc || cj < 1 || cj > mc || ck < 1 || ck > mc) continue;
                    v += w[0][a] * w[1][b] * w[2][e] *
                         ec[(ci - 1) + (long)mc * ((cj - 1) + (long)mc * (ck - 1))];
                }
                ef[i + (long)mf * (j + (long)mf * k)] += v;
            }
}

/* rc = ((mc+1)/(mf+1))^3 P^T rf on one column: the literal transpose of the
 * loop above, scattering each fine value to the coarse nodes it is
 * interpolated from.                                                       */
static void restrict_col(int mf, int mc, const double *rf, double *rc)
{
    double q = (double)(mc + 1) / (double)(mf + 1);
    double scale = q * q * q;
    memset(rc, 0, sizeof(double) * cube(mc));
    for (int k = 0; k < mf; k++)
        for (int j = 0; j < mf; j++)
            for (int i = 0; i < mf; i++) {
                int s[3]; double w[3][2];
                int t[3] = {i + 1, j + 1, k + 1};
                for (int d = 0; d < 3; d++) interp1(t[d], mf, mc, &s[d], &w[d][0], &w[d][1]);
                double r = rf[i + (long)mf * (j + (long)mf * k)];
                for (int c = 0; c < 8; c++) {
                    int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
                    int ci = s[0] + a, cj = s[1] + b, ck = s[2] + e;
                    if (ci < 1 || ci > mc || cj < 1 || cj > mc || ck < 1 || ck > mc) continue;
                    rc[(ci - 1) + (long)mc * ((cj - 1) + (long)mc * (ck - 1))] +=
                        scale * (w[0][a] * w[1][b] * w[2][e]) * r;
                }
            }
}

/* Point-major wrappers used by the parity tests. */
void orc_prolong_add(int mc, int mf, int N, const double *ec, double *ef)
{
    long nc = cube(mc), nf = cube(mf);
    for (int c = 0; c < N; c++) {
        double *a = malloc(sizeof(double) * nc), *b = malloc(sizeof(double) * nf);
        for (long p = 0; p < nc; p++) a[p] = ec[p * N + c];
        for (long p = 0; p < nf; p++) b[p] = ef[p * N + c];
        prolong_add_col(mc, mf, a, b);
        for (long p = 0; p < nf; p++) ef[p * N + c] = b[p];
        free(a); free(b);
    }
}

void orc_restrict(int mf, int mc, int N, const double *rf, double *rc)
{
    long nc = cube(mc), nf = cube(mf);
    for (int c = 0; c < N; c++) {
        double *a = malloc(sizeof(double) * nf), *b = malloc(sizeof(double) * nc);
        for (long p = 0; p < nf; p++) a[p] = rf[p * N + c];
        restrict_col(mf, mc, a, b);
        for (long p = 0; p < nc; p++) rc[p * N + c] = b[p];
        free(a); free(b);
    }
}

/* In-place dense Cholesky A = L L^T (lower triangle kept). */
static int cholesky(long n, double *A)
{
    for (long j = 0; j < n; j++) {
        double d = A[j * n + j];
        for (long k = 0; k < j; k++) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return ORC_ERR_SINGULAR;
        d = sqrt(d);
        A[j * n + j] = d;
        for (long i = j + 1; i < n; i++) {
            double s = A[i * n + j];
            for (long k = 0; k < j; k++) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / d;
        }
        for (long i = 0; i < j; i++) A[i * n + j] = 0.0;
    }
    return ORC_OK;
}

static void chol_solve(long n, const double *L, const double *b, double *x)
{
    for (long i = 0; i < n; i++) {
        double s = b[i];
        for (long k = 0; k < i; k++) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (long i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (long k = i + 1; k < n; k++) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

orc_mg *orc_mg_create(int m, double lo, double hi, const double *V, double sigma,
                      int nu1, int nu2, double omega, int coarsest)
{
    orc_mg *mg = calloc(1, sizeof(orc_mg));
    if (!mg) return NULL;
    mg->L = orc_mg_levels(m, coarsest, mg->m);
    mg->nu1 = nu1; mg->nu2 = nu2; mg->omega = omega; mg->sigma = sigma;
    mg->lo = lo; mg->hi = hi;
    for (int l = 0; l < mg->L; l++) {
        mg->h[l] = orc_grid_h(mg->m[l], lo, hi);
        mg->V[l] = malloc(sizeof(double) * cube(mg->m[l]));
        if (l == 0) memcpy(mg->V[0], V, sizeof(double) * cube(m));
        else orc_coarse_potential(mg->m[l - 1], mg->V[l - 1], mg->m[l], mg->V[l]);
    }
    int lc = mg->L - 1;
    long nc = cube(mg->m[lc]);
    mg->nc = nc;
    mg->chol = malloc(sizeof(double) * nc * nc);
    double *e = calloc(nc, sizeof(double)), *col = malloc(sizeof(double) * nc);
    for (long q = 0; q < nc; q++) {   /* assemble A_c column by column */
        e[q] = 1.0;
        apply_col(mg->m[lc], mg->h[lc], mg->V[lc], sigma, e, col);
        e[q] = 0.0;
        for (long i = 0; i < nc; i++) mg->chol[i * nc + q] = col[i];
    }
    free(e); free(col);
    if (cholesky(nc, mg->chol) != ORC_OK) {
        for (int l = 0; l < mg->L; l++) free(mg->V[l]);
        free(mg->chol); free(mg);
        return NULL;
    }
    return mg;
}

void orc_mg_destroy(orc_mg *mg)
{
    if (!mg) return;
    for (int l = 0; l < mg->L; l++) free(mg->V[l]);
    free(mg->chol);
    free(mg);
}

int orc_mg_nlevels(const orc_mg *mg) { return mg->L; }
int orc_mg_level_m(const orc_mg *mg, int l) { return mg->m[l]; }
void orc_mg_level_potential(const orc_mg *mg, int l, double *out)
{
    memcpy(out, mg->V[l], sizeof(double) * cube(mg->m[l]));
}

/* One damped-Jacobi sweep z <- z + omega D^{-1} (r - A z) on level l. */
static void jacobi_sweep(const orc_mg *mg, int l, const double *r, double *z, double *tmp)
{
    int m = mg->m[l];
    long n = cube(m);
    double h = mg->h[l];
    apply_col(m, h, mg->V[l], mg->sigma, z, tmp);
    for (long p = 0; p < n; p++) {
        double D = 3.0 / (h * h) + mg->V[l][p] + mg->sigma;
        z[p] = z[p] + mg->omega * (r[p] - tmp[p]) / D;
    }
}

static void vcycle_col(const orc_mg *mg, int l, const double *r, double *z)
{
    int m = mg->m[l];
    long n = cube(m);
    if (l == mg->L - 1) { chol_solve(n, mg->chol, r, z); return; }
    double *tmp = malloc(sizeof(double) * n);
    memset(z, 0, sizeof(double) * n);
    for (int s = 0; s < mg->nu1; s++) jacobi_sweep(mg, l, r, z, tmp);
    apply_col(m, mg->h[l], mg->V[l], mg->sigma, z, tmp);
    for (long p = 0; p < n; p++) tmp[p] = r[p] - tmp[p];        /* residual */
    long nc = cube(mg->m[l + 1]);
    double *rc = malloc(sizeof(double) * nc), *ec = malloc(sizeof(double) * nc);
    restrict_col(m, mg->m[l + 1], tmp, rc);
    vcycle_col(mg, l + 1, rc, ec);
    prolong_add_col(mg->m[l + 1], m, ec, z);
    for (int s = 0; s < mg->nu2; s++) jacobi_sweep(mg, l, r, z, tmp);
    free(tmp); free(rc); free(ec);
}

/* z = M r (one V-cycle from level 0) for each column of a point-major block. */
void orc_mg_vcycle(const orc_mg *mg, int N, const double *r, double *z)
{
    long n = cube(mg->m[0]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < N; c++) {
        double *rc = malloc(sizeof(double) * n), *zc = malloc(sizeof(double) * n);
        for (long p = 0; p < n; p++) rc[p] = r[p * N + c];
        vcycle_col(mg, 0, rc, zc);
        for (long p = 0; p < n; p++) z[p * N + c] = zc[p];
        free(rc); free(zc);
    }
}

/* One damped-Jacobi sweep on level l for a point-major block (parity tests). */
void orc_mg_smooth(const orc_mg *mg, int l, int N, const double *r, double *z)
{
    long n = cube(mg->m[l]);
    for (int c = 0; c < N; c++) {
        double *rc = malloc(sizeof(double) * n), *zc = malloc(sizeof(double) * n),
               *tmp = malloc(sizeof(double) * n);
        for (long p = 0; p < n; p++) { rc[p] = r[p * N + c]; zc[p] = z[p * N + c]; }
        jacobi_sweep(mg, l, rc, zc, tmp);
        for (long p = 0; p < n; p++) z[p * N + c] = zc[p];
        free(rc); free(zc); free(tmp);
    }
}

/* Exact coarsest-level solve for a point-major block (parity tests). */
void orc_mg_coarse_solve(const orc_mg *mg, int N, const double *r, double *z)
{
    long n = mg->nc;
    double *rc = malloc(sizeof(double) * n), *zc = malloc(sizeof(double) * n);
    for (int c = 0; c < N; c++) {
        for (long p = 0; p < n; p++) rc[p] = r[p * N + c];
        chol_solve(n, mg->chol, rc, zc);
        for (long p = 0; p < n; p++) z[p * N + c] = zc[p];
    }
    free(rc); free(zc);
}

/* Preconditioned CG with one V-cycle as preconditioner, per column:
 *   r = b - A x, z = M r, p = z
 *   repeat: q = A p, alpha = (r.z)/(p.q), x += alpha p, r -= alpha q,
 *           stop if ||r|| <= rtol ||b||, z = M r, beta = (r.z)_new/(r.z),
 *           p = z + beta p.
 * With rtol = 0 it runs exactly maxit iterations (used to compare the GPU
 * recurrence iteration by iteration).                                       */
static int pcg_col(const orc_mg *mg, const double *b, double *x, double rtol,
                   int maxit, int *iters)
{
    int m = mg->m[0];
    long n = cube(m);
    double h = mg->h[0];
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n),
           *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
    int st = ORC_ERR_NOT_CONVERGED, it = 0;
    double bn = sqrt(dot(n, b, b));
    apply_col(m, h, mg->V[0], mg->sigma, x, q);
    for (long i = 0; i < n; i++) r[i] = b[i] - q[i];
    if (sqrt(dot(n, r, r)) <= rtol * bn) st = ORC_OK;
    if (st != ORC_OK) {
        vcycle_col(mg, 0, r, z);
        memcpy(p, z, sizeof(double) * n);
    }
    double rz = dot(n, r, z);
    while (st != ORC_OK && it < maxit) {
        apply_col(m, h, mg->V[0], mg->sigma, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { st = ORC_ERR_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (long i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        it++;
        if (sqrt(dot(n, r, r)) <= rtol * bn) { st = ORC_OK; break; }
        vcycle_col(mg, 0, r, z);
        double rz1 = dot(n, r, z);
        double beta = rz1 / rz;
        for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        rz = rz1;
    }
    if (rtol == 0.0 && st == ORC_ERR_NOT_CONVERGED && it == maxit) st = ORC_OK;
    free(r); free(z); free(p); free(q);
    *iters = it;
    return st;
}

int orc_pcg_mg(const orc_mg *mg, int N, const double *b, double *x, double rtol,
               int maxit, int *iters)
{
    long n = cube(mg->m[0]);
    int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < N; c++) {
        double *bc = malloc(sizeof(double) * n), *xc = malloc(sizeof(double) * n);
        for (long p = 0; p < n; p++) { bc[p] = b[p * N + c]; xc[p] = x[p * N + c]; }
        int it = 0;
        int st = pcg_col(mg, bc, xc, rtol, maxit, &it);
        for (long p = 0; p < n; p++) x[p * N + c] = xc[p];
        if (iters) iters[c] = it;
        if (st != ORC_OK) {
#pragma omp critical
            { if (status == ORC_OK) status = st; }
        }
        free(bc); free(xc);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Inner-product matrices <A,B> = w A^T B (Section 2.1), compensated sums.  */
/* A is n x Na, B is n x Nb, both point-major; out is Na x Nb row-major.    */
/* ------------------------------------------------------------------------ */
void orc_gram(long n, int Na, const double *A, int Nb, const double *B, double w, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < Na; a++)
        for (int b = 0; b < Nb; b++) {
            ksum k = {0.0, 0.0};
            for (long p = 0; p < n; p++) kadd(&k, A[p * Na + a] * B[p * Nb + b]);
            out[a * Nb + b] = w * kval(&k);
        }
}

/* C (n x Nc) = A (n x K) * M (K x Nc), point-major blocks, plain sums. */
static void block_times_small(long n, int K, const double *A, int Nc, const double *M, double *C)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; p++)
        for (int c = 0; c < Nc; c++) {
            double s = 0.0;
            for (int k = 0; k < K; k++) s += A[p * K + k] * M[k * Nc + c];
            C[p * Nc + c] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting: solves A X = B in place (A nn x nn,      */
/* B nn x nrhs, row-major).  Returns ORC_ERR_SINGULAR on a zero pivot.      */
/* ------------------------------------------------------------------------ */
int orc_lu_solve(int nn, double *A, int nrhs, double *B)
{
    for (int k = 0; k < nn; k++) {
        int piv = k;
        double best = fabs(A[(long)k * nn + k]);
        for (int i = k + 1; i < nn; i++)
            if (fabs(A[(long)i * nn + k]) > best) { best = fabs(A[(long)i * nn + k]); piv = i; }
        if (!(best > 0.0)) return ORC_ERR_SINGULAR;
        if (piv != k) {
            for (int j = 0; j < nn; j++) {
                double t = A[(long)k * nn + j]; A[(long)k * nn + j] = A[(long)piv * nn + j]; A[(long)piv * nn + j] = t;
            }
            for (int j = 0; j < nrhs; j++) {
                double t = B[(long)k * nrhs + j]; B[(long)k * nrhs + j] = B[(long)piv * nrhs + j]; B[(long)piv * nrhs + j] = t;
            }
        }
        for (int i = k + 1; i < nn; i++) {
            double f = A[(long)i * nn + k] / A[(long)k * nn + k];
            A[(long)i * nn + k] = f;
            for (int j = k + 1; j < nn; j++) A[(long)i * nn + j] -= f * A[(long)k * nn + j];
            for (int j = 0; j < nrhs; j++) B[(long)i * nrhs + j] -= f * B[(long)k * nrhs + j];
        }
    }
    for (int i = nn - 1; i >= 0; i--)
        for (int j = 0; j < nrhs; j++) {
            double s = B[(long)i * nrhs + j];
            for (int k = i + 1; k < nn; k++) s -= A[(long)i * nn + k] * B[(long)k * nrhs + j];
            B[(long)i * nrhs + j] = s / A[(long)i * nn + i];
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigenvalue algorithm for a symmetric n x n matrix.         */
/* On exit evals ascending, evecs[:, i] (row-major, column i) the unit      */
/* eigenvector of evals[i].                                                 */
/* ------------------------------------------------------------------------ */
int orc_sym_eig(int n, const double *Ain, double *evals, double *evecs)
{
    double *A = malloc(sizeof(double) * n * n), *Vv = malloc(sizeof(double) * n * n);
    memcpy(A, Ain, sizeof(double) * n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            A[i * n + j] = 0.5 * (Ain[i * n + j] + Ain[j * n + i]);
            Vv[i * n + j] = (i == j) ? 1.0 : 0.0;
        }
    double fro = 0.0;
    for (int i = 0; i < n * n; i++) fro += A[i] * A[i];
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) off += A[i * n + j] * A[i * n + j];
        if (sqrt(off) <= 1e-15 * fro || off == 0.0) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {   /* A <- A J (columns p,q) */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {   /* A <- J^T A (rows p,q) */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                A[p * n + q] = A[q * n + p] = 0.0;
                for (int k = 0; k < n; k++) {
                    double vkp = Vv[k * n + p], vkq = Vv[k * n + q];
                    Vv[k * n + p] = c * vkp - s * vkq;
                    Vv[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    /* sort ascending (selection sort, carries eigenvectors) */
    int *idx = malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++) idx[i] = i;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++)
            if (A[idx[j] * n + idx[j]] < A[idx[i] * n + idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < n; i++) {
        evals[i] = A[idx[i] * n + idx[i]];
        if (evecs)
            for (int k = 0; k < n; k++) evecs[k * n + i] = Vv[k * n + idx[i]];
    }
    free(idx); free(A); free(Vv);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Shift rule and initial scaling (readings of Section 2.2 and Theorem 4.3) */
/* ------------------------------------------------------------------------ */
/* lb = lambda_min(-Delta_h/2) + min V; sigma = 0 if lb > 0 else 1 - lb, so
 * that the shifted operator has lambda_1 >= min(lb, 1) > 0 (Garding shift). */
double orc_auto_shift(int m, double lo, double hi, const double *V)
{
    double h = orc_grid_h(m, lo, hi);
    double s = sin(ORC_PI / (2.0 * (m + 1)));
    double lmin_lap = 3.0 * (2.0 / (h * h)) * s * s;
    double vmin = V[0];
    long n = cube(m);
    for (long p = 1; p < n; p++) if (V[p] < vmin) vmin = V[p];
    double lb = lmin_lap + vmin;
    return lb > 0.0 ? 0.0 : 1.0 - lb;
}

/* U <- U / sqrt(lambda_min(h^3 U^T U)), so that <U,U> >= I with equality in
 * one direction: U0 is put in the quasi-Stiefel set of Theorem 3.2 without
 * being orthogonalised.  Returns the scale applied.                         */
double orc_scale_initial(long n, int N, double h3, double *U)
{
    double *S = malloc(sizeof(double) * N * N), *ev = malloc(sizeof(double) * N);
    orc_gram(n, N, U, N, U, h3, S);
    orc_sym_eig(N, S, ev, NULL);
    double f = 1.0 / sqrt(ev[0]);
    for (long i = 0; i < n * N; i++) U[i] *= f;
    free(S); free(ev);
    return f;
}

/* ------------------------------------------------------------------------ */
/* One step of the quasi-orthogonal scheme, Eq. (4.1):                       */
/*   (Uh - U)/tau = G U <U, Ut> - U <G U, Ut>,   Ut = (Uh + U)/2             */
/*   (U+ - Uh)/tau = -G Uh (<Uh,Uh> - I).                                    */
/* With W = G U, X = <U,Ut>, Y = <W,Ut>, the predictor is                    */
/*   Uh = U + tau (W X - U Y),                                               */
/* and X, Y solve the 2N x 2N linear system                                  */
/*   [ I - tau/2 Puw   tau/2 S        ] [X]   [ S   ]                        */
/*   [ -tau/2 Q        I + tau/2 Pwu  ] [Y] = [ Pwu ]                        */
/* with S = <U,U>, Puw = <U,W>, Pwu = <W,U>, Q = <W,W>.                      */
/* The step also returns the Grassmann gradient norm of Remark 3.1,          */
/*   g = || W - U <G U, U> ||  (discrete L2),                                */
/* which Algorithm 1 tests against epsilon.                                  */
/*                                                                           */
/* Inputs : U (n x N), W0 (initial guess for G U, or NULL for zero),          */
/*          Z0 (initial guess for G Uh, or NULL for zero).                    */
/* Outputs (any may be NULL): W = G U, gram (2N x 2N Gram of [U W]), g,      */
/*          XY (2N x N), Uh, Shat = <Uh,Uh>, Z = G Uh, Unew.                 */
/* ------------------------------------------------------------------------ */
/* Adaptive time step (an extension: Algorithm 1 allows any tau_n <= delta_T
 * and the paper leaves adaptive stepping as future work).  From the Gram of
 * [U W] of step n:
 *   lam_hat = 1 / mu_max, mu_max the largest Ritz value of G on span(U), i.e.
 *             the largest eigenvalue of the pencil (sym <W,U>, <U,U>) -- an
 *             upper estimate of the smallest eigenvalue lambda'_1 of H + sigma;
 *   s_max   = max_i sum_j |<U,U>_ij| (Gershgorin bound on lambda_max(<U,U>));
 *   tau_n   = min(delta_T, c lam_hat / s_max, gamma tau_{n-1}),
 * with 0 < c <= 1 (0.8 by default), gamma = 1.05 and, for the first step,
 * tau_{-1} chosen so that
 * tau_0 <= c lb / s_max where lb <= lambda'_1 is the closed-form lower bound.
 * Near convergence the orthogonality error of eigenpair 1 is multiplied by
 * 1 - 2 tau / lambda'_1 per step, so tau < lambda'_1 keeps it contracting.  */
typedef struct {
    double tau_max, c, gamma, lb, tau_prev;
    int first;
} orc_adapt;

/* Cm = L^{-1} sym(K) L^{-T} with <U,U> = S = L L^T (all N x N, row-major). */
static int rr_matrix(int N, const double *K, const double *S, double *L, double *Cm, double *T)
{
    memcpy(L, S, sizeof(double) * N * N);
    int st = cholesky(N, L);
    if (st != ORC_OK) return st;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            double v = 0.5 * (K[i * N + j] + K[j * N + i]);
            for (int k = 0; k < i; k++) v -= L[i * N + k] * T[k * N + j];
            T[i * N + j] = v / L[i * N + i];
        }
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            double v = T[i * N + j];
            for (int k = 0; k < j; k++) v -= Cm[i * N + k] * L[j * N + k];
            Cm[i * N + j] = v / L[j * N + j];
        }
    return ORC_OK;
}

static double adaptive_tau(int N, const double *G2, orc_adapt *ad)
{
    int N2 = 2 * N;
    double *S = malloc(sizeof(double) * N * N), *P = malloc(sizeof(double) * N * N),
           *L = malloc(sizeof(double) * N * N), *Cm = malloc(sizeof(double) * N * N),
           *T = malloc(sizeof(double) * N * N), *ev = malloc(sizeof(double) * N);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            S[i * N + j] = G2[(long)i * N2 + j];
            P[i * N + j] = G2[(long)(N + i) * N2 + j];
        }
    /* s_max: Gershgorin bound max_i sum_j |S_ij| >= lambda_max(<U,U>) */
    double smax = 0.0;
    for (int i = 0; i < N; i++) {
        double r = 0.0;
        for (int j = 0; j < N; j++) r += fabs(S[i * N + j]);
        if (r > smax) smax = r;
    }
    double tau = ad->tau_max;
    if (rr_matrix(N, P, S, L, Cm, T) == ORC_OK) {
        orc_sym_eig(N, Cm, ev, NULL);
        double cap = ad->c * (1.0 / ev[N - 1]) / smax;
        if (cap < tau) tau = cap;
    }
    double prev = ad->first ? ad->c * ad->lb / (ad->gamma * smax) : ad->tau_prev;
    if (ad->gamma * prev < tau) tau = ad->gamma * prev;
    ad->tau_prev = tau;
    ad->first = 0;
    free(S); free(P); free(L); free(Cm); free(T); free(ev);
    return tau;
}

/* ------------------------------------------------------------------------ */
/* Step 4 and the small matrices of step 5 of Eq. (4.1), from the Gram of   */
/* [U W] (2N x 2N: S, P_uw / P_wu, Q): the 2N x 2N predictor system         */
/*   [ I - (tau/2) P_uw   (tau/2) S       ] [X]   [ S    ]                  */
/*   [ -(tau/2) Q         I + (tau/2) P_wu ] [Y] = [ P_wu ]                 */
/* solved by LU with partial pivoting (XY = [X; Y], 2N x N), and            */
/* C = [I - tau Y; tau X] (2N x N) with Uh = [U W] C.                        */
/* ------------------------------------------------------------------------ */
static int predictor_impl(int N, double tau, const double *G2, double *XY, double *C)
{
    int N2 = 2 * N;
    double *M = malloc(sizeof(double) * N2 * N2);
#define S_(i, j)   G2[(long)(i) * N2 + (j)]
#define PUW(i, j)  G2[(long)(i) * N2 + N + (j)]
#define PWU(i, j)  G2[(long)(N + (i)) * N2 + (j)]
#define Q_(i, j)   G2[(long)(N + (i)) * N2 + N + (j)]
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            double d = (i == j) ? 1.0 : 0.0;
            M[(long)i * N2 + j]           = d - 0.5 * tau * PUW(i, j);
            M[(long)i * N2 + N + j]       = 0.5 * tau * S_(i, j);
            M[(long)(N + i) * N2 + j]     = -0.5 * tau * Q_(i, j);
            M[(long)(N + i) * N2 + N + j] = d + 0.5 * tau * PWU(i, j);
            XY[(long)i * N + j]           = S_(i, j);
            XY[(long)(N + i) * N + j]     = PWU(i, j);
        }
#undef S_
#undef PUW
#undef PWU
#undef Q_
    int st = orc_lu_solve(N2, M, N, XY);
    free(M);
    if (st != ORC_OK) return st;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            C[(long)i * N + j]       = ((i == j) ? 1.0 : 0.0) - tau * XY[(long)(N + i) * N + j];
            C[(long)(N + i) * N + j] = tau * XY[(long)i * N + j];
        }
    return ORC_OK;
}

int orc_predictor(int N, double tau, const double *gram, double *XY_out, double *C_out)
{
    return predictor_impl(N, tau, gram, XY_out, C_out);
}

static int scheme_step_impl(int m, double lo, double hi, const double *V, double sigma, int N,
                            double tau, orc_adapt *ad, double *tau_used,
                            double cg_rtol, int cg_maxit,
                            const double *U, const double *W0, const double *Z0,
                            double *W_out, double *gram_out, double *g_out, double *XY_out,
                            double *Uh_out, double *Shat_out, double *Z_out, double *Unew_out,
                            int *cg_iters)
{
    long n = cube(m);
    double h = orc_grid_h(m, lo, hi), h3 = h * h * h;
    int N2 = 2 * N, st;
    double *W = malloc(sizeof(double) * n * N), *UW = malloc(sizeof(double) * n * N2),
           *G2 = malloc(sizeof(double) * N2 * N2),
           *XY = malloc(sizeof(double) * N2 * N), *C = malloc(sizeof(double) * N2 * N),
           *Uh = malloc(sizeof(double) * n * N), *Sh = malloc(sizeof(double) * N * N),
           *Z = malloc(sizeof(double) * n * N), *O = malloc(sizeof(double) * N * N),
           *ZO = malloc(sizeof(double) * n * N);
    int *it = malloc(sizeof(int) * N2);

    /* 1. W = G U */
    if (W0) memcpy(W, W0, sizeof(double) * n * N); else memset(W, 0, sizeof(double) * n * N);
    st = orc_cg(m, h, V, sigma, N, U, W, cg_rtol, cg_maxit, it);
    if (st != ORC_OK) goto done;

    /* 2. Gram of [U W]: blocks S, Puw / Pwu, Q */
    for (long p = 0; p < n; p++)
        for (int c = 0; c < N; c++) { UW[p * N2 + c] = U[p * N + c]; UW[p * N2 + N + c] = W[p * N + c]; }
    orc_gram(n, N2, UW, N2, UW, h3, G2);
#define S_(i, j)   G2[(long)(i) * N2 + (j)]
#define PUW(i, j)  G2[(long)(i) * N2 + N + (j)]
#define PWU(i, j)  G2[(long)(N + (i)) * N2 + (j)]
#define Q_(i, j)   G2[(long)(N + (i)) * N2 + N + (j)]

    /* 3. g = || W - U Pwu ||_h  (Remark 3.1, Algorithm 1) */
    if (g_out) {
        ksum k = {0.0, 0.0};
        for (long p = 0; p < n; p++)
            for (int j = 0; j < N; j++) {
                double s = 0.0;
                for (int i = 0; i < N; i++) s += U[p * N + i] * PWU(i, j);
                double r = W[p * N + j] - s;
                kadd(&k, r * r);
            }
        *g_out = sqrt(h3 * kval(&k));
    }

    /* 4. predictor system (time step fixed, or from the adaptive rule) */
    if (ad) tau = adaptive_tau(N, G2, ad);
    if (tau_used) *tau_used = tau;
    if (gram_out) memcpy(gram_out, G2, sizeof(double) * N2 * N2);
    st = predictor_impl(N, tau, G2, XY, C);
    if (st != ORC_OK) goto done;
    if (XY_out) memcpy(XY_out, XY, sizeof(double) * N2 * N);

    /* 5. Uh = U (I - tau Y) + W (tau X) = [U W] C */
    block_times_small(n, N2, UW, N, C, Uh);

    /* 6. Shat = <Uh,Uh> (computed literally), O = Shat - I */
    orc_gram(n, N, Uh, N, Uh, h3, Sh);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) O[i * N + j] = Sh[i * N + j] - ((i == j) ? 1.0 : 0.0);

    /* 7. Z = G Uh */
    if (Z0) memcpy(Z, Z0, sizeof(double) * n * N); else memset(Z, 0, sizeof(double) * n * N);
    st = orc_cg(m, h, V, sigma, N, Uh, Z, cg_rtol, cg_maxit, it + N);
    if (st != ORC_OK) goto done;

    /* 8. U+ = Uh - tau Z O */
    block_times_small(n, N, Z, N, O, ZO);
    if (Unew_out)
        for (long i = 0; i < n * N; i++) Unew_out[i] = Uh[i] - tau * ZO[i];

    if (W_out) memcpy(W_out, W, sizeof(double) * n * N);
    if (Uh_out) memcpy(Uh_out, Uh, sizeof(double) * n * N);
    if (Shat_out) memcpy(Shat_out, Sh, sizeof(double) * N * N);
    if (Z_out) memcpy(Z_out, Z, sizeof(double) * n * N);
    if (cg_iters) memcpy(cg_iters, it, sizeof(int) * N2);
#undef S_
#undef PUW
#undef PWU
#undef Q_
done:
    free(W); free(UW); free(G2); free(XY); free(C); free(Uh); free(Sh);
    free(Z); free(O); free(ZO); free(it);
    return st;
}

int orc_scheme_step(int m, double lo, double hi, const double *V, double sigma, int N,
                    double tau, double cg_rtol, int cg_maxit,
                    const double *U, const double *W0, const double *Z0,
                    double *W_out, double *gram_out, double *g_out, double *XY_out,
                    double *Uh_out, double *Shat_out, double *Z_out, double *Unew_out,
                    int *cg_iters /* 2*N or NULL */)
{
    return scheme_step_impl(m, lo, hi, V, sigma, N, tau, NULL, NULL, cg_rtol, cg_maxit, U, W0,
                            Z0, W_out, gram_out, g_out, XY_out, Uh_out, Shat_out, Z_out,
                            Unew_out, cg_iters);
}

/* Closed-form lower bound of the smallest eigenvalue of H + sigma. */
double orc_lambda1_lower_bound(int m, double lo, double hi, const double *V, double sigma)
{
    double h = orc_grid_h(m, lo, hi);
    double s = sin(ORC_PI / (2.0 * (m + 1)));
    double vmin = V[0];
    for (long p = 1; p < cube(m); p++) if (V[p] < vmin) vmin = V[p];
    return 3.0 * (2.0 / (h * h)) * s * s + vmin + sigma;
}

/* Gradient norm alone: W = G U by CG, g = || W - U <W,U> ||_h. */
int orc_grad_norm(int m, double lo, double hi, const double *V, double sigma, int N,
                  double cg_rtol, int cg_maxit, const double *U, double *W_io, double *g_out)
{
    long n = cube(m);
    double h = orc_grid_h(m, lo, hi), h3 = h * h * h;
    int st = orc_cg(m, h, V, sigma, N, U, W_io, cg_rtol, cg_maxit, NULL);
    if (st != ORC_OK) return st;
    double *P = malloc(sizeof(double) * N * N);
    orc_gram(n, N, W_io, N, U, h3, P);      /* Pwu = <W,U> */
    ksum k = {0.0, 0.0};
    for (long p = 0; p < n; p++)
        for (int j = 0; j < N; j++) {
            double s = 0.0;
            for (int i = 0; i < N; i++) s += U[p * N + i] * P[i * N + j];
            double r = W_io[p * N + j] - s;
            kadd(&k, r * r);
        }
    *g_out = sqrt(h3 * kval(&k));
    free(P);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: march Eq. (4.1) with fixed tau until g < eps.                */
/* U holds the (already scaled) initial data on entry and U_end on exit; W   */
/* receives G U_end.  The CG for G U_{n+1} starts from G Uh_n (a warm start; */
/* only the number of CG iterations depends on it).  g_hist (max_steps + 1   */
/* entries, or NULL) receives g(U_0), g(U_1), ...                            */
/* ------------------------------------------------------------------------ */
int orc_solve(int m, double lo, double hi, const double *V, double sigma, int N,
              double tau, double cg_rtol, int cg_maxit, double eps, long max_steps,
              double *U, double *W, long *steps_out, double *g_out, double *g_hist)
{
    long n = cube(m);
    double *Z = malloc(sizeof(double) * n * N), *Un = malloc(sizeof(double) * n * N);
    int have_z = 0, st = ORC_OK;
    long step = 0;
    double g = INFINITY;
    for (;;) {
        st = orc_scheme_step(m, lo, hi, V, sigma, N, tau, cg_rtol, cg_maxit, U,
                             have_z ? Z : NULL, NULL, W, NULL, &g, NULL, NULL, NULL,
                             Z, Un, NULL);
        if (st != ORC_OK) break;
        if (g_hist) g_hist[step] = g;
        if (g < eps || step >= max_steps) break;
        memcpy(U, Un, sizeof(double) * n * N);
        have_z = 1;
        step++;
    }
    if (st == ORC_OK && !(g < eps)) st = ORC_ERR_NOT_CONVERGED;
    *steps_out = step;
    *g_out = g;
    free(Z); free(Un);
    return st;
}

/* Algorithm 1 with the adaptive time step above (delta_T = tau_max).
 * tau_hist (max_steps entries or NULL) receives tau_0, tau_1, ...            */
int orc_solve_adaptive(int m, double lo, double hi, const double *V, double sigma, int N,
                       double tau_max, double c, double cg_rtol, int cg_maxit, double eps,
                       long max_steps, double *U, double *W, long *steps_out, double *g_out,
                       double *g_hist, double *tau_hist)
{
    long n = cube(m);
    if (!(c > 0.0 && c <= 1.0)) return ORC_ERR_ARG;
    double *Z = malloc(sizeof(double) * n * N), *Un = malloc(sizeof(double) * n * N);
    orc_adapt ad = {tau_max, c, 1.05, orc_lambda1_lower_bound(m, lo, hi, V, sigma), 0.0, 1};
    int have_z = 0, st = ORC_OK;
    long step = 0;
    double g = INFINITY, tau_used = 0.0;
    for (;;) {
        st = scheme_step_impl(m, lo, hi, V, sigma, N, tau_max, &ad, &tau_used, cg_rtol, cg_maxit,
                              U, have_z ? Z : NULL, NULL, W, NULL, &g, NULL, NULL, NULL, Z, Un,
                              NULL);
        if (st != ORC_OK) break;
        if (g_hist) g_hist[step] = g;
        if (g < eps || step >= max_steps) break;
        if (tau_hist) tau_hist[step] = tau_used;
        memcpy(U, Un, sizeof(double) * n * N);
        have_z = 1;
        step++;
    }
    if (st == ORC_OK && !(g < eps)) st = ORC_ERR_NOT_CONVERGED;
    *steps_out = step;
    *g_out = g;
    free(Z); free(Un);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Extraction.                                                               */
/* (a) the paper's eigenvalues (Section 5): lambda_i = eigenvalues of         */
/*     <G U, U>^{-1}, shifted back: lam_paper[i] = 1/mu_i - sigma with mu_i   */
/*     the eigenvalues of the symmetrised <W,U>, sorted ascending in lambda; */
/* (b) FP64 Rayleigh-Ritz with H (unshifted): K c = lambda S c, K = <U,HU>,  */
/*     S = <U,U>; Ritz vectors u_i = U c_i (so <u_i,u_j> = delta_ij) and     */
/*     residuals res[i] = || H u_i - lambda_i u_i ||.                         */
/* The sign of each Ritz vector is fixed so that its entry of largest        */
/* magnitude is positive.                                                    */
/* ------------------------------------------------------------------------ */
int orc_extract(int m, double lo, double hi, const double *V, double sigma, int N,
                const double *U, const double *W, double *lam_paper, double *lam_rr,
                double *evecs /* n x N or NULL */, double *res /* N or NULL */)
{
    long n = cube(m);
    double h = orc_grid_h(m, lo, hi), h3 = h * h * h;
    double *P = malloc(sizeof(double) * N * N), *mu = malloc(sizeof(double) * N);
    if (lam_paper) {
        orc_gram(n, N, W, N, U, h3, P);
        orc_sym_eig(N, P, mu, NULL);          /* ascending mu -> descending lambda */
        for (int i = 0; i < N; i++) lam_paper[i] = 1.0 / mu[N - 1 - i] - sigma;
    }
    double *HU = malloc(sizeof(double) * n * N), *K = malloc(sizeof(double) * N * N),
           *S = malloc(sizeof(double) * N * N), *L = malloc(sizeof(double) * N * N),
           *Cm = malloc(sizeof(double) * N * N), *T = malloc(sizeof(double) * N * N),
           *Y = malloc(sizeof(double) * N * N), *Cv = malloc(sizeof(double) * N * N);
    orc_apply_h(m, h, V, 0.0, N, U, HU);
    orc_gram(n, N, U, N, HU, h3, K);
    orc_gram(n, N, U, N, U, h3, S);
    memcpy(L, S, sizeof(double) * N * N);
    int st = cholesky(N, L);
    if (st != ORC_OK) goto out;
    /* T = L^{-1} K, Cm = T L^{-T}  (forward substitutions) */
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            double s = 0.5 * (K[i * N + j] + K[j * N + i]);
            for (int k = 0; k < i; k++) s -= L[i * N + k] * T[k * N + j];
            T[i * N + j] = s / L[i * N + i];
        }
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            double s = T[i * N + j];
            for (int k = 0; k < j; k++) s -= Cm[i * N + k] * L[j * N + k];
            Cm[i * N + j] = s / L[j * N + j];
        }
    double *lam = malloc(sizeof(double) * N);
    orc_sym_eig(N, Cm, lam, Y);
    /* c = L^{-T} y (back substitution) */
    for (int e = 0; e < N; e++)
        for (int i = N - 1; i >= 0; i--) {
            double s = Y[i * N + e];
            for (int k = i + 1; k < N; k++) s -= L[k * N + i] * Cv[k * N + e];
            Cv[i * N + e] = s / L[i * N + i];
        }
    if (lam_rr) memcpy(lam_rr, lam, sizeof(double) * N);
    if (evecs || res) {
        double *u = malloc(sizeof(double) * n * N), *hu = malloc(sizeof(double) * n * N);
        block_times_small(n, N, U, N, Cv, u);
        block_times_small(n, N, HU, N, Cv, hu);
        for (int e = 0; e < N; e++) {
            long arg = 0; double big = -1.0;
            for (long p = 0; p < n; p++) if (fabs(u[p * N + e]) > big) { big = fabs(u[p * N + e]); arg = p; }
            double sg = u[arg * N + e] < 0.0 ? -1.0 : 1.0;
            ksum k = {0.0, 0.0};
            for (long p = 0; p < n; p++) {
                double r = hu[p * N + e] - lam[e] * u[p * N + e];
                kadd(&k, r * r);
                u[p * N + e] *= sg;
            }
            if (res) res[e] = sqrt(h3 * kval(&k));
        }
        if (evecs) memcpy(evecs, u, sizeof(double) * n * N);
        free(u); free(hu);
    }
    free(lam);
out:
    free(P); free(mu); free(HU); free(K); free(S); free(L); free(Cm); free(T); free(Y); free(Cv);
    return st;
}

/* Energy E(U) = (1/2) (U,U)_a = (1/2) h^3 tr(U^T (H + shift) U)  (Section 2.2). */
double orc_energy(int m, double lo, double hi, const double *V, double shift, int N,
                  const double *U)
{
    long n = cube(m);
    double h = orc_grid_h(m, lo, hi), h3 = h * h * h;
    double *HU = malloc(sizeof(double) * n * N);
    orc_apply_h(m, h, V, shift, N, U, HU);
    ksum k = {0.0, 0.0};
    for (long i = 0; i < n * N; i++) kadd(&k, U[i] * HU[i]);
    free(HU);
    return 0.5 * h3 * kval(&k);
}

/* ------------------------------------------------------------------------ */
/* Differentiation through converged eigenpairs (not in the paper).         */
/* Input: eigenpairs (lam_i, u_i), i < N, of H = -Delta_h/2 + V with         */
/* <u_i,u_j> = h^3 u_i^T u_j = delta_ij, and lam_N < lam_{N+1}.              */
/*                                                                          */
/* Sum of eigenvalues: d lam_i / d V_p = <u_i, e_p u_i> = h^3 u_i(p)^2       */
/* (first-order perturbation of a simple eigenvalue), so                    */
/*   dV_p = h^3 sum_i w_i u_i(p)^2.                                         */
/*                                                                          */
/* Density loss: rho = sum_i u_i^2 (pointwise), L = (1/2) h^3 |rho - rho*|^2. */
/* A perturbation dV moves u_i by du_i = -(H - lam_i)^{-1} Q (dV u_i) with   */
/* Q = I - sum_j u_j <u_j, .> (components along the other occupied u_j      */
/* cancel in rho), and (H - lam_i) is SPD on range(Q).  With g = rho - rho*  */
/* dL = <g, d rho> = 2 sum_i <g u_i, du_i>, and the operator Q(H-lam_i)^{-1}Q */
/* is self-adjoint, so                                                      */
/*   dL/dV_p = -2 h^3 sum_i xi_i(p) u_i(p),  (H - lam_i) xi_i = Q (g u_i),  */
/* xi_i in range(Q), solved by CG with Q applied after every operator       */
/* application (the Krylov space stays in range(Q)).                        */
/* ------------------------------------------------------------------------ */
int orc_grad_eigs(int m, double lo, double hi, int N, const double *U, const double *w,
                  double *dV)
{
    long n = cube(m);
    double h = orc_grid_h(m, lo, hi), h3 = h * h * h;
    for (long p = 0; p < n; p++) {
        double s = 0.0;
        for (int i = 0; i < N; i++) s += (w ? w[i] : 1.0) * U[p * N + i] * U[p * N + i];
        dV[p] = h3 * s;
    }
    return ORC_OK;
}

/* x <- Q x = x - sum_j u_j h^3 (u_j^T x) for one column x */
static void project_out(long n, int N, double h3, const double *U, double *x)
{
    for (int j = 0; j < N; j++) {
        double s = 0.0;
        for (long p = 0; p < n; p++) s += U[p * N + j] * x[p];
        s *= h3;
        for (long p = 0; p < n; p++) x[p] -= s * U[p * N + j];
    }
}

int orc_grad_density(int m, double lo, double hi, const double *V, int N, const double *U,
                     const double *lam, const double *rho_target, double rtol, int maxit,
                     double *dV, double *loss, int *iters)
{
    long n = cube(m);
    double h = orc_grid_h(m, lo, hi), h3 = h * h * h;
    double *g = malloc(sizeof(double) * n);
    double *xi = calloc((size_t)n * N, sizeof(double));
    ksum L = {0.0, 0.0};
    for (long p = 0; p < n; p++) {
        double rho = 0.0;
        for (int i = 0; i < N; i++) rho += U[p * N + i] * U[p * N + i];
        g[p] = rho - rho_target[p];
        kadd(&L, g[p] * g[p]);
    }
    *loss = 0.5 * h3 * kval(&L);
    int status = ORC_OK, itmax = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < N; i++) {
        double *b = malloc(sizeof(double) * n), *x = calloc(n, sizeof(double));
        double *r = malloc(sizeof(double) * n), *pp = malloc(sizeof(double) * n),
               *q = malloc(sizeof(double) * n);
        for (long p = 0; p < n; p++) b[p] = g[p] * U[p * N + i];
        project_out(n, N, h3, U, b);
        /* CG on (H - lam_i) restricted to range(Q), x0 = 0 */
        double bn = sqrt(dot(n, b, b));
        for (long p = 0; p < n; p++) { r[p] = b[p]; pp[p] = b[p]; }
        double rr = dot(n, r, r);
        int st = (sqrt(rr) <= rtol * bn) ? ORC_OK : ORC_ERR_NOT_CONVERGED, it = 0;
        while (st != ORC_OK && it < maxit) {
            apply_col(m, h, V, -lam[i], pp, q);
            project_out(n, N, h3, U, q);
            double pq = dot(n, pp, q);
            if (!(pq > 0.0)) { st = ORC_ERR_BREAKDOWN; break; }
            double alpha = rr / pq;
            for (long p = 0; p < n; p++) { x[p] += alpha * pp[p]; r[p] -= alpha * q[p]; }
            double rr1 = dot(n, r, r);
            it++;
            if (sqrt(rr1) <= rtol * bn) { st = ORC_OK; break; }
            double beta = rr1 / rr;
            for (long p = 0; p < n; p++) pp[p] = r[p] + beta * pp[p];
            rr = rr1;
        }
        for (long p = 0; p < n; p++) xi[p * N + i] = x[p];
#pragma omp critical
        {
            if (st != ORC_OK && status == ORC_OK) status = st;
            if (it > itmax) itmax = it;
        }
        free(b); free(x); free(r); free(pp); free(q);
    }
    for (long p = 0; p < n; p++) {
        double s = 0.0;
        for (int i = 0; i < N; i++) s += xi[p * N + i] * U[p * N + i];
        dV[p] = -2.0 * h3 * s;
    }
    if (iters) *iters = itmax;
    free(g); free(xi);
    return status;
}

/* ------------------------------------------------------------------------ */
/* FP64 residual refinement of an approximate eigen-subspace (not in the    */
/* paper: the final refinement, in FP64, of a result computed in lower      */
/* precision).  One round, from the current U (n x N):                      */
/*   1. Rayleigh-Ritz on span(U): Ritz pairs (theta_i, u_i) of H with        */
/*      <u_i, u_j> = delta_ij (orc_extract);                                 */
/*   2. residuals r_i = H u_i - theta_i u_i, which are orthogonal to span(U) */
/*      by the Ritz conditions;                                             */
/*   3. corrections t_i in range(Q), Q = I - sum_j u_j <u_j, .>, from        */
/*        Q (H - theta_i) Q t_i = -r_i,                                     */
/*      by CG on range(Q) from t_i = 0 to ||res|| <= rtol ||r_i|| (Q applied */
/*      after every operator application).  This is Newton's equation for   */
/*      an invariant subspace written in the Ritz basis, where it decouples */
/*      into one equation per column; Q (H - theta_i) Q is positive definite */
/*      on range(Q) when every theta_i lies below the spectrum of H on the  */
/*      complement of span(U);                                              */
/*   4. U <- u + t.                                                          */
/* After `rounds` rounds a last Rayleigh-Ritz returns U = the Ritz vectors,  */
/* lam = the Ritz values (ascending) and res_i = ||H u_i - lam_i u_i||.      */
/* cg_iters (nullable) receives the largest CG count of each round.          */
/* ------------------------------------------------------------------------ */
int orc_refine(int m, double lo, double hi, const double *V, int N, double *U, int rounds,
               double rtol, int maxit, double *lam, double *res, int *cg_iters)
{
    long n = cube(m);
    double h = orc_grid_h(m, lo, hi), h3 = h * h * h;
    double *u = malloc(sizeof(double) * n * N);
    int status = ORC_OK;
    for (int k = 0; k < rounds && status == ORC_OK; k++) {
        status = orc_extract(m, lo, hi, V, 0.0, N, U, NULL, NULL, lam, u, NULL);
        if (status != ORC_OK) break;
        int itmax = 0;
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < N; i++) {
            double *ui = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n),
                   *t = calloc(n, sizeof(double)), *r = malloc(sizeof(double) * n),
                   *pp = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
            for (long p = 0; p < n; p++) ui[p] = u[p * N + i];
            apply_col(m, h, V, -lam[i], ui, b);          /* r_i = (H - theta_i) u_i */
            for (long p = 0; p < n; p++) b[p] = -b[p];
            project_out(n, N, h3, u, b);
            double bn = sqrt(dot(n, b, b));
            for (long p = 0; p < n; p++) { r[p] = b[p]; pp[p] = b[p]; }
            double rr = dot(n, r, r);
            int st = (sqrt(rr) <= rtol * bn) ? ORC_OK : ORC_ERR_NOT_CONVERGED, it = 0;
            while (st != ORC_OK && it < maxit) {
                apply_col(m, h, V, -lam[i], pp, q);
                project_out(n, N, h3, u, q);
                double pq = dot(n, pp, q);
                if (!(pq > 0.0)) { st = ORC_ERR_BREAKDOWN; break; }
                double alpha = rr / pq;
                for (long p = 0; p < n; p++) { t[p] += alpha * pp[p]; r[p] -= alpha * q[p]; }
                double rr1 = dot(n, r, r);
                it++;
                if (sqrt(rr1) <= rtol * bn) { st = ORC_OK; break; }
                double beta = rr1 / rr;
                for (long p = 0; p < n; p++) pp[p] = r[p] + beta * pp[p];
                rr = rr1;
            }
            for (long p = 0; p < n; p++) U[p * N + i] = ui[p] + t[p];
#pragma omp critical
            {
                if (st != ORC_OK && status == ORC_OK) status = st;
                if (it > itmax) itmax = it;
            }
            free(ui); free(b); free(t); free(r); free(pp); free(q);
        }
        if (cg_iters) cg_iters[k] = itmax;
    }
    if (status == ORC_OK) {
        status = orc_extract(m, lo, hi, V, 0.0, N, U, NULL, NULL, lam, u, res);
        if (status == ORC_OK) memcpy(U, u, sizeof(double) * n * N);
    }
    free(u);
    return status;
}

/* ------------------------------------------------------------------------ */
/* O'Leary's block preconditioned CG (not in the paper; an alternative inner */
/* solver for W = G U): all N columns share one block Krylov space, with    */
/* N x N step matrices instead of per-column scalars.                        */
/*   R = B - A X, Z = M R, P = Z                                             */
/*   repeat: Q = A P, alpha = (P^T Q)^{-1} (Z^T R), X += P alpha,            */
/*           R -= Q alpha, stop if every ||r_j|| <= rtol ||b_j||,            */
/*           Z' = M R, beta = (Z^T R)^{-1} (Z'^T R'), P = Z' + P beta.        */
/* P^T Q and Z^T R are symmetric positive definite while the block keeps full */
/* rank; their systems are solved by Cholesky (ORC_ERR_SINGULAR otherwise).  */
/* For N = 1 this is pcg_col.  rtol = 0 runs exactly maxit iterations.       */
/* ------------------------------------------------------------------------ */
static void apply_block(const orc_mg *mg, int N, const double *X, double *Y)
{
    orc_apply_h(mg->m[0], mg->h[0], mg->V[0], mg->sigma, N, X, Y);
}

/* C (N x N) = X^T Y, plain sums over the n points (the PCG's inner products) */
static void block_dot(long n, int N, const double *X, const double *Y, double *C)
{
    for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++) {
            double s = 0.0;
            for (long p = 0; p < n; p++) s += X[p * N + a] * Y[p * N + b];
            C[a * N + b] = s;
        }
}

/* S (N x N) <- A^{-1} S for SPD A (N x N), via its Cholesky factor L */
static int spd_solve_cols(int N, const double *A, double *S, double *L, double *tmp)
{
    memcpy(L, A, sizeof(double) * N * N);
    int st = cholesky(N, L);
    if (st != ORC_OK) return st;
    for (int c = 0; c < N; c++) {
        for (int i = 0; i < N; i++) tmp[i] = S[i * N + c];
        chol_solve(N, L, tmp, tmp + N);
        for (int i = 0; i < N; i++) S[i * N + c] = tmp[N + i];
    }
    return ORC_OK;
}

/* every column's residual within tolerance: ||r_c|| <= rtol ||b_c|| */
static int block_done(long n, int N, const double *R, double rtol, const double *bn)
{
    for (int c = 0; c < N; c++) {
        double s = 0.0;
        for (long p = 0; p < n; p++) s += R[p * N + c] * R[p * N + c];
        if (!(sqrt(s) <= rtol * bn[c])) return 0;
    }
    return 1;
}

int orc_block_pcg_mg(const orc_mg *mg, int N, const double *B, double *X, double rtol,
                     int maxit, int *iters)
{
    long n = cube(mg->m[0]);
    size_t blk = sizeof(double) * n * N, sq = sizeof(double) * N * N;
    double *R = malloc(blk), *Z = malloc(blk), *P = malloc(blk), *Q = malloc(blk), *T = malloc(blk);
    double *PQ = malloc(sq), *ZR = malloc(sq), *ZR1 = malloc(sq), *al = malloc(sq),
           *be = malloc(sq), *L = malloc(sq), *tmp = malloc(sizeof(double) * 2 * N);
    double *bn = malloc(sizeof(double) * N);
    int st = ORC_ERR_NOT_CONVERGED, it = 0;
    apply_block(mg, N, X, Q);
    for (long i = 0; i < n * N; i++) R[i] = B[i] - Q[i];
    for (int c = 0; c < N; c++) {
        double s = 0.0;
        for (long p = 0; p < n; p++) s += B[p * N + c] * B[p * N + c];
        bn[c] = sqrt(s);
    }
    if (rtol > 0.0 && block_done(n, N, R, rtol, bn)) st = ORC_OK;
    if (st != ORC_OK) {
        orc_mg_vcycle(mg, N, R, Z);
        memcpy(P, Z, blk);
        block_dot(n, N, Z, R, ZR);
    }
    while (st != ORC_OK && it < maxit) {
        apply_block(mg, N, P, Q);
        block_dot(n, N, P, Q, PQ);
        memcpy(al, ZR, sq);
        if (spd_solve_cols(N, PQ, al, L, tmp) != ORC_OK) { st = ORC_ERR_BREAKDOWN; break; }
        for (long p = 0; p < n; p++)
            for (int j = 0; j < N; j++) {
                double sx = 0.0, sr = 0.0;
                for (int k = 0; k < N; k++) {
                    sx += P[p * N + k] * al[k * N + j];
                    sr += Q[p * N + k] * al[k * N + j];
                }
                X[p * N + j] += sx;
                R[p * N + j] -= sr;
            }
        it++;
        if (rtol > 0.0 && block_done(n, N, R, rtol, bn)) { st = ORC_OK; break; }
        orc_mg_vcycle(mg, N, R, Z);
        block_dot(n, N, Z, R, ZR1);
        memcpy(be, ZR1, sq);
        if (spd_solve_cols(N, ZR, be, L, tmp) != ORC_OK) { st = ORC_ERR_BREAKDOWN; break; }
        for (long p = 0; p < n; p++)
            for (int j = 0; j < N; j++) {
                double s = 0.0;
                for (int k = 0; k < N; k++) s += P[p * N + k] * be[k * N + j];
                T[p * N + j] = Z[p * N + j] + s;
            }
        memcpy(P, T, blk);
        memcpy(ZR, ZR1, sq);
    }
    if (rtol == 0.0 && st == ORC_ERR_NOT_CONVERGED && it == maxit) st = ORC_OK;
    if (iters) *iters = it;
    free(R); free(Z); free(P); free(Q); free(T); free(PQ); free(ZR); free(ZR1); free(al);
    free(be); free(L); free(tmp); free(bn);
    return st;
}
