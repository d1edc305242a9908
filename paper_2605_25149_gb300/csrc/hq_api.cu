// libhq: host orchestration and the C ABI declared in include/hq.h.
//
// One step of the scheme Eq. (4.1) (Wang & Zhou, arXiv 2605.25149):
//   A1  W = G U_n                   block PCG with a multigrid V-cycle
//   A2  G2 = <[U W], [U W]>         split-K Gram, fixed-order reduction
//   A3  g = || W - U <W,U> ||        Grassmann gradient (Remark 3.1), the
//                                   quantity Algorithm 1 tests
//   B1  [X; Y] from the 2N x 2N predictor system (LU, partial pivoting)
//   B2  Uh = U (I - tau Y) + W (tau X)
//   B3  Shat = <Uh,Uh> = C^T G2 C    (C = [I - tau Y; tau X]: the Gram of Uh
//                                   by bilinearity, no extra pass over Uh)
//   B4  Z = G Uh                    second block PCG
//   B5  U_{n+1} = Uh - tau Z (Shat - I)
// Every step runs on the caller's stream inside the caller's workspace; the
// host reads back one scalar per PCG iteration (number of active columns) and
// one per step (g) and never allocates device memory after hq_init.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hq.h"
#include "hq_internal.cuh"

using namespace hq;

namespace {

constexpr int MAXLEV = 24;

struct Level {
    int m = 0;
    long n = 0;
    double h = 0, c = 0;
    double *V = nullptr, *D = nullptr, *wD = nullptr;   // FP64
    void *Dt = nullptr, *wDt = nullptr;                 // working precision
    // FP64 V-cycle (FP64 contexts): wD c per point and the pre-scaled
    // right-hand side rt = wD r of the level (the first sweep from zero)
    double *wcD = nullptr;
    void *rt = nullptr;
    void *r = nullptr, *z = nullptr, *t = nullptr;      // level buffers (l >= 1)
    XferTab tab{};                                       // transfer tables to level l + 1
    GridGeom g;
};

}  // namespace

namespace {
constexpr int MAXGRAPH = 4;
// a captured PCG loop (conditional WHILE node) for one solution block
struct PcgGraph {
    const void *X = nullptr;
    double rtol = 0.0;
    int maxit = 0;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    long body_launches[HQ_K_NCLASS] = {};
    bool ok = false;
};
}  // namespace

// a captured phase of the scheme (A: W = G U, Gram, g; B: predictor,
// updates, Z = G Uh, corrector) with its PCG loop as a conditional WHILE node
struct StepGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = false, tried = false;
    long fixed[HQ_K_NCLASS] = {};   // launches outside the PCG loop
    long part1[HQ_K_NCLASS] = {};   // per loop iteration
    long part2[HQ_K_NCLASS] = {};   // per executed IF body (V-cycle, beta, p)
    long launches = 0;              // graph launches not yet folded into the counters
    long long seen[2] = {0, 0};     // device counters already folded
};

struct hq_ctx {
    hq_config cfg;
    bool mixed = false;
    size_t esz = 8;
    int m = 0, N = 0;
    long n = 0;
    double h = 0, h3 = 0, sigma = 0;
    cudaStream_t st = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    int L = 0;
    Level lev[MAXLEV];
    long nc = 0;
    double *Acoarse = nullptr, *Ainv = nullptr;
    void *xt1 = nullptr, *xt2 = nullptr;   // transfer-pass scratch
    // the V-cycle's view of the levels: lev itself, or (mg32: an FP64 context
    // with an FP32 preconditioner) FP32 copies of D, omega/D, level buffers,
    // geometries and transfer scratch
    Level mg[MAXLEV];
    void *mxt1 = nullptr, *mxt2 = nullptr;
    bool mg32 = false;
    // FP64 V-cycle smoothing from the pre-scaled right-hand side (Level::rt)
    bool rtilde = false;
    // FP32 V-cycles: levels fuse_l0 .. L-1 run as one launch (k_vcoarse); -1: off.
    // no_fuse: set while a batch graph of several problems is captured (their
    // separate small kernels interleave better across concurrent problems)
    int fuse_l0 = -1;
    bool no_fuse = false;
    // whether level 0 of an FP32 V-cycle fits one launch, whatever
    // HQ_FUSED_COARSE says (selects the FP64 <-> FP32 interface of mg_fp32,
    // so the switch leaves every value unchanged)
    bool level0_fits = false;
    float *R32 = nullptr, *Z32 = nullptr, *T32 = nullptr;
    // n x N blocks in the working precision
    void *U = nullptr, *W = nullptr, *Uh = nullptr, *Z = nullptr;
    void *R = nullptr, *Zp = nullptr, *P = nullptr, *Q = nullptr, *Tt = nullptr;
    // FP64 n x N blocks for extraction / staging (aliases in FP64 mode)
    double *E1 = nullptr, *E2 = nullptr, *E3 = nullptr;
    PcgScalars sc;
    double *part = nullptr, *part2 = nullptr;
    GramPlan gplan_uw, gplan_max;
    double *gpart = nullptr;
    float *tcpart = nullptr;   // tensor-core Gram partials (HQ_MIXED)
    unsigned char *tcimg = nullptr;   // split small matrix of the tensor-core block products
    TallPlan tplan;
    double *tpart = nullptr;   // gy x N
    double *G2 = nullptr, *Mw = nullptr, *XY = nullptr, *C = nullptr, *T1 = nullptr;
    double *Shat = nullptr, *Om = nullptr, *Msm = nullptr, *Ksm = nullptr, *Ssm = nullptr;
    double *Lm = nullptr, *Cm = nullptr, *Ym = nullptr, *Cv = nullptr, *Cv2 = nullptr;
    double *eigwork = nullptr, *evals = nullptr, *mu = nullptr, *lam_p = nullptr;
    double *lam_r = nullptr, *resn = nullptr, *scal = nullptr, *signwork = nullptr;
    int *status = nullptr;
    int *ipiv = nullptr;   // pivots of the small eliminations (2N)
    float *lu32 = nullptr;  // FP32 factors of the small systems (mixed precision)
    unsigned char *ozimg = nullptr;   // FP64 tensor-core block products: digit planes
    double *ozgram = nullptr;         // FP64 tensor-core Gram: chunk partials, exponents
    double *pB = nullptr, *pR = nullptr;   // predictor right-hand side / residual
    // the warm-start solve's own FP32 factors, pivots and residual: it runs
    // on `side`, beside the predictor system (fork / join by the two events)
    int *ipivw = nullptr;
    float *lu32w = nullptr;
    double *pRw = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t evside[2] = {nullptr, nullptr};
    double *vn[3] = {nullptr, nullptr, nullptr};   // FP64 n-vectors (density, adjoint)
    double *pvec = nullptr;                        // power-iteration vector (N)
    // host state
    bool have_V = false, have_U = false, w_valid = false, z_valid = false;
    long step = 0;
    double last_g = NAN;
    double lambda1_lb = 0.0;   // closed-form lower bound of lambda_1(H + sigma)
    std::string err;
    // instrumentation
    long launches[HQ_K_NCLASS] = {};
    double work[HQ_K_NCLASS] = {};
    long stat_solves = 0, stat_iters = 0;
    bool timing = false;
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    std::vector<std::pair<int, size_t>> evrec;
    size_t pending_start = 0;
    // captured PCG loops
    bool use_graphs = true, capturing = false;
    long *cap_counts = nullptr;
    PcgGraph pgraph[MAXGRAPH];
    int npgraph = 0;
    cudaStream_t cap = nullptr;
    // whole-phase graphs
    StepGraph sg[2];
    cudaStream_t capA = nullptr, capB = nullptr, capC = nullptr, capD = nullptr;
    // device words: [0..3] PCG loop counters of the phase graphs, [4..7] the
    // same in batch graphs, [8..16] the batch time-loop state (BS_*)
    long long *dcount = nullptr;
    // batched form: launch counts of the phases as captured in a batch graph
    StepGraph bsg[2];
    long long bseen[4] = {0, 0, 0, 0};
    int gen = 0;   // incremented whenever the captured graphs are dropped
    // hq_solve's device-side time loop: a one-member batch graph on this
    // context's stream (created at the first graph-replayed hq_solve; freed by
    // hq_destroy); solo_failed: its capture failed, use the host loop
    hq_batch *solo = nullptr;
    bool solo_failed = false;
    ~hq_ctx() {
        for (cudaEvent_t e : evpool) cudaEventDestroy(e);
        for (int i = 0; i < npgraph; i++) {
            if (pgraph[i].exec) cudaGraphExecDestroy(pgraph[i].exec);
            if (pgraph[i].g) cudaGraphDestroy(pgraph[i].g);
        }
        if (cap) cudaStreamDestroy(cap);
        for (int i = 0; i < 2; i++) {
            if (sg[i].exec) cudaGraphExecDestroy(sg[i].exec);
            if (sg[i].g) cudaGraphDestroy(sg[i].g);
        }
        if (capA) cudaStreamDestroy(capA);
        if (capB) cudaStreamDestroy(capB);
        if (capC) cudaStreamDestroy(capC);
        if (capD) cudaStreamDestroy(capD);
        if (side) cudaStreamDestroy(side);
        for (cudaEvent_t e : evside)
            if (e) cudaEventDestroy(e);
    }
};

namespace hq {
namespace {
thread_local hq_ctx *g_prof = nullptr;
thread_local int g_level = 0;   // multigrid level of the launches being issued
}
void hook_before(int cls) {
    (void)cls;
    hq_ctx *x = g_prof;
    if (!x || !x->timing || x->capturing) return;
    while (x->evpool.size() < x->evused + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        x->evpool.push_back(e);
    }
    x->pending_start = x->evused;
    cudaEventRecord(x->evpool[x->evused], x->st);
    x->evused += 2;
}
void hook_after(int cls, double work) {
    hq_ctx *x = g_prof;
    if (!x) return;
    if (g_level > 0 && (cls == HQ_K_STENCIL || cls == HQ_K_RESIDUAL || cls == HQ_K_SMOOTH ||
                        cls == HQ_K_TRANSFER || cls == HQ_K_VECTOR))
        cls = HQ_K_COARSE_GRIDS;
    if (x->capturing) {
        if (x->cap_counts && cls >= 0 && cls < HQ_K_NCLASS) x->cap_counts[cls]++;
        return;
    }
    if (cls >= 0 && cls < HQ_K_NCLASS) {
        x->launches[cls]++;
        x->work[cls] += work;
    }
    if (!x->timing || x->evused < 2) return;
    cudaEventRecord(x->evpool[x->pending_start + 1], x->st);
    x->evrec.emplace_back(cls, x->pending_start);
}
}  // namespace hq

namespace {
// tags the launches issued in its lifetime with a multigrid level
struct LevelScope {
    int prev;
    explicit LevelScope(int l) : prev(hq::g_level) { hq::g_level = l; }
    ~LevelScope() { hq::g_level = prev; }
};

// binds the instrumentation hooks to a context for the duration of a call
struct ProfScope {
    hq_ctx *prev;
    explicit ProfScope(hq_ctx *x) : prev(hq::g_prof) { hq::g_prof = x; }
    ~ProfScope() { hq::g_prof = prev; }
};
}  // namespace

namespace {

// ---------------------------------------------------------------------------
// workspace carving (identical in the sizing pass and the real pass)
// ---------------------------------------------------------------------------
struct Carver {
    char *base;
    size_t off = 0;
    template <typename P>
    P *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        P *p = base ? reinterpret_cast<P *>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

bool valid_config(const hq_config *c, std::string *why) {
    auto fail = [&](const char *s) {
        if (why) *why = s;
        return false;
    };
    if (!c) return fail("null config");
    if (c->m < 3) return fail("m must be >= 3");
    if (c->m > 1024) return fail("m must be <= 1024");
    long n = (long)c->m * c->m * c->m;
    if (c->nev < 1 || c->nev > 512 || c->nev > n) return fail("nev must satisfy 1 <= N <= min(n, 512)");
    if (!(c->hi > c->lo)) return fail("box: hi must exceed lo");
    if (!(c->tau > 0.0) || !std::isfinite(c->tau)) return fail("tau must be positive and finite");
    if (c->precision != HQ_FP64 && c->precision != HQ_MIXED) return fail("unknown precision");
    if (!(c->cg_rtol >= 0.0)) return fail("cg_rtol must be >= 0");
    if (c->cg_maxit < 1) return fail("cg_maxit must be >= 1");
    if (c->mg_nu1 < 1 || c->mg_nu2 < 1 || c->mg_nu1 > 16 || c->mg_nu2 > 16)
        return fail("mg_nu1, mg_nu2 must be in [1, 16]");
    if (c->mg_coarsest < 1 || c->mg_coarsest > 4) return fail("mg_coarsest must be in [1, 4]");
    if (!(c->mg_omega > 0.0 && c->mg_omega < 2.0)) return fail("mg_omega must be in (0, 2)");
    if (c->grid_block != 0 && c->grid_block != 64 && c->grid_block != 128 && c->grid_block != 256)
        return fail("grid_block must be 0, 64, 128 or 256");
    if (c->grid_ctas < 0 || c->grid_ctas > 64) return fail("grid_ctas must be in [0, 64]");
    if (c->fp64_tc < 0 || c->fp64_tc > 2) return fail("fp64_tc must be 0, 1 or 2");
    if (c->mg_fp32 != 0 && c->mg_fp32 != 1) return fail("mg_fp32 must be 0 or 1");
    if (!(c->tau_safety > 0.0 && c->tau_safety <= 1.0)) return fail("tau_safety must be in (0, 1]");
    return true;
}

int level_sizes(int m, int coarsest, int *ms) {
    int L = 0;
    ms[L++] = m;
    while (ms[L - 1] > coarsest && ms[L - 1] >= 2 && L < MAXLEV) {
        ms[L] = ms[L - 1] / 2;
        L++;
    }
    return L;
}

// z-marching CTAs for a finest level whose block reaches 100 MB (beyond
// about three quarters of L2); HQ_ZMARCH=1 / 0 forces them on / off
void zmarch_rule(GridGeom &g, double block_bytes) {
    const char *zm = std::getenv("HQ_ZMARCH");
    const bool force = zm && zm[0] == '1', off = zm && zm[0] == '0';
    if (!off && (force || block_bytes >= 100e6)) enable_zmarch(g);
}

size_t carve(hq_ctx *x, const hq_config *c, char *base) {
    Carver cv{base};
    const int m = c->m, N = c->nev;
    const long n = (long)m * m * m;
    const bool mixed = c->precision == HQ_MIXED;
    const size_t esz = mixed ? 4 : 8;
    const size_t blk = (size_t)n * N * esz;
    int ms[MAXLEV];
    const int L = level_sizes(m, c->mg_coarsest, ms);
    void *U = cv.take<char>(blk), *W = cv.take<char>(blk), *Uh = cv.take<char>(blk),
         *Z = cv.take<char>(blk), *R = cv.take<char>(blk), *Zp = cv.take<char>(blk),
         *P = cv.take<char>(blk), *Q = cv.take<char>(blk), *Tt = cv.take<char>(blk);
    double *E1, *E2, *E3;
    if (mixed) {
        E1 = cv.take<double>(sizeof(double) * n * N);
        E2 = cv.take<double>(sizeof(double) * n * N);
        E3 = cv.take<double>(sizeof(double) * n * N);
    } else {
        E1 = (double *)Q;
        E2 = (double *)Tt;
        E3 = (double *)Uh;
    }
    Level lev[MAXLEV];
    for (int l = 0; l < L; l++) {
        Level &v = lev[l];
        v.m = ms[l];
        v.n = (long)ms[l] * ms[l] * ms[l];
        v.h = (c->hi - c->lo) / (ms[l] + 1);
        v.c = 0.5 / (v.h * v.h);
        v.g = make_geom(ms[l], N, (int)esz, c->grid_block, c->grid_ctas);
        // finest-level blocks of 100 MB or more: z-marching smoothing sweeps
        // (HQ_ZMARCH=0 keeps the linear point order, HQ_ZMARCH=1 forces the
        // z-marching order at any size; both for comparisons)
        if (l == 0 && L > 1) zmarch_rule(v.g, (double)v.n * N * esz);
        v.V = cv.take<double>(sizeof(double) * v.n);
        v.D = cv.take<double>(sizeof(double) * v.n);
        v.wD = cv.take<double>(sizeof(double) * v.n);
        if (!mixed && !c->mg_fp32 && l + 1 < L) {
            v.wcD = cv.take<double>(sizeof(double) * v.n);
            v.rt = cv.take<char>((size_t)v.n * N * esz);
        }
        if (mixed) {
            v.Dt = cv.take<float>(sizeof(float) * v.n);
            v.wDt = cv.take<float>(sizeof(float) * v.n);
        } else {
            v.Dt = v.D;
            v.wDt = v.wD;
        }
        if (l > 0) {
            size_t lb = (size_t)v.n * N * esz;
            v.r = cv.take<char>(lb);
            v.z = cv.take<char>(lb);
            v.t = cv.take<char>(lb);
        } else {
            v.r = R;
            v.z = Zp;
            v.t = Tt;
        }
    }
    for (int l = 0; l + 1 < L; l++) {
        const int mc = ms[l + 1], mf = ms[l];
        lev[l].tab.ridx = cv.take<int>(sizeof(int) * mc * XFER_RTAPS);
        lev[l].tab.rw = cv.take<double>(sizeof(double) * mc * XFER_RTAPS);
        lev[l].tab.rwf = cv.take<float>(sizeof(float) * mc * XFER_RTAPS);
        lev[l].tab.pidx = cv.take<int>(sizeof(int) * mf * 2);
        lev[l].tab.pw = cv.take<double>(sizeof(double) * mf * 2);
        lev[l].tab.pwf = cv.take<float>(sizeof(float) * mf * 2);
    }
    // scratch of the separable transfers: (mf^2 mc + mf mc^2) x N elements on the finest level
    const size_t xs = (L > 1) ? (size_t)ms[0] * ms[0] * ms[1] : 1;
    const size_t xs2 = (L > 1) ? (size_t)ms[0] * ms[1] * ms[1] : 1;
    void *xt1 = cv.take<char>(xs * N * esz);
    void *xt2 = cv.take<char>(xs2 * N * esz);
    // FP32 preconditioner of an FP64 context: FP32 level copies and buffers
    const bool mg32 = !mixed && c->mg_fp32;
    Level mgv[MAXLEV];
    void *mxt1 = xt1, *mxt2 = xt2;
    float *R32 = nullptr, *Z32 = nullptr, *T32 = nullptr;
    for (int l = 0; l < L; l++) mgv[l] = lev[l];
    if (mg32) {
        R32 = cv.take<float>(sizeof(float) * n * N);
        Z32 = cv.take<float>(sizeof(float) * n * N);
        T32 = cv.take<float>(sizeof(float) * n * N);
        for (int l = 0; l < L; l++) {
            Level &w = mgv[l];
            w.g = make_geom(ms[l], N, 4, c->grid_block, c->grid_ctas);
            if (l == 0 && L > 1) zmarch_rule(w.g, (double)w.n * N * 4);
            w.Dt = cv.take<float>(sizeof(float) * w.n);
            w.wDt = cv.take<float>(sizeof(float) * w.n);
            if (l > 0) {
                w.r = cv.take<float>(sizeof(float) * w.n * N);
                w.z = cv.take<float>(sizeof(float) * w.n * N);
                w.t = cv.take<float>(sizeof(float) * w.n * N);
            } else {
                w.r = R32;
                w.z = Z32;
                w.t = T32;
            }
        }
        mxt1 = cv.take<float>(sizeof(float) * xs * N);
        mxt2 = cv.take<float>(sizeof(float) * xs2 * N);
    }
    const long nc = lev[L - 1].n;
    double *Acoarse = cv.take<double>(sizeof(double) * nc * nc);
    double *Ainv = cv.take<double>(sizeof(double) * nc * nc);
    PcgScalars sc;
    sc.rz = cv.take<double>(sizeof(double) * N);
    sc.alpha = cv.take<double>(sizeof(double) * N);
    sc.beta = cv.take<double>(sizeof(double) * N);
    sc.bnorm = cv.take<double>(sizeof(double) * N);
    sc.rnorm = cv.take<double>(sizeof(double) * N);
    sc.active = cv.take<int>(sizeof(int) * N);
    sc.iters = cv.take<int>(sizeof(int) * N);
    sc.num_active = cv.take<int>(sizeof(int) * 4);
    sc.status = cv.take<int>(sizeof(int) * 4);
    // partial rows: the working-precision geometry of the finest level, or the
    // FP64 geometry used by the FP64 extraction / monitoring kernels
    int gy0 = std::max(std::max(lev[0].g.gy, part_rows(lev[0].g)), make_geom(m, N, 8).gy);
    if (!mixed && c->mg_fp32) {
        GridGeom g32 = make_geom(m, N, 4, c->grid_block, c->grid_ctas);
        gy0 = std::max(gy0, std::max(g32.gy, part_rows(g32)));
    }
    double *part = cv.take<double>(sizeof(double) * (size_t)gy0 * N);
    double *part2 = cv.take<double>(sizeof(double) * (size_t)gy0 * N);
    sc.fpart = cv.take<double>(sizeof(double) * 2 * (size_t)finalize_chunks(gy0) * N);
    sc.fcount = cv.take<unsigned>(sizeof(unsigned) * 16);
    float *tcpart = mixed ? cv.take<float>(gram_tc_partial_bytes(n, 2 * N)) : nullptr;
    unsigned char *tcimg = mixed ? cv.take<unsigned char>(tall_tc_image_bytes(N, N, N)) : nullptr;
    GramPlan guw = make_gram_plan(n, 2 * N, 2 * N, true);
    GramPlan gmax = make_gram_plan(n, 2 * N, 2 * N, false);
    double *gpart = cv.take<double>(std::max(gram_partial_bytes(guw), gram_partial_bytes(gmax)));
    TallPlan tp = make_tall_plan(n, N, 2 * N, 0);
    const size_t tparts = std::max((size_t)tp.gy * std::max(N, tp.gx),
                                   mixed ? (size_t)tall_tc_partials(n, N) : (size_t)0);
    double *tpart = cv.take<double>(sizeof(double) * tparts);
    const size_t N2 = (size_t)N * N;
    double *G2 = cv.take<double>(sizeof(double) * 4 * N2);
    double *Mw = cv.take<double>(sizeof(double) * 4 * N2);
    double *XY = cv.take<double>(sizeof(double) * 2 * N2);
    int *ipiv = cv.take<int>(sizeof(int) * 2 * N);
    // the predictor system by FP32 elimination and FP64 refinement (both
    // precisions): FP32 factors and FP64 right-hand side / residual
    float *lu32 = cv.take<float>(sizeof(float) * 4 * N2);
    // digit planes of the small matrices of the FP64 tensor-core block products
    unsigned char *ozimg = (!mixed && c->fp64_tc && tall_oz_supported(2 * N, 0))
                               ? cv.take<unsigned char>(tall_oz_image_bytes(n, 2 * N, N))
                               : nullptr;
    double *ozgram = (!mixed && c->fp64_tc && gram_oz_supported(2 * N))
                         ? cv.take<double>(gram_oz_scratch_bytes(n, 2 * N))
                         : nullptr;
    double *pB = cv.take<double>(sizeof(double) * 2 * N2);
    double *pR = cv.take<double>(sizeof(double) * 2 * N2);
    int *ipivw = cv.take<int>(sizeof(int) * N);
    float *lu32w = cv.take<float>(sizeof(float) * N2);
    double *pRw = cv.take<double>(sizeof(double) * N2);
    double *Cc = cv.take<double>(sizeof(double) * 2 * N2);
    double *T1 = cv.take<double>(sizeof(double) * 2 * N2);
    double *Shat = cv.take<double>(sizeof(double) * N2);
    double *Om = cv.take<double>(sizeof(double) * N2);
    double *Msm = cv.take<double>(sizeof(double) * N2);
    double *Ksm = cv.take<double>(sizeof(double) * N2);
    double *Ssm = cv.take<double>(sizeof(double) * N2);
    double *Lm = cv.take<double>(sizeof(double) * N2);
    double *Cm = cv.take<double>(sizeof(double) * N2);
    double *Ym = cv.take<double>(sizeof(double) * N2);
    double *Cvv = cv.take<double>(sizeof(double) * N2);
    double *Cv2 = cv.take<double>(sizeof(double) * N2);
    const size_t P2 = (size_t)((N + 1) & ~1) * ((N + 1) & ~1);
    double *eigwork = cv.take<double>(sizeof(double) * 2 * P2);
    double *evals = cv.take<double>(sizeof(double) * N);
    double *mu = cv.take<double>(sizeof(double) * N);
    double *lam_p = cv.take<double>(sizeof(double) * N);
    double *lam_r = cv.take<double>(sizeof(double) * N);
    double *resn = cv.take<double>(sizeof(double) * N);
    double *scal = cv.take<double>(sizeof(double) * 16);
    double *signwork = cv.take<double>(sizeof(double) * 2 * 64 * N);
    int *status = cv.take<int>(sizeof(int) * 4);
    double *vn0 = cv.take<double>(sizeof(double) * n);
    double *vn1 = cv.take<double>(sizeof(double) * n);
    double *vn2 = cv.take<double>(sizeof(double) * n);
    double *pvec = cv.take<double>(sizeof(double) * N);
    long long *dcount = cv.take<long long>(sizeof(long long) * 24);
    if (x) {
        x->pvec = pvec;
        x->dcount = dcount;
        x->vn[0] = vn0; x->vn[1] = vn1; x->vn[2] = vn2;
        x->U = U; x->W = W; x->Uh = Uh; x->Z = Z; x->R = R; x->Zp = Zp; x->P = P; x->Q = Q;
        x->Tt = Tt; x->E1 = E1; x->E2 = E2; x->E3 = E3;
        x->L = L;
        for (int l = 0; l < L; l++) x->lev[l] = lev[l];
        x->nc = nc; x->Acoarse = Acoarse; x->Ainv = Ainv; x->xt1 = xt1; x->xt2 = xt2;
        for (int l = 0; l < L; l++) x->mg[l] = mgv[l];
        x->mxt1 = mxt1; x->mxt2 = mxt2; x->mg32 = mg32;
        x->rtilde = !mixed && !mg32 && L > 1;
        x->R32 = R32; x->Z32 = Z32; x->T32 = T32;
        x->sc = sc; x->part = part; x->part2 = part2;
        x->gplan_uw = guw; x->gplan_max = gmax; x->gpart = gpart; x->tcpart = tcpart; x->tcimg = tcimg;
        x->tplan = tp; x->tpart = tpart;
        x->ipiv = ipiv;
        x->lu32 = lu32;
        x->ozimg = ozimg;
        x->ozgram = ozgram;
        x->pB = pB;
        x->pR = pR;
        x->ipivw = ipivw;
        x->lu32w = lu32w;
        x->pRw = pRw;
        x->G2 = G2; x->Mw = Mw; x->XY = XY; x->C = Cc; x->T1 = T1; x->Shat = Shat; x->Om = Om;
        x->Msm = Msm; x->Ksm = Ksm; x->Ssm = Ssm; x->Lm = Lm; x->Cm = Cm; x->Ym = Ym;
        x->Cv = Cvv; x->Cv2 = Cv2; x->eigwork = eigwork; x->evals = evals; x->mu = mu;
        x->lam_p = lam_p; x->lam_r = lam_r; x->resn = resn; x->scal = scal;
        x->signwork = signwork; x->status = status;
    }
    return cv.off + 256;
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define HQ_CUDA(call)                                                          \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            x->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return HQ_ERR_CUDA;                                                \
        }                                                                      \
    } while (0)

#define HQ_TRY(expr)                    \
    do {                                \
        hq_status s_ = (expr);          \
        if (s_ != HQ_OK) return s_;     \
    } while (0)

hq_status fail(hq_ctx *x, hq_status s, const std::string &msg) {
    if (x) x->err = msg;
    return s;
}

hq_status check_launch(hq_ctx *x) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(x, HQ_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return HQ_OK;
}

hq_status sync_status(hq_ctx *x, int *dev_status_word, const char *where) {
    int st = 0;
    HQ_CUDA(cudaMemcpyAsync(&st, dev_status_word, sizeof(int), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    HQ_TRY(check_launch(x));
    if (st & ST_BREAKDOWN) return fail(x, HQ_ERR_BREAKDOWN, std::string(where) + ": CG breakdown (p^T A p <= 0)");
    if (st & ST_SINGULAR) return fail(x, HQ_ERR_SINGULAR, std::string(where) + ": singular small system");
    if (st & ST_NONFINITE) return fail(x, HQ_ERR_NONFINITE, std::string(where) + ": non-finite value");
    if (st & ST_GJ_FAIL) return fail(x, HQ_ERR_ARG, std::string(where) + ": coarsest operator not positive definite (shift too small)");
    if (st & ST_TC_TIMEOUT) return fail(x, HQ_ERR_TIMEOUT, std::string(where) + ": tensor-core wait expired");
    if (st & ST_PCG_MAXIT) return fail(x, HQ_ERR_NOT_CONVERGED, std::string(where) + ": inner PCG reached cg_maxit");
    return HQ_OK;
}

hq_status clear_status(hq_ctx *x) {
    HQ_CUDA(cudaMemsetAsync(x->sc.status, 0, sizeof(int), x->st));
    HQ_CUDA(cudaMemsetAsync(x->status, 0, sizeof(int), x->st));
    return HQ_OK;
}

// copy of an n x N block, count elements
template <typename T>
hq_status copy_blk(hq_ctx *x, T *dst, const T *src, size_t count) {
    if (dst != src) HQ_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToDevice, x->st));
    return HQ_OK;
}

// ---------------------------------------------------------------------------
// multigrid V-cycle
// ---------------------------------------------------------------------------
int cycle_writes(const hq_ctx *x) { return (x->cfg.mg_nu1 - 1) + 1 + x->cfg.mg_nu2; }

template <typename T>
T *first_target(hq_ctx *x, int l, T *Zfinal, T *Tbuf) {
    (void)l;
    return (cycle_writes(x) % 2 == 0) ? Zfinal : Tbuf;
}

template <typename T>
hq_status vcycle(hq_ctx *x, int l, const T *r, T *Zf, T *Tb, bool first_done, double *part_final,
                 const double *r64dot = nullptr);

// The FP64 V-cycle of level l with the smoothing sweeps from the pre-scaled
// right-hand side rt = wD r (launch_jacobi_rt): the first sweep from zero is
// rt itself (written by launch_jacobi_first, or by the PCG update when
// first_done), so the sweeps read rt instead of r and form
// wc nbrsum(z) + ((1 - omega) z + rt); rt stays untouched for the post
// sweeps.  Iterates and the residual alternate between Zf and Tb, starting
// so that the last write lands in Zf (no copy).
hq_status vcycle_rt(hq_ctx *x, int l, const double *r, double *Zf, double *Tb, bool first_done,
                    double *part_final) {
    Level &v = x->mg[l];
    const double c = v.c, omw = 1.0 - x->cfg.mg_omega;
    double *rt = (double *)v.rt;
    if (!first_done) launch_jacobi_first<double>(v.g, v.wD, r, rt, x->st);
    // writes after the first sweep: nu1 - 1 pre sweeps, the residual, the
    // prolongation (into the residual's buffer), nu2 post sweeps
    const int nu1 = x->cfg.mg_nu1, nu2 = x->cfg.mg_nu2;
    auto final_is_first = [&]() {
        // simulate with the first written buffer labelled 0
        int cur = -1, k = 0;
        auto next = [&](int c0) { return c0 < 0 ? 0 : 1 - c0; };
        for (int s = 1; s < nu1; s++) cur = next(cur);
        k = next(cur);   // residual buffer, the prolongation writes into it
        cur = k;
        for (int s = 0; s < nu2; s++) cur = next(cur);
        return cur == 0;
    };
    double *b0 = final_is_first() ? Zf : Tb;
    auto next = [&](const double *cb) -> double * {
        return cb == rt ? b0 : (cb == Zf ? Tb : Zf);
    };
    double *cur = rt;
    for (int s = 1; s < nu1; s++) {
        double *o = next(cur);
        launch_jacobi_rt<double>(v.g, v.wcD, omw, r, rt, cur, o, nullptr, x->st);
        cur = o;
    }
    double *res = next(cur);
    launch_resid<double>(v.g, v.D, c, cur, r, res, nullptr, nullptr, x->st);
    Level &w = x->mg[l + 1];
    launch_restrict<double>(v.m, w.m, x->N, v.tab, res, (double *)x->mxt1, (double *)x->mxt2,
                            (double *)w.r, x->st);
    HQ_TRY(vcycle<double>(x, l + 1, (const double *)w.r, (double *)w.z, (double *)w.t, false,
                          nullptr));
    launch_prolong<double>(v.m, w.m, x->N, v.tab, (const double *)w.z, (double *)x->mxt1,
                           (double *)x->mxt2, cur, res, x->st);
    cur = res;
    for (int s = 0; s < nu2; s++) {
        const bool last = (s == nu2 - 1);
        double *o = next(cur);
        launch_jacobi_rt<double>(v.g, v.wcD, omw, r, rt, cur, o, last ? part_final : nullptr,
                                 x->st);
        cur = o;
    }
    if (cur != Zf) HQ_TRY(copy_blk<double>(x, Zf, cur, (size_t)v.n * x->N));
    return HQ_OK;
}

// the FP32 V-cycle of levels l .. L-1 as one launch's description
VCoarse make_vcoarse(const hq_ctx *x, int l) {
    VCoarse vc;
    std::memset(&vc, 0, sizeof(vc));
    vc.levels = x->L - l;
    for (int k = 0; k < vc.levels; k++) {
        const Level &v = x->mg[l + k];
        vc.m[k] = v.m;
        vc.c[k] = (float)v.c;
        vc.D[k] = (const float *)v.Dt;
        vc.wD[k] = (const float *)v.wDt;
        if (k + 1 < vc.levels) {
            vc.ridx[k] = v.tab.ridx;
            vc.rw[k] = v.tab.rwf;
            vc.pidx[k] = v.tab.pidx;
            vc.pw[k] = v.tab.pwf;
            const double q = (double)(x->mg[l + k + 1].m + 1) / (double)(v.m + 1);
            vc.rscale[k] = (float)(q * q * q);
        }
    }
    vc.Ainv = x->Ainv;
    vc.nc = (int)x->nc;
    vc.omw = (float)(1.0 - x->cfg.mg_omega);
    vc.nu1 = x->cfg.mg_nu1;
    vc.nu2 = x->cfg.mg_nu2;
    return vc;
}

// first level from which the FP32 V-cycle fits one launch (-1: none), or -1
// when HQ_FUSED_COARSE=0 (the multi-kernel V-cycle, for comparisons)
int fuse_level(const hq_ctx *x, bool honour_switch = true) {
    const char *e = std::getenv("HQ_FUSED_COARSE");
    if (honour_switch && e && e[0] == '0') return -1;
    if (!x->mixed && !x->mg32) return -1;
    if (x->nc > 64) return -1;   // k_vcoarse's coarsest solve: at most 64 points (4^3)
    for (int l = 0; l + 1 < x->L; l++) {
        if (x->L - l > VC_MAXLEV) continue;
        if (vcoarse_smem_bytes(make_vcoarse(x, l)) <= (size_t)VC_MAX_SMEM) return l;
    }
    return -1;
}

// r64dot (FP32 V-cycle of an FP64 PCG, level 0, linear point order only):
// the last sweep forms part_final as the FP64 partials of r64dot . z
template <typename T>
hq_status vcycle(hq_ctx *x, int l, const T *r, T *Zf, T *Tb, bool first_done, double *part_final,
                 const double *r64dot) {
    LevelScope lvl_(l);
    if constexpr (std::is_same<T, float>::value) {
        if (x->fuse_l0 >= 0 && !x->no_fuse && l >= x->fuse_l0 && l + 1 < x->L && !first_done &&
            !part_final) {
            launch_vcoarse(make_vcoarse(x, l), x->N, r, Zf, x->st);
            return HQ_OK;
        }
    }
    Level &v = x->mg[l];
    const T c = (T)v.c, omw = (T)(1.0 - x->cfg.mg_omega);
    if (l == x->L - 1) {
        launch_coarse_solve<T>(v.g, x->Ainv, r, Zf, x->st);
        if (part_final) launch_dot<T>(v.g, r, Zf, part_final, x->st);
        return HQ_OK;
    }
    if constexpr (std::is_same<T, double>::value) {
        if (x->rtilde) return vcycle_rt(x, l, r, Zf, Tb, first_done, part_final);
    }
    T *cur = first_target<T>(x, l, Zf, Tb);
    T *oth = (cur == Zf) ? Tb : Zf;
    if (!first_done) launch_jacobi_first<T>(v.g, (const T *)v.wDt, r, cur, x->st);
    for (int s = 1; s < x->cfg.mg_nu1; s++) {
        launch_jacobi<T>(v.g, (const T *)v.Dt, (const T *)v.wDt, c, omw, r, cur, oth, nullptr, x->st);
        std::swap(cur, oth);
    }
    launch_resid<T>(v.g, (const T *)v.Dt, c, cur, r, oth, nullptr, nullptr, x->st);
    Level &w = x->mg[l + 1];
    launch_restrict<T>(v.m, w.m, x->N, v.tab, oth, (T *)x->mxt1, (T *)x->mxt2, (T *)w.r, x->st);
    HQ_TRY(vcycle<T>(x, l + 1, (const T *)w.r, (T *)w.z, (T *)w.t, false, nullptr));
    launch_prolong<T>(v.m, w.m, x->N, v.tab, (const T *)w.z, (T *)x->mxt1, (T *)x->mxt2, cur, oth,
                      x->st);
    std::swap(cur, oth);
    for (int s = 0; s < x->cfg.mg_nu2; s++) {
        bool last = (s == x->cfg.mg_nu2 - 1);
        if constexpr (std::is_same<T, float>::value) {
            if (last && part_final && r64dot) {
                launch_jacobi_dot64(v.g, (const float *)v.wDt, c, omw, r, r64dot, cur, oth,
                                    part_final, x->st);
                std::swap(cur, oth);
                continue;
            }
        }
        launch_jacobi<T>(v.g, (const T *)v.Dt, (const T *)v.wDt, c, omw, r, cur, oth,
                         last ? part_final : nullptr, x->st);
        std::swap(cur, oth);
    }
    if (cur != Zf) HQ_TRY(copy_blk<T>(x, Zf, cur, (size_t)v.n * x->N));
    return HQ_OK;
}

// z = M r (one V-cycle) and, if part is non-null, the partials of r.z in the
// finest level's layout.  In mg32 contexts (FP64 PCG, FP32 preconditioner)
// r is rounded to FP32, the V-cycle runs on the FP32 level copies, and z is
// widened back to FP64 while r.z is formed in FP64.
template <typename T>
hq_status precondition(hq_ctx *x, const T *r, T *z, T *tbuf, bool first_done, double *part) {
    if constexpr (std::is_same<T, double>::value) {
        if (x->mg32) {
            // the whole V-cycle fits one launch: conversion, V-cycle, widening
            // and r.z in that launch (the same values as the three launches)
            if (x->fuse_l0 == 0 && !x->no_fuse) {
                const VCoarse vc = make_vcoarse(x, 0);
                if (vcoarse64_smem_bytes(vc, x->lev[0].g) <= (size_t)VC_MAX_SMEM) {
                    launch_vcoarse64(vc, x->lev[0].g, r, z, part, x->st);
                    return HQ_OK;
                }
            }
            const size_t cnt = (size_t)x->n * x->N;
            launch_convert_d2f(cnt, r, x->R32, x->st);
            HQ_TRY(vcycle<float>(x, 0, x->R32, x->Z32, x->T32, false, nullptr));
            launch_widen_dot(x->lev[0].g, x->Z32, r, z, part, x->st);
            return HQ_OK;
        }
    }
    return vcycle<T>(x, 0, r, z, tbuf, first_done, part);
}

// the first damped-Jacobi sweep can be fused into the x / r update when the
// V-cycle runs on the PCG's own buffers (more than one level, same precision)
bool fuse_first_sweep(hq_ctx *x) { return x->L > 1 && !x->mg32; }

// FP64 block PCG with an FP32 V-cycle whose finest level runs as separate
// kernels in linear point order: the FP64 <-> FP32 interface is fused into the
// PCG's passes (k_pcg_xr_mg writes r32 and the first sweep, the last sweep
// forms r.z in FP64, k_pcg_p_mg reads z in FP32) instead of k_d2f,
// k_jacobi_first and k_widen_dot
bool mgf(const hq_ctx *x) {
    return x->mg32 && x->L > 1 && !x->level0_fits && x->mg[0].g.zch == 0;
}

// rows of the r.z partials precondition() leaves: the last smoothing sweep
// of the finest level, or the FP64 widening kernel of an FP32 V-cycle, or the
// fused FP32 sweep
int prec_rows(hq_ctx *x) {
    if (mgf(x)) return x->mg[0].g.gy;
    return x->mg32 ? x->lev[0].g.gy : part_rows(x->lev[0].g);
}

// the block PCG's preconditioner in mgf contexts: z (FP32, in Z32) = M r with
// r32 written here (first_done false) or by k_pcg_xr_mg together with the
// first sweep (first_done true); part: the FP64 partials of r.z
hq_status precondition_mgf(hq_ctx *x, const double *r, bool first_done, double *part) {
    if (!first_done) launch_convert_d2f((size_t)x->n * x->N, r, x->R32, x->st);
    return vcycle<float>(x, 0, x->R32, x->Z32, x->T32, first_done, part, r);
}

// ---------------------------------------------------------------------------
// block PCG: X = G B, per-column stopping ||r_j|| <= rtol ||b_j||
//
// Per column (columns that have stopped are frozen by alpha = beta = 0):
//   r = b - A x, z = M r, p = z, rz = r.z
//   iterate: q = A p, alpha = rz / p.q, x += alpha p, r -= alpha q,
//            stop if ||r|| <= rtol ||b||; z = M r, beta = (r.z)/rz, p = z + beta p
// The first iteration runs from the host; the remaining ones run as the body
// of a CUDA graph with a conditional WHILE node (body: V-cycle, beta, p, A p,
// alpha, x / r update, stopping test, and a kernel that sets the loop
// condition from the number of active columns and the iteration count), so
// a whole solve costs two host round trips.  With per-launch event timing on,
// the same body is launched from the host instead.
// ---------------------------------------------------------------------------
// PCG start: z = M r, rz = r.z, p = z
template <typename T>
hq_status pcg_first_direction(hq_ctx *x, double rtol) {
    const int N = x->N;
    T *R = (T *)x->R, *Zp = (T *)x->Zp, *P = (T *)x->P, *Tt = (T *)x->Tt;
    PcgScalars sc = x->sc;
    if constexpr (std::is_same<T, double>::value) {
        if (mgf(x)) {
            HQ_TRY(precondition_mgf(x, R, false, x->part));
            launch_finalize(FIN_RZ, N, prec_rows(x), x->part, nullptr, sc, rtol, x->st);
            launch_convert_f2d((size_t)x->n * N, x->Z32, P, x->st);
            return HQ_OK;
        }
    }
    HQ_TRY(precondition<T>(x, R, Zp, Tt, false, x->part));
    launch_finalize(FIN_RZ, N, prec_rows(x), x->part, nullptr, sc, rtol, x->st);
    return copy_blk<T>(x, P, Zp, (size_t)x->n * N);
}

template <typename T>
hq_status pcg_body(hq_ctx *x, T *X, double rtol) {
    Level &v = x->lev[0];
    const GridGeom &g = v.g;
    const int N = x->N;
    T *R = (T *)x->R, *Zp = (T *)x->Zp, *P = (T *)x->P, *Q = (T *)x->Q, *Tt = (T *)x->Tt;
    PcgScalars sc = x->sc;
    if constexpr (std::is_same<T, double>::value) {
        if (mgf(x)) {
            HQ_TRY(precondition_mgf(x, R, true, x->part));
            launch_finalize(FIN_BETA, N, prec_rows(x), x->part, nullptr, sc, rtol, x->st);
            launch_pcg_p_mg(g, sc.beta, x->Z32, P, x->st);
            return HQ_OK;
        }
    }
    HQ_TRY(precondition<T>(x, R, Zp, Tt, fuse_first_sweep(x), x->part));
    launch_finalize(FIN_BETA, N, prec_rows(x), x->part, nullptr, sc, rtol, x->st);
    launch_pcg_p<T>(g, sc.beta, Zp, P, x->st);
    return HQ_OK;
}

template <typename T>
hq_status pcg_half(hq_ctx *x, T *X, double rtol) {
    Level &v = x->lev[0];
    const GridGeom &g = v.g;
    const int N = x->N;
    T *R = (T *)x->R, *Zp = (T *)x->Zp, *P = (T *)x->P, *Q = (T *)x->Q, *Tt = (T *)x->Tt;
    PcgScalars sc = x->sc;
    T *zfirst = x->rtilde ? (T *)x->mg[0].rt : first_target<T>(x, 0, Zp, Tt);
    launch_apply<T>(g, (const T *)v.Dt, (T)v.c, P, Q, x->part, x->st);
    launch_finalize(FIN_ALPHA, N, part_rows(g), x->part, nullptr, sc, rtol, x->st);
    bool done = false;
    if constexpr (std::is_same<T, double>::value) {
        if (mgf(x)) {
            launch_pcg_xr_mg(g, sc.alpha, P, Q, X, R, x->part, (const float *)x->mg[0].wDt,
                             x->R32, first_target<float>(x, 0, x->Z32, x->T32), x->st);
            done = true;
        }
    }
    if (!done)
        launch_pcg_xr<T>(g, sc.alpha, P, Q, X, R, x->part, (const T *)v.wDt,
                         fuse_first_sweep(x) ? zfirst : nullptr, x->st);
    HQ_CUDA(cudaMemsetAsync(sc.num_active, 0, sizeof(int), x->st));
    launch_finalize(FIN_RR, N, g.gy, x->part, nullptr, sc, rtol, x->st);
    return HQ_OK;
}

void destroy_graph(PcgGraph &pg) {
    if (pg.exec) cudaGraphExecDestroy(pg.exec);
    if (pg.g) cudaGraphDestroy(pg.g);
    pg = PcgGraph();
}

template <typename T>
PcgGraph *pcg_graph(hq_ctx *x, T *X, double rtol, int maxit) {
    for (int i = 0; i < x->npgraph; i++) {
        PcgGraph &pg = x->pgraph[i];
        if (pg.X == X && pg.rtol == rtol && pg.maxit == maxit) return pg.ok ? &pg : nullptr;
    }
    if (x->npgraph == MAXGRAPH) {
        destroy_graph(x->pgraph[0]);
        for (int i = 1; i < MAXGRAPH; i++) x->pgraph[i - 1] = x->pgraph[i];
        x->pgraph[MAXGRAPH - 1] = PcgGraph();
        x->npgraph--;
    }
    PcgGraph &pg = x->pgraph[x->npgraph++];
    pg.X = X;
    pg.rtol = rtol;
    pg.maxit = maxit;
    pg.ok = false;
    if (!x->cap && cudaStreamCreateWithFlags(&x->cap, cudaStreamNonBlocking) != cudaSuccess) {
        x->cap = nullptr;
        return nullptr;
    }
    cudaGraphConditionalHandle h;
    if (cudaGraphCreate(&pg.g, 0) != cudaSuccess) return nullptr;
    if (cudaGraphConditionalHandleCreate(&h, pg.g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return nullptr;
    // zero-initialised node parameters (the struct has no default constructor)
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    std::memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(npbuf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, pg.g, nullptr, nullptr, 0, &np) != cudaSuccess) return nullptr;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(x->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return nullptr;
    cudaStream_t saved = x->st;
    x->st = x->cap;
    x->capturing = true;
    for (int i = 0; i < HQ_K_NCLASS; i++) pg.body_launches[i] = 0;
    x->cap_counts = pg.body_launches;
    hq_status st = pcg_body<T>(x, X, rtol);
    if (st == HQ_OK) st = pcg_half<T>(x, X, rtol);
    if (st == HQ_OK) launch_pcg_cond(x->sc.num_active, x->sc.num_active + 1, maxit, h, x->st);
    x->capturing = false;
    x->cap_counts = nullptr;
    x->st = saved;
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(x->cap, &out);
    if (st != HQ_OK || e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaGraphInstantiate(&pg.exec, pg.g, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    pg.ok = true;
    return &pg;
}

template <typename T>
hq_status pcg(hq_ctx *x, const T *B, T *X, double rtol, int maxit, int *iters_host) {
    Level &v = x->lev[0];
    const GridGeom &g = v.g;
    const int N = x->N;
    T *R = (T *)x->R, *Zp = (T *)x->Zp, *P = (T *)x->P, *Tt = (T *)x->Tt;
    const T c = (T)v.c;
    PcgScalars sc = x->sc;
    HQ_CUDA(cudaMemsetAsync(sc.num_active, 0, sizeof(int), x->st));
    launch_resid<T>(g, (const T *)v.Dt, c, X, B, R, x->part, x->part2, x->st);
    launch_finalize(FIN_BNORM_RNORM, N, part_rows(g), x->part, x->part2, sc, rtol, x->st);
    int nact = 0;
    HQ_CUDA(cudaMemcpyAsync(&nact, sc.num_active, sizeof(int), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    hq_status st = HQ_OK;
    long it_done = 0;
    if (nact > 0 && maxit > 0) {
        HQ_TRY(pcg_first_direction<T>(x, rtol));
        HQ_TRY(pcg_half<T>(x, X, rtol));   // iteration 1
        it_done = 1;
        HQ_CUDA(cudaMemcpyAsync(&nact, sc.num_active, sizeof(int), cudaMemcpyDeviceToHost, x->st));
        HQ_CUDA(cudaStreamSynchronize(x->st));
        if (nact > 0 && maxit > 1) {
            PcgGraph *pg = (x->use_graphs && !x->timing) ? pcg_graph<T>(x, X, rtol, maxit) : nullptr;
            if (pg) {
                int it[2] = {nact, 1};
                HQ_CUDA(cudaMemcpyAsync(sc.num_active, it, sizeof(it), cudaMemcpyHostToDevice, x->st));
                HQ_CUDA(cudaGraphLaunch(pg->exec, x->st));
                HQ_CUDA(cudaMemcpyAsync(it, sc.num_active, sizeof(it), cudaMemcpyDeviceToHost, x->st));
                HQ_CUDA(cudaStreamSynchronize(x->st));
                nact = it[0];
                it_done = it[1];
                for (int i = 0; i < HQ_K_NCLASS; i++)
                    x->launches[i] += pg->body_launches[i] * (long)(it[1] - 1);
            } else {
                for (int it = 2; it <= maxit; it++) {
                    HQ_TRY(pcg_body<T>(x, X, rtol));
                    HQ_TRY(pcg_half<T>(x, X, rtol));
                    it_done = it;
                    HQ_CUDA(cudaMemcpyAsync(&nact, sc.num_active, sizeof(int), cudaMemcpyDeviceToHost, x->st));
                    HQ_CUDA(cudaStreamSynchronize(x->st));
                    if (nact == 0) break;
                }
            }
        }
        if (nact > 0 && rtol > 0.0) st = HQ_ERR_NOT_CONVERGED;
    }
    x->stat_solves++;
    x->stat_iters += it_done;
    if (iters_host) HQ_CUDA(cudaMemcpyAsync(iters_host, sc.iters, sizeof(int) * N, cudaMemcpyDeviceToHost, x->st));
    HQ_TRY(sync_status(x, sc.status, "inner PCG"));
    if (st == HQ_ERR_NOT_CONVERGED) return fail(x, st, "inner PCG reached cg_maxit");
    return HQ_OK;
}

// Symmetric Gram of [X1 X2] into out (FP64): SIMT FP64 in HQ_FP64 contexts,
// tcgen05 3xTF32 in HQ_MIXED contexts.
template <typename T>
void gram_sym(hq_ctx *x, const T *X1, int n1, const T *X2, int n2, double *out);
// fp64_tc = 1 sends an FP64 product to the digit-sliced tensor-core kernels
// only from this many multiply-adds on: below it their splitting passes and
// one-CTA-per-SM schedule cost more than the SIMT FP64 kernels (a 4096 x 8
// block: 23 us per product on tensor cores against a few us in SIMT)
constexpr double OZ_MIN_MACS = 33554432.0;
bool use_oz(const hq_ctx *x, double macs) {
    return x->cfg.fp64_tc == 2 || (x->cfg.fp64_tc == 1 && macs >= OZ_MIN_MACS);
}

template <>
void gram_sym<double>(hq_ctx *x, const double *X1, int n1, const double *X2, int n2, double *out) {
    const double na = n1 + n2;
    if (x->ozgram && gram_oz_supported(n1 + n2) && use_oz(x, 0.5 * (double)x->n * na * na)) {
        launch_gram_oz(x->n, X1, n1, X2, n2, x->h3, x->ozgram, out, x->status, x->st);
        return;
    }
    GramPlan gp = make_gram_plan(x->n, n1 + n2, n1 + n2, true);
    launch_gram<double>(gp, X1, n1, X2, n2, X1, n1, X2, n2, x->h3, x->gpart, out, x->st);
}
template <>
void gram_sym<float>(hq_ctx *x, const float *X1, int n1, const float *X2, int n2, double *out) {
    launch_gram_tc(x->n, X1, n1, X2, n2, x->h3, x->tcpart, out, x->status, x->st);
}

// Out = A1 M1 (+ A2 M2) (+ Cin) (n x N); part_sq: sum of squares of Out into
// x->tpart and the number of partials into *np.  FP64: SIMT register-tiled;
// HQ_MIXED: tcgen05 3xTF32.
template <typename T>
void block_gemm(hq_ctx *x, const T *A1, int k1, const double *M1, const T *A2, int k2,
                const double *M2, const T *Cin, T *Out, bool sq, int *np);
template <>
void block_gemm<double>(hq_ctx *x, const double *A1, int k1, const double *M1, const double *A2,
                        int k2, const double *M2, const double *Cin, double *Out, bool sq, int *np) {
    const double K = k1 + (A2 ? k2 : 0);
    if (x->ozimg && tall_oz_supported(k1, A2 ? k2 : 0) && use_oz(x, (double)x->n * K * x->N)) {
        launch_tall_oz(x->n, A1, k1, M1, A2, k2, M2, x->N, Cin, Out, sq ? x->tpart : nullptr,
                       x->ozimg, x->status, x->st);
        if (np) *np = tall_oz_partials(x->n, x->N);
        return;
    }
    TallPlan tp = make_tall_plan(x->n, x->N, k1, k2);
    launch_tall_gemm<double>(tp, A1, M1, A2, M2, Cin, Out, sq ? x->tpart : nullptr, x->st);
    if (np) *np = tp.gy * tp.gx;
}
template <>
void block_gemm<float>(hq_ctx *x, const float *A1, int k1, const double *M1, const float *A2,
                       int k2, const double *M2, const float *Cin, float *Out, bool sq, int *np) {
    launch_tall_tc(x->n, A1, k1, M1, A2, k2, M2, x->N, Cin, Out, sq ? x->tpart : nullptr, x->tcimg,
                   x->status, x->st);
    if (np) *np = tall_tc_partials(x->n, x->N);
}

// ---------------------------------------------------------------------------
// the scheme
// ---------------------------------------------------------------------------
// Appends a conditional node with handle h to the capture sequence of s and
// returns its body graph; the capture continues after the node.
bool add_cond_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                   cudaGraph_t *body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &ed, &nd) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return false;
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    std::memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(npbuf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, ed, nd, &np) != cudaSuccess) return false;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
        cudaSuccess)
        return false;
    *body = np.conditional.phGraph_out[0];
    return true;
}

bool capture_graph_of(cudaStream_t s, cudaGraph_t *g) {
    cudaStreamCaptureStatus cs;
    return cudaStreamGetCaptureInfo(s, &cs, nullptr, g, nullptr, nullptr, nullptr) == cudaSuccess &&
           cs == cudaStreamCaptureStatusActive;
}

// Block PCG recorded into the phase graph being captured on x->st: the
// prologue, then WHILE(active && it < maxit) { q = A p, alpha, x / r update,
// stopping test, IF(active) { z = M r, beta, p = z + beta p } }.  The
// operation sequence equals that of pcg(); nothing is read back on the host.
template <typename T>
hq_status pcg_device(hq_ctx *x, const T *B, T *X, double rtol, int maxit, StepGraph &sgr,
                     long long *counters) {
    Level &v = x->lev[0];
    const GridGeom &g = v.g;
    const int N = x->N;
    T *R = (T *)x->R, *Zp = (T *)x->Zp, *P = (T *)x->P, *Tt = (T *)x->Tt;
    PcgScalars sc = x->sc;
    cudaStream_t main = x->st;
    HQ_CUDA(cudaMemsetAsync(sc.num_active, 0, 2 * sizeof(int), main));
    launch_resid<T>(g, (const T *)v.Dt, (T)v.c, X, B, R, x->part, x->part2, main);
    launch_finalize(FIN_BNORM_RNORM, N, part_rows(g), x->part, x->part2, sc, rtol, main);
    HQ_TRY(pcg_first_direction<T>(x, rtol));
    cudaGraph_t gmain;
    if (!capture_graph_of(main, &gmain)) return fail(x, HQ_ERR_CUDA, "capture state");
    cudaGraphConditionalHandle hw, hif;
    if (cudaGraphConditionalHandleCreate(&hw, gmain, 0, cudaGraphCondAssignDefault) != cudaSuccess)
        return fail(x, HQ_ERR_CUDA, "conditional handle");
    launch_pcg_cond_init(sc.num_active, maxit, hw, main);
    cudaGraph_t body;
    if (!add_cond_node(main, hw, cudaGraphCondTypeWhile, &body))
        return fail(x, HQ_ERR_CUDA, "WHILE node");
    // loop body, captured on capB
    x->st = x->capB;
    if (cudaStreamBeginCaptureToGraph(x->capB, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        x->st = main;
        return fail(x, HQ_ERR_CUDA, "body capture");
    }
    x->cap_counts = sgr.part1;
    hq_status st = pcg_half<T>(x, X, rtol);
    cudaGraph_t ifbody = nullptr;
    bool ok = st == HQ_OK &&
              cudaGraphConditionalHandleCreate(&hif, body, 0, cudaGraphCondAssignDefault) ==
                  cudaSuccess;
    if (ok) {
        launch_pcg_cond2(sc.num_active, sc.num_active + 1, maxit, hw, hif, counters, sc.status,
                         rtol > 0.0 ? 1 : 0, x->st);
        ok = add_cond_node(x->capB, hif, cudaGraphCondTypeIf, &ifbody);
    }
    if (ok) {
        x->st = x->capC;
        ok = cudaStreamBeginCaptureToGraph(x->capC, ifbody, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            x->cap_counts = sgr.part2;
            st = pcg_body<T>(x, X, rtol);
            cudaGraph_t tmp;
            if (cudaStreamEndCapture(x->capC, &tmp) != cudaSuccess) ok = false;
        }
        x->st = x->capB;
    }
    cudaGraph_t tmpb;
    if (cudaStreamEndCapture(x->capB, &tmpb) != cudaSuccess) ok = false;
    x->st = main;
    x->cap_counts = sgr.fixed;
    if (!ok || st != HQ_OK) return fail(x, HQ_ERR_CUDA, "PCG loop capture");
    return HQ_OK;
}

// A1-A3: W = G U (warm start from the previous G Uh), Gram of [U W], g.
// sgr == nullptr: host-driven PCG; otherwise recorded into a phase graph.
template <typename T>
hq_status enqueue_a(hq_ctx *x, StepGraph *sgr, long long *counters) {
    const int N = x->N;
    const size_t cnt = (size_t)x->n * N;
    T *U = (T *)x->U, *W = (T *)x->W;
    if (x->z_valid || sgr) HQ_TRY(copy_blk<T>(x, W, (const T *)x->Z, cnt));
    else HQ_CUDA(cudaMemsetAsync(W, 0, cnt * sizeof(T), x->st));
    if (sgr) HQ_TRY(pcg_device<T>(x, U, W, x->cfg.cg_rtol, x->cfg.cg_maxit, *sgr, counters));
    else HQ_TRY(pcg<T>(x, U, W, x->cfg.cg_rtol, x->cfg.cg_maxit, nullptr));
    gram_sym<T>(x, U, N, W, N, x->G2);
    // Msm = -Pwu (rows N..2N-1, columns 0..N-1 of G2); g = || W - U Pwu ||_h
    launch_extract(N, N, -1.0, x->G2 + (size_t)N * 2 * N, 2 * N, x->Msm, N, x->st);
    int np = 0;
    block_gemm<T>(x, U, N, x->Msm, nullptr, 0, nullptr, W, nullptr, true, &np);
    launch_sum_sqrt(np, x->tpart, x->h3, x->scal, x->st);
    return HQ_OK;
}

// the side stream and fork / join events of phase B
bool ensure_side(hq_ctx *x) {
    if (!x->side && cudaStreamCreateWithFlags(&x->side, cudaStreamNonBlocking) != cudaSuccess) {
        x->side = nullptr;
        return false;
    }
    for (cudaEvent_t &e : x->evside)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            e = nullptr;
            return false;
        }
    return true;
}

// B1-B5: predictor system, Uh, Shat, Z = G Uh, corrector (U <- U_{n+1}).
template <typename T>
hq_status enqueue_b(hq_ctx *x, StepGraph *sgr, long long *counters) {
    const int N = x->N;
    const size_t cnt = (size_t)x->n * N;
    const double tau = x->cfg.tau;
    T *U = (T *)x->U, *W = (T *)x->W, *Uh = (T *)x->Uh, *Z = (T *)x->Z;
    const double *tau_dev = nullptr;
    // the warm start's N x N solve needs only the Gram: it runs on the side
    // stream beside the step size and the predictor system (not in the
    // per-launch timing mode, whose events are on the main stream)
    const bool ws_fork = x->cfg.z_warm_start && x->lu32w && x->ipivw && x->pRw &&
                         lu32_fits(N, N) && !x->timing && ensure_side(x);
    if (ws_fork) {
        HQ_CUDA(cudaEventRecord(x->evside[0], x->st));
        HQ_CUDA(cudaStreamWaitEvent(x->side, x->evside[0], 0));
        if (x->mixed)
            launch_spd_solve(N, x->G2, 2 * N, x->G2 + N, 2 * N, x->Mw, x->Lm, x->Ym, x->ipivw,
                             x->status, x->side, x->lu32w);
        else
            launch_solve32_refined(N, N, x->G2, 2 * N, x->G2 + N, 2 * N, x->Ym, x->lu32w,
                                   x->ipivw, x->pRw, 2, x->status, x->side);
        HQ_CUDA(cudaEventRecord(x->evside[1], x->side));
    }
    if (x->cfg.adaptive_tau) {
        // tau_n from the Gram of step n (Ritz estimate of lambda_1, bound on lambda_max<U,U>)
        launch_extract(N, N, 1.0, x->G2, 2 * N, x->Ssm, N, x->st);
        launch_extract(N, N, 1.0, x->G2 + (size_t)N * 2 * N, 2 * N, x->Ksm, N, x->st);
        if (x->mixed && lam_hat32_fits(N)) {
            launch_lam_hat32(N, x->Ksm, x->Ssm, x->pvec, x->scal + 12, x->status, x->st);
        } else {
            launch_rr_reduce(N, x->Ksm, x->Ssm, x->Lm, x->Cm, x->status, x->st);
            launch_top_eig(N, x->Cm, N, x->pvec, x->scal + 12, x->st);
        }
        launch_gersh(N, x->Ssm, N, x->scal + 13, x->st);
        const double tmax = x->cfg.tau_max > 0.0 ? x->cfg.tau_max : 1e300;
        launch_adapt_tau(x->scal + 12, x->scal + 13, tmax, x->cfg.tau_safety, 1.05, x->lambda1_lb,
                         x->scal + 8,
                         x->st);
        tau_dev = x->scal + 8;
    }
    launch_predictor_solve(N, tau, x->G2, x->Mw, x->XY, x->C, x->status, x->st, tau_dev, x->ipiv,
                           x->lu32, x->pB, x->pR);
    block_gemm<T>(x, U, N, x->C, W, N, x->C + (size_t)N * N, nullptr, Uh, false, nullptr);
    // Shat = C^T G2 C, Om = -tau (Shat - I)
    launch_small_gemm(2 * N, N, 2 * N, 1.0, x->G2, 2 * N, false, x->C, N, false, 0.0, x->T1, N,
                      x->st);
    launch_small_gemm(N, N, 2 * N, 1.0, x->C, N, true, x->T1, N, false, 0.0, x->Shat, N, x->st);
    launch_corrector_matrix(N, x->Shat, tau_dev, tau, x->Om, x->st);
    if (x->cfg.z_warm_start) {
        // G Uh = W C1 + G W C2 and G W ~ W M with M = S^{-1} Puw (exact when
        // span(U) is G-invariant): start from Z0 = W (C1 + M C2)
        // mixed: FP32 elimination (a warm start needs no more); FP64: FP32
        // elimination and two FP64 refinement steps where the factors fit
        // shared memory (the FP64 solution to rounding level)
        if (ws_fork)
            HQ_CUDA(cudaStreamWaitEvent(x->st, x->evside[1], 0));
        else if (!x->mixed && x->lu32 && x->pR && x->ipiv && lu32_fits(N, N))
            launch_solve32_refined(N, N, x->G2, 2 * N, x->G2 + N, 2 * N, x->Ym, x->lu32, x->ipiv,
                                   x->pR, 2, x->status, x->st);
        else
            launch_spd_solve(N, x->G2, 2 * N, x->G2 + N, 2 * N, x->Mw, x->Lm, x->Ym, x->ipiv,
                             x->status, x->st, x->mixed ? x->lu32 : nullptr);
        launch_extract(N, N, 1.0, x->C, N, x->Cm, N, x->st);
        launch_small_gemm(N, N, N, 1.0, x->Ym, N, false, x->C + (size_t)N * N, N, false, 1.0,
                          x->Cm, N, x->st);
    }
    if (!sgr) HQ_TRY(sync_status(x, x->status, "predictor system"));
    if (x->cfg.z_warm_start) {
        block_gemm<T>(x, W, N, x->Cm, nullptr, 0, nullptr, nullptr, Z, false, nullptr);
    } else {
        HQ_CUDA(cudaMemsetAsync(Z, 0, cnt * sizeof(T), x->st));
    }
    if (sgr) HQ_TRY(pcg_device<T>(x, Uh, Z, x->cfg.cg_rtol, x->cfg.cg_maxit, *sgr, counters + 2));
    else HQ_TRY(pcg<T>(x, Uh, Z, x->cfg.cg_rtol, x->cfg.cg_maxit, nullptr));
    block_gemm<T>(x, Z, N, x->Om, nullptr, 0, nullptr, Uh, U, false, nullptr);
    return HQ_OK;
}

// the private streams the captures of a context are recorded on
bool ensure_cap_streams(hq_ctx *x) {
    for (cudaStream_t *c : {&x->capA, &x->capB, &x->capC, &x->capD})
        if (!*c && cudaStreamCreateWithFlags(c, cudaStreamNonBlocking) != cudaSuccess) {
            *c = nullptr;
            return false;
        }
    return true;
}

// Captures phase `which` (0: A, 1: B) once; later calls replay it.
template <typename T>
StepGraph *phase_graph(hq_ctx *x, int which) {
    StepGraph &sgr = x->sg[which];
    if (sgr.tried) return sgr.ok ? &sgr : nullptr;
    sgr.tried = true;
    if (!ensure_cap_streams(x)) return nullptr;
    if (cudaStreamSynchronize(x->st) != cudaSuccess) return nullptr;
    cudaStream_t saved = x->st;
    x->st = x->capA;
    if (cudaStreamBeginCapture(x->capA, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        x->st = saved;
        return nullptr;
    }
    x->capturing = true;
    x->cap_counts = sgr.fixed;
    hq_status st = which == 0 ? enqueue_a<T>(x, &sgr, x->dcount) : enqueue_b<T>(x, &sgr, x->dcount);
    x->capturing = false;
    x->cap_counts = nullptr;
    x->st = saved;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(x->capA, &g);
    if (st != HQ_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        x->err.clear();
        return nullptr;
    }
    sgr.g = g;
    if (cudaGraphInstantiate(&sgr.exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    sgr.ok = true;
    return &sgr;
}

// adds the launches of the replayed phase graphs to the counters
hq_status fold_graph_counts(hq_ctx *x) {
    if (!x->sg[0].launches && !x->sg[1].launches) return HQ_OK;
    long long c[4];
    HQ_CUDA(cudaMemcpyAsync(c, x->dcount, sizeof(c), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    for (int w = 0; w < 2; w++) {
        StepGraph &sgr = x->sg[w];
        const long long it = c[2 * w] - sgr.seen[0], ifs = c[2 * w + 1] - sgr.seen[1];
        sgr.seen[0] = c[2 * w];
        sgr.seen[1] = c[2 * w + 1];
        for (int k = 0; k < HQ_K_NCLASS; k++)
            x->launches[k] += sgr.fixed[k] * sgr.launches + sgr.part1[k] * it + sgr.part2[k] * ifs;
        // each replay runs one solve of 1 + (loop iterations) PCG iterations
        x->stat_solves += sgr.launches;
        x->stat_iters += (long)it;
        sgr.launches = 0;
    }
    return HQ_OK;
}

// Graphs hold the shift constants and the lower bound of lambda_1 by value:
// a new potential discards them (after folding their launch counts).
hq_status drop_graphs(hq_ctx *x) {
    HQ_TRY(fold_graph_counts(x));
    x->gen++;
    for (int i = 0; i < x->npgraph; i++) destroy_graph(x->pgraph[i]);
    x->npgraph = 0;
    for (StepGraph &sgr : x->sg) {
        if (sgr.exec) cudaGraphExecDestroy(sgr.exec);
        if (sgr.g) cudaGraphDestroy(sgr.g);
        const long long s0 = sgr.seen[0], s1 = sgr.seen[1];
        sgr = StepGraph();
        sgr.seen[0] = s0;
        sgr.seen[1] = s1;
    }
    return HQ_OK;
}

bool use_phase_graphs(hq_ctx *x) { return x->use_graphs && !x->timing && x->z_valid; }

template <typename T>
hq_status phase_a(hq_ctx *x) {
    StepGraph *sgr = use_phase_graphs(x) ? phase_graph<T>(x, 0) : nullptr;
    if (sgr) {
        HQ_CUDA(cudaGraphLaunch(sgr->exec, x->st));
        sgr->launches++;
    } else {
        HQ_TRY(enqueue_a<T>(x, nullptr, nullptr));
    }
    HQ_TRY(check_launch(x));
    x->w_valid = true;
    return HQ_OK;
}

// restart the adaptive time step (first step from the lower bound)
hq_status reset_tau(hq_ctx *x) {
    double st[3] = {x->cfg.tau, x->cfg.tau, 1.0};
    HQ_CUDA(cudaMemcpyAsync(x->scal + 8, st, sizeof(st), cudaMemcpyHostToDevice, x->st));
    HQ_CUDA(cudaMemsetAsync(x->pvec, 0, sizeof(double) * x->N, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return HQ_OK;
}

hq_status read_g(hq_ctx *x, double *g) {
    HQ_CUDA(cudaMemcpyAsync(g, x->scal, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    HQ_TRY(check_launch(x));
    x->last_g = *g;
    if (!std::isfinite(*g)) return fail(x, HQ_ERR_NONFINITE, "gradient norm is not finite");
    return HQ_OK;
}

template <typename T>
hq_status phase_b(hq_ctx *x) {
    StepGraph *sgr = use_phase_graphs(x) ? phase_graph<T>(x, 1) : nullptr;
    if (sgr) {
        HQ_CUDA(cudaGraphLaunch(sgr->exec, x->st));
        sgr->launches++;
    } else {
        HQ_TRY(enqueue_b<T>(x, nullptr, nullptr));
    }
    HQ_TRY(check_launch(x));
    x->w_valid = false;
    x->z_valid = true;
    x->step++;
    return HQ_OK;
}

// status words of the replayed graphs (read at the end of hq_step / each
// hq_solve iteration)
hq_status graph_status(hq_ctx *x) {
    HQ_TRY(sync_status(x, x->sc.status, "inner PCG"));
    return sync_status(x, x->status, "step");
}

}  // namespace

// ===========================================================================
// Batched form: the time loop of Algorithm 1 for many contexts in one graph.
//
//   init (steps, flags, start time)
//   WHILE (some problem running) {
//     arm: h_k = problem k running
//     IF (h_k) { phase A_k; check g_k / cap / errors; IF (running) { phase B_k; ++steps } }
//     ... one IF node per problem, all in parallel ...
//     cond: wall-clock limit, loop condition
//   }
// Each phase holds its PCG loop as nested WHILE / IF nodes (pcg_device), so a
// whole batched solve is one graph launch and one host synchronisation.
// Phases of different problems share no buffers and run concurrently.
// ===========================================================================
struct hq_batch {
    std::vector<hq_ctx *> ctx;
    std::vector<int> gen;
    cudaStream_t st = nullptr;                      // caller's stream
    cudaStream_t capT = nullptr, capW = nullptr;    // captures: top graph, loop body
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
    long launches = 0;   // batch-level kernels (init, arm, cond)
    long loop_iters = 0;
    ~hq_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        if (capT) cudaStreamDestroy(capT);
        if (capW) cudaStreamDestroy(capW);
    }
};

namespace {

hq_status bfail(hq_batch *b, hq_status st, const std::string &msg) {
    b->err = msg;
    return st;
}

long long *slot_of(hq_ctx *x) { return x->dcount + 8; }

// Records problem x (phase A, the stopping test, phase B under an IF node)
// into `body`, the IF body graph of this problem in the time-loop body.
template <typename T>
hq_status capture_problem(hq_ctx *x, cudaGraph_t body) {
    ProfScope ps_(x);
    for (StepGraph &c : x->bsg) c = StepGraph();
    cudaStream_t saved = x->st;
    x->st = x->capA;
    if (cudaStreamBeginCaptureToGraph(x->capA, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        x->st = saved;
        return fail(x, HQ_ERR_CUDA, "batch capture");
    }
    x->capturing = true;
    x->cap_counts = x->bsg[0].fixed;
    hq_status st = enqueue_a<T>(x, &x->bsg[0], x->dcount + 4);
    bool ok = st == HQ_OK;
    cudaGraph_t gA = nullptr, bodyB = nullptr;
    cudaGraphConditionalHandle hB;
    ok = ok && capture_graph_of(x->capA, &gA) &&
         cudaGraphConditionalHandleCreate(&hB, gA, 0, 0) == cudaSuccess;
    if (ok) {
        launch_batch_check(slot_of(x), x->scal, x->status, x->sc.status, hB, x->capA);
        ok = add_cond_node(x->capA, hB, cudaGraphCondTypeIf, &bodyB);
    }
    if (ok) {
        x->st = x->capD;
        ok = cudaStreamBeginCaptureToGraph(x->capD, bodyB, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            x->cap_counts = x->bsg[1].fixed;
            st = enqueue_b<T>(x, &x->bsg[1], x->dcount + 4);
            launch_batch_count(slot_of(x), x->capD);
            cudaGraph_t tmp;
            if (cudaStreamEndCapture(x->capD, &tmp) != cudaSuccess) ok = false;
        }
        x->st = x->capA;
    }
    cudaGraph_t tmpA;
    if (cudaStreamEndCapture(x->capA, &tmpA) != cudaSuccess) ok = false;
    x->st = saved;
    x->capturing = false;
    x->cap_counts = nullptr;
    if (!ok || st != HQ_OK) {
        cudaGetLastError();
        return fail(x, HQ_ERR_CUDA, "batch capture of a problem");
    }
    return HQ_OK;
}

void batch_drop(hq_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->g) cudaGraphDestroy(b->g);
    b->exec = nullptr;
    b->g = nullptr;
}

hq_status batch_build(hq_batch *b) {
    batch_drop(b);
    const int K = (int)b->ctx.size();
    for (hq_ctx *x : b->ctx)
        if (!ensure_cap_streams(x)) return bfail(b, HQ_ERR_CUDA, "stream creation");
    for (cudaStream_t *c : {&b->capT, &b->capW})
        if (!*c && cudaStreamCreateWithFlags(c, cudaStreamNonBlocking) != cudaSuccess) {
            *c = nullptr;
            return bfail(b, HQ_ERR_CUDA, "stream creation");
        }
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.count = K;
    for (int k = 0; k < K; k++) a.slot[k] = slot_of(b->ctx[k]);
    if (cudaStreamBeginCapture(b->capT, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(b, HQ_ERR_CUDA, "batch capture");
    bool ok = true;
    cudaGraph_t top = nullptr, wbody = nullptr;
    cudaGraphConditionalHandle hT;
    std::vector<cudaGraph_t> bodies(K, nullptr);
    ok = capture_graph_of(b->capT, &top) &&
         cudaGraphConditionalHandleCreate(&hT, top, 0, 0) == cudaSuccess;
    if (ok) {
        launch_batch_init(a, hT, b->capT);
        ok = add_cond_node(b->capT, hT, cudaGraphCondTypeWhile, &wbody);
    }
    if (ok) {
        ok = cudaStreamBeginCaptureToGraph(b->capW, wbody, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            for (int k = 0; k < K && ok; k++)
                ok = cudaGraphConditionalHandleCreate(&a.h[k], wbody, 0, 0) == cudaSuccess;
            if (ok) launch_batch_arm(a, b->capW);
            // one IF node per problem, all depending on the arm kernel only
            cudaStreamCaptureStatus cs;
            cudaGraph_t gW = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            const cudaGraphEdgeData *ed = nullptr;
            size_t nd = 0;
            ok = ok && cudaStreamGetCaptureInfo(b->capW, &cs, nullptr, &gW, &deps, &ed, &nd) ==
                           cudaSuccess &&
                 cs == cudaStreamCaptureStatusActive;
            std::vector<cudaGraphNode_t> dv, ifn(K);
            std::vector<cudaGraphEdgeData> ev;
            if (ok) {
                dv.assign(deps, deps + nd);
                if (ed) ev.assign(ed, ed + nd);
            }
            for (int k = 0; k < K && ok; k++) {
                alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
                std::memset(npbuf, 0, sizeof(npbuf));
                cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(npbuf);
                np.type = cudaGraphNodeTypeConditional;
                np.conditional.handle = a.h[k];
                np.conditional.type = cudaGraphCondTypeIf;
                np.conditional.size = 1;
                ok = cudaGraphAddNode(&ifn[k], gW, dv.data(), ed ? ev.data() : nullptr, nd, &np) ==
                     cudaSuccess;
                if (ok) bodies[k] = np.conditional.phGraph_out[0];
            }
            ok = ok && cudaStreamUpdateCaptureDependencies(b->capW, ifn.data(), nullptr, K,
                                                           cudaStreamSetCaptureDependencies) ==
                           cudaSuccess;
            if (ok) launch_batch_cond(a, hT, b->capW);
            cudaGraph_t tmp;
            if (cudaStreamEndCapture(b->capW, &tmp) != cudaSuccess) ok = false;
        }
    }
    hq_status st = HQ_OK;
    for (int k = 0; k < K && ok; k++) {
        hq_ctx *x = b->ctx[k];
        // several concurrent problems: the coarse levels of a larger grid as
        // separate kernels (the same values bit for bit, see k_vcoarse.cu);
        // a V-cycle that fits one launch whole stays one launch
        x->no_fuse = K > 1 && x->fuse_l0 > 0;
        st = x->mixed ? capture_problem<float>(x, bodies[k]) : capture_problem<double>(x, bodies[k]);
        x->no_fuse = false;
        if (st != HQ_OK) {
            ok = false;
            b->err = "problem " + std::to_string(k) + ": " + x->err;
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capT, &g);
    if (!ok || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (b->err.empty()) b->err = "batch graph capture failed";
        return st != HQ_OK ? st : HQ_ERR_CUDA;
    }
    b->g = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        batch_drop(b);
        return bfail(b, HQ_ERR_CUDA, "batch graph instantiation failed");
    }
    for (int k = 0; k < K; k++) b->gen[k] = b->ctx[k]->gen;
    return HQ_OK;
}

// mode 0: Algorithm 1 per problem (stop at g < eps[k] or max_steps);
// mode 1: max_steps steps per problem
hq_status batch_run(hq_batch *b, int mode, const double *eps, long max_steps, double timeout_s,
                    long *steps_out, double *resid_out, int *status_out) {
    const int K = (int)b->ctx.size();
    b->err.clear();
    for (int k = 0; k < K; k++) {
        hq_ctx *x = b->ctx[k];
        if (!x->have_V || !x->have_U)
            return bfail(b, HQ_ERR_STATE, "problem " + std::to_string(k) +
                                              ": potential or initial block not set");
    }
    bool stale = !b->exec;
    for (int k = 0; k < K; k++) stale = stale || b->gen[k] != b->ctx[k]->gen;
    // the contexts' own streams may still hold work (uploads)
    for (hq_ctx *x : b->ctx)
        if (cudaStreamSynchronize(x->st) != cudaSuccess) return bfail(b, HQ_ERR_CUDA, "sync");
    if (stale) HQ_TRY(batch_build(b));
    for (int k = 0; k < K; k++) {
        hq_ctx *x = b->ctx[k];
        if (!x->z_valid) {
            // a zero warm start of W = G U, as the host path uses before the first step
            if (cudaMemsetAsync(x->Z, 0, (size_t)x->n * x->N * x->esz, b->st) != cudaSuccess)
                return bfail(b, HQ_ERR_CUDA, "memset");
            x->z_valid = true;
        }
        long long w[9];
        const double e = mode == 0 ? eps[k] : 0.0;
        std::memcpy(&w[BS_EPS], &e, sizeof(double));
        w[BS_STEPS] = 0;
        w[BS_DONE] = 0;
        w[BS_AEXEC] = 0;
        w[BS_MODE] = mode;
        w[BS_MAXSTEPS] = max_steps;
        w[BS_T0] = 0;
        w[BS_TIMEOUT] = (k == 0 && timeout_s > 0) ? (long long)(timeout_s * 1e9) : 0;
        w[BS_ITERS] = 0;
        if (cudaMemcpyAsync(slot_of(x), w, sizeof(w), cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
            cudaMemsetAsync(x->status, 0, sizeof(int), b->st) != cudaSuccess ||
            cudaMemsetAsync(x->sc.status, 0, sizeof(int), b->st) != cudaSuccess)
            return bfail(b, HQ_ERR_CUDA, "batch staging");
    }
    if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, HQ_ERR_CUDA, "batch graph launch failed");
    }
    // read back: loop state, PCG counters, g
    std::vector<long long> words((size_t)K * 13);
    std::vector<double> g(K);
    for (int k = 0; k < K; k++) {
        hq_ctx *x = b->ctx[k];
        if (cudaMemcpyAsync(&words[(size_t)k * 13], x->dcount + 4, 13 * sizeof(long long),
                            cudaMemcpyDeviceToHost, b->st) != cudaSuccess ||
            cudaMemcpyAsync(&g[k], x->scal, sizeof(double), cudaMemcpyDeviceToHost, b->st) !=
                cudaSuccess)
            return bfail(b, HQ_ERR_CUDA, "batch read-back");
    }
    cudaError_t ce = cudaStreamSynchronize(b->st);
    if (ce != cudaSuccess) return bfail(b, HQ_ERR_CUDA, cudaGetErrorString(ce));
    hq_status first = HQ_OK;
    long iters = 0;
    for (int k = 0; k < K; k++) {
        hq_ctx *x = b->ctx[k];
        const long long *c = &words[(size_t)k * 13];   // c[0..3] PCG counters, c[4..12] slot
        const long long *sl = c + 4;
        const long steps = (long)sl[BS_STEPS], aexec = (long)sl[BS_AEXEC];
        if (k == 0) iters = (long)sl[BS_ITERS];
        x->step += steps;
        x->w_valid = aexec > steps;
        x->last_g = g[k];
        // launch accounting (see fold_graph_counts)
        long long d[4];
        for (int i = 0; i < 4; i++) {
            d[i] = c[i] - x->bseen[i];
            x->bseen[i] = c[i];
        }
        for (int cl = 0; cl < HQ_K_NCLASS; cl++)
            x->launches[cl] += x->bsg[0].fixed[cl] * aexec + x->bsg[1].fixed[cl] * steps +
                               x->bsg[0].part1[cl] * d[0] + x->bsg[0].part2[cl] * d[1] +
                               x->bsg[1].part1[cl] * d[2] + x->bsg[1].part2[cl] * d[3];
        x->stat_solves += aexec + steps;
        x->stat_iters += (long)(d[0] + d[2]);
        hq_status stk = HQ_OK;
        switch (sl[BS_DONE]) {
            case BD_CONVERGED: stk = HQ_OK; break;
            case BD_MAXSTEPS:
                stk = mode == 0 ? fail(x, HQ_ERR_NOT_CONVERGED, "Algorithm 1 reached max_steps")
                                : HQ_OK;
                break;
            case BD_TIMEOUT: stk = fail(x, HQ_ERR_TIMEOUT, "batch wall-clock limit reached"); break;
            default: {
                stk = graph_status(x);
                if (stk == HQ_OK)
                    stk = std::isfinite(g[k]) ? fail(x, HQ_ERR_STATE, "batch loop ended early")
                                              : fail(x, HQ_ERR_NONFINITE, "gradient norm is not finite");
            }
        }
        if (stk == HQ_OK && sl[BS_DONE] != BD_ERROR) stk = graph_status(x);
        if (steps_out) steps_out[k] = steps;
        if (resid_out) resid_out[k] = g[k];
        if (status_out) status_out[k] = stk;
        if (stk != HQ_OK && first == HQ_OK) {
            first = stk;
            b->err = "problem " + std::to_string(k) + ": " + x->err;
        }
    }
    b->loop_iters += iters;
    b->launches += 1 + 2 * iters;
    return first;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {

hq_status guard(hq_ctx *x) {
    if (!x) return HQ_ERR_ARG;
    return HQ_OK;
}

hq_status need_ready(hq_ctx *x) {
    if (!x->have_V) return fail(x, HQ_ERR_STATE, "hq_set_potential has not been called");
    if (!x->have_U) return fail(x, HQ_ERR_STATE, "hq_set_initial / hq_set_state has not been called");
    return HQ_OK;
}

cudaMemcpyKind kind_in(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

template <typename T>
hq_status set_potential_impl(hq_ctx *x, const double *V, int on_device) {
    Level &v0 = x->lev[0];
    x->have_V = false;
    HQ_TRY(drop_graphs(x));
    HQ_TRY(clear_status(x));
    HQ_CUDA(cudaMemcpyAsync(v0.V, V, sizeof(double) * x->n, kind_in(on_device), x->st));
    launch_minmax(x->n, v0.V, x->scal + 2, x->st);
    double mm[2] = {0, 0};
    HQ_CUDA(cudaMemcpyAsync(mm, x->scal + 2, sizeof(mm), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    HQ_TRY(check_launch(x));
    if (mm[1] != 0.0) return fail(x, HQ_ERR_NONFINITE, "potential contains NaN or Inf");
    const double PI = 3.14159265358979323846;
    double s = std::sin(PI / (2.0 * (x->m + 1)));
    double lb = 3.0 * (2.0 / (x->h * x->h)) * s * s + mm[0];
    x->sigma = std::isnan(x->cfg.shift) ? (lb > 0.0 ? 0.0 : 1.0 - lb) : x->cfg.shift;
    x->lambda1_lb = lb + x->sigma;
    for (int l = 1; l < x->L; l++) {
        launch_coarse_potential(x->lev[l - 1].m, x->lev[l - 1].V, x->lev[l].m, x->lev[l].V, x->st);
        launch_xfer_tables(x->lev[l - 1].m, x->lev[l].m, x->lev[l - 1].tab, x->st);
    }
    for (int l = 0; l < x->L; l++) {
        Level &v = x->lev[l];
        launch_level_diag(v.n, v.V, x->sigma, v.c, x->cfg.mg_omega, v.D, v.wD, v.wcD, x->st);
        if (x->mixed) {
            launch_convert_d2f(v.n, v.D, (float *)v.Dt, x->st);
            launch_convert_d2f(v.n, v.wD, (float *)v.wDt, x->st);
        }
        if (x->mg32) {
            launch_convert_d2f(v.n, v.D, (float *)x->mg[l].Dt, x->st);
            launch_convert_d2f(v.n, v.wD, (float *)x->mg[l].wDt, x->st);
        }
    }
    Level &vc = x->lev[x->L - 1];
    launch_assemble_dense(vc.m, vc.c, vc.V, x->sigma, x->Acoarse, x->st);
    launch_gauss_jordan((int)x->nc, x->Acoarse, x->Ainv, x->status, x->st);
    HQ_TRY(sync_status(x, x->status, "potential setup"));
    x->have_V = true;
    x->w_valid = x->z_valid = false;
    x->step = 0;
    return reset_tau(x);
}

template <typename T>
hq_status load_block(hq_ctx *x, T *dst, const double *src, int on_device) {
    const size_t cnt = (size_t)x->n * x->N;
    if (!x->mixed) {
        HQ_CUDA(cudaMemcpyAsync(dst, src, cnt * sizeof(double), kind_in(on_device), x->st));
    } else {
        const double *s64 = src;
        if (!on_device) {
            HQ_CUDA(cudaMemcpyAsync(x->E1, src, cnt * sizeof(double), cudaMemcpyHostToDevice, x->st));
            s64 = x->E1;
        }
        launch_convert_d2f(cnt, s64, (float *)dst, x->st);
    }
    return check_launch(x);
}

template <typename T>
hq_status store_block(hq_ctx *x, double *dst, const T *src, int on_device) {
    const size_t cnt = (size_t)x->n * x->N;
    if (!x->mixed) {
        HQ_CUDA(cudaMemcpyAsync(dst, src, cnt * sizeof(double), kind_out(on_device), x->st));
    } else {
        double *d64 = on_device ? dst : x->E1;
        launch_convert_f2d(cnt, (const float *)src, d64, x->st);
        if (!on_device)
            HQ_CUDA(cudaMemcpyAsync(dst, d64, cnt * sizeof(double), cudaMemcpyDeviceToHost, x->st));
    }
    return check_launch(x);
}

template <typename T>
hq_status set_initial_impl(hq_ctx *x, const double *U0, int on_device) {
    const int N = x->N;
    x->have_U = false;
    HQ_TRY(clear_status(x));
    T *U = (T *)x->U;
    HQ_TRY(load_block<T>(x, U, U0, on_device));
    gram_sym<T>(x, U, N, (const T *)nullptr, 0, x->Ssm);
    launch_sym_eig(N, x->Ssm, x->eigwork, x->evals, nullptr, x->st);
    launch_inv_sqrt_first(x->evals, x->scal + 1, x->st);
    double lmin = 0;
    HQ_CUDA(cudaMemcpyAsync(&lmin, x->evals, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    HQ_TRY(check_launch(x));
    if (!(lmin > 0.0) || !std::isfinite(lmin))
        return fail(x, HQ_ERR_ARG, "initial block is rank deficient or not finite");
    launch_scale<T>((size_t)x->n * N, x->scal + 1, U, x->st);
    HQ_TRY(check_launch(x));
    x->have_U = true;
    x->w_valid = x->z_valid = false;
    x->step = 0;
    return reset_tau(x);
}

template <typename T>
hq_status step_impl(hq_ctx *x, int nsteps, double *resid_out) {
    HQ_TRY(need_ready(x));
    HQ_TRY(clear_status(x));
    double g = NAN;
    for (int s = 0; s < nsteps; s++) {
        HQ_TRY(phase_a<T>(x));
        if (s == nsteps - 1 || !use_phase_graphs(x)) HQ_TRY(read_g(x, &g));
        HQ_TRY(phase_b<T>(x));
    }
    HQ_TRY(graph_status(x));
    if (resid_out) *resid_out = g;
    return HQ_OK;
}

// Algorithm 1 on the device: the time loop of a one-member batch graph (the
// batched form's WHILE node, stopping test g < eps and step cap decided on
// the device), one graph launch and one host synchronisation per call.  The
// trajectory equals the host loop's bit for bit.  Returns false (nothing
// launched) when the graph cannot be captured; the caller then runs the host
// loop.
bool solve_device(hq_ctx *x, double eps, long max_steps, long *steps_out, double *resid_out,
                  hq_status *st_out) {
    if (x->solo_failed || !x->use_graphs || x->timing) return false;
    if (!x->solo) {
        x->solo = new hq_batch();
        x->solo->ctx.assign(1, x);
        x->solo->gen.assign(1, -1);
        x->solo->st = x->st;
    }
    hq_batch *b = x->solo;
    if (!b->exec || b->gen[0] != x->gen) {
        if (cudaStreamSynchronize(x->st) != cudaSuccess) return false;
        if (batch_build(b) != HQ_OK) {
            x->solo_failed = true;
            cudaGetLastError();
            x->err.clear();
            return false;
        }
    }
    long steps = 0;
    double g = NAN;
    int stk = HQ_OK;
    const double tmo = x->cfg.timeout_s > 0 ? x->cfg.timeout_s : 0.0;
    hq_status st = batch_run(b, 0, &eps, max_steps, tmo, &steps, &g, &stk);
    if (st == HQ_OK || stk != HQ_OK) st = (hq_status)stk;
    else if (x->err.empty()) x->err = b->err;
    if (steps_out) *steps_out = steps;
    if (resid_out) *resid_out = g;
    *st_out = st;
    return true;
}

template <typename T>
hq_status solve_impl(hq_ctx *x, double eps, long max_steps, long *steps_out, double *resid_out) {
    HQ_TRY(need_ready(x));
    HQ_TRY(clear_status(x));
    hq_status dst = HQ_OK;
    if (solve_device(x, eps, max_steps, steps_out, resid_out, &dst)) return dst;
    auto t0 = std::chrono::steady_clock::now();
    long taken = 0;
    double g = NAN;
    hq_status st = HQ_OK;
    for (;;) {
        st = phase_a<T>(x);
        if (st != HQ_OK) break;
        st = read_g(x, &g);
        if (st != HQ_OK) break;
        if (g < eps) break;
        if (taken >= max_steps) {
            st = fail(x, HQ_ERR_NOT_CONVERGED, "Algorithm 1 reached max_steps");
            break;
        }
        if (x->cfg.timeout_s > 0) {
            double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > x->cfg.timeout_s) {
                st = fail(x, HQ_ERR_TIMEOUT, "hq_solve wall-clock limit reached");
                break;
            }
        }
        st = phase_b<T>(x);
        if (st != HQ_OK) break;
        taken++;
    }
    if (st == HQ_OK) st = graph_status(x);
    if (steps_out) *steps_out = taken;
    if (resid_out) *resid_out = g;
    return st;
}

template <typename T>
hq_status eigen_impl(hq_ctx *x, double *evals_paper, double *evals_rr, double *evecs,
                     int evecs_on_device, double *resid) {
    HQ_TRY(need_ready(x));
    HQ_TRY(clear_status(x));
    const int N = x->N;
    const size_t cnt = (size_t)x->n * N;
    if (!x->w_valid) HQ_TRY(phase_a<T>(x));
    // eigenvalues of <G U, U>^{-1} (Section 5), shifted back
    launch_extract(N, N, 1.0, x->G2 + (size_t)N * 2 * N, 2 * N, x->Ksm, N, x->st);
    launch_sym_eig(N, x->Ksm, x->eigwork, x->mu, nullptr, x->st);
    launch_paper_evals(N, x->mu, x->sigma, x->lam_p, x->st);
    // FP64 Rayleigh-Ritz of H on span(U)
    double *U64 = (double *)x->U;
    if (x->mixed) {
        launch_convert_f2d(cnt, (const float *)x->U, x->E1, x->st);
        U64 = x->E1;
    }
    Level &v0 = x->lev[0];
    GridGeom g64 = make_geom(x->m, N, 8);
    launch_apply<double>(g64, v0.D, v0.c, U64, x->E2, nullptr, x->st);   // (H + sigma) U
    GramPlan gk = make_gram_plan(x->n, N, N, false);
    GramPlan gs = make_gram_plan(x->n, N, N, true);
    launch_gram<double>(gk, U64, N, nullptr, 0, x->E2, N, nullptr, 0, x->h3, x->gpart, x->Ksm, x->st);
    launch_gram<double>(gs, U64, N, nullptr, 0, U64, N, nullptr, 0, x->h3, x->gpart, x->Ssm, x->st);
    launch_axpy_small(N * N, -x->sigma, x->Ssm, x->Ksm, x->st);   // <U, H U>
    launch_rr_reduce(N, x->Ksm, x->Ssm, x->Lm, x->Cm, x->status, x->st);
    HQ_TRY(sync_status(x, x->status, "Rayleigh-Ritz (Cholesky of <U,U>)"));
    launch_sym_eig(N, x->Cm, x->eigwork, x->lam_r, x->Ym, x->st);
    launch_rr_back(N, x->Lm, x->Ym, x->Cv, x->st);
    TallPlan tp = make_tall_plan(x->n, N, N, N);
    if (evecs || resid) {
        double *X = (evecs && evecs_on_device) ? evecs : x->E3;
        launch_tall_gemm<double>(tp, U64, x->Cv, nullptr, nullptr, nullptr, X, nullptr, x->st);
        launch_fix_signs<double>(x->n, N, X, x->signwork, x->st);
        if (evecs && !evecs_on_device)
            HQ_CUDA(cudaMemcpyAsync(evecs, X, cnt * sizeof(double), cudaMemcpyDeviceToHost, x->st));
        if (resid) {
            launch_scale_cols(N, x->Cv, x->lam_r, x->sigma, x->Cv2, x->st);
            launch_tall_gemm_colsq<double>(tp, x->E2, x->Cv, U64, x->Cv2, nullptr, nullptr,
                                           x->tpart, x->st);
            launch_colsum_sqrt(tp.gy, N, x->tpart, x->h3, x->resn, x->st);
            HQ_CUDA(cudaMemcpyAsync(resid, x->resn, sizeof(double) * N, cudaMemcpyDeviceToHost, x->st));
        }
    }
    if (evals_paper)
        HQ_CUDA(cudaMemcpyAsync(evals_paper, x->lam_p, sizeof(double) * N, cudaMemcpyDeviceToHost, x->st));
    if (evals_rr)
        HQ_CUDA(cudaMemcpyAsync(evals_rr, x->lam_r, sizeof(double) * N, cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return check_launch(x);
}

template <typename T>
hq_status monitor_impl(hq_ctx *x, double *energy, double *onorm, double *smin, double *smax) {
    HQ_TRY(need_ready(x));
    HQ_TRY(clear_status(x));
    const int N = x->N;
    const size_t cnt = (size_t)x->n * N;
    double *U64 = (double *)x->U;
    if (x->mixed) {
        launch_convert_f2d(cnt, (const float *)x->U, x->E1, x->st);
        U64 = x->E1;
    }
    Level &v0 = x->lev[0];
    GridGeom g64 = make_geom(x->m, N, 8);
    // tr(U^T (H + sigma) U) as per-column partial dots, fused into the operator
    launch_apply<double>(g64, v0.D, v0.c, U64, x->E2, x->part, x->st);
    GramPlan gs = make_gram_plan(x->n, N, N, true);
    launch_gram<double>(gs, U64, N, nullptr, 0, U64, N, nullptr, 0, x->h3, x->gpart, x->Ssm, x->st);
    launch_monitor_finish(g64.gy * N, x->part, x->h3, N, x->Ssm, x->scal + 4, x->st);
    launch_sym_eig(N, x->Ssm, x->eigwork, x->evals, nullptr, x->st);
    double e2[2], ev_lo = 0, ev_hi = 0;
    HQ_CUDA(cudaMemcpyAsync(e2, x->scal + 4, sizeof(e2), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaMemcpyAsync(&ev_lo, x->evals, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaMemcpyAsync(&ev_hi, x->evals + N - 1, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    HQ_TRY(check_launch(x));
    // (1/2) h^3 tr(U^T H U) = (1/2) (h^3 tr(U^T (H + sigma) U) - sigma tr<U,U>)
    double trS = 0.0;
    {
        std::vector<double> S((size_t)N * N);
        HQ_CUDA(cudaMemcpyAsync(S.data(), x->Ssm, sizeof(double) * N * N, cudaMemcpyDeviceToHost, x->st));
        HQ_CUDA(cudaStreamSynchronize(x->st));
        for (int i = 0; i < N; i++) trS += S[(size_t)i * N + i];
    }
    if (energy) *energy = 0.5 * (e2[0] - x->sigma * trS);
    if (onorm) *onorm = e2[1];
    if (smin) *smin = ev_lo;
    if (smax) *smax = ev_hi;
    return HQ_OK;
}

template <typename T>
hq_status trace_impl(hq_ctx *x, void *W, double *gram, double *g, double *XY, void *Uh,
                     double *Shat, void *Z, void *Unew) {
    HQ_TRY(need_ready(x));
    HQ_TRY(clear_status(x));
    const int N = x->N;
    const size_t cnt = (size_t)x->n * N;
    HQ_TRY(phase_a<T>(x));
    double gh;
    HQ_TRY(read_g(x, &gh));
    if (W) HQ_CUDA(cudaMemcpyAsync(W, x->W, cnt * sizeof(T), cudaMemcpyDeviceToDevice, x->st));
    if (gram) HQ_CUDA(cudaMemcpyAsync(gram, x->G2, sizeof(double) * 4 * N * N, cudaMemcpyDeviceToDevice, x->st));
    if (g) HQ_CUDA(cudaMemcpyAsync(g, x->scal, sizeof(double), cudaMemcpyDeviceToDevice, x->st));
    HQ_TRY(phase_b<T>(x));
    if (XY) HQ_CUDA(cudaMemcpyAsync(XY, x->XY, sizeof(double) * 2 * N * N, cudaMemcpyDeviceToDevice, x->st));
    if (Uh) HQ_CUDA(cudaMemcpyAsync(Uh, x->Uh, cnt * sizeof(T), cudaMemcpyDeviceToDevice, x->st));
    if (Shat) HQ_CUDA(cudaMemcpyAsync(Shat, x->Shat, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, x->st));
    if (Z) HQ_CUDA(cudaMemcpyAsync(Z, x->Z, cnt * sizeof(T), cudaMemcpyDeviceToDevice, x->st));
    if (Unew) HQ_CUDA(cudaMemcpyAsync(Unew, x->U, cnt * sizeof(T), cudaMemcpyDeviceToDevice, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return check_launch(x);
}

template <typename T>
hq_status level_check(hq_ctx *x, int level, bool need_next) {
    if (!x->have_V) return fail(x, HQ_ERR_STATE, "hq_set_potential has not been called");
    if (level < 0 || level >= x->L || (need_next && level + 1 >= x->L))
        return fail(x, HQ_ERR_ARG, "multigrid level out of range");
    return HQ_OK;
}

// ---------------------------------------------------------------------------
// differentiation (FP64 contexts)
// ---------------------------------------------------------------------------
// y <- P y = y - u (h^3 u^T y), u = Ritz vectors (in Uh).  u^T y by the
// SIMT FP64 Gram for solves to rtol below 1e-8: y is kept in range(P), so
// u^T y is at the rounding level of |u| |y|, while the digit-sliced
// tensor-core Gram's error is bounded by the columns' largest entries times
// the number of points (~3e-11 of |u| |y| at 64^3 for localised u), which let
// the Krylov space of a 1e-11 adjoint solve leak into span(u) and stall.  A
// looser solve (the refinement's inexact Newton steps) takes the tensor-core
// Gram of [u y] (rows 0..N-1, columns N..2N-1 of the 2N x 2N result, in the
// predictor scratch, unused outside a step).
hq_status project(hq_ctx *x, double *y, double rtol = 0.0) {
    const int N = x->N;
    const double *u = (const double *)x->Uh;
    const double na = 2.0 * N;
    if (rtol >= 1e-8 && x->ozgram && gram_oz_supported(2 * N) &&
        use_oz(x, 0.5 * (double)x->n * na * na)) {
        // only the block <u, y> is used: the Gram's columns of y (the column
        // tiles from y's first column on)
        launch_gram_oz(x->n, u, N, y, N, x->h3, x->ozgram, x->Mw, x->status, x->st, N);
        launch_extract(N, N, -1.0, x->Mw + N, 2 * N, x->Msm, N, x->st);
    } else {
        GramPlan gp = make_gram_plan(x->n, N, N, false);
        launch_gram<double>(gp, u, N, nullptr, 0, y, N, nullptr, 0, x->h3, x->gpart, x->Ksm, x->st);
        launch_extract(N, N, -1.0, x->Ksm, N, x->Msm, N, x->st);
    }
    block_gemm<double>(x, u, N, x->Msm, nullptr, 0, nullptr, y, y, false, nullptr);
    return check_launch(x);
}

hq_status need_fp64(hq_ctx *x) {
    if (x->mixed) return fail(x, HQ_ERR_STATE, "differentiation needs an HQ_FP64 context");
    return need_ready(x);
}

// Ritz vectors into Uh, Ritz values into lam_r (device)
hq_status ritz(hq_ctx *x) {
    return eigen_impl<double>(x, nullptr, nullptr, (double *)x->Uh, 1, nullptr);
}

hq_status density_impl(hq_ctx *x, double *rho_out, int on_device) {
    HQ_TRY(need_fp64(x));
    HQ_TRY(ritz(x));
    launch_rowreduce(0, x->n, x->N, (const double *)x->Uh, nullptr, nullptr, 1.0, x->vn[0], x->st);
    HQ_CUDA(cudaMemcpyAsync(rho_out, x->vn[0], sizeof(double) * x->n, kind_out(on_device), x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return check_launch(x);
}

hq_status grad_eigs_impl(hq_ctx *x, const double *w, double *dV, int on_device) {
    HQ_TRY(need_fp64(x));
    HQ_TRY(ritz(x));
    const double *wd = nullptr;
    if (w) {
        HQ_CUDA(cudaMemcpyAsync(x->mu, w, sizeof(double) * x->N, cudaMemcpyHostToDevice, x->st));
        wd = x->mu;
    }
    launch_rowreduce(0, x->n, x->N, (const double *)x->Uh, nullptr, wd, x->h3, x->vn[0], x->st);
    HQ_CUDA(cudaMemcpyAsync(dV, x->vn[0], sizeof(double) * x->n, kind_out(on_device), x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return check_launch(x);
}

// Projected, column-shifted block PCG (FP64 contexts): xi_i in range(P) with
//   P (A - s_i) P xi_i = b_i,   b_i in range(P),   A = H + sigma,
// P = I - u (h^3 u^T) the projector onto the complement of the Ritz vectors u
// (in Uh), shifts s (device, N values), preconditioner P M P with M the
// V-cycle of A, xi_0 = 0, column i stopped at ||r_i|| <= rtol ||b_i||.  b is
// kept; the PCG blocks R, Zp, P, Q, Tt are overwritten.  P (A - s_i) P is
// positive definite on range(P) when s_i lies below the spectrum of A on the
// complement of span(u).  *iters: iterations run.
hq_status projected_pcg(hq_ctx *x, const double *b, double *xi, const double *shifts, double rtol,
                        int maxit, int *iters, const char *what) {
    const int N = x->N;
    const long n = x->n;
    const size_t cnt = (size_t)n * N;
    Level &v = x->lev[0];
    const GridGeom &g = v.g;
    double *R = (double *)x->R, *Zp = (double *)x->Zp, *P = (double *)x->P, *Q = (double *)x->Q,
           *Tt = (double *)x->Tt;
    PcgScalars sc = x->sc;
    HQ_CUDA(cudaMemsetAsync(xi, 0, cnt * sizeof(double), x->st));
    HQ_TRY(copy_blk<double>(x, R, b, cnt));
    HQ_CUDA(cudaMemsetAsync(sc.num_active, 0, sizeof(int), x->st));
    launch_dot<double>(g, R, R, x->part, x->st);
    launch_dot<double>(g, b, b, x->part2, x->st);
    launch_finalize(FIN_BNORM_RNORM, N, g.gy, x->part, x->part2, sc, rtol, x->st);
    int nact = 0, it = 0;
    HQ_CUDA(cudaMemcpyAsync(&nact, sc.num_active, sizeof(int), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    if (nact > 0) {
        HQ_TRY(precondition<double>(x, R, Zp, Tt, false, nullptr));
        HQ_TRY(project(x, Zp, rtol));
        launch_dot<double>(g, R, Zp, x->part, x->st);
        launch_finalize(FIN_RZ, N, g.gy, x->part, nullptr, sc, rtol, x->st);
        HQ_TRY(copy_blk<double>(x, P, Zp, cnt));
        for (it = 1; it <= maxit; it++) {
            launch_apply<double>(g, v.D, v.c, P, Q, nullptr, x->st);
            launch_shift_cols(n, N, shifts, P, Q, x->st);
            HQ_TRY(project(x, Q, rtol));
            launch_dot<double>(g, P, Q, x->part, x->st);
            launch_finalize(FIN_ALPHA, N, g.gy, x->part, nullptr, sc, rtol, x->st);
            launch_pcg_xr<double>(g, sc.alpha, P, Q, xi, R, x->part, v.wD, nullptr, x->st);
            HQ_CUDA(cudaMemsetAsync(sc.num_active, 0, sizeof(int), x->st));
            launch_finalize(FIN_RR, N, g.gy, x->part, nullptr, sc, rtol, x->st);
            HQ_CUDA(cudaMemcpyAsync(&nact, sc.num_active, sizeof(int), cudaMemcpyDeviceToHost, x->st));
            HQ_CUDA(cudaStreamSynchronize(x->st));
            if (nact == 0) break;
            HQ_TRY(precondition<double>(x, R, Zp, Tt, false, nullptr));
            HQ_TRY(project(x, Zp, rtol));
            launch_dot<double>(g, R, Zp, x->part, x->st);
            launch_finalize(FIN_BETA, N, g.gy, x->part, nullptr, sc, rtol, x->st);
            launch_pcg_p<double>(g, sc.beta, Zp, P, x->st);
        }
    }
    if (iters) *iters = it > maxit ? maxit : it;
    HQ_TRY(sync_status(x, sc.status, what));
    HQ_TRY(sync_status(x, x->status, what));   // tensor-core projections
    if (nact > 0) return fail(x, HQ_ERR_NOT_CONVERGED, std::string(what) + " reached maxit");
    return HQ_OK;
}

hq_status grad_density_impl(hq_ctx *x, const double *G, const double *rho_target, int on_device,
                            double rtol, int maxit, double *dV, double *loss, int *iters) {
    HQ_TRY(need_fp64(x));
    HQ_TRY(clear_status(x));
    HQ_TRY(ritz(x));
    const int N = x->N;
    const long n = x->n;
    const double *u = (const double *)x->Uh;
    double *Gd = x->vn[1];
    if (rho_target) {
        // G = h^3 (rho - rho_target), L = (1/2) h^3 sum (rho - rho_target)^2
        launch_rowreduce(0, n, N, u, nullptr, nullptr, 1.0, x->vn[0], x->st);
        HQ_CUDA(cudaMemcpyAsync(x->vn[2], rho_target, sizeof(double) * n, kind_in(on_device), x->st));
        int np = launch_diff_sq(n, x->vn[0], x->vn[2], Gd, x->tpart, x->st);
        launch_monitor_finish(np, x->tpart, 0.5 * x->h3, 0, nullptr, x->scal + 6, x->st);
        launch_dscale((int)n, x->h3, Gd, Gd, x->st);
    } else {
        if (!G) return fail(x, HQ_ERR_ARG, "G and rho_target are both null");
        HQ_CUDA(cudaMemcpyAsync(Gd, G, sizeof(double) * n, kind_in(on_device), x->st));
    }
    // right-hand sides b_i = P (G o u_i) in Z; shifts s_i = lambda_i + sigma
    double *b = (double *)x->Z, *xi = (double *)x->W;
    launch_scale_rows(n, N, Gd, u, b, x->st);
    HQ_TRY(project(x, b));
    launch_add_scalar(N, x->lam_r, x->sigma, x->mu, x->st);
    int it = 0;
    hq_status st = projected_pcg(x, b, xi, x->mu, rtol, maxit, &it, "adjoint PCG");
    // the step buffers W and Z now hold adjoint data
    x->w_valid = false;
    x->z_valid = false;
    if (iters) *iters = it;
    HQ_TRY(st);
    // dL/dV = -2 sum_i u_i o xi_i
    launch_rowreduce(1, n, N, u, xi, nullptr, -2.0, x->vn[0], x->st);
    HQ_CUDA(cudaMemcpyAsync(dV, x->vn[0], sizeof(double) * n, kind_out(on_device), x->st));
    if (loss) {
        *loss = 0.0;
        if (rho_target)
            HQ_CUDA(cudaMemcpyAsync(loss, x->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    }
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return check_launch(x);
}

// FP64 Rayleigh-Ritz of H on span(U) without the phase-A solve that
// hq_eigenpairs runs for Section 5's values: Ritz values (ascending) into
// lam_r, <.,.>-orthonormal, sign-fixed Ritz vectors into Uh.  FP64 contexts.
hq_status rayleigh_ritz_vectors(hq_ctx *x) {
    const int N = x->N;
    double *U64 = (double *)x->U;
    Level &v0 = x->lev[0];
    launch_apply<double>(v0.g, v0.D, v0.c, U64, x->E2, nullptr, x->st);   // (H + sigma) U
    GramPlan gk = make_gram_plan(x->n, N, N, false);
    GramPlan gs = make_gram_plan(x->n, N, N, true);
    launch_gram<double>(gk, U64, N, nullptr, 0, x->E2, N, nullptr, 0, x->h3, x->gpart, x->Ksm, x->st);
    launch_gram<double>(gs, U64, N, nullptr, 0, U64, N, nullptr, 0, x->h3, x->gpart, x->Ssm, x->st);
    launch_axpy_small(N * N, -x->sigma, x->Ssm, x->Ksm, x->st);   // <U, H U>
    launch_rr_reduce(N, x->Ksm, x->Ssm, x->Lm, x->Cm, x->status, x->st);
    HQ_TRY(sync_status(x, x->status, "Rayleigh-Ritz (Cholesky of <U,U>)"));
    launch_sym_eig(N, x->Cm, x->eigwork, x->lam_r, x->Ym, x->st);
    launch_rr_back(N, x->Lm, x->Ym, x->Cv, x->st);
    TallPlan tp = make_tall_plan(x->n, N, N, N);
    launch_tall_gemm<double>(tp, U64, x->Cv, nullptr, nullptr, nullptr, (double *)x->Uh, nullptr,
                             x->st);
    launch_fix_signs<double>(x->n, N, (double *)x->Uh, x->signwork, x->st);
    return check_launch(x);
}

// FP64 residual refinement (not in the paper; the final FP64 refinement of a
// lower-precision result).  Each round: Ritz pairs (theta_i, u_i) of span(U);
// r_i = H u_i - theta_i u_i; corrections t_i in the complement of span(u)
// from P (A - s_i) P t_i = -r_i, s_i = theta_i + sigma (Newton's equation for
// an invariant subspace in the Ritz basis, one equation per column), by the
// projected PCG; U <- u + t.  A last Rayleigh-Ritz leaves U = the Ritz
// vectors.  The warm start of the next inner solve is dropped.
hq_status refine_impl(hq_ctx *x, int rounds, double rtol, int maxit, double *resid,
                      int *iters_out) {
    HQ_TRY(need_ready(x));
    if (x->mixed) return fail(x, HQ_ERR_STATE, "hq_refine needs an HQ_FP64 context");
    if (rounds < 0 || maxit < 1 || !(rtol > 0.0)) return fail(x, HQ_ERR_ARG, "rounds >= 0, maxit >= 1, rtol > 0");
    HQ_TRY(clear_status(x));
    const int N = x->N;
    const long n = x->n;
    const size_t cnt = (size_t)n * N;
    Level &v = x->lev[0];
    double *u = (double *)x->Uh, *b = (double *)x->Z, *t = (double *)x->W;
    int total = 0;
    hq_status st = HQ_OK;
    for (int k = 0; k < rounds && st == HQ_OK; k++) {
        st = rayleigh_ritz_vectors(x);
        if (st != HQ_OK) break;
        launch_add_scalar(N, x->lam_r, x->sigma, x->mu, x->st);
        // b = -(A u - s u) = -(H u_i - theta_i u_i), projected
        launch_apply<double>(v.g, v.D, v.c, u, b, nullptr, x->st);
        launch_shift_cols(n, N, x->mu, u, b, x->st);
        launch_axpby(cnt, -1.0, b, 0.0, b, b, x->st);
        st = project(x, b, rtol);
        if (st != HQ_OK) break;
        int it = 0;
        st = projected_pcg(x, b, t, x->mu, rtol, maxit, &it, "refinement PCG");
        total += it;
        if (st != HQ_OK) break;
        launch_axpby(cnt, 1.0, u, 1.0, t, (double *)x->U, x->st);
    }
    x->w_valid = false;
    x->z_valid = false;
    if (iters_out) *iters_out = total;
    HQ_TRY(st);
    HQ_TRY(rayleigh_ritz_vectors(x));
    HQ_TRY(copy_blk<double>(x, (double *)x->U, u, cnt));
    if (resid) {
        // ||H u_i - theta_i u_i|| of the final Ritz pairs
        launch_add_scalar(N, x->lam_r, x->sigma, x->mu, x->st);
        launch_apply<double>(v.g, v.D, v.c, u, b, nullptr, x->st);
        launch_shift_cols(n, N, x->mu, u, b, x->st);
        GramPlan gp = make_gram_plan(n, N, N, true);
        launch_gram<double>(gp, b, N, nullptr, 0, b, N, nullptr, 0, x->h3, x->gpart, x->Ksm, x->st);
        std::vector<double> K((size_t)N * N);
        HQ_CUDA(cudaMemcpyAsync(K.data(), x->Ksm, sizeof(double) * N * N, cudaMemcpyDeviceToHost, x->st));
        HQ_CUDA(cudaStreamSynchronize(x->st));
        for (int i = 0; i < N; i++) resid[i] = std::sqrt(std::max(0.0, K[(size_t)i * N + i]));
    }
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return check_launch(x);
}

#define HQ_DISPATCH(x, fn, ...) ((x)->mixed ? fn<float>(__VA_ARGS__) : fn<double>(__VA_ARGS__))

template <typename T>
hq_status apply_impl(hq_ctx *x, const void *in, void *out, int ncol) {
    Level &v = x->lev[0];
    // N columns: the block PCG's own operator launch (its launch shape, the
    // per-column x.y partial sums formed into the PCG scratch); a plain launch
    // otherwise
    const bool own = ncol == x->N;
    GridGeom g = own ? v.g : make_geom(x->m, ncol, (int)sizeof(T));
    launch_apply<T>(g, (const T *)v.Dt, (T)v.c, (const T *)in, (T *)out, own ? x->part : nullptr,
                    x->st);
    return check_launch(x);
}
template <typename T>
hq_status vcycle_impl(hq_ctx *x, const void *r, void *z) {
    HQ_TRY(precondition<T>(x, (const T *)r, (T *)z, (T *)x->Tt, false, nullptr));
    return check_launch(x);
}
template <typename T>
hq_status pcg_impl(hq_ctx *x, const void *B, void *X, double rtol, int maxit, int *iters) {
    HQ_TRY(clear_status(x));
    return pcg<T>(x, (const T *)B, (T *)X, rtol, maxit, iters);
}
// The split over grid points of a Gram must fit the workspace's partial sums
// (sized for the step's own Gram shapes): otherwise fewer, longer point chunks.
hq_status fit_gram_plan(hq_ctx *x, GramPlan &gp) {
    const size_t avail = std::max(gram_partial_bytes(x->gplan_max), gram_partial_bytes(x->gplan_uw));
    if (gram_partial_bytes(gp) <= avail) return HQ_OK;
    const size_t per_chunk = sizeof(double) * (size_t)gp.ntiles * 64 * 64;
    const long max_chunks = (long)(avail / per_chunk);
    if (max_chunks < 1) return fail(x, HQ_ERR_ARG, "Gram shape exceeds the workspace plan");
    long rows = (x->n + max_chunks - 1) / max_chunks;
    rows = (rows + 15) / 16 * 16;
    gp.chunk_rows = rows;
    gp.chunks = (int)((x->n + rows - 1) / rows);
    if (gram_partial_bytes(gp) > avail)
        return fail(x, HQ_ERR_ARG, "Gram shape exceeds the workspace plan");
    return HQ_OK;
}

// O'Leary's block PCG (not in the paper; an alternative to the per-column
// recurrences of pcg()): X = G B with all N columns in one block Krylov space,
// N x N step matrices alpha = (P^T Q)^-1 (Z^T R), beta = (Z^T R)^-1 (Z'^T R'):
//   R = B - A X, Z = M R, P = Z
//   repeat: Q = A P, X += P alpha, R -= Q alpha, stop when every column has
//           ||r_j|| <= rtol ||b_j||, Z' = M R, P = Z' + P beta.
// The inner products are plain sums over the points (as the per-column
// PCG's), formed by the SIMT Gram with FP64 accumulation; the N x N systems
// by the FP64 SPD solves; the block updates by the step's block products.
// Host-driven (one synchronisation per iteration for the stopping test).
// rtol = 0 runs exactly maxit iterations.
template <typename T>
hq_status coupled_pcg_impl(hq_ctx *x, const T *B, T *X, double rtol, int maxit, int *iters_out) {
    HQ_TRY(clear_status(x));
    const int N = x->N;
    const long n = x->n;
    Level &v = x->lev[0];
    const GridGeom &g = v.g;
    T *R = (T *)x->R, *Z = (T *)x->Zp, *P = (T *)x->P, *Q = (T *)x->Q, *Tt = (T *)x->Tt;
    GramPlan gp = make_gram_plan(n, N, N, false);
    HQ_TRY(fit_gram_plan(x, gp));
    auto inner = [&](const T *A, const T *Bm, double *out) {
        launch_gram<T>(gp, A, N, nullptr, 0, Bm, N, nullptr, 0, 1.0, x->gpart, out, x->st);
    };
    std::vector<double> rn(N), bn(N);
    // R = B - A X with the partial sums of r.r and b.b
    launch_resid<T>(g, (const T *)v.Dt, (T)v.c, X, B, R, x->part, x->part2, x->st);
    launch_colsum_sqrt(part_rows(g), N, x->part, 1.0, x->resn, x->st);
    launch_colsum_sqrt(part_rows(g), N, x->part2, 1.0, x->mu, x->st);
    HQ_CUDA(cudaMemcpyAsync(rn.data(), x->resn, sizeof(double) * N, cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaMemcpyAsync(bn.data(), x->mu, sizeof(double) * N, cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    auto done = [&]() {
        if (!(rtol > 0.0)) return false;
        for (int c = 0; c < N; c++)
            if (!(rn[c] <= rtol * bn[c])) return false;
        return true;
    };
    int it = 0;
    if (!done() && maxit > 0) {
        HQ_TRY(precondition<T>(x, R, Z, Tt, false, nullptr));
        HQ_TRY(copy_blk<T>(x, P, Z, (size_t)n * N));
        inner(Z, R, x->Ssm);   // Z^T R
        for (it = 1; it <= maxit; it++) {
            launch_apply<T>(g, (const T *)v.Dt, (T)v.c, P, Q, nullptr, x->st);
            inner(P, Q, x->Ksm);   // P^T A P
            launch_spd_solve(N, x->Ksm, N, x->Ssm, N, x->Mw, x->Lm, x->Ym, x->ipiv, x->status,
                             x->st);   // alpha
            // X and R in place: the block products' epilogues read Cin and
            // write Out element by element in the same thread
            block_gemm<T>(x, P, N, x->Ym, nullptr, 0, nullptr, X, X, false, nullptr);
            launch_dscale(N * N, -1.0, x->Ym, x->Cm, x->st);
            block_gemm<T>(x, Q, N, x->Cm, nullptr, 0, nullptr, R, R, false, nullptr);
            launch_dot<T>(g, R, R, x->part, x->st);
            launch_colsum_sqrt(g.gy, N, x->part, 1.0, x->resn, x->st);
            HQ_CUDA(cudaMemcpyAsync(rn.data(), x->resn, sizeof(double) * N, cudaMemcpyDeviceToHost,
                                    x->st));
            HQ_TRY(sync_status(x, x->status, "block PCG (P^T A P)"));
            if (done()) break;
            HQ_TRY(precondition<T>(x, R, Z, Tt, false, nullptr));
            inner(Z, R, x->Msm);   // Z'^T R'
            launch_spd_solve(N, x->Ssm, N, x->Msm, N, x->Mw, x->Lm, x->Cv, x->ipiv, x->status,
                             x->st);   // beta
            // P' = Z' + P beta into Q's buffer (P is read while P' is written),
            // then the two buffers swap roles
            block_gemm<T>(x, P, N, x->Cv, nullptr, 0, nullptr, Z, Q, false, nullptr);
            std::swap(P, Q);
            HQ_CUDA(cudaMemcpyAsync(x->Ssm, x->Msm, sizeof(double) * N * N,
                                    cudaMemcpyDeviceToDevice, x->st));
        }
        if (it > maxit) it = maxit;
    }
    if (iters_out) *iters_out = it;
    HQ_TRY(sync_status(x, x->status, "block PCG"));
    // the step's warm starts refer to the PCG buffers no longer
    x->w_valid = false;
    if (rtol > 0.0 && !done()) return fail(x, HQ_ERR_NOT_CONVERGED, "block PCG reached maxit");
    return check_launch(x);
}

template <typename T>
hq_status gram_impl(hq_ctx *x, const void *A, int Na, const void *B, int Nb, double w, double *out) {
    if (x->mixed && A == B && Na == Nb) {
        // symmetric case of a mixed context: the tensor-core path of the step
        launch_gram_tc(x->n, (const float *)A, Na, nullptr, 0, w, x->tcpart, out, x->status, x->st);
        HQ_TRY(check_launch(x));
        return sync_status(x, x->status, "tensor-core Gram");
    }
    GramPlan gp = make_gram_plan(x->n, Na, Nb, A == B && Na == Nb);
    HQ_TRY(fit_gram_plan(x, gp));
    launch_gram<T>(gp, (const T *)A, Na, nullptr, 0, (const T *)B, Nb, nullptr, 0, w, x->gpart, out, x->st);
    return check_launch(x);
}
template <typename T>
hq_status block_gemm_impl(hq_ctx *x, const void *A1, int k1, const double *M1, const void *A2,
                          int k2, const double *M2, const void *Cin, void *Out) {
    HQ_TRY(clear_status(x));
    block_gemm<T>(x, (const T *)A1, k1, M1, (const T *)A2, k2, M2, (const T *)Cin, (T *)Out, false,
                  nullptr);
    HQ_TRY(check_launch(x));
    return sync_status(x, x->status, "block gemm");
}

template <typename T>
hq_status smooth_impl(hq_ctx *x, int l, const void *r, const void *zin, void *zout) {
    Level &v = x->lev[l];
    launch_jacobi<T>(v.g, (const T *)v.Dt, (const T *)v.wDt, (T)v.c, (T)(1.0 - x->cfg.mg_omega),
                     (const T *)r, (const T *)zin, (T *)zout, nullptr, x->st);
    return check_launch(x);
}
template <typename T>
hq_status restrict_impl(hq_ctx *x, int l, const void *rf, void *rc) {
    launch_restrict<T>(x->lev[l].m, x->lev[l + 1].m, x->N, x->lev[l].tab, (const T *)rf,
                       (T *)x->xt1, (T *)x->xt2, (T *)rc, x->st);
    return check_launch(x);
}
template <typename T>
hq_status prolong_impl(hq_ctx *x, int l, const void *ec, const void *efin, void *efout) {
    launch_prolong<T>(x->lev[l].m, x->lev[l + 1].m, x->N, x->lev[l].tab, (const T *)ec,
                      (T *)x->xt1, (T *)x->xt2, (const T *)efin, (T *)efout, x->st);
    return check_launch(x);
}
template <typename T>
hq_status coarse_impl(hq_ctx *x, const void *r, void *z) {
    launch_coarse_solve<T>(x->lev[x->L - 1].g, x->Ainv, (const T *)r, (T *)z, x->st);
    return check_launch(x);
}
template <typename T>
hq_status get_state_impl(hq_ctx *x, double *U, double *Zw, int on_device) {
    if (U) HQ_TRY(store_block<T>(x, U, (const T *)x->U, on_device));
    if (Zw) {
        if (!x->z_valid) return fail(x, HQ_ERR_STATE, "no warm-start block yet (no step taken)");
        HQ_TRY(store_block<T>(x, Zw, (const T *)x->Z, on_device));
    }
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return HQ_OK;
}
template <typename T>
hq_status set_state_impl(hq_ctx *x, const double *U, const double *Zw, int on_device) {
    HQ_TRY(load_block<T>(x, (T *)x->U, U, on_device));
    x->have_U = true;
    x->w_valid = false;
    x->z_valid = false;
    if (Zw) {
        HQ_TRY(load_block<T>(x, (T *)x->Z, Zw, on_device));
        x->z_valid = true;
    }
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return HQ_OK;
}

}  // namespace

// HQ_LOG=<path>: every hq_step call appends one JSON line to <path> (the
// context, its step counter, the steps taken, the gradient norm g, the inner
// PCG solves and iterations of the call, its wall time in ms, the status).
struct StepLog {
    FILE *f = nullptr;
    std::mutex mu;
    StepLog() {
        const char *p = std::getenv("HQ_LOG");
        if (p && *p) f = std::fopen(p, "a");
    }
    ~StepLog() {
        if (f) std::fclose(f);
    }
};
StepLog &step_log() {
    static StepLog l;
    return l;
}

// Every public call is an NVTX range named after the call (header-only NVTX:
// a no-op unless a profiler is attached), so a timeline shows the library's
// calls around their kernels.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#define HQ_API_BEGIN      \
    NvtxRange nvtx_(__func__); \
    try {
#define HQ_API_END                                                   \
    }                                                                \
    catch (...) {                                                    \
        return HQ_ERR_NOMEM;                                         \
    }

extern "C" {

void hq_default_config(hq_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->m = 0;
    c->lo = -6.0;
    c->hi = 6.0;
    c->nev = 0;
    c->tau = 0.4;
    c->shift = NAN;
    c->precision = HQ_FP64;
    c->cg_rtol = 1e-10;
    c->cg_maxit = 200;
    c->mg_nu1 = 2;
    c->mg_nu2 = 2;
    c->mg_coarsest = 4;
    c->mg_omega = 0.8;
    c->timeout_s = 0.0;
    c->z_warm_start = 1;
    c->adaptive_tau = 0;
    c->fp64_tc = 1;
    c->mg_fp32 = 0;
    c->tau_safety = 0.8;
    c->tau_max = 0.0;
}

size_t hq_workspace_bytes(const hq_config *cfg) {
    if (!valid_config(cfg, nullptr)) return 0;
    try {
        return carve(nullptr, cfg, nullptr);
    } catch (...) {
        return 0;
    }
}

hq_status hq_init(const hq_config *cfg, void *d_workspace, size_t bytes, void *cuda_stream,
                  hq_ctx **out) {
    HQ_API_BEGIN
    if (!out) return HQ_ERR_ARG;
    *out = nullptr;
    std::string why;
    if (!valid_config(cfg, &why)) return HQ_ERR_ARG;
    size_t need = carve(nullptr, cfg, nullptr);
    if (!d_workspace || bytes < need) return HQ_ERR_NOMEM;
    if (((uintptr_t)d_workspace & 255u) != 0) return HQ_ERR_ARG;
    hq_ctx *x = new hq_ctx();
    x->cfg = *cfg;
    x->mixed = cfg->precision == HQ_MIXED;
    x->esz = x->mixed ? 4 : 8;
    x->m = cfg->m;
    x->N = cfg->nev;
    x->n = (long)cfg->m * cfg->m * cfg->m;
    x->h = (cfg->hi - cfg->lo) / (cfg->m + 1);
    x->h3 = x->h * x->h * x->h;
    x->st = (cudaStream_t)cuda_stream;
    x->ws = (char *)d_workspace;
    x->ws_bytes = bytes;
    {
        const char *e = std::getenv("HQ_NO_GRAPHS");
        x->use_graphs = !(e && e[0] == '1');
    }
    carve(x, cfg, x->ws);
    x->fuse_l0 = fuse_level(x);
    x->level0_fits = fuse_level(x, false) == 0;
    // the status words and counters start cleared
    cudaError_t e = cudaMemsetAsync(x->sc.status, 0, sizeof(int), x->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->status, 0, sizeof(int), x->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->dcount, 0, sizeof(long long) * 24, x->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->sc.fcount, 0, sizeof(unsigned) * 16, x->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->st);
    if (x->mixed) hq::tc_prepare();
    hq::lu_prepare();
    hq::vcoarse_prepare();
    hq::lu32_prepare();
    if (x->ozimg || x->ozgram) hq::oz_prepare();
    if (e != cudaSuccess) {
        delete x;
        return HQ_ERR_CUDA;
    }
    *out = x;
    return HQ_OK;
    HQ_API_END
}

hq_status hq_set_potential(hq_ctx *x, const double *V, int on_device) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!V) return fail(x, HQ_ERR_ARG, "V is null");
    return HQ_DISPATCH(x, set_potential_impl, x, V, on_device);
    HQ_API_END
}

hq_status hq_set_initial(hq_ctx *x, const double *U0, int on_device) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!U0) return fail(x, HQ_ERR_ARG, "U0 is null");
    return HQ_DISPATCH(x, set_initial_impl, x, U0, on_device);
    HQ_API_END
}

hq_status hq_step(hq_ctx *x, int nsteps, double *resid_out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (nsteps < 0) return fail(x, HQ_ERR_ARG, "nsteps < 0");
    StepLog &lg = step_log();
    if (!lg.f) return HQ_DISPATCH(x, step_impl, x, nsteps, resid_out);
    // per-call record: the gradient norm is read back (one synchronisation)
    HQ_TRY(fold_graph_counts(x));
    const long s0 = x->stat_solves, i0 = x->stat_iters;
    const auto t0 = std::chrono::steady_clock::now();
    double g = NAN;
    const hq_status st = HQ_DISPATCH(x, step_impl, x, nsteps, &g);
    if (st == HQ_OK) HQ_CUDA(cudaStreamSynchronize(x->st));
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st == HQ_OK) HQ_TRY(fold_graph_counts(x));
    if (resid_out) *resid_out = g;
    std::lock_guard<std::mutex> lk(lg.mu);
    std::fprintf(lg.f,
                 "{\"ctx\": \"%p\", \"step\": %ld, \"nsteps\": %d, \"g\": %.17g, "
                 "\"pcg_solves\": %ld, \"pcg_iterations\": %ld, \"ms\": %.4f, \"status\": %d}\n",
                 (void *)x, x->step, nsteps, std::isfinite(g) ? g : -1.0, x->stat_solves - s0,
                 x->stat_iters - i0, ms, (int)st);
    std::fflush(lg.f);
    return st;
    HQ_API_END
}

hq_status hq_solve(hq_ctx *x, double eps, long max_steps, long *steps_out, double *resid_out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!(eps > 0.0) || max_steps < 0) return fail(x, HQ_ERR_ARG, "eps must be > 0, max_steps >= 0");
    return HQ_DISPATCH(x, solve_impl, x, eps, max_steps, steps_out, resid_out);
    HQ_API_END
}

hq_status hq_eigenpairs(hq_ctx *x, double *evals_paper, double *evals_rr, double *evecs,
                        int evecs_on_device, double *resid) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    return HQ_DISPATCH(x, eigen_impl, x, evals_paper, evals_rr, evecs, evecs_on_device, resid);
    HQ_API_END
}

hq_status hq_monitor(hq_ctx *x, double *energy, double *onorm, double *smin, double *smax) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    return HQ_DISPATCH(x, monitor_impl, x, energy, onorm, smin, smax);
    HQ_API_END
}

hq_status hq_density(hq_ctx *x, double *rho_out, int on_device) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!rho_out) return fail(x, HQ_ERR_ARG, "rho_out is null");
    return density_impl(x, rho_out, on_device);
    HQ_API_END
}

hq_status hq_grad_eigs(hq_ctx *x, const double *w, double *dV, int on_device) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!dV) return fail(x, HQ_ERR_ARG, "dV is null");
    return grad_eigs_impl(x, w, dV, on_device);
    HQ_API_END
}

hq_status hq_grad_density(hq_ctx *x, const double *G, const double *rho_target, int on_device,
                          double rtol, int maxit, double *dV, double *loss, int *iters) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!dV || !(rtol > 0.0) || maxit < 1) return fail(x, HQ_ERR_ARG, "bad argument");
    return grad_density_impl(x, G, rho_target, on_device, rtol, maxit, dV, loss, iters);
    HQ_API_END
}

hq_status hq_refine(hq_ctx *x, int rounds, double rtol, int maxit, double *resid, int *iters) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    return refine_impl(x, rounds, rtol, maxit, resid, iters);
    HQ_API_END
}

hq_status hq_get_state(hq_ctx *x, double *U, double *Zwarm, int on_device, long *step) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!x->have_U) return fail(x, HQ_ERR_STATE, "no iterate");
    HQ_TRY(HQ_DISPATCH(x, get_state_impl, x, U, Zwarm, on_device));
    if (step) *step = x->step;
    return HQ_OK;
    HQ_API_END
}

hq_status hq_set_state(hq_ctx *x, const double *U, const double *Zwarm, int on_device, long step) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!U || step < 0) return fail(x, HQ_ERR_ARG, "U is null or step < 0");
    HQ_TRY(HQ_DISPATCH(x, set_state_impl, x, U, Zwarm, on_device));
    x->step = step;
    return HQ_OK;
    HQ_API_END
}

hq_status hq_time_step(hq_ctx *x, double *tau) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    if (!tau) return fail(x, HQ_ERR_ARG, "tau is null");
    if (!x->cfg.adaptive_tau) {
        *tau = x->cfg.tau;
        return HQ_OK;
    }
    HQ_CUDA(cudaMemcpyAsync(tau, x->scal + 8, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    return HQ_OK;
    HQ_API_END
}

hq_status hq_problem_info(hq_ctx *x, double *h, double *sigma, int *levels, int *level_m) {
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (h) *h = x->h;
    if (sigma) *sigma = x->sigma;
    if (levels) *levels = x->L;
    if (level_m)
        for (int l = 0; l < x->L; l++) level_m[l] = x->lev[l].m;
    return HQ_OK;
}

hq_status hq_apply_operator(hq_ctx *x, const void *in, void *out, int ncol) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!x->have_V) return fail(x, HQ_ERR_STATE, "hq_set_potential has not been called");
    if (!in || !out || ncol < 1 || ncol > x->N) return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, apply_impl, x, in, out, ncol);
    HQ_API_END
}

hq_status hq_mg_vcycle(hq_ctx *x, const void *r, void *z) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!x->have_V) return fail(x, HQ_ERR_STATE, "hq_set_potential has not been called");
    if (!r || !z) return fail(x, HQ_ERR_ARG, "null operand");
    return HQ_DISPATCH(x, vcycle_impl, x, r, z);
    HQ_API_END
}

hq_status hq_block_pcg(hq_ctx *x, const void *B, void *X, double rtol, int maxit, int *iters) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!x->have_V) return fail(x, HQ_ERR_STATE, "hq_set_potential has not been called");
    if (!B || !X || maxit < 0 || !(rtol >= 0.0)) return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, pcg_impl, x, B, X, rtol, maxit, iters);
    HQ_API_END
}

hq_status hq_block_pcg_coupled(hq_ctx *x, const void *B, void *X, double rtol, int maxit,
                               int *iters) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!x->have_V) return fail(x, HQ_ERR_STATE, "hq_set_potential has not been called");
    if (!B || !X || maxit < 0 || !(rtol >= 0.0)) return fail(x, HQ_ERR_ARG, "bad operand");
    if (x->mixed) return coupled_pcg_impl<float>(x, (const float *)B, (float *)X, rtol, maxit, iters);
    return coupled_pcg_impl<double>(x, (const double *)B, (double *)X, rtol, maxit, iters);
    HQ_API_END
}

hq_status hq_gram(hq_ctx *x, const void *A, int Na, const void *B, int Nb, double w, double *out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!A || !B || !out || Na < 1 || Nb < 1 || Na > 2 * x->N || Nb > 2 * x->N)
        return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, gram_impl, x, A, Na, B, Nb, w, out);
    HQ_API_END
}

hq_status hq_block_gemm(hq_ctx *x, const void *A1, int k1, const double *M1, const void *A2,
                        int k2, const double *M2, const void *Cin, void *Out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!A1 || !M1 || !Out || k1 < 1 || k1 > x->N || k2 < 0 || k2 > x->N || (k2 > 0 && (!A2 || !M2)))
        return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, block_gemm_impl, x, A1, k1, M1, k2 > 0 ? A2 : nullptr, k2,
                       k2 > 0 ? M2 : nullptr, Cin, Out);
    HQ_API_END
}

hq_status hq_step_trace(hq_ctx *x, void *W, double *gram, double *g, double *XY, void *Uh,
                        double *Shat, void *Z, void *Unew) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    return HQ_DISPATCH(x, trace_impl, x, W, gram, g, XY, Uh, Shat, Z, Unew);
    HQ_API_END
}

hq_status hq_mg_smooth(hq_ctx *x, int level, const void *r, const void *z_in, void *z_out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    HQ_TRY(HQ_DISPATCH(x, level_check, x, level, false));
    if (!r || !z_in || !z_out || z_in == z_out) return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, smooth_impl, x, level, r, z_in, z_out);
    HQ_API_END
}

hq_status hq_mg_smooth_prescaled(hq_ctx *x, int level, const void *rt, const void *z_in,
                                 void *z_out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!x->rtilde) return fail(x, HQ_ERR_STATE, "the context's V-cycle does not pre-scale (mixed or mg_fp32)");
    HQ_TRY(level_check<double>(x, level, true));
    if (!rt || !z_in || !z_out || z_in == z_out) return fail(x, HQ_ERR_ARG, "bad operand");
    Level &v = x->mg[level];
    launch_jacobi_rt<double>(v.g, v.wcD, 1.0 - x->cfg.mg_omega, nullptr, (const double *)rt,
                             (const double *)z_in, (double *)z_out, nullptr, x->st);
    return check_launch(x);
    HQ_API_END
}

hq_status hq_mg_restrict(hq_ctx *x, int level, const void *rf, void *rc) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    HQ_TRY(HQ_DISPATCH(x, level_check, x, level, true));
    if (!rf || !rc) return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, restrict_impl, x, level, rf, rc);
    HQ_API_END
}

hq_status hq_mg_prolong(hq_ctx *x, int level, const void *ec, const void *ef_in, void *ef_out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    HQ_TRY(HQ_DISPATCH(x, level_check, x, level, true));
    if (!ec || !ef_in || !ef_out) return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, prolong_impl, x, level, ec, ef_in, ef_out);
    HQ_API_END
}

hq_status hq_mg_coarse_solve(hq_ctx *x, const void *r, void *z) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    if (!x->have_V) return fail(x, HQ_ERR_STATE, "hq_set_potential has not been called");
    if (!r || !z) return fail(x, HQ_ERR_ARG, "bad operand");
    return HQ_DISPATCH(x, coarse_impl, x, r, z);
    HQ_API_END
}

hq_status hq_mg_level_potential(hq_ctx *x, int level, double *V_out) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    ProfScope ps_(x);
    HQ_TRY(HQ_DISPATCH(x, level_check, x, level, false));
    if (!V_out) return fail(x, HQ_ERR_ARG, "bad operand");
    HQ_CUDA(cudaMemcpyAsync(V_out, x->lev[level].V, sizeof(double) * x->lev[level].n,
                            cudaMemcpyDeviceToDevice, x->st));
    return HQ_OK;
    HQ_API_END
}

hq_status hq_profile(hq_ctx *x, int timing) {
    HQ_TRY(guard(x));
    HQ_TRY(fold_graph_counts(x));
    for (int i = 0; i < HQ_K_NCLASS; i++) {
        x->launches[i] = 0;
        x->work[i] = 0.0;
    }
    x->stat_solves = x->stat_iters = 0;
    x->timing = timing != 0;
    x->evused = 0;
    x->evrec.clear();
    return HQ_OK;
}

hq_status hq_profile_read(hq_ctx *x, long *launches, double *ms, double *elements) {
    HQ_API_BEGIN
    HQ_TRY(guard(x));
    HQ_TRY(fold_graph_counts(x));
    HQ_CUDA(cudaStreamSynchronize(x->st));
    if (launches)
        for (int i = 0; i < HQ_K_NCLASS; i++) launches[i] = x->launches[i];
    if (elements)
        for (int i = 0; i < HQ_K_NCLASS; i++) elements[i] = x->work[i];
    if (ms) {
        for (int i = 0; i < HQ_K_NCLASS; i++) ms[i] = 0.0;
        for (auto &r : x->evrec) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, x->evpool[r.second], x->evpool[r.second + 1]) == cudaSuccess)
                ms[r.first] += t;
        }
    }
    return HQ_OK;
    HQ_API_END
}

hq_status hq_pcg_stats(hq_ctx *x, long *solves, long *iterations) {
    HQ_TRY(guard(x));
    HQ_TRY(fold_graph_counts(x));
    if (solves) *solves = x->stat_solves;
    if (iterations) *iterations = x->stat_iters;
    return HQ_OK;
}

const char *hq_last_error(hq_ctx *x) { return x ? x->err.c_str() : "null context"; }

const char *hq_status_string(hq_status s) {
    switch (s) {
    case HQ_OK: return "ok";
    case HQ_ERR_ARG: return "invalid argument";
    case HQ_ERR_STATE: return "call out of order";
    case HQ_ERR_CUDA: return "CUDA error";
    case HQ_ERR_NOMEM: return "insufficient workspace or host memory";
    case HQ_ERR_BREAKDOWN: return "inner CG breakdown";
    case HQ_ERR_SINGULAR: return "singular predictor system";
    case HQ_ERR_NOT_CONVERGED: return "not converged";
    case HQ_ERR_TIMEOUT: return "timeout";
    case HQ_ERR_NONFINITE: return "non-finite value";
    }
    return "unknown status";
}

void hq_destroy(hq_ctx *x) {
    if (!x) return;
    delete x->solo;
    delete x;
}

// ---------------------------------------------------------------------------
// launch-shape autotuner
// ---------------------------------------------------------------------------
static const int TUNE_BLOCKS[] = {64, 128, 256};
static const int TUNE_CTAS[] = {4, 8, 16, 32};

size_t hq_tune_workspace_bytes(const hq_config *cfg) {
    if (!valid_config(cfg, nullptr)) return 0;
    size_t need = 0;
    try {
        for (int b : TUNE_BLOCKS)
            for (int c : TUNE_CTAS) {
                hq_config t = *cfg;
                t.grid_block = b;
                t.grid_ctas = c;
                need = std::max(need, carve(nullptr, &t, nullptr));
            }
    } catch (...) {
        return 0;
    }
    return need;
}

hq_status hq_tune(const hq_config *cfg, void *d_workspace, size_t bytes, void *cuda_stream,
                  hq_config *tuned, double *ms_out) {
    HQ_API_BEGIN
    if (!cfg || !tuned) return HQ_ERR_ARG;
    const size_t need = hq_tune_workspace_bytes(cfg);
    if (need == 0) return HQ_ERR_ARG;
    if (!d_workspace || bytes < need) return HQ_ERR_NOMEM;
    const int m = cfg->m;
    const long n = (long)m * m * m;
    // harmonic potential on the configured box (timing input)
    std::vector<double> V((size_t)n);
    const double h = (cfg->hi - cfg->lo) / (m + 1);
    for (int k = 0; k < m; k++)
        for (int j = 0; j < m; j++)
            for (int i = 0; i < m; i++) {
                const double xx = cfg->lo + h * (i + 1), yy = cfg->lo + h * (j + 1),
                             zz = cfg->lo + h * (k + 1);
                V[(size_t)i + (size_t)m * (j + (size_t)m * k)] = 0.5 * (xx * xx + yy * yy + zz * zz);
            }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HQ_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HQ_ERR_CUDA;
    }
    const int iters = 10;
    double best = 1e300;
    hq_config best_cfg = *cfg;
    hq_status st = HQ_OK;
    for (int b : TUNE_BLOCKS) {
        for (int c : TUNE_CTAS) {
            hq_config t = *cfg;
            t.grid_block = b;
            t.grid_ctas = c;
            hq_ctx *x = nullptr;
            st = hq_init(&t, d_workspace, bytes, cuda_stream, &x);
            if (st != HQ_OK) break;
            {
                ProfScope ps_(x);
                st = hq_set_potential(x, V.data(), 0);
                const size_t cnt = (size_t)n * x->N;
                if (st == HQ_OK) {
                    if (x->mixed) launch_fill_hash<float>((long)cnt, 12345u, (float *)x->U, s);
                    else launch_fill_hash<double>((long)cnt, 12345u, (double *)x->U, s);
                    if (cudaMemsetAsync(x->W, 0, cnt * x->esz, s) != cudaSuccess) st = HQ_ERR_CUDA;
                }
                // one untimed solve (captures the PCG graph), then the timed one
                float ms = 0.f;
                for (int rep = 0; rep < 2 && st == HQ_OK; rep++) {
                    if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = HQ_ERR_CUDA;
                    if (st == HQ_OK)
                        st = x->mixed ? pcg<float>(x, (const float *)x->U, (float *)x->W, 0.0, iters, nullptr)
                                      : pcg<double>(x, (const double *)x->U, (double *)x->W, 0.0, iters, nullptr);
                    if (rep == 1 && st == HQ_OK) {
                        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                            st = HQ_ERR_CUDA;
                    }
                }
                if (st == HQ_OK && ms / iters < best) {
                    best = ms / iters;
                    best_cfg = t;
                }
            }
            hq_destroy(x);
            if (st != HQ_OK) break;
        }
        if (st != HQ_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HQ_OK) return st;
    *tuned = best_cfg;
    if (ms_out) *ms_out = best;
    return HQ_OK;
    HQ_API_END
}

hq_status hq_batch_create(hq_ctx *const *ctxs, int count, void *cuda_stream, hq_batch **out) {
    HQ_API_BEGIN
    if (!out) return HQ_ERR_ARG;
    *out = nullptr;
    if (!ctxs || count < 1 || count > BATCH_MAX) return HQ_ERR_ARG;
    for (int i = 0; i < count; i++) {
        if (!ctxs[i]) return HQ_ERR_ARG;
        for (int j = 0; j < i; j++)
            if (ctxs[j] == ctxs[i]) return HQ_ERR_ARG;
    }
    hq_batch *b = new hq_batch();
    b->ctx.assign(ctxs, ctxs + count);
    b->gen.assign(count, -1);
    b->st = (cudaStream_t)cuda_stream;
    *out = b;
    return HQ_OK;
    HQ_API_END
}

hq_status hq_batch_solve(hq_batch *b, const double *eps, long max_steps, double timeout_s,
                         long *steps_out, double *resid_out, int *status_out) {
    HQ_API_BEGIN
    if (!b) return HQ_ERR_ARG;
    if (!eps || max_steps < 0 || timeout_s < 0 || !std::isfinite(timeout_s))
        return bfail(b, HQ_ERR_ARG, "bad argument");
    for (size_t k = 0; k < b->ctx.size(); k++)
        if (!(eps[k] > 0.0)) return bfail(b, HQ_ERR_ARG, "eps must be > 0");
    return batch_run(b, 0, eps, max_steps, timeout_s, steps_out, resid_out, status_out);
    HQ_API_END
}

hq_status hq_batch_step(hq_batch *b, long nsteps, double *resid_out, int *status_out) {
    HQ_API_BEGIN
    if (!b) return HQ_ERR_ARG;
    if (nsteps < 0) return bfail(b, HQ_ERR_ARG, "nsteps must be >= 0");
    return batch_run(b, 1, nullptr, nsteps, 0.0, nullptr, resid_out, status_out);
    HQ_API_END
}

hq_status hq_batch_launches(const hq_batch *b, long *batch_kernels, long *loop_iterations) {
    if (!b) return HQ_ERR_ARG;
    if (batch_kernels) *batch_kernels = b->launches;
    if (loop_iterations) *loop_iterations = b->loop_iters;
    return HQ_OK;
}

const char *hq_batch_last_error(const hq_batch *b) { return b ? b->err.c_str() : "null batch"; }

void hq_batch_destroy(hq_batch *b) { delete b; }

}  // extern "C"
