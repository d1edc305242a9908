// Dense kernels of the scheme: inner-product matrices <A,B> = w A^T B of
// tall-skinny blocks (split over grid points, fixed-order reduction), the
// block x small-matrix products of the predictor / corrector updates, and
// the small FP64 algebra (predictor system of Eq. (4.1) by LU with partial
// pivoting, cyclic Jacobi eigensolver, Rayleigh-Ritz reduction).
#include "hq_internal.cuh"

#include <algorithm>

namespace hq {

// ---------------------------------------------------------------------------
// Gram: out = w [A1 A2]^T [B1 B2], tiles of 64 x 64, split over point chunks.
// ---------------------------------------------------------------------------
constexpr int GT = 64;   // tile edge
constexpr int GK = 16;   // points per smem stage

GramPlan make_gram_plan(long n, int na, int nb, bool sym) {
    GramPlan p;
    p.n = n;
    p.na = na;
    p.nb = nb;
    p.sym = sym;
    p.tiles_a = (na + GT - 1) / GT;
    p.tiles_b = (nb + GT - 1) / GT;
    p.ntiles = sym ? p.tiles_a * (p.tiles_a + 1) / 2 : p.tiles_a * p.tiles_b;
    long target = std::max(1L, (long)(2 * 152) / p.ntiles);
    long maxchunks = std::max(1L, (n + GT - 1) / GT);
    long chunks = std::min(target, maxchunks);
    long rows = (n + chunks - 1) / chunks;
    rows = (rows + GK - 1) / GK * GK;
    p.chunk_rows = rows;
    p.chunks = (int)((n + rows - 1) / rows);
    return p;
}

size_t gram_partial_bytes(const GramPlan &p) {
    return sizeof(double) * (size_t)p.chunks * p.ntiles * GT * GT;
}

__device__ __forceinline__ void tile_of(int t, int tiles_a, bool sym, int &ta, int &tb) {
    if (!sym) {
        ta = t % tiles_a;
        tb = t / tiles_a;
        return;
    }
    // upper triangle, row-major over (ta <= tb)
    int r = 0, rem = t;
    while (rem >= tiles_a - r) {
        rem -= tiles_a - r;
        r++;
    }
    ta = r;
    tb = r + rem;
}

template <typename T>
__device__ __forceinline__ T gat(const T *X1, int n1, const T *X2, int n2, long p, int c) {
    return c < n1 ? X1[(size_t)p * n1 + c] : X2[(size_t)p * n2 + (c - n1)];
}

template <typename T>
__global__ void __launch_bounds__(256) k_gram_partial(GramPlan P, const T *A1, int na1,
                                                      const T *A2, int na2, const T *B1,
                                                      int nb1, const T *B2, int nb2,
                                                      double *partials) {
    __shared__ T As[GK][GT + 1];
    __shared__ T Bs[GK][GT + 1];
    const int tile = blockIdx.x, chunk = blockIdx.y;
    int ta, tb;
    tile_of(tile, P.tiles_a, P.sym, ta, tb);
    const int a0 = ta * GT, b0 = tb * GT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long r0 = (long)chunk * P.chunk_rows;
    const long r1 = (P.n < r0 + P.chunk_rows) ? P.n : r0 + P.chunk_rows;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);
    for (long p0 = r0; p0 < r1; p0 += GK) {
        for (int idx = threadIdx.x; idx < GK * GT; idx += 256) {
            int kk = idx / GT, c = idx % GT;
            long p = p0 + kk;
            int ca = a0 + c, cb = b0 + c;
            As[kk][c] = (p < r1 && ca < P.na) ? gat(A1, na1, A2, na2, p, ca) : T(0);
            Bs[kk][c] = (p < r1 && cb < P.nb) ? gat(B1, nb1, B2, nb2, p, cb) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk++) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
    double *dst = partials + ((size_t)chunk * P.ntiles + tile) * GT * GT;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) dst[(ty + 16 * i) * GT + tx + 16 * j] = (double)acc[i][j];
}

// one thread per tile entry (grid: tiles x entry blocks), chunks summed in order
__global__ void k_gram_reduce(GramPlan P, const double *partials, double w, double *out) {
    const int tile = blockIdx.x;
    int ta, tb;
    tile_of(tile, P.tiles_a, P.sym, ta, tb);
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= GT * GT) return;
    const int la = e / GT, lb = e % GT;
    const int a = ta * GT + la, b = tb * GT + lb;
    if (a >= P.na || b >= P.nb) return;
    double s = ordered_sum(partials + (size_t)tile * GT * GT + e, P.chunks, (size_t)P.ntiles * GT * GT);
    s *= w;
    out[(size_t)a * P.nb + b] = s;
    if (P.sym && ta != tb) out[(size_t)b * P.nb + a] = s;
}

template <typename T>
void launch_gram(const GramPlan &p, const T *A1, int na1, const T *A2, int na2, const T *B1,
                 int nb1, const T *B2, int nb2, double w, double *partials, double *out,
                 cudaStream_t s) {
    HQ_LAUNCH(HQ_K_GRAM, k_gram_partial<T><<<dim3(p.ntiles, p.chunks), 256, 0, s>>>(p, A1, na1, A2, na2, B1, nb1,
                                                               B2, nb2, partials));
    HQ_LAUNCH(HQ_K_GRAM, k_gram_reduce<<<dim3(p.ntiles, (GT * GT + 255) / 256), 256, 0, s>>>(
                             p, partials, w, out));
}

// ---------------------------------------------------------------------------
// Tall GEMM: Out = A1 M1 + A2 M2 + Cin (64 x 64 output tiles)
// ---------------------------------------------------------------------------
constexpr int TBP = 64, TBN = 64, TKC = 16;

TallPlan make_tall_plan(long n, int ncol, int k1, int k2) {
    TallPlan p;
    p.n = n;
    p.ncol = ncol;
    p.k1 = k1;
    p.k2 = k2;
    p.gx = (ncol + TBN - 1) / TBN;
    p.gy = (int)((n + TBP - 1) / TBP);
    return p;
}

template <typename T>
__global__ void __launch_bounds__(256) k_tall_gemm(TallPlan P, const T *A1, const double *M1,
                                                   const T *A2, const double *M2, const T *Cin,
                                                   T *Out, double *part_sq, int colwise) {
    __shared__ T As[TBP][TKC + 1];
    __shared__ T Ms[TKC][TBN + 1];
    __shared__ double red[256];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long p0 = (long)blockIdx.y * TBP;
    const int c0 = blockIdx.x * TBN;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);
    for (int pass = 0; pass < 2; pass++) {
        const T *A = pass == 0 ? A1 : A2;
        const double *M = pass == 0 ? M1 : M2;
        const int K = pass == 0 ? P.k1 : P.k2;
        if (A == nullptr || K == 0) continue;
        for (int k0 = 0; k0 < K; k0 += TKC) {
            for (int idx = threadIdx.x; idx < TBP * TKC; idx += 256) {
                int r = idx / TKC, kk = idx % TKC;
                long p = p0 + r;
                As[r][kk] = (p < P.n && k0 + kk < K) ? A[(size_t)p * K + k0 + kk] : T(0);
            }
            for (int idx = threadIdx.x; idx < TKC * TBN; idx += 256) {
                int kk = idx / TBN, c = idx % TBN;
                Ms[kk][c] = (k0 + kk < K && c0 + c < P.ncol)
                                ? (T)M[(size_t)(k0 + kk) * P.ncol + c0 + c]
                                : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < TKC; kk++) {
                T a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = As[ty + 16 * i][kk];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = Ms[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] += a[i] * b[j];
            }
            __syncthreads();
        }
    }
    double sq = 0.0;
    double sqc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        long p = p0 + ty + 16 * i;
        if (p >= P.n) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int c = c0 + tx + 16 * j;
            if (c >= P.ncol) continue;
            size_t e = (size_t)p * P.ncol + c;
            T v = acc[i][j];
            if (Cin) v = Cin[e] + v;
            if (Out) Out[e] = v;
            if (part_sq) {
                double dv = (double)v;
                sq += dv * dv;
                sqc[j] += dv * dv;
            }
        }
    }
    if (part_sq) {
        if (!colwise) {
            red[threadIdx.x] = sq;
            __syncthreads();
            for (int w = 128; w > 0; w >>= 1) {
                if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
                __syncthreads();
            }
            if (threadIdx.x == 0) part_sq[(size_t)blockIdx.y * P.gx + blockIdx.x] = red[0];
        } else {
            // per column: reduce over ty (16 rows of threads) in order
            for (int j = 0; j < 4; j++) {
                red[threadIdx.x] = sqc[j];
                __syncthreads();
                if (ty == 0) {
                    double s = 0.0;
                    for (int y = 0; y < 16; y++) s += red[y * 16 + tx];
                    int c = c0 + tx + 16 * j;
                    if (c < P.ncol) part_sq[(size_t)blockIdx.y * P.ncol + c] = s;
                }
                __syncthreads();
            }
        }
    }
}

template <typename T>
void launch_tall_gemm(const TallPlan &p, const T *A1, const double *M1, const T *A2,
                      const double *M2, const T *Cin, T *Out, double *part_sq,
                      cudaStream_t s) {
    HQ_LAUNCH(HQ_K_BLOCKGEMM, k_tall_gemm<T><<<dim3(p.gx, p.gy), 256, 0, s>>>(p, A1, M1, A2, M2, Cin, Out, part_sq, 0));
}
template <typename T>
void launch_tall_gemm_colsq(const TallPlan &p, const T *A1, const double *M1, const T *A2,
                            const double *M2, const T *Cin, T *Out, double *part_sq,
                            cudaStream_t s) {
    HQ_LAUNCH(HQ_K_BLOCKGEMM, k_tall_gemm<T><<<dim3(p.gx, p.gy), 256, 0, s>>>(p, A1, M1, A2, M2, Cin, Out, part_sq, 1));
}

__global__ void k_sum_sqrt(int np, const double *part, double w, double *out) {
    __shared__ double red[256];
    double s = strided_sum(part, np, threadIdx.x, 256);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(w * red[0]);
}
void launch_sum_sqrt(int np, const double *part, double w, double *out, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_REDUCE, k_sum_sqrt<<<1, 256, 0, s>>>(np, part, w, out));
}

__global__ void k_colsum_sqrt(int np, int ncol, const double *part, double w, double *out) {
    __shared__ double red[128];
    const int c = blockIdx.x;
    double s = strided_sum(part + c, np, threadIdx.x, 128, (size_t)ncol);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 64; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sqrt(w * red[0]);
}
void launch_colsum_sqrt(int np, int ncol, const double *part, double w, double *out,
                        cudaStream_t s) {
    HQ_LAUNCH(HQ_K_REDUCE, k_colsum_sqrt<<<ncol, 128, 0, s>>>(np, ncol, part, w, out));
}

// ---------------------------------------------------------------------------
// small FP64 algebra
// ---------------------------------------------------------------------------
__global__ void k_small_gemm(int M, int Nc, int K, double alpha, const double *A, int lda,
                             int ta, const double *B, int ldb, int tb, double beta, double *C,
                             int ldc) {
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)M * Nc;
         idx += (long)gridDim.x * blockDim.x) {
        int i = (int)(idx / Nc), j = (int)(idx % Nc);
        const double *ap = ta ? A + i : A + (size_t)i * lda;
        const double *bp = tb ? B + (size_t)j * ldb : B + j;
        const size_t as = ta ? (size_t)lda : 1, bs = tb ? 1 : (size_t)ldb;
        // k in order; the loads of eight terms issued ahead of their FMAs
        double s = 0.0;
        for (int k0 = 0; k0 < K; k0 += 8) {
            double a[8], b[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                a[u] = k0 + u < K ? ap[(size_t)(k0 + u) * as] : 0.0;
                b[u] = k0 + u < K ? bp[(size_t)(k0 + u) * bs] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (k0 + u < K) s += a[u] * b[u];
        }
        double c = beta == 0.0 ? 0.0 : beta * C[(size_t)i * ldc + j];
        C[(size_t)i * ldc + j] = c + alpha * s;
    }
}
void launch_small_gemm(int M, int Ncol, int K, double alpha, const double *A, int lda, bool ta,
                       const double *B, int ldb, bool tb, double beta, double *C, int ldc,
                       cudaStream_t s) {
    long tot = (long)M * Ncol;
    int blocks = (int)std::min<long>((tot + 255) / 256, 1024);
    HQ_LAUNCH(HQ_K_SMALL, k_small_gemm<<<blocks, 256, 0, s>>>(M, Ncol, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc));
}

// Predictor system of Eq. (4.1) (one CTA).
__global__ void __launch_bounds__(1024) k_predictor_solve(int N, double tau_arg, const double *G2,
                                                          double *Mw, double *XY, double *C,
                                                          int *status, const double *tau_dev) {
    const double tau = tau_dev ? tau_dev[0] : tau_arg;
    extern __shared__ double sh[];
    double *lcol = sh;                       // 2N
    double *rv = sh + 2 * N;                 // 1024 reduction values
    int *ri = (int *)(rv + 1024);            // 1024 reduction indices
    const int nn = 2 * N, ld2 = 2 * N;
    const int T = blockDim.x, tid = threadIdx.x;
    const int lx = tid & 31, wy = tid >> 5, NW = T >> 5;
    const double ht = 0.5 * tau;
    // build [I - tau/2 Puw, tau/2 S; -tau/2 Q, I + tau/2 Pwu] and [S; Pwu]
    for (long idx = tid; idx < (long)nn * nn; idx += T) {
        int i = (int)(idx / nn), j = (int)(idx % nn);
        double d = (i == j) ? 1.0 : 0.0;   // G2 rows / columns: [U W]
        double v;
        if (i < N && j < N) v = ht * G2[(size_t)i * ld2 + N + j] * -1.0 + d;     // I - tau/2 Puw
        else if (i < N) v = ht * G2[(size_t)i * ld2 + (j - N)];                  // tau/2 S
        else if (j < N) v = -ht * G2[(size_t)i * ld2 + N + j];                   // -tau/2 Q
        else v = d + ht * G2[(size_t)i * ld2 + (j - N)];                         // I + tau/2 Pwu
        Mw[idx] = v;
    }
    for (long idx = tid; idx < (long)nn * N; idx += T) {
        int i = (int)(idx / N), j = (int)(idx % N);
        XY[idx] = G2[(size_t)i * ld2 + j];   // rows 0..N-1: S; rows N..2N-1: Pwu
    }
    __syncthreads();
    for (int k = 0; k < nn; k++) {
        // pivot: max |M[i][k]|, i >= k, first index on ties
        double best = -1.0;
        int bi = nn;
        for (int i = k + tid; i < nn; i += T) {
            double v = fabs(Mw[(size_t)i * nn + k]);
            if (v > best) { best = v; bi = i; }
        }
        rv[tid] = best;
        ri[tid] = bi;
        __syncthreads();
        for (int w = T / 2; w > 0; w >>= 1) {
            if (tid < w) {
                double v2 = rv[tid + w];
                int i2 = ri[tid + w];
                if (v2 > rv[tid] || (v2 == rv[tid] && i2 < ri[tid])) { rv[tid] = v2; ri[tid] = i2; }
            }
            __syncthreads();
        }
        const int piv = ri[0];
        const double pval = rv[0];
        __syncthreads();
        if (!(pval > 0.0) || !isfinite(pval)) {
            if (tid == 0) atomicOr(status, ST_SINGULAR);
            return;
        }
        if (piv != k) {
            for (int j = tid; j < nn; j += T) {
                double t = Mw[(size_t)k * nn + j];
                Mw[(size_t)k * nn + j] = Mw[(size_t)piv * nn + j];
                Mw[(size_t)piv * nn + j] = t;
            }
            for (int j = tid; j < N; j += T) {
                double t = XY[(size_t)k * N + j];
                XY[(size_t)k * N + j] = XY[(size_t)piv * N + j];
                XY[(size_t)piv * N + j] = t;
            }
        }
        __syncthreads();
        const double dkk = Mw[(size_t)k * nn + k];
        for (int i = k + 1 + tid; i < nn; i += T) {
            double f = Mw[(size_t)i * nn + k] / dkk;
            Mw[(size_t)i * nn + k] = f;
            lcol[i] = f;
        }
        __syncthreads();
        // trailing update: rows by warp, columns by lane
        for (int i = k + 1 + wy; i < nn; i += NW) {
            const double f = lcol[i];
            for (int j = k + 1 + lx; j < nn; j += 32) Mw[(size_t)i * nn + j] -= f * Mw[(size_t)k * nn + j];
            for (int j = lx; j < N; j += 32) XY[(size_t)i * N + j] -= f * XY[(size_t)k * N + j];
        }
        __syncthreads();
    }
    // back substitution (column-oriented)
    for (int i = nn - 1; i >= 0; i--) {
        const double dii = Mw[(size_t)i * nn + i];
        for (int j = tid; j < N; j += T) XY[(size_t)i * N + j] /= dii;
        __syncthreads();
        for (int r = wy; r < i; r += NW) {
            const double u = Mw[(size_t)r * nn + i];
            for (int j = lx; j < N; j += 32) XY[(size_t)r * N + j] -= u * XY[(size_t)i * N + j];
        }
        __syncthreads();
    }
    // C = [I - tau Y; tau X]
    for (long idx = tid; idx < (long)N * N; idx += T) {
        int i = (int)(idx / N), j = (int)(idx % N);
        C[idx] = ((i == j) ? 1.0 : 0.0) - tau * XY[(size_t)(N + i) * N + j];
        C[(size_t)(N + i) * N + j] = tau * XY[idx];
    }
}

// ---------------------------------------------------------------------------
// Dense FP64 solve A X = B (A nn x nn, B nn x nrhs, both row-major and
// contiguous, overwritten): Gaussian elimination with partial pivoting on the
// augmented matrix [A | B] in panels of PB columns (pivot: largest |entry| in
// the column, first row on ties, as in the one-CTA kernels), then blocked
// back substitution.  Per panel: the panel factorisation (one CTA), row swaps
// + unit-lower triangular solve of the panel rows for every column to the
// right (one thread per column), the trailing update (64 x 64 tiles over many
// CTAs); per block of the back substitution: the diagonal triangle (one
// thread per right-hand side) and the update of the rows above (tiles).
// ---------------------------------------------------------------------------
constexpr int PB = 32;

__global__ void k_pred_build(int N, double tau_arg, const double *tau_dev, const double *G2,
                             double *Mw, double *XY) {
    const double tau = tau_dev ? tau_dev[0] : tau_arg;
    const double ht = 0.5 * tau;
    const int nn = 2 * N, ld2 = 2 * N;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)nn * nn + (long)nn * N;
         idx += (long)gridDim.x * blockDim.x) {
        if (idx < (long)nn * nn) {
            int i = (int)(idx / nn), j = (int)(idx % nn);
            double d = (i == j) ? 1.0 : 0.0;
            double v;
            if (i < N && j < N) v = ht * G2[(size_t)i * ld2 + N + j] * -1.0 + d;
            else if (i < N) v = ht * G2[(size_t)i * ld2 + (j - N)];
            else if (j < N) v = -ht * G2[(size_t)i * ld2 + N + j];
            else v = d + ht * G2[(size_t)i * ld2 + (j - N)];
            Mw[idx] = v;
        } else {
            long r = idx - (long)nn * nn;
            int i = (int)(r / N), j = (int)(r % N);
            XY[r] = G2[(size_t)i * ld2 + j];
        }
    }
}

// factorise columns [k0, k0 + nb) of rows [k0, nn): the panel is staged in
// shared memory (row stride nb + 1), pivots into ipiv
__global__ void __launch_bounds__(512) k_lu_panel(int nn, int k0, int nb, double *Mw, int *ipiv,
                                                  int *status) {
    extern __shared__ double P[];
    __shared__ double wv[16];
    __shared__ int wi[16];
    __shared__ int piv_s;
    __shared__ double pval_s;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = nn - k0, ld = nb + 1;
    for (int idx = tid; idx < R * nb; idx += T) {
        const int r = idx / nb, c = idx % nb;
        P[r * ld + c] = Mw[(size_t)(k0 + r) * nn + k0 + c];
    }
    __syncthreads();
    for (int jj = 0; jj < nb; jj++) {
        // pivot: largest |P[i][jj]|, i >= jj, first row on ties
        double best = -1.0;
        int bi = R;
        for (int r = jj + tid; r < R; r += T) {
            const double v = fabs(P[r * ld + jj]);
            if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_down_sync(0xffffffffu, best, o);
            const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
            if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
        }
        if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            const int nw = T >> 5;
            best = lane < nw ? wv[lane] : -1.0;
            bi = lane < nw ? wi[lane] : R;
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_down_sync(0xffffffffu, best, o);
                const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
            }
            if (lane == 0) { piv_s = bi; pval_s = best; }
        }
        __syncthreads();
        const int piv = piv_s;
        const double pval = pval_s;
        if (!(pval > 0.0) || !isfinite(pval)) {
            if (tid == 0) {
                atomicOr(status, ST_SINGULAR);
                for (int t = jj; t < nb; t++) ipiv[k0 + t] = k0 + t;
            }
            break;
        }
        if (tid == 0) ipiv[k0 + jj] = k0 + piv;
        if (piv != jj && tid < nb) {
            const double t = P[jj * ld + tid];
            P[jj * ld + tid] = P[piv * ld + tid];
            P[piv * ld + tid] = t;
        }
        __syncthreads();
        const double djj = P[jj * ld + jj];
        for (int r = jj + 1 + tid; r < R; r += T) P[r * ld + jj] = P[r * ld + jj] / djj;
        __syncthreads();
        // trailing part of the panel: lane = column, warps stride the rows, so
        // all warps share the FP64 work (each element sees the same
        // multiply-subtract sequence over jj as a row-per-thread loop)
        const int c = jj + 1 + lane;
        if (c < nb) {
            const double u = P[jj * ld + c];
            for (int r = jj + 1 + warp; r < R; r += (T >> 5)) P[r * ld + c] -= P[r * ld + jj] * u;
        }
        __syncthreads();
    }
    __syncthreads();
    for (int idx = tid; idx < R * nb; idx += T) {
        const int r = idx / nb, c = idx % nb;
        Mw[(size_t)(k0 + r) * nn + k0 + c] = P[r * ld + c];
    }
}

size_t lu_panel_smem(int nn, int nb) { return sizeof(double) * (size_t)nn * (nb + 1); }
int lu_block(int nn) { return nn > 768 ? 16 : PB; }

// columns right of the panel (matrix columns [k0+nb, nn), then the N RHS
// columns): the panel's row swaps in order, then the unit-lower solve with
// the panel's L11 staged in shared memory
__global__ void __launch_bounds__(128) k_lu_trsm(int nn, int N, int k0, int nb, double *Mw,
                                                 double *XY, const int *ipiv) {
    __shared__ double L[PB][PB + 1];
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int r = idx / nb, q = idx % nb;
        L[r][q] = Mw[(size_t)(k0 + r) * nn + k0 + q];
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncm = nn - k0 - nb;
    if (t >= ncm + N) return;
    double *col;
    size_t ld;
    if (t < ncm) { col = Mw + k0 + nb + t; ld = nn; }
    else { col = XY + (t - ncm); ld = N; }
    for (int j = 0; j < nb; j++) {
        const int piv = ipiv[k0 + j];
        if (piv != k0 + j) {
            double a = col[(size_t)(k0 + j) * ld], b = col[(size_t)piv * ld];
            col[(size_t)(k0 + j) * ld] = b;
            col[(size_t)piv * ld] = a;
        }
    }
    // the column's nb entries are loaded together, solved in registers and
    // stored together (same arithmetic as row-by-row)
    double x[PB];
#pragma unroll
    for (int r = 0; r < PB; r++)
        if (r < nb) x[r] = col[(size_t)(k0 + r) * ld];
#pragma unroll
    for (int r = 0; r < PB; r++) {
        if (r < nb) {
            double v = x[r];
#pragma unroll
            for (int q = 0; q < r; q++) v -= L[r][q] * x[q];
            x[r] = v;
        }
    }
#pragma unroll
    for (int r = 0; r < PB; r++)
        if (r < nb) col[(size_t)(k0 + r) * ld] = x[r];
}

// trailing update: rows [k0+nb, nn) of every column right of the panel
// (matrix and RHS) -= L21 (rows x nb) * U12 (nb x cols); 64 x 64 tiles
__global__ void __launch_bounds__(256) k_lu_update(int nn, int N, int k0, int nb, double *Mw,
                                                     double *XY) {
    __shared__ double Ls[64][PB + 1];
    __shared__ double Us[PB][64 + 1];
    const int r0 = k0 + nb + blockIdx.y * 64;
    const int ncm = nn - k0 - nb;
    const int c0 = blockIdx.x * 64;   // index over [matrix cols right of panel | RHS cols]
    const int tid = threadIdx.x;
    for (int idx = tid; idx < 64 * PB; idx += 256) {
        const int rr = idx / PB, q = idx % PB;
        const int row = r0 + rr;
        Ls[rr][q] = (row < nn && q < nb) ? Mw[(size_t)row * nn + k0 + q] : 0.0;
    }
    for (int idx = tid; idx < PB * 64; idx += 256) {
        const int q = idx / 64, cc = idx % 64;
        const int t = c0 + cc;
        double v = 0.0;
        if (q < nb && t < ncm + N)
            v = t < ncm ? Mw[(size_t)(k0 + q) * nn + k0 + nb + t] : XY[(size_t)(k0 + q) * N + (t - ncm)];
        Us[q][cc] = v;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    for (int a = 0; a < 4; a++) {
        const int rr = ty * 4 + a, row = r0 + rr;
        if (row >= nn) continue;
        for (int b = 0; b < 4; b++) {
            const int cc = tx * 4 + b, t = c0 + cc;
            if (t >= ncm + N) continue;
            double acc = 0.0;
            for (int q = 0; q < nb; q++) acc += Ls[rr][q] * Us[q][cc];
            double *dst = t < ncm ? &Mw[(size_t)row * nn + k0 + nb + t] : &XY[(size_t)row * N + (t - ncm)];
            *dst -= acc;
        }
    }
}

// back substitution, diagonal block [k0, k0+nb): X_b = U_bb^-1 Y_b (one thread
// per RHS column, U_bb staged in shared memory)
__global__ void __launch_bounds__(128) k_lu_back_diag(int nn, int N, int k0, int nb,
                                                      const double *Mw, double *XY) {
    __shared__ double Ub[PB][PB + 1];
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int r = idx / nb, q = idx % nb;
        Ub[r][q] = Mw[(size_t)(k0 + r) * nn + k0 + q];
    }
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    // loads first, the substitution in registers, stores last (same arithmetic)
    double x[PB];
#pragma unroll
    for (int r = 0; r < PB; r++)
        if (r < nb) x[r] = XY[(size_t)(k0 + r) * N + c];
#pragma unroll
    for (int r = PB - 1; r >= 0; r--) {
        if (r < nb) {
            double v = x[r];
#pragma unroll
            for (int q = r + 1; q < PB; q++)
                if (q < nb) v -= Ub[r][q] * x[q];
            x[r] = v / Ub[r][r];
        }
    }
#pragma unroll
    for (int r = 0; r < PB; r++)
        if (r < nb) XY[(size_t)(k0 + r) * N + c] = x[r];
}

// rows [0, k0): Y -= U[0:k0, k0:k0+nb] X_b (64 x 64 tiles)
__global__ void __launch_bounds__(256) k_lu_back_update(int nn, int N, int k0, int nb,
                                                          const double *Mw, double *XY) {
    __shared__ double Ls[64][PB + 1];
    __shared__ double Xs[PB][64 + 1];
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64, tid = threadIdx.x;
    for (int idx = tid; idx < 64 * PB; idx += 256) {
        const int rr = idx / PB, q = idx % PB, row = r0 + rr;
        Ls[rr][q] = (row < k0 && q < nb) ? Mw[(size_t)row * nn + k0 + q] : 0.0;
    }
    for (int idx = tid; idx < PB * 64; idx += 256) {
        const int q = idx / 64, cc = idx % 64, c = c0 + cc;
        Xs[q][cc] = (q < nb && c < N) ? XY[(size_t)(k0 + q) * N + c] : 0.0;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    for (int a = 0; a < 4; a++) {
        const int row = r0 + ty * 4 + a;
        if (row >= k0) continue;
        for (int b = 0; b < 4; b++) {
            const int c = c0 + tx * 4 + b;
            if (c >= N) continue;
            double acc = 0.0;
            for (int q = 0; q < nb; q++) acc += Ls[ty * 4 + a][q] * Xs[q][tx * 4 + b];
            XY[(size_t)row * N + c] -= acc;
        }
    }
}

// C = [I - tau Y; tau X]
__global__ void k_pred_c(int N, double tau_arg, const double *tau_dev, const double *XY,
                         double *C) {
    const double tau = tau_dev ? tau_dev[0] : tau_arg;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)N * N;
         idx += (long)gridDim.x * blockDim.x) {
        int i = (int)(idx / N), j = (int)(idx % N);
        C[idx] = ((i == j) ? 1.0 : 0.0) - tau * XY[(size_t)(N + i) * N + j];
        C[(size_t)(N + i) * N + j] = tau * XY[idx];
    }
}

void small_prepare();   // shared-memory limits of the staged small kernels (below)

void lu_prepare() {
    static bool done = false;
    if (done) return;
    small_prepare();
    cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)lu_panel_smem(768, PB));
    done = true;
}

void launch_lu_solve(int nn, int N, double *Mw, double *XY, int *ipiv, int *status,
                     cudaStream_t s) {
    const int bs = lu_block(nn);
    for (int k0 = 0; k0 < nn; k0 += bs) {
        const int nb = std::min(bs, nn - k0);
        HQ_LAUNCH(HQ_K_SMALL, k_lu_panel<<<1, 512, lu_panel_smem(nn - k0, nb), s>>>(nn, k0, nb, Mw,
                                                                                   ipiv, status));
        const int ncols = nn - k0 - nb + N;
        HQ_LAUNCH(HQ_K_SMALL, k_lu_trsm<<<(ncols + 127) / 128, 128, 0, s>>>(nn, N, k0, nb, Mw, XY,
                                                                             ipiv));
        const int rows = nn - k0 - nb;
        if (rows > 0)
            HQ_LAUNCH(HQ_K_SMALL, k_lu_update<<<dim3((ncols + 63) / 64, (rows + 63) / 64), 256, 0, s>>>(
                                      nn, N, k0, nb, Mw, XY));
    }
    for (int k0 = ((nn - 1) / bs) * bs; k0 >= 0; k0 -= bs) {
        const int nb = std::min(bs, nn - k0);
        HQ_LAUNCH(HQ_K_SMALL, k_lu_back_diag<<<(N + 127) / 128, 128, 0, s>>>(nn, N, k0, nb, Mw, XY));
        if (k0 > 0)
            HQ_LAUNCH(HQ_K_SMALL, k_lu_back_update<<<dim3((N + 63) / 64, (k0 + 63) / 64), 256, 0, s>>>(
                                      nn, N, k0, nb, Mw, XY));
    }
}

// ---------------------------------------------------------------------------
// Small solves of the mixed-precision path: FP32 Gaussian elimination with
// partial pivoting in one CTA's shared memory, followed by FP64 iterative
// refinement (residual in FP64 over many CTAs, correction with the stored
// FP32 factors).  GB300 issues about two FP64 lane operations per clock per
// SM, so a one-SM FP64 elimination is bound by that rate; FP32 runs 64x
// faster per SM and the FP64 residuals restore FP64 accuracy (each
// refinement multiplies the error by about cond(A) * 2^-24).
// ---------------------------------------------------------------------------
constexpr int LU32_THREADS = 1024;

size_t lu32_smem(int nn, int nr) { return sizeof(float) * ((size_t)nn * (nn + 1) + (size_t)nn * nr); }
bool lu32_fits(int nn, int nr) { return lu32_smem(nn, nr) <= 200 * 1024; }

__device__ __forceinline__ void lu32_argmax(float v, int i, float *wv, int *wi, int *piv_s,
                                            float *pval_s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_down_sync(0xffffffffu, v, o);
        const int i2 = __shfl_down_sync(0xffffffffu, i, o);
        if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
    }
    if (lane == 0) { wv[warp] = v; wi[warp] = i; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? wv[lane] : -1.0f;
        i = lane < nw ? wi[lane] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const float v2 = __shfl_down_sync(0xffffffffu, v, o);
            const int i2 = __shfl_down_sync(0xffffffffu, i, o);
            if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
        }
        if (lane == 0) { *piv_s = i; *pval_s = v; }
    }
    __syncthreads();
}

// A (nn x nn, lda) and B (nn x nr, ldb) in FP64; factors LU (nn x nn FP32,
// L unit lower below the diagonal, rows permuted) and ipiv to global memory;
// X (nn x nr, FP64) = the FP32 solution (nr = 0: factors only).  Work is mapped row = warp, column =
// lane (no integer division in the loops).
__global__ void __launch_bounds__(LU32_THREADS) k_lu32_factor_solve(int nn, int nr, const double *A,
                                                                  int lda, const double *B, int ldb,
                                                                  float *LU, int *ipiv, double *X,
                                                                  int *status) {
    extern __shared__ float sm32[];
    float *sA = sm32;                          // nn x (nn + 1)
    float *sB = sm32 + (size_t)nn * (nn + 1);  // nn x nr
    __shared__ float wv[32];
    __shared__ int wi[32];
    __shared__ int piv_s;
    __shared__ float pval_s;
    const int T = blockDim.x, tid = threadIdx.x, la = nn + 1;
    const int lx = tid & 31, wy = tid >> 5, NW = T >> 5;
    for (int r = wy; r < nn; r += NW) {
        for (int c = lx; c < nn; c += 32) sA[r * la + c] = (float)A[(size_t)r * lda + c];
        for (int c = lx; c < nr; c += 32) sB[r * nr + c] = (float)B[(size_t)r * ldb + c];
    }
    __syncthreads();
    for (int k = 0; k < nn; k++) {
        float best = -1.0f;
        int bi = 0x7fffffff;
        for (int r = k + tid; r < nn; r += T) {
            const float v = fabsf(sA[r * la + k]);
            if (v > best) { best = v; bi = r; }
        }
        lu32_argmax(best, bi, wv, wi, &piv_s, &pval_s);
        const int piv = piv_s;
        if (!(pval_s > 0.0f) || !isfinite(pval_s)) {
            if (tid == 0) atomicOr(status, ST_SINGULAR);
            for (int t = k + tid; t < nn; t += T) ipiv[t] = t;
            return;
        }
        if (tid == 0) ipiv[k] = piv;
        if (piv != k) {
            for (int c = tid; c < nn; c += T) {
                const float t = sA[k * la + c];
                sA[k * la + c] = sA[piv * la + c];
                sA[piv * la + c] = t;
            }
            for (int c = tid; c < nr; c += T) {
                const float t = sB[k * nr + c];
                sB[k * nr + c] = sB[piv * nr + c];
                sB[piv * nr + c] = t;
            }
        }
        __syncthreads();
        const float inv = 1.0f / sA[k * la + k];
        for (int r = k + 1 + wy; r < nn; r += NW) {
            const float l = sA[r * la + k] * inv;   // every lane of the warp computes it
            for (int c = k + 1 + lx; c < nn; c += 32) sA[r * la + c] -= l * sA[k * la + c];
            for (int c = lx; c < nr; c += 32) sB[r * nr + c] -= l * sB[k * nr + c];
        }
        __syncthreads();
        for (int r = k + 1 + tid; r < nn; r += T) sA[r * la + k] *= inv;
        // (column k below the diagonal is read by no later step of this loop)
    }
    __syncthreads();
    // nr == 0: factors only (the solves run in k_lu32_resolve)
    if (nr > 0) {
        for (int k = nn - 1; k >= 0; k--) {
            const float inv = 1.0f / sA[k * la + k];
            for (int r = wy; r < k; r += NW) {
                const float u = sA[r * la + k] * inv;
                for (int c = lx; c < nr; c += 32) sB[r * nr + c] -= u * sB[k * nr + c];
            }
            __syncthreads();
            for (int c = tid; c < nr; c += T) sB[k * nr + c] *= inv;
            // row k is read by no later step
        }
        __syncthreads();
    }
    for (int r = wy; r < nn; r += NW) {
        for (int c = lx; c < nn; c += 32) LU[(size_t)r * nn + c] = sA[r * la + c];
        for (int c = lx; c < nr; c += 32) X[(size_t)r * nr + c] = (double)sB[r * nr + c];
    }
}

// R = B - A X in FP64.  CTA = one row r of R and 64 of its columns; the
// four threads of a column (one per 64-thread group) split k into four
// contiguous ranges (each a chain of nn/4 FMAs in k order), whose sums are
// added in range order.
constexpr int RES_COLS = 64, RES_KG = 4;
__global__ void __launch_bounds__(RES_COLS * RES_KG) k_resid64(int nn, int nr, const double *A,
                                                              int lda, const double *B, int ldb,
                                                              const double *X, double *R) {
    __shared__ double ps[RES_KG][RES_COLS];
    const int r = blockIdx.x, cl = threadIdx.x % RES_COLS, kg = threadIdx.x / RES_COLS;
    const int c = blockIdx.y * RES_COLS + cl;
    const int kc = (nn + RES_KG - 1) / RES_KG, k0 = kg * kc, k1 = min(nn, k0 + kc);
    double s = 0.0;
    if (c < nr)
        for (int k = k0; k < k1; k++) s += A[(size_t)r * lda + k] * X[(size_t)k * nr + c];
    ps[kg][cl] = s;
    __syncthreads();
    if (kg == 0 && c < nr) {
        double t = ps[0][cl];
#pragma unroll
        for (int g = 1; g < RES_KG; g++) t += ps[g][cl];
        R[(size_t)r * nr + c] = B[(size_t)r * ldb + c] - t;
    }
}

// X = (LU)^-1 P R, or X += (LU)^-1 P R (accumulate), with the stored FP32
// factors; R has leading dimension ldr, X is dense nn x nr.  The solves of
// the first solution and of every refinement step run here.  One warp per
// right-hand side (the CTA's warps share the factors in shared memory):
// lane l holds rows l + 32 i in registers, the pivot value of step k comes
// by a shuffle from its owner, so the 2 nn steps of the two substitutions
// need no barrier.  P R is gathered through the composed row permutation
// (the swaps of the elimination applied in reverse to each row index), and
// every element sees the same operations in the same order as the
// elimination with the swaps applied in place.
constexpr int RS_WARPS = 8, RS_THREADS = 32 * RS_WARPS;
size_t lu32_resolve_smem(int nn) {
    return sizeof(float) * (size_t)nn * (nn + 1) + sizeof(int) * (size_t)nn * 2;
}
template <int NI>
__global__ void __launch_bounds__(RS_THREADS) k_lu32_resolve(int nn, int nr, const float *LU,
                                                           const int *ipiv, const double *R,
                                                           int ldr, double *X, int accumulate) {
    extern __shared__ float sm32[];
    float *sA = sm32;
    int *piv = reinterpret_cast<int *>(sm32 + (size_t)nn * (nn + 1));
    int *perm = piv + nn;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, la = nn + 1;
    for (int idx = tid; idx < nn * nn; idx += RS_THREADS) {
        const int r = idx / nn, q = idx - r * nn;
        sA[r * la + q] = LU[idx];
    }
    for (int k = tid; k < nn; k += RS_THREADS) piv[k] = ipiv[k];
    __syncthreads();
    for (int i = tid; i < nn; i += RS_THREADS) {
        int idx = i;
        for (int k = nn - 1; k >= 0; k--) {
            const int p = piv[k];
            idx = idx == k ? p : (idx == p ? k : idx);
        }
        perm[i] = idx;
    }
    __syncthreads();
    const int c = blockIdx.x * RS_WARPS + warp;
    if (c >= nr) return;
    float x[NI];
#pragma unroll
    for (int i = 0; i < NI; i++) {
        const int row = lane + 32 * i;
        x[i] = row < nn ? (float)R[(size_t)perm[row] * ldr + c] : 0.f;
    }
    // forward substitution with the unit lower factor
#pragma unroll
    for (int kb = 0; kb < NI; kb++)
        for (int kk = 0; kk < 32; kk++) {
            const int k = 32 * kb + kk;
            if (k >= nn - 1) break;
            const float bk = __shfl_sync(0xffffffffu, x[kb], kk);
#pragma unroll
            for (int i = kb; i < NI; i++) {
                const int row = lane + 32 * i;
                if (row > k && row < nn) x[i] -= sA[row * la + k] * bk;
            }
        }
    // backward substitution with the upper factor
#pragma unroll
    for (int kb = NI - 1; kb >= 0; kb--)
        for (int kk = 31; kk >= 0; kk--) {
            const int k = 32 * kb + kk;
            if (k >= nn) continue;
            const float inv = 1.0f / sA[k * la + k];
            const float bk = __shfl_sync(0xffffffffu, x[kb], kk);
#pragma unroll
            for (int i = 0; i <= kb; i++) {
                const int row = lane + 32 * i;
                if (row < k) {
                    const float u = sA[row * la + k] * inv;
                    x[i] -= u * bk;
                }
            }
            if (lane == kk) x[kb] *= inv;
        }
#pragma unroll
    for (int i = 0; i < NI; i++) {
        const int row = lane + 32 * i;
        if (row < nn) {
            const double v = (double)x[i];
            X[(size_t)row * nr + c] = accumulate ? X[(size_t)row * nr + c] + v : v;
        }
    }
}

static void launch_resolve(int nn, int nr, const float *LU, const int *ipiv, const double *R,
                           int ldr, double *X, int accumulate, cudaStream_t s) {
    const dim3 grid((nr + RS_WARPS - 1) / RS_WARPS);
    const size_t sm = lu32_resolve_smem(nn);
    switch ((nn + 31) / 32) {
#define RS_CASE(K)                                                                                 \
    case K:                                                                                        \
        HQ_LAUNCH(HQ_K_SMALL, k_lu32_resolve<K><<<grid, RS_THREADS, sm, s>>>(nn, nr, LU, ipiv, R,  \
                                                                            ldr, X, accumulate));  \
        break;
        RS_CASE(1) RS_CASE(2) RS_CASE(3) RS_CASE(4) RS_CASE(5) RS_CASE(6) RS_CASE(7) RS_CASE(8)
#undef RS_CASE
    default: break;   // lu32_fits bounds nn well below 256
    }
}

void lu32_prepare() {
    static bool done = false;
    if (done) return;
    const int lim = 200 * 1024;
    cudaFuncSetAttribute(k_lu32_factor_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_lu32_resolve<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    done = true;
}

// FP32 factors of A in one CTA, then X = (LU)^-1 P B over RS_WARPS-column CTAs
static void lu32_factor_then_solve(int nn, int nr, const double *A, int lda, const double *B,
                                   int ldb, double *X, float *LU, int *ipiv, int *status,
                                   cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_lu32_factor_solve<<<1, LU32_THREADS, lu32_smem(nn, 0), s>>>(
                              nn, 0, A, lda, nullptr, 0, LU, ipiv, nullptr, status));
    launch_resolve(nn, nr, LU, ipiv, B, ldb, X, 0, s);
}

// X = A^-1 B (A nn x nn, B nn x nr, FP64 in and out) by FP32 elimination and
// `refine` FP64 refinement steps; LU (nn^2 floats), ipiv (nn) and R (nn x nr
// doubles) are scratch.  Requires lu32_fits(nn, nr).
void launch_solve32_refined(int nn, int nr, const double *A, int lda, const double *B, int ldb,
                            double *X, float *LU, int *ipiv, double *R, int refine, int *status,
                            cudaStream_t s) {
    lu32_factor_then_solve(nn, nr, A, lda, B, ldb, X, LU, ipiv, status, s);
    for (int it = 0; it < refine; it++) {
        HQ_LAUNCH(HQ_K_SMALL, k_resid64<<<dim3(nn, (nr + RES_COLS - 1) / RES_COLS), RES_COLS * RES_KG,
                                           0, s>>>(nn, nr, A, lda, B, ldb, X, R));
        launch_resolve(nn, nr, LU, ipiv, R, nr, X, 1, s);
    }
}

void launch_predictor_solve(int N, double tau, const double *G2, double *Mw, double *XY,
                            double *C, int *status, cudaStream_t s, const double *tau_dev,
                            int *ipiv, float *lu32, double *pB, double *pR) {
    const int nn = 2 * N;
    if (lu32 && pB && pR && ipiv && lu32_fits(nn, N)) {
        // mixed-precision path: FP32 elimination + 2 FP64 refinement steps
        const long tot = (long)nn * nn + (long)nn * N;
        HQ_LAUNCH(HQ_K_SMALL, k_pred_build<<<(int)std::min<long>((tot + 255) / 256, 1024), 256, 0, s>>>(
                                  N, tau, tau_dev, G2, Mw, pB));
        launch_solve32_refined(nn, N, Mw, nn, pB, N, XY, lu32, ipiv, pR, 2, status, s);
        HQ_LAUNCH(HQ_K_SMALL, k_pred_c<<<(int)std::min<long>(((long)N * N + 255) / 256, 1024), 256, 0, s>>>(
                                  N, tau, tau_dev, XY, C));
        return;
    }
    if (nn <= 64 || !ipiv) {
        size_t shm = sizeof(double) * (2 * N + 1024) + sizeof(int) * 1024;
        HQ_LAUNCH(HQ_K_SMALL, k_predictor_solve<<<1, 1024, shm, s>>>(N, tau, G2, Mw, XY, C, status,
                                                                      tau_dev));
        return;
    }
    const long tot = (long)nn * nn + (long)nn * N;
    HQ_LAUNCH(HQ_K_SMALL, k_pred_build<<<(int)std::min<long>((tot + 255) / 256, 1024), 256, 0, s>>>(
                              N, tau, tau_dev, G2, Mw, XY));
    launch_lu_solve(nn, N, Mw, XY, ipiv, status, s);
    HQ_LAUNCH(HQ_K_SMALL, k_pred_c<<<(int)std::min<long>(((long)N * N + 255) / 256, 1024), 256, 0, s>>>(
                              N, tau, tau_dev, XY, C));
}

// X = A^-1 B for an N x N matrix A and N right-hand sides (leading dimensions
// lda, ldb); Mw: N x N scratch.  Blocked elimination for N > 32, else the
// one-CTA Cholesky kernel (A symmetric positive definite there).
__global__ void k_copy2(int N, const double *A, int lda, const double *B, int ldb, double *Mw,
                        double *X) {
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < 2L * N * N;
         idx += (long)gridDim.x * blockDim.x) {
        const long e = idx % ((long)N * N);
        const int i = (int)(e / N), j = (int)(e % N);
        if (idx < (long)N * N) Mw[e] = A[(size_t)i * lda + j];
        else X[e] = B[(size_t)i * ldb + j];
    }
}
void launch_spd_solve(int N, const double *A, int lda, const double *B, int ldb, double *Mw,
                      double *L, double *X, int *ipiv, int *status, cudaStream_t s, float *lu32) {
    if (lu32 && ipiv && lu32_fits(N, N)) {
        // mixed-precision path (a warm start only needs FP32 accuracy)
        lu32_factor_then_solve(N, N, A, lda, B, ldb, X, lu32, ipiv, status, s);
        return;
    }
    if (N <= 32 || !ipiv) {
        launch_chol_solve(N, A, lda, B, ldb, L, X, status, s);
        return;
    }
    HQ_LAUNCH(HQ_K_SMALL, k_copy2<<<(int)std::min<long>((2L * N * N + 255) / 256, 1024), 256, 0, s>>>(
                              N, A, lda, B, ldb, Mw, X));
    launch_lu_solve(N, N, Mw, X, ipiv, status, s);
}

// Largest eigenvalue of the symmetric part of A (N x N, leading dimension
// lda) by power iteration with Rayleigh quotients, one CTA; out[0] = value.
// vec (N, device): start vector on entry (all zero: a fixed start), final
// iterate on exit, so successive calls on slowly changing matrices restart
// close to the answer.
__global__ void __launch_bounds__(256) k_top_eig(int N, const double *A, int lda, double *vec,
                                                 double *out) {
    extern __shared__ double sh[];
    double *v = sh, *w = sh + N, *red = sh + 2 * N;
    const int tid = threadIdx.x;
    __shared__ int fresh;
    if (tid == 0) {
        double nv = 0.0;
        for (int i = 0; i < N; i++) nv += vec[i] * vec[i];
        fresh = !(nv > 0.0);
    }
    __syncthreads();
    for (int i = tid; i < N; i += blockDim.x) v[i] = fresh ? 1.0 + 0.125 * (double)(i % 7) : vec[i];
    __syncthreads();
    double mu = 0.0, mu_prev = 0.0;
    for (int it = 0; it < 1000; it++) {
        for (int i = tid; i < N; i += blockDim.x) {
            double acc = 0.0;
            for (int j = 0; j < N; j++)
                acc += 0.5 * (A[(size_t)i * lda + j] + A[(size_t)j * lda + i]) * v[j];
            w[i] = acc;
        }
        __syncthreads();
        double vw = 0.0, vv = 0.0, ww = 0.0;
        for (int i = tid; i < N; i += blockDim.x) {
            vw += v[i] * w[i];
            vv += v[i] * v[i];
            ww += w[i] * w[i];
        }
        red[tid] = vw;
        red[256 + tid] = vv;
        red[512 + tid] = ww;
        __syncthreads();
        for (int k = 128; k > 0; k >>= 1) {
            if (tid < k) {
                red[tid] += red[tid + k];
                red[256 + tid] += red[256 + tid + k];
                red[512 + tid] += red[512 + tid + k];
            }
            __syncthreads();
        }
        mu = red[0] / red[256];
        const double nw = sqrt(red[512]);
        __syncthreads();
        if (!(nw > 0.0)) break;
        for (int i = tid; i < N; i += blockDim.x) v[i] = w[i] / nw;
        __syncthreads();
        if (it > 1 && fabs(mu - mu_prev) <= 1e-14 * fabs(mu)) break;
        mu_prev = mu;
    }
    for (int i = tid; i < N; i += blockDim.x) vec[i] = v[i];
    if (tid == 0) out[0] = mu;
}
// The same power iteration with the symmetric part B = (A + A^T) / 2 staged
// in shared memory (N <= TE_SMEM_N): each product reads B from shared memory
// instead of A and A^T from L2 (the transposed reads uncoalesced), and the
// three inner products of an iteration are reduced by warp butterflies and
// one pass over the warps (three barriers instead of ten).
constexpr int TE_SMEM_N = 120;
size_t te_smem_bytes(int N) { return sizeof(double) * ((size_t)N * N + 2 * N + 768); }
__global__ void __launch_bounds__(256) k_top_eig_sm(int N, const double *A, int lda, double *vec,
                                                    double *out) {
    extern __shared__ double sh[];
    double *B = sh, *v = sh + (size_t)N * N, *w = v + N, *red = w + N;   // red: 3 x 8 warps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ int fresh;
    __shared__ double mu_sh, nw_sh;
    for (long idx = tid; idx < (long)N * N; idx += blockDim.x) {
        const int i = (int)(idx / N), j = (int)(idx % N);
        B[idx] = 0.5 * (A[(size_t)i * lda + j] + A[(size_t)j * lda + i]);
    }
    if (tid == 0) {
        double nv = 0.0;
        for (int i = 0; i < N; i++) nv += vec[i] * vec[i];
        fresh = !(nv > 0.0);
    }
    __syncthreads();
    for (int i = tid; i < N; i += blockDim.x) v[i] = fresh ? 1.0 + 0.125 * (double)(i % 7) : vec[i];
    __syncthreads();
    double mu = 0.0, mu_prev = 0.0;
    for (int it = 0; it < 1000; it++) {
        for (int i = tid; i < N; i += blockDim.x) {
            double acc = 0.0;
            for (int j = 0; j < N; j++) acc += B[(size_t)i * N + j] * v[j];
            w[i] = acc;
        }
        __syncthreads();
        // v.w, v.v, w.w: per-warp butterflies, then the eight warps in order
        double vw = 0.0, vv = 0.0, ww = 0.0;
        for (int i = tid; i < N; i += blockDim.x) {
            vw += v[i] * w[i];
            vv += v[i] * v[i];
            ww += w[i] * w[i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vw += __shfl_xor_sync(0xffffffffu, vw, o);
            vv += __shfl_xor_sync(0xffffffffu, vv, o);
            ww += __shfl_xor_sync(0xffffffffu, ww, o);
        }
        if (lane == 0) {
            red[warp] = vw;
            red[8 + warp] = vv;
            red[16 + warp] = ww;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0, c = 0.0;
            for (int q = 0; q < 8; q++) {
                a += red[q];
                b += red[8 + q];
                c += red[16 + q];
            }
            mu_sh = a / b;
            nw_sh = sqrt(c);
        }
        __syncthreads();
        mu = mu_sh;
        const double nw = nw_sh;
        if (!(nw > 0.0)) break;
        const double rnw = 1.0 / nw;
        for (int i = tid; i < N; i += blockDim.x) v[i] = w[i] * rnw;
        __syncthreads();
        if (it > 1 && fabs(mu - mu_prev) <= 1e-14 * fabs(mu)) break;
        mu_prev = mu;
    }
    for (int i = tid; i < N; i += blockDim.x) vec[i] = v[i];
    if (tid == 0) out[0] = mu;
}

void launch_top_eig(int N, const double *A, int lda, double *vec, double *out, cudaStream_t s) {
    if (N <= TE_SMEM_N) {
        HQ_LAUNCH(HQ_K_SMALL, k_top_eig_sm<<<1, 256, te_smem_bytes(N), s>>>(N, A, lda, vec, out));
        return;
    }
    size_t shm = sizeof(double) * (2 * N + 768);
    HQ_LAUNCH(HQ_K_SMALL, k_top_eig<<<1, 256, shm, s>>>(N, A, lda, vec, out));
}

// out[0] = max_i sum_j |A_ij| (N x N, leading dimension lda): Gershgorin bound
__global__ void k_gersh(int N, const double *A, int lda, double *out) {
    __shared__ double red[256];
    double best = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double r = 0.0;
        for (int j = 0; j < N; j++) r += fabs(A[(size_t)i * lda + j]);
        best = fmax(best, r);
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}
void launch_gersh(int N, const double *A, int lda, double *out, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_gersh<<<1, 256, 0, s>>>(N, A, lda, out));
}

// Adaptive time step: st[0] = tau_n written from mu_max = mm[0] (largest Ritz
// value of G), smax = sm[0] (lambda_max<U,U>) and the previous tau st[1];
// st[2] != 0 marks the first step (tau_{-1} from the lower bound lb).
__global__ void k_adapt_tau(const double *mm, const double *sm, double tau_max, double c,
                            double gamma, double lb, double *st) {
    const double smax = sm[0];
    double tau = tau_max;
    const double cap = c * (1.0 / mm[0]) / smax;
    if (mm[0] > 0.0 && cap < tau) tau = cap;
    const double prev = (st[2] != 0.0) ? c * lb / (gamma * smax) : st[1];
    if (gamma * prev < tau) tau = gamma * prev;
    st[0] = tau;
    st[1] = tau;
    st[2] = 0.0;
}
void launch_adapt_tau(const double *mm, const double *sm, double tau_max, double c, double gamma,
                      double lb, double *st, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_adapt_tau<<<1, 1, 0, s>>>(mm, sm, tau_max, c, gamma, lb, st));
}

// Om = -tau (Shat - I) with tau from device memory
__global__ void k_corrector_matrix(int N, const double *Shat, const double *tau_dev, double tau,
                                   double *Om) {
    const double t = tau_dev ? tau_dev[0] : tau;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * N; i += gridDim.x * blockDim.x)
        Om[i] = -t * (Shat[i] - ((i / N == i % N) ? 1.0 : 0.0));
}
void launch_corrector_matrix(int N, const double *Shat, const double *tau_dev, double tau,
                             double *Om, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_corrector_matrix<<<std::min((N * N + 255) / 256, 1024), 256, 0, s>>>(
                              N, Shat, tau_dev, tau, Om));
}

__global__ void k_add_diag(int N, double *A, double v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        A[(size_t)i * N + i] += v;
}
void launch_add_diag(int N, double *A, double v, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_add_diag<<<(N + 255) / 256, 256, 0, s>>>(N, A, v));
}

__global__ void k_dscale(int count, double alpha, const double *in, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = alpha * in[i];
}
void launch_dscale(int count, double alpha, const double *in, double *out, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_dscale<<<std::min((count + 255) / 256, 1024), 256, 0, s>>>(count, alpha, in, out));
}

__global__ void k_axpy_small(int count, double a, const double *x, double *y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        y[i] += a * x[i];
}
void launch_axpy_small(int count, double a, const double *x, double *y, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_axpy_small<<<std::min((count + 255) / 256, 1024), 256, 0, s>>>(count, a, x, y));
}

// Cyclic Jacobi with a parallel (round-robin) ordering, one CTA.  work: 2 N^2
// (+ padding to even order).  Rotation: theta = (a_qq - a_pp) / (2 a_pq),
// t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1/sqrt(t^2 + 1), s = t c,
// A <- J^T A J, V <- V J with J = [c s; -s c] on (p, q).
__global__ void __launch_bounds__(1024) k_sym_eig(int N, const double *Ain, double *work,
                                                  double *evals, double *evecs) {
    extern __shared__ double sh[];
    const int P = (N + 1) & ~1;          // even order (index N is a dummy when N is odd)
    double *A = work;                    // P x P
    double *Vv = work + (size_t)P * P;   // P x P
    double *cs = sh;                     // P/2 c
    double *sn = sh + P / 2;             // P/2 s
    int *pp = (int *)(sh + P);           // P/2
    int *qq = pp + P / 2;                // P/2
    double *red = (double *)(pp + P);    // 1024 (pp + P is 8-byte aligned: P even)
    const int tid = threadIdx.x, T = blockDim.x;
    for (long idx = tid; idx < (long)P * P; idx += T) {
        int i = (int)(idx / P), j = (int)(idx % P);
        double v = 0.0;
        if (i < N && j < N) v = 0.5 * (Ain[(size_t)i * N + j] + Ain[(size_t)j * N + i]);
        A[idx] = v;
        Vv[idx] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    double fro;
    {
        double s = 0.0;
        for (long idx = tid; idx < (long)P * P; idx += T) s += A[idx] * A[idx];
        red[tid] = s;
        __syncthreads();
        for (int w = T / 2; w > 0; w >>= 1) {
            if (tid < w) red[tid] += red[tid + w];
            __syncthreads();
        }
        fro = sqrt(red[0]);
        __syncthreads();
    }
    for (int sweep = 0; sweep < 100; sweep++) {
        double s = 0.0;
        for (long idx = tid; idx < (long)P * P; idx += T) {
            int i = (int)(idx / P), j = (int)(idx % P);
            if (i < j) s += A[idx] * A[idx];
        }
        red[tid] = s;
        __syncthreads();
        for (int w = T / 2; w > 0; w >>= 1) {
            if (tid < w) red[tid] += red[tid + w];
            __syncthreads();
        }
        double off = red[0];
        __syncthreads();
        if (sqrt(off) <= 1e-15 * fro || off == 0.0) break;
        for (int r = 0; r < P - 1; r++) {
            for (int k = tid; k < P / 2; k += T) {
                int a, b;
                if (k == 0) { a = P - 1; b = r; }
                else { a = (r + k) % (P - 1); b = (r - k + (P - 1)) % (P - 1); }
                int p = a < b ? a : b, q = a < b ? b : a;
                pp[k] = p;
                qq[k] = q;
                double c = 1.0, sv = 0.0;
                if (q < N) {
                    double apq = A[(size_t)p * P + q];
                    if (apq != 0.0) {
                        double app = A[(size_t)p * P + p], aqq = A[(size_t)q * P + q];
                        double theta = (aqq - app) / (2.0 * apq);
                        double t = (theta >= 0.0 ? 1.0 : -1.0) /
                                   (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sv = t * c;
                    }
                }
                cs[k] = c;
                sn[k] = sv;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (long idx = tid; idx < (long)(P / 2) * P; idx += T) {
                int k = (int)(idx / P), j = (int)(idx % P);
                double c = cs[k], sv = sn[k];
                if (sv == 0.0) continue;
                int p = pp[k], q = qq[k];
                double apj = A[(size_t)p * P + j], aqj = A[(size_t)q * P + j];
                A[(size_t)p * P + j] = c * apj - sv * aqj;
                A[(size_t)q * P + j] = sv * apj + c * aqj;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (long idx = tid; idx < (long)(P / 2) * P; idx += T) {
                int k = (int)(idx / P), i = (int)(idx % P);
                double c = cs[k], sv = sn[k];
                if (sv == 0.0) continue;
                int p = pp[k], q = qq[k];
                double aip = A[(size_t)i * P + p], aiq = A[(size_t)i * P + q];
                A[(size_t)i * P + p] = c * aip - sv * aiq;
                A[(size_t)i * P + q] = sv * aip + c * aiq;
                double vip = Vv[(size_t)i * P + p], viq = Vv[(size_t)i * P + q];
                Vv[(size_t)i * P + p] = c * vip - sv * viq;
                Vv[(size_t)i * P + q] = sv * vip + c * viq;
            }
            __syncthreads();
            for (int k = tid; k < P / 2; k += T) {
                if (sn[k] != 0.0) {
                    A[(size_t)pp[k] * P + qq[k]] = 0.0;
                    A[(size_t)qq[k] * P + pp[k]] = 0.0;
                }
            }
            __syncthreads();
        }
    }
    // sort ascending (rank sort, ties by index)
    for (int i = tid; i < N; i += T) {
        double di = A[(size_t)i * P + i];
        int rank = 0;
        for (int j = 0; j < N; j++) {
            double dj = A[(size_t)j * P + j];
            if (dj < di || (dj == di && j < i)) rank++;
        }
        evals[rank] = di;
        if (evecs)
            for (int k = 0; k < N; k++) evecs[(size_t)k * N + rank] = Vv[(size_t)k * P + i];
    }
}

void launch_sym_eig(int N, const double *A, double *work, double *evals, double *evecs,
                    cudaStream_t s) {
    int P = (N + 1) & ~1;
    size_t shm = sizeof(double) * (P + 1024) + sizeof(int) * (P + 2) + 16;
    HQ_LAUNCH(HQ_K_SMALL, k_sym_eig<<<1, 1024, shm, s>>>(N, A, work, evals, evecs));
}

// Rayleigh-Ritz reduction: S = L L^T, Cm = L^{-1} sym(K) L^{-T}.  One CTA.
__global__ void __launch_bounds__(1024) k_rr_reduce(int N, const double *K, const double *S,
                                                    double *L, double *Cm, int *status) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (long idx = tid; idx < (long)N * N; idx += T) L[idx] = S[idx];
    __syncthreads();
    for (int k = 0; k < N; k++) {
        double d = L[(size_t)k * N + k];
        if (!(d > 0.0)) {
            if (tid == 0) atomicOr(status, ST_SINGULAR);
            return;
        }
        d = sqrt(d);
        __syncthreads();
        for (int i = k + tid; i < N; i += T) L[(size_t)i * N + k] = (i == k) ? d : L[(size_t)i * N + k] / d;
        __syncthreads();
        for (int i = k + 1 + (tid >> 5); i < N; i += (T >> 5)) {
            const double lik = L[(size_t)i * N + k];
            for (int j = k + 1 + (tid & 31); j <= i; j += 32)
                L[(size_t)i * N + j] -= lik * L[(size_t)j * N + k];
        }
        __syncthreads();
    }
    for (long idx = tid; idx < (long)N * N; idx += T) {
        int i = (int)(idx / N), j = (int)(idx % N);
        if (j > i) L[idx] = 0.0;
    }
    __syncthreads();
    // T1 = L^{-1} sym(K) into Cm (column j by thread), then Cm = L^{-1} T1^T
    for (int j = tid; j < N; j += T) {
        for (int i = 0; i < N; i++) {
            double s = 0.5 * (K[(size_t)i * N + j] + K[(size_t)j * N + i]);
            for (int k = 0; k < i; k++) s -= L[(size_t)i * N + k] * Cm[(size_t)k * N + j];
            Cm[(size_t)i * N + j] = s / L[(size_t)i * N + i];
        }
    }
    __syncthreads();
    // transpose in place
    for (long idx = tid; idx < (long)N * N; idx += T) {
        int i = (int)(idx / N), j = (int)(idx % N);
        if (i < j) {
            double a = Cm[idx], b = Cm[(size_t)j * N + i];
            Cm[idx] = b;
            Cm[(size_t)j * N + i] = a;
        }
    }
    __syncthreads();
    for (int j = tid; j < N; j += T) {
        for (int i = 0; i < N; i++) {
            double s = Cm[(size_t)i * N + j];
            for (int k = 0; k < i; k++) s -= L[(size_t)i * N + k] * Cm[(size_t)k * N + j];
            Cm[(size_t)i * N + j] = s / L[(size_t)i * N + i];
        }
    }
}
// The same reduction in three launches for N <= RR_SMEM_N.  GB300 retires
// about two FP64 operations per clock per SM, so one CTA doing the whole
// reduction (N^3/6 for the Cholesky, N^3 for the two triangular solves, N^2
// divisions) is bound by that single SM's FP64 pipe and by its dependency
// chains (~0.5 ms at N = 64).  Here one CTA factors S = L L^T in shared
// memory (reciprocal of each pivot once), and the two triangular solves
// run one column per CTA on N SMs, each row's dot product split over the
// warp's lanes: T1 = L^{-1} sym(K) stored transposed, then Cm = L^{-1} T1^T.
// Same quantities as k_rr_reduce; rounded in a different order.
constexpr int RR_SMEM_N = 96;
size_t rr_chol_smem(int N) { return sizeof(double) * (size_t)N * N; }
// Cholesky S = L L^T in shared memory by one CTA of 1024 threads (the
// pivot's reciprocal once per step; the trailing update with rows across the
// warps and columns across the lanes).  A one-warp form took twice as long:
// GB300's FP64 latency needs the warps in flight more than the barriers cost.
__global__ void __launch_bounds__(1024) k_chol_sm(int N, const double *S, double *Lg, int *status) {
    extern __shared__ double L[];
    __shared__ double d_sh, rd_sh;
    const int tid = threadIdx.x, T = blockDim.x;
    for (long idx = tid; idx < (long)N * N; idx += T) L[idx] = S[idx];
    __syncthreads();
    for (int k = 0; k < N; k++) {
        const double dk = L[(size_t)k * N + k];
        if (!(dk > 0.0)) {
            if (tid == 0) atomicOr(status, ST_SINGULAR);
            return;
        }
        if (tid == 0) {
            d_sh = sqrt(dk);
            rd_sh = 1.0 / d_sh;
        }
        __syncthreads();
        const double d = d_sh, rd = rd_sh;
        for (int i = k + tid; i < N; i += T) L[(size_t)i * N + k] = (i == k) ? d : L[(size_t)i * N + k] * rd;
        __syncthreads();
        for (int i = k + 1 + (tid >> 5); i < N; i += (T >> 5)) {
            const double lik = L[(size_t)i * N + k];
            for (int j = k + 1 + (tid & 31); j <= i; j += 32)
                L[(size_t)i * N + j] -= lik * L[(size_t)j * N + k];
        }
        __syncthreads();
    }
    for (long idx = tid; idx < (long)N * N; idx += T) {
        const int i = (int)(idx / N), j = (int)(idx % N);
        Lg[idx] = j > i ? 0.0 : L[idx];
    }
}
// x = L^{-1} b for column j = blockIdx.x (one warp, L staged in shared
// memory), each row's dot product split over the lanes: mode 0:
// b_i = (K_ij + K_ji) / 2, x stored as row j of Out (the transpose); mode 1:
// b_i = In_ij, x stored as column j of Out
__global__ void __launch_bounds__(32) k_trsv_col(int N, const double *L, const double *In,
                                                 int mode, double *Out) {
    extern __shared__ double tsm[];
    double *Ls = tsm, *x = tsm + (size_t)N * N;
    const int j = blockIdx.x, lane = threadIdx.x;
    for (long idx = lane; idx < (long)N * N; idx += 32) Ls[idx] = L[idx];
    for (int i = lane; i < N; i += 32)
        x[i] = mode == 0 ? 0.5 * (In[(size_t)i * N + j] + In[(size_t)j * N + i]) : In[(size_t)i * N + j];
    __syncwarp();
    for (int i = 0; i < N; i++) {
        double part = 0.0;
        for (int k = lane; k < i; k += 32) part += Ls[(size_t)i * N + k] * x[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) x[i] = (x[i] - part) / Ls[(size_t)i * N + i];
        __syncwarp();
    }
    for (int i = lane; i < N; i += 32) {
        if (mode == 0) Out[(size_t)j * N + i] = x[i];
        else Out[(size_t)i * N + j] = x[i];
    }
}

// The largest eigenvalue mu of the pencil (sym(K), S) in FP32, one CTA, for
// the adaptive time step of mixed-precision contexts (a step-size estimate
// needs ~1e-6, not FP64's 1e-14): C = L^{-1} sym(K) L^{-T} from the FP32
// Cholesky S = L L^T, then the power iteration of k_top_eig_sm on C from
// the warm vector vec (FP64, updated), stopped when mu changes by less than
// 1e-6 of itself.  FP32 runs about sixty times FP64's lane rate here, and
// the whole estimate is one launch instead of four.  N <= LH_MAX_N.
constexpr int LH_MAX_N = 96;
size_t lam_hat32_smem(int N) { return sizeof(float) * (2 * (size_t)N * (N + 1) + 2 * N + 64); }
__global__ void __launch_bounds__(1024) k_lam_hat32(int N, const double *K, const double *S,
                                                   double *vec, double *out, int *status) {
    extern __shared__ float lsm[];
    const int LD = N + 1;   // row stride: a column read by consecutive threads spans all banks
    float *L = lsm, *C = lsm + (size_t)N * LD, *v = C + (size_t)N * LD, *w = v + N, *red = w + N;
    __shared__ float d_sh, rd_sh, mu_sh, nw_sh;
    __shared__ int fresh;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (long idx = tid; idx < (long)N * N; idx += T) {
        const int i = (int)(idx / N), j = (int)(idx % N);
        L[i * LD + j] = (float)S[idx];
        C[i * LD + j] = (float)(0.5 * (K[(size_t)i * N + j] + K[(size_t)j * N + i]));
    }
    if (tid == 0) {
        double nv = 0.0;
        for (int i = 0; i < N; i++) nv += vec[i] * vec[i];
        fresh = !(nv > 0.0);
    }
    __syncthreads();
    for (int k = 0; k < N; k++) {
        const float dk = L[k * LD + k];
        if (!(dk > 0.f)) {
            if (tid == 0) atomicOr(status, ST_SINGULAR);
            return;
        }
        if (tid == 0) {
            d_sh = sqrtf(dk);
            rd_sh = 1.f / d_sh;
        }
        __syncthreads();
        const float d = d_sh, rd = rd_sh;
        for (int i = k + tid; i < N; i += T) L[i * LD + k] = (i == k) ? d : L[i * LD + k] * rd;
        __syncthreads();
        for (int i = k + 1 + (tid >> 5); i < N; i += (T >> 5)) {
            const float lik = L[i * LD + k];
            for (int j = k + 1 + lane; j <= i; j += 32) L[i * LD + j] -= lik * L[j * LD + k];
        }
        __syncthreads();
    }
    // C <- L^{-1} C (column j by thread), transpose, and again: L^{-1} C L^{-T}
    for (int pass = 0; pass < 2; pass++) {
        for (int j = tid; j < N; j += T)
            for (int i = 0; i < N; i++) {
                float acc = C[i * LD + j];
                for (int k = 0; k < i; k++) acc -= L[i * LD + k] * C[k * LD + j];
                C[i * LD + j] = acc / L[i * LD + i];
            }
        __syncthreads();
        for (long idx = tid; idx < (long)N * N; idx += T) {
            const int i = (int)(idx / N), j = (int)(idx % N);
            if (i < j) {
                const float a = C[i * LD + j], b = C[j * LD + i];
                C[i * LD + j] = b;
                C[j * LD + i] = a;
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < N; i += T) v[i] = fresh ? 1.f + 0.125f * (float)(i % 7) : (float)vec[i];
    __syncthreads();
    float mu = 0.f, mu_prev = 0.f;
    for (int it = 0; it < 500; it++) {
        // w = C v: a warp per row, the lanes split the row and a butterfly
        // of shuffles adds their sums
        for (int i = warp; i < N; i += (T >> 5)) {
            float acc = 0.f;
            for (int j = lane; j < N; j += 32) acc += C[i * LD + j] * v[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) w[i] = acc;
        }
        __syncthreads();
        float vw = 0.f, vv = 0.f, ww = 0.f;
        for (int i = tid; i < N; i += T) {
            vw += v[i] * w[i];
            vv += v[i] * v[i];
            ww += w[i] * w[i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vw += __shfl_xor_sync(0xffffffffu, vw, o);
            vv += __shfl_xor_sync(0xffffffffu, vv, o);
            ww += __shfl_xor_sync(0xffffffffu, ww, o);
        }
        if (lane == 0 && warp < 4) {   // the N <= 96 values live in the first warps
            red[warp] = vw;
            red[4 + warp] = vv;
            red[8 + warp] = ww;
        }
        __syncthreads();
        if (tid == 0) {
            float a = 0.f, b = 0.f, c = 0.f;
            for (int q = 0; q < 4; q++) {
                a += red[q];
                b += red[4 + q];
                c += red[8 + q];
            }
            mu_sh = a / b;
            nw_sh = sqrtf(c);
        }
        __syncthreads();
        mu = mu_sh;
        const float nw = nw_sh;
        if (!(nw > 0.f)) break;
        for (int i = tid; i < N; i += T) v[i] = w[i] / nw;
        __syncthreads();
        if (it > 1 && fabsf(mu - mu_prev) <= 1e-6f * fabsf(mu)) break;
        mu_prev = mu;
    }
    for (int i = tid; i < N; i += T) vec[i] = (double)v[i];
    if (tid == 0) out[0] = (double)mu;
}

bool lam_hat32_fits(int N) { return N <= LH_MAX_N; }
void launch_lam_hat32(int N, const double *K, const double *S, double *vec, double *out,
                      int *status, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_lam_hat32<<<1, 1024, lam_hat32_smem(N), s>>>(N, K, S, vec, out, status));
}

void small_prepare() {
    cudaFuncSetAttribute(k_lam_hat32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)lam_hat32_smem(LH_MAX_N));
    cudaFuncSetAttribute(k_chol_sm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rr_chol_smem(RR_SMEM_N));
    cudaFuncSetAttribute(k_trsv_col, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(rr_chol_smem(RR_SMEM_N) + sizeof(double) * RR_SMEM_N));

    cudaFuncSetAttribute(k_top_eig_sm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)te_smem_bytes(TE_SMEM_N));
}

void launch_rr_reduce(int N, const double *K, const double *S, double *L, double *Cm,
                      int *status, cudaStream_t s) {
    if (N <= RR_SMEM_N) {
        // T1^T into Cm, then Cm = L^{-1} T1^T in place: CTA j of the second
        // solve reads only column j of Cm (into shared memory, before any
        // write) and writes only column j
        const size_t tsm = rr_chol_smem(N) + sizeof(double) * N;
        HQ_LAUNCH(HQ_K_SMALL, k_chol_sm<<<1, 1024, rr_chol_smem(N), s>>>(N, S, L, status));
        HQ_LAUNCH(HQ_K_SMALL, k_trsv_col<<<N, 32, tsm, s>>>(N, L, K, 0, Cm));
        HQ_LAUNCH(HQ_K_SMALL, k_trsv_col<<<N, 32, tsm, s>>>(N, L, Cm, 1, Cm));
        return;
    }
    HQ_LAUNCH(HQ_K_SMALL, k_rr_reduce<<<1, 1024, 0, s>>>(N, K, S, L, Cm, status));
}

// X = A^{-1} B for SPD A (N x N, leading dimension lda) and N right-hand
// sides B (leading dimension ldb) by Cholesky; L: N x N work.  One CTA.
__global__ void __launch_bounds__(1024) k_chol_solve(int N, const double *A, int lda,
                                                     const double *B, int ldb, double *L,
                                                     double *X, int *status) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (long idx = tid; idx < (long)N * N; idx += T) {
        int i = (int)(idx / N), j = (int)(idx % N);
        L[idx] = A[(size_t)i * lda + j];
        X[idx] = B[(size_t)i * ldb + j];
    }
    __syncthreads();
    for (int k = 0; k < N; k++) {
        double d = L[(size_t)k * N + k];
        if (!(d > 0.0)) {
            if (tid == 0) atomicOr(status, ST_SINGULAR);
            return;
        }
        d = sqrt(d);
        __syncthreads();
        for (int i = k + tid; i < N; i += T) L[(size_t)i * N + k] = (i == k) ? d : L[(size_t)i * N + k] / d;
        __syncthreads();
        for (int i = k + 1 + (tid >> 5); i < N; i += (T >> 5)) {
            const double lik = L[(size_t)i * N + k];
            for (int j = k + 1 + (tid & 31); j <= i; j += 32)
                L[(size_t)i * N + j] -= lik * L[(size_t)j * N + k];
        }
        __syncthreads();
    }
    // forward then backward substitution, one right-hand side per thread
    for (int c = tid; c < N; c += T) {
        for (int i = 0; i < N; i++) {
            double s = X[(size_t)i * N + c];
            for (int k = 0; k < i; k++) s -= L[(size_t)i * N + k] * X[(size_t)k * N + c];
            X[(size_t)i * N + c] = s / L[(size_t)i * N + i];
        }
        for (int i = N - 1; i >= 0; i--) {
            double s = X[(size_t)i * N + c];
            for (int k = i + 1; k < N; k++) s -= L[(size_t)k * N + i] * X[(size_t)k * N + c];
            X[(size_t)i * N + c] = s / L[(size_t)i * N + i];
        }
    }
}
void launch_chol_solve(int N, const double *A, int lda, const double *B, int ldb, double *L,
                       double *X, int *status, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_chol_solve<<<1, 1024, 0, s>>>(N, A, lda, B, ldb, L, X, status));
}

__global__ void k_rr_back(int N, const double *L, const double *Y, double *Cv) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        for (int i = N - 1; i >= 0; i--) {
            double s = Y[(size_t)i * N + e];
            for (int k = i + 1; k < N; k++) s -= L[(size_t)k * N + i] * Cv[(size_t)k * N + e];
            Cv[(size_t)i * N + e] = s / L[(size_t)i * N + i];
        }
    }
}
void launch_rr_back(int N, const double *L, const double *Y, double *Cv, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_rr_back<<<(N + 127) / 128, 128, 0, s>>>(N, L, Y, Cv));
}

__global__ void k_inv_sqrt_first(const double *ev, double *out) { out[0] = 1.0 / sqrt(ev[0]); }
void launch_inv_sqrt_first(const double *evals, double *out, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_inv_sqrt_first<<<1, 1, 0, s>>>(evals, out));
}

__global__ void k_paper_evals(int N, const double *mu, double sigma, double *lam) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) lam[i] = 1.0 / mu[N - 1 - i] - sigma;
}
void launch_paper_evals(int N, const double *mu, double sigma, double *lam, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_paper_evals<<<1, 256, 0, s>>>(N, mu, sigma, lam));
}

__global__ void k_add_scalar(int N, const double *in, double add, double *out) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) out[i] = in[i] + add;
}
void launch_add_scalar(int N, const double *in, double add, double *out, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_add_scalar<<<1, 256, 0, s>>>(N, in, add, out));
}

// Ritz-vector sign: per column, entry of largest magnitude (first on ties)
// made positive.  Pass 1: per-CTA (max, index) over a slab of points.
template <typename T>
__global__ void k_sign_pass1(long n, int N, const T *U, long rows, double *work) {
    __shared__ double bv[256];
    __shared__ long bi[256];
    const int c = blockIdx.x;
    const long r0 = (long)blockIdx.y * rows, r1 = min(n, r0 + rows);
    double best = -1.0;
    long idx = -1;
    for (long p = r0 + threadIdx.x; p < r1; p += blockDim.x) {
        double v = fabs((double)U[(size_t)p * N + c]);
        if (v > best) { best = v; idx = p; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            double v2 = bv[threadIdx.x + w];
            long i2 = bi[threadIdx.x + w];
            if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 >= 0 && (bi[threadIdx.x] < 0 || i2 < bi[threadIdx.x]))) {
                bv[threadIdx.x] = v2;
                bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        work[((size_t)blockIdx.y * N + c) * 2] = bv[0];
        work[((size_t)blockIdx.y * N + c) * 2 + 1] = (double)bi[0];
    }
}
template <typename T>
__global__ void k_sign_pass2(long n, int N, T *U, int gy, const double *work) {
    const int c = blockIdx.x;
    __shared__ double sgn;
    if (threadIdx.x == 0) {
        double best = -1.0;
        long idx = -1;
        for (int y = 0; y < gy; y++) {
            double v = work[((size_t)y * N + c) * 2];
            long i = (long)work[((size_t)y * N + c) * 2 + 1];
            if (v > best) { best = v; idx = i; }
        }
        sgn = (idx >= 0 && U[(size_t)idx * N + c] < T(0)) ? -1.0 : 1.0;
    }
    __syncthreads();
    if (sgn > 0) return;
    for (long p = threadIdx.x; p < n; p += blockDim.x) U[(size_t)p * N + c] = -U[(size_t)p * N + c];
}
template <typename T>
void launch_fix_signs(long n, int N, T *U, double *work, cudaStream_t s) {
    int gy = (int)std::min<long>(64, (n + 1023) / 1024);
    long rows = (n + gy - 1) / gy;
    HQ_LAUNCH(HQ_K_SMALL, k_sign_pass1<T><<<dim3(N, gy), 256, 0, s>>>(n, N, U, rows, work));
    HQ_LAUNCH(HQ_K_SMALL, k_sign_pass2<T><<<N, 256, 0, s>>>(n, N, U, gy, work));
}

__global__ void k_extract(int rows, int cols, double alpha, const double *src, int lds,
                          double *dst, int ldd) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * cols;
         idx += gridDim.x * blockDim.x) {
        int i = idx / cols, j = idx % cols;
        dst[(size_t)i * ldd + j] = alpha * src[(size_t)i * lds + j];
    }
}
void launch_extract(int rows, int cols, double alpha, const double *src, int lds, double *dst,
                    int ldd, cudaStream_t s) {
    int tot = rows * cols;
    HQ_LAUNCH(HQ_K_SMALL, k_extract<<<std::min((tot + 255) / 256, 1024), 256, 0, s>>>(rows, cols, alpha, src, lds, dst,
                                                                ldd));
}

__global__ void k_scale_cols(int N, const double *Cv, const double *lam, double add,
                             double *out) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * N;
         idx += gridDim.x * blockDim.x) {
        int j = idx % N;
        out[idx] = -Cv[idx] * (lam[j] + add);
    }
}
void launch_scale_cols(int N, const double *Cv, const double *lam, double add, double *out,
                       cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_scale_cols<<<std::min((N * N + 255) / 256, 1024), 256, 0, s>>>(N, Cv, lam, add, out));
}

// out[0] = w * sum of all np*ncol partials (fixed order); out[1] = ||A - I||_F
// of the N x N matrix A (nullable)
__global__ void k_monitor_finish(int np, const double *part, double w, int N, const double *A,
                                 double *out) {
    __shared__ double red[256];
    double s = strided_sum(part, np, threadIdx.x, 256);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    double tot = red[0];
    __syncthreads();
    double o = 0.0;
    if (A)
        for (int i = threadIdx.x; i < N * N; i += 256) {
            double d = A[i] - ((i / N == i % N) ? 1.0 : 0.0);
            o += d * d;
        }
    red[threadIdx.x] = o;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = w * tot;
        out[1] = sqrt(red[0]);
    }
}
void launch_monitor_finish(int np, const double *part, double w, int N, const double *A,
                           double *out, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_REDUCE, k_monitor_finish<<<1, 256, 0, s>>>(np, part, w, N, A, out));
}

#define HQ_DINST(T)                                                                          \
    template void launch_gram<T>(const GramPlan &, const T *, int, const T *, int, const T *, \
                                 int, const T *, int, double, double *, double *,            \
                                 cudaStream_t);                                              \
    template void launch_tall_gemm<T>(const TallPlan &, const T *, const double *, const T *, \
                                      const double *, const T *, T *, double *,              \
                                      cudaStream_t);                                         \
    template void launch_tall_gemm_colsq<T>(const TallPlan &, const T *, const double *,      \
                                            const T *, const double *, const T *, T *,        \
                                            double *, cudaStream_t);                         \
    template void launch_fix_signs<T>(long, int, T *, double *, cudaStream_t);

HQ_DINST(double)
HQ_DINST(float)

}  // namespace hq
