// The coarse levels of the FP32 multigrid V-cycle in one launch.
//
// Below a few thousand points per level the V-cycle's kernels are bound by
// launch latency: on a 16^3 level each of its ~20 launches (sweeps, residual,
// three restriction and three prolongation passes per level, the coarsest
// solve) runs for about as long as it takes to start.  The V-cycle acts on
// every column independently, so here one CTA carries one column through all
// levels from l0 down to the coarsest and back, with every level's right-hand
// side, iterates and transfer temporaries in shared memory: no grid-wide
// synchronisation, one launch per V-cycle.
//
// Each operation repeats the expression of its multi-kernel counterpart in
// k_grid.cu (damped-Jacobi sweep, residual, the 1-D transfer passes with the
// same tap tables in the same order, the coarsest solve's FP64 sums in the
// same grouping), so a column's values follow the same roundings.
#include "hq_internal.cuh"

#include <algorithm>

namespace hq {

namespace {

constexpr int VC_THREADS = 1024;

// sum of the six neighbours of point p = i + m (j + m k) in one column stored
// contiguously (zero outside the grid), grouped as nbr_sum groups them
__device__ __forceinline__ float nbr6(const float *x, int p, int i, int j, int k, int m) {
    const int sy = m, sz = m * m;
    const bool bw = i > 0, be = i < m - 1, bs = j > 0, bn = j < m - 1, bb = k > 0, bt = k < m - 1;
    const float a0 = bw ? x[p - 1] : 0.f, a1 = be ? x[p + 1] : 0.f;
    const float a2 = bs ? x[p - sy] : 0.f, a3 = bn ? x[p + sy] : 0.f;
    const float a4 = bb ? x[p - sz] : 0.f, a5 = bt ? x[p + sz] : 0.f;
    return ((a0 + a1) + (a2 + a3)) + (a4 + a5);
}

// a / d for 0 <= a < 2^22 and 1 <= d < 2^12: the quotient through the FP32
// reciprocal (relative error below 2^-23, so at most one off) and one
// correction step; a few instructions instead of an integer division's
// sequence, which dominated this kernel's index set-up per pass
__device__ __forceinline__ int fdiv(int a, int d) {
    int q = __float2int_rz(__int2float_rn(a) * __frcp_rn(__int2float_rn(d)));
    const int r = a - q * d;
    q += r < 0 ? -1 : (r >= d ? 1 : 0);
    return q;
}

__device__ __forceinline__ void decomp(int p, int m, int &i, int &j, int &k) {
    const int q = fdiv(p, m);
    i = p - q * m;
    k = fdiv(q, m);
    j = q - k * m;
}

// The points p = t, t + S, t + 2S, ... of an m^3 grid with their (i, j, k):
// the divisions happen once per pass, each step adds the precomputed
// decomposition of S with carries (the index arithmetic per point would
// otherwise be two integer divisions, more instructions than the update)
struct GridWalk {
    int p, i, j, k, di, dj, dk, m;
    __device__ __forceinline__ GridWalk(int t, int S, int m_) : p(t), m(m_) {
        decomp(t, m, i, j, k);
        decomp(S, m, di, dj, dk);
    }
    __device__ __forceinline__ void next(int S) {
        p += S;
        i += di;
        int ci = i >= m;
        i -= ci ? m : 0;
        j += dj + ci;
        int cj = j >= m;
        j -= cj ? m : 0;
        k += dk + cj;
    }
};

// z = wD r (the first sweep from zero)
__device__ void sm_first(int m, const float *wD, const float *r, float *z) {
    const int n = m * m * m;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const float w = wD[p];
        z[p] = w * r[p];
    }
}

// zout = (1 - omega) zin + wD (r + c nbrsum(zin))
__device__ void sm_jacobi(int m, const float *wD, float c, float omw, const float *r,
                          const float *zin, float *zout) {
    const int n = m * m * m;
    for (GridWalk g(threadIdx.x, blockDim.x, m); g.p < n; g.next(blockDim.x)) {
        const int p = g.p, i = g.i, j = g.j, k = g.k;
        const float s = nbr6(zin, p, i, j, k, m);
        const float w = wD[p];
        const float zc = zin[p], rv = r[p];
        zout[p] = omw * zc + w * (rv + c * s);
    }
}

// y = (b - D x) + c nbrsum(x)
__device__ void sm_resid(int m, const float *D, float c, const float *x, const float *b,
                         float *y) {
    const int n = m * m * m;
    for (GridWalk g(threadIdx.x, blockDim.x, m); g.p < n; g.next(blockDim.x)) {
        const int p = g.p, i = g.i, j = g.j, k = g.k;
        const float s = nbr6(x, p, i, j, k, m);
        const float d = D[p];
        const float xc = x[p], bb = b[p];
        y[p] = (bb - d * xc) + c * s;
    }
}

// one 1-D transfer pass on a single column (k_axis_pass with N = 1): output
// dims (o2, o1, o0), input dims equal except along `axis` (ilen); output
// index o along the axis takes taps idx[o NT + t] (-1 = none) with weights
// w[o NT + t]; out = scale sum (no add) or add + sum (scale = 1)
template <int NT>
__device__ void sm_axis(int o2, int o1, int o0, int ilen, int axis, const int *idx, const float *w,
                        float scale, const float *in, const float *add, float *out) {
    const int nout = o2 * o1 * o0;
    const int d0 = axis == 0 ? ilen : o0;
    const int d1 = axis == 1 ? ilen : o1;
    const int s1 = d0, s2 = d1 * d0;
    const int sa = axis == 0 ? 1 : (axis == 1 ? s1 : s2);
    const bool unit = scale == 1.f;
    // (i0, i1, i2) of p = t, t + S, ... by carries (one set of divisions)
    const int S = blockDim.x;
    const int t = threadIdx.x;
    const int tq = fdiv(t, o0), sq = fdiv(S, o0);
    int i0 = t - tq * o0, i2 = fdiv(tq, o1), i1 = tq - i2 * o1;
    const int s0 = S - sq * o0, s2d = fdiv(sq, o1), s1d = sq - s2d * o1;
    for (int p = threadIdx.x; p < nout; p += S) {
        if (p != (int)threadIdx.x) {
            i0 += s0;
            const int c0 = i0 >= o0;
            i0 -= c0 ? o0 : 0;
            i1 += s1d + c0;
            const int c1 = i1 >= o1;
            i1 -= c1 ? o1 : 0;
            i2 += s2d + c1;
        }
        const int oa = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
        const int ib = (axis == 0 ? 0 : i0) + (axis == 1 ? 0 : i1 * s1) + (axis == 2 ? 0 : i2 * s2);
        int ii[NT];
        float wt[NT], a[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) {
            ii[t] = idx[oa * NT + t];
            wt[t] = w[oa * NT + t];
            a[t] = ii[t] >= 0 ? in[ib + ii[t] * sa] : 0.f;
        }
        float e = 0.f;
        if (add) e = add[p];
        float acc = (add && unit) ? e : 0.f;
#pragma unroll
        for (int t = 0; t < NT; t++) {
            if (ii[t] < 0) continue;
            acc += wt[t] * a[t];
        }
        out[p] = unit ? acc : (add ? e + scale * acc : scale * acc);
    }
}

// z = Ainv r on the coarsest level: per point, eight FP64 partial sums over
// the terms qq = y, y + 8, ... (y = 0..7; one thread each), added in y order
// (the grouping of k_coarse_solve), rounded to FP32; part: 8 nc doubles
__device__ void sm_coarse(int nc, const double *__restrict__ Ainv, const float *r, float *z,
                          double *part) {
    for (int t = threadIdx.x; t < 8 * nc; t += blockDim.x) {
        const int p = t >> 3, y = t & 7;
        // nc <= 64: at most eight terms, their loads issued together
        double a[8], rv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int qq = y + 8 * u;
            a[u] = qq < nc ? __ldg(Ainv + (size_t)p * nc + qq) : 0.0;
            rv[u] = qq < nc ? (double)r[qq] : 0.0;
        }
        double acc = 0.0;
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (y + 8 * u < nc) acc += a[u] * rv[u];
        part[t] = acc;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < nc; p += blockDim.x) {
        double s = 0.0;
        for (int y = 0; y < 8; y++) s += part[p * 8 + y];
        z[p] = (float)s;
    }
}

// shared-memory layout of one column (floats unless stated): per level l the
// right-hand side r, two iterates a, b (3 n_l), then per level D and wD
// (2 n_l), the transfer temporaries (m0^2 m1 + m0 m1^2), per level pair the
// restriction taps (ridx: 6 m_{l+1} ints, rw: 6 m_{l+1}) and prolongation
// taps (pidx: 2 m_l ints, pw: 2 m_l), padding to 8 bytes, and 8 nc doubles of
// coarse-solve partials
__host__ __device__ inline size_t vc_floats(const VCoarse &v) {
    size_t f = 0;
    for (int l = 0; l < v.levels; l++) f += 5 * (size_t)v.m[l] * v.m[l] * v.m[l];
    if (v.levels > 1) f += (size_t)v.m[0] * v.m[0] * v.m[1] + (size_t)v.m[0] * v.m[1] * v.m[1];
    for (int l = 0; l + 1 < v.levels; l++) f += 12 * (size_t)v.m[l + 1] + 4 * (size_t)v.m[l];
    return (f + 1) & ~(size_t)1;
}

// Shared-memory offsets (floats) of the layout above, computed where they
// are used: the pointers the sweeps get are then visibly derived from the
// shared array (shared-memory loads and stores, no per-level pointer tables
// in local memory)
__device__ __forceinline__ int vc_n(const VCoarse &v, int l) { return v.m[l] * v.m[l] * v.m[l]; }
__device__ __forceinline__ int vc_ntot(const VCoarse &v) {
    int s = 0;
    for (int l = 0; l < v.levels; l++) s += vc_n(v, l);
    return s;
}
// r, a, b of level l: 3 sum_{i<l} n_i + {0, n_l, 2 n_l}
__device__ __forceinline__ int vc_rab(const VCoarse &v, int l) {
    int s = 0;
    for (int i = 0; i < l; i++) s += vc_n(v, i);
    return 3 * s;
}
// D, wD of level l: 3 n_tot + 2 sum_{i<l} n_i + {0, n_l}
__device__ __forceinline__ int vc_dw(const VCoarse &v, int l, int ntot) {
    int s = 0;
    for (int i = 0; i < l; i++) s += vc_n(v, i);
    return 3 * ntot + 2 * s;
}
// transfer temporaries
__device__ __forceinline__ int vc_tmp1(int ntot) { return 5 * ntot; }
__device__ __forceinline__ int vc_tmp2(const VCoarse &v, int ntot) {
    return 5 * ntot + (v.levels > 1 ? v.m[0] * v.m[0] * v.m[1] : 0);
}
// taps of level pair l -> l + 1: ridx (6 m_{l+1} ints), rw (6 m_{l+1}),
// pidx (2 m_l ints), pw (2 m_l)
__device__ __forceinline__ int vc_taps(const VCoarse &v, int l, int ntot) {
    int s = vc_tmp2(v, ntot) + (v.levels > 1 ? v.m[0] * v.m[1] * v.m[1] : 0);
    for (int i = 0; i < l; i++) s += 2 * XFER_RTAPS * v.m[i + 1] + 4 * v.m[i];
    return s;
}

// MG64 = false: r, z are FP32 blocks (rin, zout).  MG64 = true (the whole
// V-cycle of an FP32 preconditioner inside an FP64 PCG): r is read from the
// FP64 block r64 and rounded (the value k_d2f writes), z is written widened
// to the FP64 block z64, and the partial sums of r64 . z are formed as
// k_widen_dot forms them in the FP64 level geometry (TY points per row chunk
// per thread row, ppt chunks, gy partial rows: the same terms in the same
// order, so the values equal d2f + V-cycle + widen bit for bit)
template <bool MG64>
__global__ void __launch_bounds__(VC_THREADS)
    k_vcoarse(const __grid_constant__ VCoarse v, int N, const float *__restrict__ rin,
              float *__restrict__ zout, const double *__restrict__ r64, double *__restrict__ z64,
              double *part, int TY, int ppt, int gy) {
    extern __shared__ __align__(16) float vsm[];
    const int col = blockIdx.x;
    const int Lf = v.levels;   // levels in this launch: l0 .. l0 + Lf - 1 (last = coarsest)
    const int ntot = vc_ntot(v);
    int *const vsi = reinterpret_cast<int *>(vsm);
    // level tables: D and omega / D of every level, the transfer taps
    for (int l = 0; l < Lf; l++) {
        const int n = vc_n(v, l);
        float *d = vsm + vc_dw(v, l, ntot), *w = d + n;
        // four points per thread in flight: loads first, then the stores
        for (int p0 = threadIdx.x; p0 < n; p0 += 4 * blockDim.x) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int p = p0 + u * blockDim.x;
                a[u] = p < n ? __ldg(v.D[l] + p) : 0.f;
                b[u] = p < n ? __ldg(v.wD[l] + p) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int p = p0 + u * blockDim.x;
                if (p < n) {
                    d[p] = a[u];
                    w[p] = b[u];
                }
            }
        }
    }
    for (int l = 0; l + 1 < Lf; l++) {
        const int mf = v.m[l], mc = v.m[l + 1];
        const int o = vc_taps(v, l, ntot);
        int *ri = vsi + o;
        float *rw = vsm + o + XFER_RTAPS * mc;
        int *pi = vsi + o + 2 * XFER_RTAPS * mc;
        float *pw = vsm + o + 2 * XFER_RTAPS * mc + 2 * mf;
        for (int t = threadIdx.x; t < XFER_RTAPS * mc; t += blockDim.x) {
            ri[t] = __ldg(v.ridx[l] + t);
            rw[t] = __ldg(v.rw[l] + t);
        }
        for (int t = threadIdx.x; t < 2 * mf; t += blockDim.x) {
            pi[t] = __ldg(v.pidx[l] + t);
            pw[t] = __ldg(v.pw[l] + t);
        }
    }
    double *cpart = reinterpret_cast<double *>(vsm + vc_floats(v));
    float *const tmp1 = vsm + vc_tmp1(ntot);
    float *const tmp2 = vsm + vc_tmp2(v, ntot);
    // right-hand side of level l0 (column `col` of a point-major n0 x N block)
    {
        const int n0 = vc_n(v, 0);
        float *r0 = vsm + vc_rab(v, 0);
        for (int p0 = threadIdx.x; p0 < n0; p0 += 4 * blockDim.x) {
            float a[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int p = p0 + u * blockDim.x;
                if (MG64) a[u] = p < n0 ? (float)r64[(size_t)p * N + col] : 0.f;
                else a[u] = p < n0 ? rin[(size_t)p * N + col] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int p = p0 + u * blockDim.x;
                if (p < n0) r0[p] = a[u];
            }
        }
    }
    __syncthreads();
    // down: pre-smoothing, residual, restriction.  in_b: bit l set when
    // level l's pre-smoothed iterate ended in b (else in a)
    unsigned in_b = 0;
    for (int l = 0; l + 1 < Lf; l++) {
        const int m = v.m[l], mc = v.m[l + 1], n = vc_n(v, l);
        const int orab = vc_rab(v, l), odw = vc_dw(v, l, ntot), ot = vc_taps(v, l, ntot);
        const float *r = vsm + orab, *D = vsm + odw, *wD = vsm + odw + n;
        float *c0 = vsm + orab + n, *o0 = vsm + orab + 2 * n;
        bool cb = false;
        sm_first(m, wD, r, c0);
        __syncthreads();
        for (int s = 1; s < v.nu1; s++) {
            sm_jacobi(m, wD, v.c[l], v.omw, r, c0, o0);
            __syncthreads();
            float *t = c0;
            c0 = o0;
            o0 = t;
            cb = !cb;
        }
        sm_resid(m, D, v.c[l], c0, r, o0);
        __syncthreads();
        const int *ri = vsi + ot;
        const float *rw = vsm + ot + XFER_RTAPS * mc;
        sm_axis<XFER_RTAPS>(m, m, mc, m, 0, ri, rw, 1.f, o0, nullptr, tmp1);
        __syncthreads();
        sm_axis<XFER_RTAPS>(m, mc, mc, m, 1, ri, rw, 1.f, tmp1, nullptr, tmp2);
        __syncthreads();
        sm_axis<XFER_RTAPS>(mc, mc, mc, m, 2, ri, rw, v.rscale[l], tmp2, nullptr,
                            vsm + vc_rab(v, l + 1));
        __syncthreads();
        if (cb) in_b |= 1u << l;
    }
    // coarsest solve
    {
        const int oc = vc_rab(v, Lf - 1), nc = vc_n(v, Lf - 1);
        sm_coarse(v.nc, v.Ainv, vsm + oc, vsm + oc + nc, cpart);
    }
    __syncthreads();
    // the finished correction of the level below
    float *zc = vsm + vc_rab(v, Lf - 1) + vc_n(v, Lf - 1);
    // up: prolongation added to the pre-smoothed iterate, post-smoothing
    for (int l = Lf - 2; l >= 0; l--) {
        const int m = v.m[l], mc = v.m[l + 1], n = vc_n(v, l);
        const int orab = vc_rab(v, l), odw = vc_dw(v, l, ntot), ot = vc_taps(v, l, ntot);
        const float *r = vsm + orab, *wD = vsm + odw + n;
        float *a = vsm + orab + n, *b = vsm + orab + 2 * n;
        float *c0 = ((in_b >> l) & 1u) ? b : a;
        float *o0 = ((in_b >> l) & 1u) ? a : b;
        const int *pi = vsi + ot + 2 * XFER_RTAPS * mc;
        const float *pw = vsm + ot + 2 * XFER_RTAPS * mc + 2 * m;
        sm_axis<2>(m, mc, mc, mc, 2, pi, pw, 1.f, zc, nullptr, tmp2);
        __syncthreads();
        sm_axis<2>(m, m, mc, mc, 1, pi, pw, 1.f, tmp2, nullptr, tmp1);
        __syncthreads();
        sm_axis<2>(m, m, m, mc, 0, pi, pw, 1.f, tmp1, c0, o0);
        __syncthreads();
        {
            float *t = c0;
            c0 = o0;
            o0 = t;
        }
        for (int s = 0; s < v.nu2; s++) {
            sm_jacobi(m, wD, v.c[l], v.omw, r, c0, o0);
            __syncthreads();
            float *t = c0;
            c0 = o0;
            o0 = t;
        }
        zc = c0;
    }
    const int n0 = vc_n(v, 0);
    if (!MG64) {
        for (int p = threadIdx.x; p < n0; p += blockDim.x) zout[(size_t)p * N + col] = zc[p];
        return;
    }
    for (int p = threadIdx.x; p < n0; p += blockDim.x) z64[(size_t)p * N + col] = (double)zc[p];
    if (!part) return;
    // partial row `row` of column col = sum over thread rows y (in order) of
    // the sum over chunks k (in order) of r . z at p = row TY ppt + k TY + y
    double *red = cpart + 8 * v.nc;
    for (int t = threadIdx.x; t < gy * TY; t += blockDim.x) {
        const int row = fdiv(t, TY), y = t - row * TY;
        double acc = 0.0;
        for (int k = 0; k < ppt; k++) {
            const long p = (long)row * TY * ppt + (long)k * TY + y;
            if (p >= n0) continue;
            const double o = (double)zc[p];
            acc += r64[(size_t)p * N + col] * o;
        }
        red[t] = acc;
    }
    __syncthreads();
    for (int row = threadIdx.x; row < gy; row += blockDim.x) {
        double sacc = 0.0;
        for (int y = 0; y < TY; y++) sacc += red[row * TY + y];
        part[(size_t)row * N + col] = sacc;
    }
}

}  // namespace

size_t vcoarse_smem_bytes(const VCoarse &v) {
    return vc_floats(v) * sizeof(float) + 8 * sizeof(double) * (size_t)v.nc;
}

size_t vcoarse64_smem_bytes(const VCoarse &v, const GridGeom &g64) {
    return vcoarse_smem_bytes(v) + sizeof(double) * (size_t)g64.gy * g64.ty;
}

void vcoarse_prepare() {
    cudaFuncSetAttribute(k_vcoarse<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, VC_MAX_SMEM);
    cudaFuncSetAttribute(k_vcoarse<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, VC_MAX_SMEM);
}

void launch_vcoarse(const VCoarse &v, int N, const float *r, float *z, cudaStream_t s) {
    const size_t bytes = vcoarse_smem_bytes(v);
    HQ_LAUNCH_W(HQ_K_COARSE, (double)v.m[0] * v.m[0] * v.m[0] * N,
                k_vcoarse<false><<<N, VC_THREADS, bytes, s>>>(v, N, r, z, nullptr, nullptr,
                                                              nullptr, 0, 0, 0));
}

void launch_vcoarse64(const VCoarse &v, const GridGeom &g64, const double *r64, double *z64,
                      double *part, cudaStream_t s) {
    const size_t bytes = vcoarse64_smem_bytes(v, g64);
    HQ_LAUNCH_W(HQ_K_COARSE, (double)v.m[0] * v.m[0] * v.m[0] * g64.N,
                k_vcoarse<true><<<g64.N, VC_THREADS, bytes, s>>>(v, g64.N, nullptr, nullptr, r64,
                                                                 z64, part, g64.ty, g64.ppt,
                                                                 g64.gy));
}

}  // namespace hq
