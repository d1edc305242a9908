// Grid kernels of the inner solve: 7-point operator, block-PCG vector
// updates, damped-Jacobi smoothing, trilinear transfer operators, coarsest
// solve and the per-column reductions that drive the PCG recurrences.
//
// All blocks are point-major (n x N, columns fastest), so each stencil tap is
// a contiguous N-vector: a thread owns VEC consecutive columns of one point
// and every load/store is a 16-byte (or 8-byte) vector access, coalesced
// across the threads of a warp.  Reductions are per CTA in a fixed order,
// then over CTAs in a fixed order (deterministic, bit-reproducible).
#include "hq_internal.cuh"

#include <algorithm>

namespace hq {

template <typename T, int V>
struct alignas(sizeof(T) * V) VT {
    T v[V];
};

template <typename T, int V>
__device__ __forceinline__ VT<T, V> ldv(const T *p) {
    return *reinterpret_cast<const VT<T, V> *>(p);
}
template <typename T, int V>
__device__ __forceinline__ void stv(T *p, const VT<T, V> &x) {
    *reinterpret_cast<VT<T, V> *>(p) = x;
}

GridGeom make_geom(int m, int N, int elem_bytes, int block, int ctas_per_sm) {
    GridGeom g;
    g.m = m;
    g.n = (long)m * m * m;
    g.N = N;
    if (block <= 0) block = 256;
    if (ctas_per_sm <= 0) ctas_per_sm = 16;
    if (elem_bytes == 8)
        g.vec = (N % 2 == 0) ? 2 : 1;
    else
        g.vec = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 1);
    int tpr = N / g.vec;
    g.tx = tpr <= 32 ? tpr : 32;
    g.ty = std::max(1, block / g.tx);
    g.gx = (tpr + g.tx - 1) / g.tx;
    long target_gy = std::max(1L, 152L * ctas_per_sm / g.gx);
    long ppt = (g.n + (long)g.ty * target_gy - 1) / ((long)g.ty * target_gy);
    g.ppt = (int)std::max(1L, ppt);
    g.gy = (int)((g.n + (long)g.ty * g.ppt - 1) / ((long)g.ty * g.ppt));
    g.zch = 0;
    return g;
}

void enable_zmarch(GridGeom &g) {
    const long per_chunk = (long)g.gx * ((g.m + g.ty - 1) / g.ty) * g.m;   // CTAs per z-chunk
    long zch = (152L * 8 + per_chunk - 1) / per_chunk;
    zch = std::max(1L, std::min(zch, (long)std::max(1, g.m / 8)));
    g.zch = (int)zch;
}

// Per-column partial sums: each thread holds acc[V] for its columns; reduce
// over threadIdx.y in order and store one row of the partial array.  One
// thread per output (column group, slot) sums the thread rows, so the chains
// run side by side.  FP64 partials are summed in FP64 (row order as ever);
// FP32 partials in FP32 and widened once per output (the thread partials
// are FP32 sums already; widening each one made the reduction an FP64-pipe
// cost comparable to the sweep itself at GB300's FP64 rate).
template <int V, typename A>
__device__ __forceinline__ void block_col_reduce(A (&acc)[V], double *red, double *part,
                                                 int N, int col, bool cv) {
    (void)col;
    (void)cv;
    const int tx = threadIdx.x, ty = threadIdx.y, TX = blockDim.x, TY = blockDim.y;
    A *ra = reinterpret_cast<A *>(red);
#pragma unroll
    for (int v = 0; v < V; v++) ra[(ty * TX + tx) * V + v] = acc[v];
    __syncthreads();
    // TX V outputs over TX TY threads (64-thread CTAs of 32 column groups of
    // four: two outputs per thread)
    if (part)
        for (int o = ty * TX + tx; o < TX * V; o += TX * TY) {
            const int cx = o / V, vv = o - cx * V;
            const int c = (blockIdx.x * TX + cx) * V;   // the column group's first column
            if (c < N) {
                A s = A(0);
#pragma unroll 4
                for (int y = 0; y < TY; y++) s += ra[(y * TX + cx) * V + vv];
                part[(size_t)blockIdx.y * N + c + vv] = (double)s;
            }
        }
    __syncthreads();
}

// Grid coordinates of point p (p = i + m (j + m k), n = m^3 < 2^31): one 32-bit
// decomposition per thread, then an increment per visited point (the loops
// below step p by the block height), which keeps integer division out of the
// per-point work.
__device__ __forceinline__ void grid_decomp(unsigned p, unsigned m, int &i, int &j, int &kk) {
    const unsigned q = p / m;
    i = (int)(p - q * m);
    kk = (int)(q / m);
    j = (int)(q - (unsigned)kk * m);
}
__device__ __forceinline__ void grid_advance(int d, int m, int &i, int &j, int &kk) {
    i += d;
    while (i >= m) {
        i -= m;
        if (++j == m) {
            j = 0;
            ++kk;
        }
    }
}

// Sum of the six neighbours of element e (point (i, j, k) of an m^3 grid) with
// zero Dirichlet values outside.  Every load uses a clamped, always valid
// address and is masked afterwards by a select, so the compiler can issue all
// six loads back to back (no branch between them).
template <typename T, int V>
__device__ __forceinline__ VT<T, V> nbr_sum(const T *__restrict__ x, size_t e, int i, int j, int kk,
                                            int m, size_t sx, size_t sy, size_t sz) {
    const bool bw = i > 0, be = i < m - 1, bs = j > 0, bn = j < m - 1, bb = kk > 0, bt = kk < m - 1;
    VT<T, V> a0 = ldv<T, V>(x + (bw ? e - sx : e)), a1 = ldv<T, V>(x + (be ? e + sx : e));
    VT<T, V> a2 = ldv<T, V>(x + (bs ? e - sy : e)), a3 = ldv<T, V>(x + (bn ? e + sy : e));
    VT<T, V> a4 = ldv<T, V>(x + (bb ? e - sz : e)), a5 = ldv<T, V>(x + (bt ? e + sz : e));
    VT<T, V> s;
#pragma unroll
    for (int v = 0; v < V; v++)
        s.v[v] = (((bw ? a0.v[v] : T(0)) + (be ? a1.v[v] : T(0))) +
                  ((bs ? a2.v[v] : T(0)) + (bn ? a3.v[v] : T(0)))) +
                 ((bb ? a4.v[v] : T(0)) + (bt ? a5.v[v] : T(0)));
    return s;
}

// ---------------------------------------------------------------------------
// 7-point operator.  MODE 0: y = A x (+ x.y);  MODE 1: y = b - A x (+ y.y, b.b)
// A x = D x - c (x_w + x_e + x_s + x_n + x_b + x_t),  D = 6c + V + sigma.
// The residual is formed as (b - D x) + c s: two FMAs after the neighbour
// sum, one FP64-pipe instruction fewer than b - (D x - c s).
// PART: form the partial sums (a compile-time switch: in FP64 the extra
// products are a measurable share of the FP64-pipe work of a sweep).
// ---------------------------------------------------------------------------
template <typename T, int V, int MODE, bool PART>
__global__ void __launch_bounds__(256) k_stencil(int m, long n, int N, int ppt,
                                                 const T *__restrict__ D, T c,
                                                 const T *__restrict__ x,
                                                 const T *__restrict__ b, T *__restrict__ y,
                                                 double *part1, double *part2) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int col = t * V;
    const bool cv = col < N;
    T a1[V], a2[V];   // per-thread partials in the working precision
#pragma unroll
    for (int v = 0; v < V; v++) a1[v] = a2[v] = T(0);
    const size_t sx = (size_t)N, sy = (size_t)m * N, sz = (size_t)m * m * N;
    const long base = (long)blockIdx.y * TY * ppt;
    long p = base + threadIdx.y;
    int i, j, kk;
    grid_decomp((unsigned)p, (unsigned)m, i, j, kk);
    for (int k = 0; k < ppt; k++, p += TY, grid_advance(TY, m, i, j, kk)) {
        if (!cv || p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<T, V> xc = ldv<T, V>(x + e);
        VT<T, V> s = nbr_sum<T, V>(x, e, i, j, kk, m, sx, sy, sz);
        T d = D[p];
        VT<T, V> o;
        VT<T, V> bb;
        if (MODE == 1) bb = ldv<T, V>(b + e);
#pragma unroll
        for (int v = 0; v < V; v++)
            o.v[v] = MODE == 1 ? (bb.v[v] - d * xc.v[v]) + c * s.v[v] : d * xc.v[v] - c * s.v[v];
        if (MODE == 1) {
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (PART) {
                    a1[v] += o.v[v] * o.v[v];
                    a2[v] += bb.v[v] * bb.v[v];
                }
            }
        } else if (PART) {
#pragma unroll
            for (int v = 0; v < V; v++) a1[v] += xc.v[v] * o.v[v];
        }
        stv<T, V>(y + e, o);
    }
    if (PART) {
        block_col_reduce<V, T>(a1, red, part1, N, col, cv);
        if (MODE == 1 && part2) block_col_reduce<V, T>(a2, red, part2, N, col, cv);
    }
}

// x += alpha p; r -= alpha q; partial r.r; optional zf = wD r
template <typename T, int V>
__global__ void __launch_bounds__(256) k_pcg_xr(int m, long n, int N, int ppt,
                                                const double *__restrict__ alpha,
                                                const T *__restrict__ p_, const T *__restrict__ q_,
                                                T *__restrict__ x, T *__restrict__ r,
                                                double *part, const T *__restrict__ wD,
                                                T *__restrict__ zf) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    T acc[V];
    T a[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
        acc[v] = T(0);
        a[v] = cv ? (T)alpha[col + v] : T(0);
    }
    const long base = (long)blockIdx.y * TY * ppt;
    for (int k = 0; k < ppt; k++) {
        long p = base + (long)k * TY + threadIdx.y;
        if (!cv || p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<T, V> pv = ldv<T, V>(p_ + e), qv = ldv<T, V>(q_ + e), xv = ldv<T, V>(x + e),
                 rv = ldv<T, V>(r + e);
#pragma unroll
        for (int v = 0; v < V; v++) {
            xv.v[v] += a[v] * pv.v[v];
            rv.v[v] -= a[v] * qv.v[v];
            acc[v] += rv.v[v] * rv.v[v];
        }
        stv<T, V>(x + e, xv);
        stv<T, V>(r + e, rv);
        if (zf) {
            T w = wD[p];
            VT<T, V> zv;
#pragma unroll
            for (int v = 0; v < V; v++) zv.v[v] = w * rv.v[v];
            stv<T, V>(zf + e, zv);
        }
    }
    block_col_reduce<V, T>(acc, red, part, N, col, cv);
}

template <typename T, int V>
__global__ void __launch_bounds__(256) k_pcg_p(long n, int N, int ppt,
                                               const double *__restrict__ beta,
                                               const T *__restrict__ z, T *__restrict__ p_) {
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (col >= N) return;
    T bt[V];
#pragma unroll
    for (int v = 0; v < V; v++) bt[v] = (T)beta[col + v];
    const long base = (long)blockIdx.y * TY * ppt;
    for (int k = 0; k < ppt; k++) {
        long p = base + (long)k * TY + threadIdx.y;
        if (p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<T, V> zv = ldv<T, V>(z + e), pv = ldv<T, V>(p_ + e);
#pragma unroll
        for (int v = 0; v < V; v++) pv.v[v] = zv.v[v] + bt[v] * pv.v[v];
        stv<T, V>(p_ + e, pv);
    }
}

// z_out = z_in + wD (r - A z_in) = (1 - omega) z_in + wD (r + c * nbrsum(z_in))
// (wD = omega / D, so wD * D = omega); PART: partial r.z_out.
// RT: the same sweep from the pre-scaled right-hand side rt = wD r (the
// first sweep from zero, kept by the V-cycle) and wc = wD c per point:
// z_out = wc nbrsum(z_in) + ((1 - omega) z_in + rt), two FMAs after the
// neighbour sum instead of a multiply and two FMAs (FP64 levels, where the
// FP64 pipe bounds the sweep).
template <typename T, int V, bool PART, bool RT = false>
__global__ void __launch_bounds__(256) k_jacobi(int m, long n, int N, int ppt,
                                                const T *__restrict__ wD, T c, T omw,
                                                const T *__restrict__ r,
                                                const T *__restrict__ zin,
                                                T *__restrict__ zout, double *part,
                                                const T *__restrict__ rt = nullptr) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = T(0);
    const size_t sx = (size_t)N, sy = (size_t)m * N, sz = (size_t)m * m * N;
    const long base = (long)blockIdx.y * TY * ppt;
    long p = base + threadIdx.y;
    int i, j, kk;
    grid_decomp((unsigned)p, (unsigned)m, i, j, kk);
    for (int k = 0; k < ppt; k++, p += TY, grid_advance(TY, m, i, j, kk)) {
        if (!cv || p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<T, V> zc = ldv<T, V>(zin + e), rv;
        if (!RT || PART) rv = ldv<T, V>(r + e);
        VT<T, V> s = nbr_sum<T, V>(zin, e, i, j, kk, m, sx, sy, sz);
        T w = wD[p];
        VT<T, V> o;
        if (RT) {
            VT<T, V> tv = ldv<T, V>(rt + e);
#pragma unroll
            for (int v = 0; v < V; v++) o.v[v] = w * s.v[v] + (omw * zc.v[v] + tv.v[v]);
        } else {
#pragma unroll
            for (int v = 0; v < V; v++) o.v[v] = omw * zc.v[v] + w * (rv.v[v] + c * s.v[v]);
        }
#pragma unroll
        for (int v = 0; v < V; v++)
            if (PART) acc[v] += rv.v[v] * o.v[v];
        stv<T, V>(zout + e, o);
    }
    if (PART) block_col_reduce<V, T>(acc, red, part, N, col, cv);
}

// The same sweep with z-marching CTAs for blocks larger than L2: a CTA owns
// TY consecutive x-points of one y-row and walks a range of z-planes, keeping
// the z-1, z, z+1 values of its points in registers, so the z-neighbours are
// read once from memory instead of being re-read from other CTAs' rows.  The
// six-neighbour sum is formed in the same order with the same zero masks as
// nbr_sum, so the swept values are bit-identical to k_jacobi.  The optional
// partial r.z is reduced over the CTA's points (one partial row per CTA:
// part_rows() rows in all), so its summation order differs from k_jacobi's.
template <typename T, int V, bool PART, bool RT = false>
__global__ void __launch_bounds__(256) k_jacobi_zm(int m, int N, int nseg, int mz,
                                                   const T *__restrict__ wD, T c, T omw,
                                                   const T *__restrict__ r,
                                                   const T *__restrict__ zin,
                                                   T *__restrict__ zout, double *part,
                                                   const T *__restrict__ rt = nullptr) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    const int b = blockIdx.y;
    const int seg = b % nseg, rest = b / nseg;
    const int j = rest % m, zc = rest / m;
    const int i = seg * TY + threadIdx.y;
    const int k0 = zc * mz, k1 = min(m, k0 + mz);
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = T(0);
    if (cv && i < m && k0 < k1) {
        const size_t sx = (size_t)N, sy = (size_t)m * N, sz = (size_t)m * m * N;
        long p = i + (long)m * (j + (long)m * k0);
        size_t e = (size_t)p * N + col;
        const bool bw = i > 0, be = i < m - 1, bs = j > 0, bn = j < m - 1;
        VT<T, V> zero;
#pragma unroll
        for (int v = 0; v < V; v++) zero.v[v] = T(0);
        VT<T, V> zcur = ldv<T, V>(zin + e);
        VT<T, V> zprev = k0 > 0 ? ldv<T, V>(zin + e - sz) : zero;
        for (int kk = k0; kk < k1; kk++, e += sz, p += (long)m * m) {
            VT<T, V> znext = kk + 1 < m ? ldv<T, V>(zin + e + sz) : zero;
            VT<T, V> a0 = ldv<T, V>(zin + (bw ? e - sx : e)), a1 = ldv<T, V>(zin + (be ? e + sx : e));
            VT<T, V> a2 = ldv<T, V>(zin + (bs ? e - sy : e)), a3 = ldv<T, V>(zin + (bn ? e + sy : e));
            VT<T, V> rv, tv;
            if (!RT || PART) rv = ldv<T, V>(r + e);
            if (RT) tv = ldv<T, V>(rt + e);
            const T w = wD[p];
            VT<T, V> o;
#pragma unroll
            for (int v = 0; v < V; v++) {
                const T sum = (((bw ? a0.v[v] : T(0)) + (be ? a1.v[v] : T(0))) +
                               ((bs ? a2.v[v] : T(0)) + (bn ? a3.v[v] : T(0)))) +
                              (zprev.v[v] + znext.v[v]);
                if (RT) o.v[v] = w * sum + (omw * zcur.v[v] + tv.v[v]);
                else o.v[v] = omw * zcur.v[v] + w * (rv.v[v] + c * sum);
                if (PART) acc[v] += rv.v[v] * o.v[v];
            }
            stv<T, V>(zout + e, o);
            zprev = zcur;
            zcur = znext;
        }
    }
    if (PART) block_col_reduce<V, T>(acc, red, part, N, col, cv);
}

// The 7-point operator of k_stencil (MODE 0: y = A x with partial x.y;
// MODE 1: y = b - A x with partials y.y and b.b) on the z-marching CTAs of
// k_jacobi_zm: the same element values, partials reduced per CTA.
template <typename T, int V, int MODE, bool PART>
__global__ void __launch_bounds__(256) k_stencil_zm(int m, int N, int nseg, int mz,
                                                    const T *__restrict__ D, T c,
                                                    const T *__restrict__ x,
                                                    const T *__restrict__ b, T *__restrict__ y,
                                                    double *part1, double *part2) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    const int bl = blockIdx.y;
    const int seg = bl % nseg, rest = bl / nseg;
    const int j = rest % m, zc = rest / m;
    const int i = seg * TY + threadIdx.y;
    const int k0 = zc * mz, k1 = min(m, k0 + mz);
    T s1[V], s2[V];
#pragma unroll
    for (int v = 0; v < V; v++) s1[v] = s2[v] = T(0);
    if (cv && i < m && k0 < k1) {
        const size_t sx = (size_t)N, sy = (size_t)m * N, sz = (size_t)m * m * N;
        long p = i + (long)m * (j + (long)m * k0);
        size_t e = (size_t)p * N + col;
        const bool bw = i > 0, be = i < m - 1, bs = j > 0, bn = j < m - 1;
        VT<T, V> zero;
#pragma unroll
        for (int v = 0; v < V; v++) zero.v[v] = T(0);
        VT<T, V> xcur = ldv<T, V>(x + e);
        VT<T, V> xprev = k0 > 0 ? ldv<T, V>(x + e - sz) : zero;
        for (int kk = k0; kk < k1; kk++, e += sz, p += (long)m * m) {
            VT<T, V> xnext = kk + 1 < m ? ldv<T, V>(x + e + sz) : zero;
            VT<T, V> a0 = ldv<T, V>(x + (bw ? e - sx : e)), a1 = ldv<T, V>(x + (be ? e + sx : e));
            VT<T, V> a2 = ldv<T, V>(x + (bs ? e - sy : e)), a3 = ldv<T, V>(x + (bn ? e + sy : e));
            const T d = D[p];
            VT<T, V> o;
            VT<T, V> bb;
            if (MODE == 1) bb = ldv<T, V>(b + e);
#pragma unroll
            for (int v = 0; v < V; v++) {
                const T sum = (((bw ? a0.v[v] : T(0)) + (be ? a1.v[v] : T(0))) +
                               ((bs ? a2.v[v] : T(0)) + (bn ? a3.v[v] : T(0)))) +
                              (xprev.v[v] + xnext.v[v]);
                o.v[v] = MODE == 1 ? (bb.v[v] - d * xcur.v[v]) + c * sum
                                   : d * xcur.v[v] - c * sum;
            }
            if (MODE == 1) {
#pragma unroll
                for (int v = 0; v < V; v++) {
                    if (PART) {
                        s1[v] += o.v[v] * o.v[v];
                        s2[v] += bb.v[v] * bb.v[v];
                    }
                }
            } else if (PART) {
#pragma unroll
                for (int v = 0; v < V; v++) s1[v] += xcur.v[v] * o.v[v];
            }
            stv<T, V>(y + e, o);
            xprev = xcur;
            xcur = xnext;
        }
    }
    if (PART) {
        block_col_reduce<V, T>(s1, red, part1, N, col, cv);
        if (MODE == 1 && part2) block_col_reduce<V, T>(s2, red, part2, N, col, cv);
    }
}

// z = (double) z32 and partial r.z per column (FP64 geometry of the level):
// the exit of an FP32 preconditioner inside an FP64 block PCG
template <int V>
__global__ void __launch_bounds__(256) k_widen_dot(long n, int N, int ppt,
                                                   const float *__restrict__ z32,
                                                   const double *__restrict__ r,
                                                   double *__restrict__ z, double *part) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    double acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 0.0;
    const long base = (long)blockIdx.y * TY * ppt;
    for (int k = 0; k < ppt; k++) {
        long p = base + (long)k * TY + threadIdx.y;
        if (!cv || p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<double, V> rv = ldv<double, V>(r + e), o;
#pragma unroll
        for (int v = 0; v < V; v++) {
            o.v[v] = (double)z32[e + v];
            acc[v] += rv.v[v] * o.v[v];
        }
        stv<double, V>(z + e, o);
    }
    if (part) block_col_reduce<V, double>(acc, red, part, N, col, cv);
}

template <typename T, int V>
__global__ void __launch_bounds__(256) k_jacobi_first(long n, int N, int ppt,
                                                      const T *__restrict__ wD,
                                                      const T *__restrict__ r,
                                                      T *__restrict__ z) {
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (col >= N) return;
    const long base = (long)blockIdx.y * TY * ppt;
    for (int k = 0; k < ppt; k++) {
        long p = base + (long)k * TY + threadIdx.y;
        if (p >= n) continue;
        size_t e = (size_t)p * N + col;
        T w = wD[p];
        VT<T, V> rv = ldv<T, V>(r + e), o;
#pragma unroll
        for (int v = 0; v < V; v++) o.v[v] = w * rv.v[v];
        stv<T, V>(z + e, o);
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(256) k_dot(long n, int N, int ppt, const T *__restrict__ x,
                                             const T *__restrict__ y, double *part) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = T(0);
    const long base = (long)blockIdx.y * TY * ppt;
    for (int k = 0; k < ppt; k++) {
        long p = base + (long)k * TY + threadIdx.y;
        if (!cv || p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<T, V> xv = ldv<T, V>(x + e), yv = ldv<T, V>(y + e);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] += xv.v[v] * yv.v[v];
    }
    block_col_reduce<V, T>(acc, red, part, N, col, cv);
}

// ---------------------------------------------------------------------------
// Transfer operators between a grid of mf and one of mc nodes per side on the
// same box.  Fine node f (1-based) has coarse coordinate f (mc+1)/(mf+1); the
// 1-D hat weight of coarse node c for fine node f is
//   w(f, c) = (den - |f (mc+1) - c den|) / den,  den = mf + 1,
// a ratio of two integers, so every implementation obtains the same doubles.
// P = Pz (x) Py (x) Px and R = ((mc+1)/(mf+1))^3 P^T are tensor products, so
// both are applied as three 1-D passes (x, y, z), each reading its weights
// from small per-level tables built once per potential.
// ---------------------------------------------------------------------------
__global__ void k_xfer_tables(int mf, int mc, int *ridx, double *rw, float *rwf, int *pidx,
                              double *pw, float *pwf) {
    const long den = mf + 1, mcp = mc + 1;
    for (int c = threadIdx.x; c < mc; c += blockDim.x) {
        const int c1 = c + 1;
        long lo = ((long)(c1 - 1) * den) / mcp, hi = ((long)(c1 + 1) * den + mcp - 1) / mcp;
        if (lo < 1) lo = 1;
        if (hi > mf) hi = mf;
        int cnt = 0;
        for (long f = lo; f <= hi && cnt < XFER_RTAPS; f++) {
            long a = f * mcp - (long)c1 * den;
            if (a < 0) a = -a;
            if (a < den) {
                double w = (double)(den - a) / (double)den;
                ridx[c * XFER_RTAPS + cnt] = (int)(f - 1);
                rw[c * XFER_RTAPS + cnt] = w;
                rwf[c * XFER_RTAPS + cnt] = (float)w;
                cnt++;
            }
        }
        for (; cnt < XFER_RTAPS; cnt++) {
            ridx[c * XFER_RTAPS + cnt] = -1;
            rw[c * XFER_RTAPS + cnt] = 0.0;
            rwf[c * XFER_RTAPS + cnt] = 0.f;
        }
    }
    for (int f = threadIdx.x; f < mf; f += blockDim.x) {
        const long num = (long)(f + 1) * mcp;
        const int s0 = (int)(num / den);
        const long rem = num % den;
        const double w1 = (double)rem / (double)den, w0 = (double)(den - rem) / (double)den;
        const int c0 = s0, c1 = s0 + 1;   // 1-based coarse nodes
        const bool v0 = c0 >= 1 && c0 <= mc && w0 > 0.0, v1 = c1 >= 1 && c1 <= mc && w1 > 0.0;
        pidx[f * 2] = v0 ? c0 - 1 : -1;
        pw[f * 2] = v0 ? w0 : 0.0;
        pwf[f * 2] = v0 ? (float)w0 : 0.f;
        pidx[f * 2 + 1] = v1 ? c1 - 1 : -1;
        pw[f * 2 + 1] = v1 ? w1 : 0.0;
        pwf[f * 2 + 1] = v1 ? (float)w1 : 0.f;
    }
}

template <typename T>
__device__ __forceinline__ const T *wsel(const double *wd, const float *wf);
template <>
__device__ __forceinline__ const double *wsel<double>(const double *wd, const float *) { return wd; }
template <>
__device__ __forceinline__ const float *wsel<float>(const double *, const float *wf) { return wf; }

// One 1-D pass along `axis` (0 = x, fastest; 1 = y; 2 = z).  Output dims
// (o2, o1, o0), input dims equal except along the axis (ilen).  Output index
// o along the axis takes taps idx[o*NT + t] (input index, -1 = none; the
// valid taps come first) with weights w[o*NT + t]:
//   out = scale * sum_t w in          (no add)
//   out = add + sum_t w in            (scale = 1: the sum starts from add)
// With scale = 1 no multiply is issued (the restriction's x and y passes,
// every prolongation pass): in FP64 these passes are bound by the FP64 pipe,
// and a tap costs one FMA.  The taps' loads are issued before their FMAs.
template <typename T, int V, int NT>
__global__ void __launch_bounds__(256) k_axis_pass(int o2, int o1, int o0, int ilen, int axis,
                                                   int N, int ppt, const int *__restrict__ idx,
                                                   const double *__restrict__ wd,
                                                   const float *__restrict__ wf, T scale,
                                                   const T *__restrict__ in,
                                                   const T *__restrict__ add,
                                                   T *__restrict__ out) {
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (col >= N) return;
    const T *w = wsel<T>(wd, wf);
    const bool unit = scale == T(1);
    const unsigned nout = (unsigned)o2 * (unsigned)o1 * (unsigned)o0;   // m <= 1024: < 2^30
    const int d0 = axis == 0 ? ilen : o0;
    const int d1 = axis == 1 ? ilen : o1;
    const size_t s0 = (size_t)N, s1 = (size_t)d0 * N, s2 = (size_t)d1 * d0 * N;
    const size_t sa = axis == 0 ? s0 : (axis == 1 ? s1 : s2);
    const unsigned base = blockIdx.y * (unsigned)TY * (unsigned)ppt;
    for (int k = 0; k < ppt; k++) {
        const unsigned p = base + (unsigned)k * TY + threadIdx.y;
        if (p >= nout) continue;
        const unsigned i0 = p % (unsigned)o0;
        const unsigned q = p / (unsigned)o0;
        const unsigned i1 = q % (unsigned)o1;
        const unsigned i2 = q / (unsigned)o1;
        const unsigned oa = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
        const size_t ib = (axis == 0 ? 0 : (size_t)i0 * s0) + (axis == 1 ? 0 : (size_t)i1 * s1) +
                          (axis == 2 ? 0 : (size_t)i2 * s2) + col;
        const size_t oe = (size_t)p * N + col;
        int ii[NT];
        T wt[NT];
        VT<T, V> a[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) {
            ii[t] = idx[oa * NT + t];
            wt[t] = w[oa * NT + t];
            if (ii[t] >= 0) a[t] = ldv<T, V>(in + ib + (size_t)ii[t] * sa);
        }
        VT<T, V> e;
        if (add) e = ldv<T, V>(add + oe);
        T acc[V];
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = (add && unit) ? e.v[v] : T(0);
#pragma unroll
        for (int t = 0; t < NT; t++) {
            if (ii[t] < 0) continue;
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] += wt[t] * a[t].v[v];
        }
        VT<T, V> o;
#pragma unroll
        for (int v = 0; v < V; v++)
            o.v[v] = unit ? acc[v] : (add ? e.v[v] + scale * acc[v] : scale * acc[v]);
        stv<T, V>(out + oe, o);
    }
}

// z = Ainv r on the coarsest level, one coarse point per CTA: thread (x, y)
// sums the terms qq = y, y + CS_Y, ... of its column vector x in FP64, then
// the CS_Y partials are added in y order (fixed order: deterministic)
constexpr int CS_Y = 8;
template <typename T, int V>
__global__ void __launch_bounds__(256) k_coarse_solve(long nc, int N, const double *__restrict__ Ainv,
                                                      const T *__restrict__ r,
                                                      T *__restrict__ z) {
    __shared__ double red[CS_Y][256];
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    const long p = blockIdx.y;
    double acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 0.0;
    if (cv)
        for (long qq = threadIdx.y; qq < nc; qq += CS_Y) {
            const double a = Ainv[p * nc + qq];
            VT<T, V> rv = ldv<T, V>(r + (size_t)qq * N + col);
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] += a * (double)rv.v[v];
        }
#pragma unroll
    for (int v = 0; v < V; v++) red[threadIdx.y][threadIdx.x * V + v] = acc[v];
    __syncthreads();
    if (threadIdx.y == 0 && cv) {
        VT<T, V> o;
#pragma unroll
        for (int v = 0; v < V; v++) {
            double s = 0.0;
            for (int y = 0; y < CS_Y; y++) s += red[y][threadIdx.x * V + v];
            o.v[v] = (T)s;
        }
        stv<T, V>(z + (size_t)p * N + col, o);
    }
}

// ---------------------------------------------------------------------------
// per-column finalisation of the PCG recurrences.  Grid: ceil(N/32) column
// tiles x ceil(gy/FIN_ROWS) row chunks; lanes are columns (coalesced reads of
// the gy x N partials), warps split a chunk's rows.  Each CTA stores its chunk
// sums; the last CTA of a column tile to arrive (arrival counter) adds the
// chunk sums in chunk order, so the result does not depend on scheduling,
// applies the PCG update for its 32 columns and resets the counter.
// ---------------------------------------------------------------------------
constexpr int FIN_ROWS = 128;

__global__ void __launch_bounds__(256) k_finalize(int mode, int N, int gy, const double *part,
                                                  const double *part2, PcgScalars sc,
                                                  double rtol) {
    __shared__ double red[2][8][32];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int R = gridDim.y, y0 = blockIdx.y * FIN_ROWS;
    const int y1 = min(gy, y0 + FIN_ROWS);
    // all loads of a thread are issued before the additions (an add after
    // each load would serialise their latencies); the sums run in row order
    constexpr int PER = FIN_ROWS / 8;
    double v1[PER], v2[PER];
#pragma unroll
    for (int t = 0; t < PER; t++) {
        const int i = y0 + warp + 8 * t;
        const bool in = col < N && i < y1;
        v1[t] = in ? part[(size_t)i * N + col] : 0.0;
        v2[t] = (in && part2) ? part2[(size_t)i * N + col] : 0.0;
    }
    double s = 0.0, s2 = 0.0;
#pragma unroll
    for (int t = 0; t < PER; t++)
        if (y0 + warp + 8 * t < y1) {
            s += v1[t];
            s2 += v2[t];
        }
    red[0][warp][lane] = s;
    red[1][warp][lane] = s2;
    __syncthreads();
    if (warp == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; w++) {
            a += red[0][w][lane];
            b += red[1][w][lane];
        }
        if (col < N) {
            sc.fpart[(size_t)blockIdx.y * N + col] = a;
            sc.fpart[(size_t)(R + blockIdx.y) * N + col] = b;
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&sc.fcount[blockIdx.x], 1u) == (unsigned)(R - 1));
    __syncthreads();
    if (!last || warp != 0) return;
    __threadfence();
    if (lane == 0) sc.fcount[blockIdx.x] = 0u;
    if (col >= N) return;
    s = 0.0;
    s2 = 0.0;
    for (int c0 = 0; c0 < R; c0 += 8) {
        double a[8], b[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int c = c0 + u;
            a[u] = c < R ? __ldcg(&sc.fpart[(size_t)c * N + col]) : 0.0;
            b[u] = c < R ? __ldcg(&sc.fpart[(size_t)(R + c) * N + col]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (c0 + u < R) {
                s += a[u];
                s2 += b[u];
            }
    }
    switch (mode) {
    case FIN_BNORM_RNORM: {
        double rn = sqrt(s), bn = sqrt(s2);
        sc.rnorm[col] = rn;
        sc.bnorm[col] = bn;
        sc.iters[col] = 0;
        if (!isfinite(rn) || !isfinite(bn)) atomicOr(sc.status, ST_NONFINITE);
        int act = (rn > rtol * bn) ? 1 : 0;
        sc.active[col] = act;
        if (act) atomicAdd(sc.num_active, 1);
        break;
    }
    case FIN_RZ:
        sc.rz[col] = s;
        break;
    case FIN_ALPHA: {
        double a = 0.0;
        if (sc.active[col]) {
            if (!(s > 0.0) || !isfinite(s)) {
                atomicOr(sc.status, ST_BREAKDOWN);
                sc.active[col] = 0;
            } else {
                a = sc.rz[col] / s;
            }
        }
        sc.alpha[col] = a;
        break;
    }
    case FIN_RR: {
        double rn = sqrt(s);
        sc.rnorm[col] = rn;
        if (!isfinite(rn)) atomicOr(sc.status, ST_NONFINITE);
        if (sc.active[col]) {
            sc.iters[col] += 1;
            if (rn <= rtol * sc.bnorm[col] || !isfinite(rn))
                sc.active[col] = 0;
            else
                atomicAdd(sc.num_active, 1);
        }
        break;
    }
    case FIN_BETA: {
        double b = 0.0;
        if (sc.active[col]) {
            b = s / sc.rz[col];
            sc.rz[col] = s;
        }
        sc.beta[col] = b;
        break;
    }
    }
}

// Row-wise kernels of the adjoint (FP64, point-major n x N blocks):
//   mode 0: out[p] = scale * sum_c w[c] u[p][c]^2            (w nullable: 1)
//   mode 1: out[p] = scale * sum_c u[p][c] v[p][c]
__global__ void k_rowreduce(int mode, long n, int N, const double *u, const double *v,
                            const double *w, double scale, double *out) {
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x) {
        const double *ur = u + (size_t)p * N;
        double s = 0.0;
        if (mode == 0) {
            for (int c = 0; c < N; c++) s += (w ? w[c] : 1.0) * ur[c] * ur[c];
        } else {
            const double *vr = v + (size_t)p * N;
            for (int c = 0; c < N; c++) s += ur[c] * vr[c];
        }
        out[p] = scale * s;
    }
}
void launch_rowreduce(int mode, long n, int N, const double *u, const double *v, const double *w,
                      double scale, double *out, cudaStream_t s) {
    int blocks = (int)std::min<long>((n + 255) / 256, 152 * 8);
    HQ_LAUNCH(HQ_K_VECTOR, k_rowreduce<<<blocks, 256, 0, s>>>(mode, n, N, u, v, w, scale, out));
}

//   y[p][c] = g[p] * u[p][c]               (scale rows)
__global__ void k_scale_rows(long n, int N, const double *g, const double *u, double *y) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * N;
         e += (size_t)gridDim.x * blockDim.x)
        y[e] = g[e / N] * u[e];
}
void launch_scale_rows(long n, int N, const double *g, const double *u, double *y, cudaStream_t s) {
    int blocks = (int)std::min<size_t>(((size_t)n * N + 255) / 256, 152 * 16);
    HQ_LAUNCH(HQ_K_VECTOR, k_scale_rows<<<blocks, 256, 0, s>>>(n, N, g, u, y));
}

//   y[p][c] -= s[c] * x[p][c]              (per-column shift)
__global__ void k_shift_cols(long n, int N, const double *sft, const double *x, double *y) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * N;
         e += (size_t)gridDim.x * blockDim.x)
        y[e] -= sft[e % N] * x[e];
}
void launch_shift_cols(long n, int N, const double *sft, const double *x, double *y,
                       cudaStream_t s) {
    int blocks = (int)std::min<size_t>(((size_t)n * N + 255) / 256, 152 * 16);
    HQ_LAUNCH(HQ_K_VECTOR, k_shift_cols<<<blocks, 256, 0, s>>>(n, N, sft, x, y));
}

//   out[e] = a * x[e] + b * y[e]            (whole blocks, FP64)
__global__ void k_axpby(size_t count, double a, const double *x, double b, const double *y,
                        double *out) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
         e += (size_t)gridDim.x * blockDim.x)
        out[e] = a * x[e] + b * y[e];
}
void launch_axpby(size_t count, double a, const double *x, double b, const double *y, double *out,
                  cudaStream_t s) {
    int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
    HQ_LAUNCH(HQ_K_VECTOR, k_axpby<<<blocks, 256, 0, s>>>(count, a, x, b, y, out));
}

// d[p] = a[p] - b[p]; part[block] = sum of d^2 (one partial per block)
__global__ void k_diff_sq(long n, const double *a, const double *b, double *d, double *part) {
    __shared__ double red[256];
    double s = 0.0;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x) {
        const double v = a[p] - b[p];
        d[p] = v;
        s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
int launch_diff_sq(long n, const double *a, const double *b, double *d, double *part,
                   cudaStream_t s) {
    int blocks = (int)std::min<long>((n + 255) / 256, 512);
    HQ_LAUNCH(HQ_K_VECTOR, k_diff_sq<<<blocks, 256, 0, s>>>(n, a, b, d, part));
    return blocks;
}

// loop condition of the captured PCG: one more iteration was completed;
// continue while columns are active and the cap is not reached
__global__ void k_pcg_cond(const int *num_active, int *iter, int maxit,
                           cudaGraphConditionalHandle h) {
    const int it = iter[0] + 1;
    iter[0] = it;
    cudaGraphSetConditional(h, (num_active[0] > 0 && it < maxit) ? 1u : 0u);
}

// deterministic pseudo-random values in [-1, 1) (a 64-bit integer hash of
// the index; timing inputs of the autotuner, no part of the method)
template <typename T>
__global__ void k_fill_hash(long count, unsigned long long seed, T *out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
         i += (long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

// whole-phase graphs: enter the WHILE node only if a column is active
__global__ void k_pcg_cond_init(const int *num_active, int maxit, cudaGraphConditionalHandle hw) {
    cudaGraphSetConditional(hw, (num_active[0] > 0 && maxit > 0) ? 1u : 0u);
}

// whole-phase graphs, end of a loop iteration (x / r update and stopping
// test done): the IF node that follows (z = M r, beta, p) and the next
// iteration run only while columns are active and the cap is not reached
__global__ void k_pcg_cond2(const int *num_active, int *iter, int maxit,
                            cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hif,
                            long long *counters, int *status, int check_maxit) {
    const int it = iter[0] + 1;
    iter[0] = it;
    const bool act = num_active[0] > 0;
    const bool more = act && it < maxit;
    counters[0] += 1;
    if (more) counters[1] += 1;
    if (act && it >= maxit && check_maxit) atomicOr(status, ST_PCG_MAXIT);
    cudaGraphSetConditional(hif, more ? 1u : 0u);
    cudaGraphSetConditional(hw, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// setup kernels (once per potential)
// ---------------------------------------------------------------------------
__global__ void k_coarse_potential(int mf, const double *__restrict__ Vf, int mc,
                                   double *__restrict__ Vc) {
    long nc = (long)mc * mc * mc;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < nc;
         p += (long)gridDim.x * blockDim.x) {
        int t[3];
        t[0] = (int)(p % mc) + 1;
        long q = p / mc;
        t[1] = (int)(q % mc) + 1;
        t[2] = (int)(q / mc) + 1;
        int s0[3];
        double w[3][2];
        for (int d = 0; d < 3; d++) {
            long num = (long)t[d] * (mf + 1), den = mc + 1;
            s0[d] = (int)(num / den);
            long rem = num % den;
            w[d][1] = (double)rem / (double)den;
            w[d][0] = (double)(den - rem) / (double)den;
        }
        double v = 0.0;
        for (int c = 0; c < 8; c++) {
            int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
            double wt = w[0][a] * w[1][b] * w[2][e];
            if (wt == 0.0) continue;
            int fi = s0[0] + a, fj = s0[1] + b, fk = s0[2] + e;
            if (fi < 1 || fi > mf || fj < 1 || fj > mf || fk < 1 || fk > mf) continue;
            v += wt * Vf[(fi - 1) + (long)mf * ((fj - 1) + (long)mf * (fk - 1))];
        }
        Vc[p] = v;
    }
}

__global__ void k_level_diag(long n, const double *V, double sigma, double c, double omega,
                             double *D, double *wD, double *wcD) {
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n;
         p += (long)gridDim.x * blockDim.x) {
        double d = 6.0 * c + V[p] + sigma;
        D[p] = d;
        wD[p] = omega / d;
        if (wcD) wcD[p] = (omega / d) * c;
    }
}

__global__ void k_assemble_dense(int mc, double c, const double *V, double sigma, double *A) {
    long nc = (long)mc * mc * mc;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < nc * nc;
         idx += (long)gridDim.x * blockDim.x) {
        long p = idx / nc, q = idx % nc;
        double a = 0.0;
        if (p == q) {
            a = 6.0 * c + V[p] + sigma;
        } else {
            int pi = p % mc, pj = (p / mc) % mc, pk = p / (mc * mc);
            int qi = q % mc, qj = (q / mc) % mc, qk = q / (mc * mc);
            int d = abs(pi - qi) + abs(pj - qj) + abs(pk - qk);
            if (d == 1) a = -c;
        }
        A[idx] = a;
    }
}

// Gauss-Jordan inverse of an SPD matrix (no pivoting needed), one CTA.
__global__ void __launch_bounds__(256) k_gauss_jordan(int nc, double *A, double *Ainv,
                                                      int *status) {
    extern __shared__ double fcol[];
    const long n2 = (long)nc * nc;
    for (long i = threadIdx.x; i < n2; i += blockDim.x)
        Ainv[i] = (i / nc == i % nc) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < nc; k++) {
        double piv = A[(long)k * nc + k];
        if (!(piv > 0.0) || !isfinite(piv)) {
            if (threadIdx.x == 0) atomicOr(status, ST_GJ_FAIL);
            return;  // uniform: every thread reads the same pivot
        }
        __syncthreads();
        double inv = 1.0 / piv;
        for (int j = threadIdx.x; j < nc; j += blockDim.x) {
            A[(long)k * nc + j] *= inv;
            Ainv[(long)k * nc + j] *= inv;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += blockDim.x) fcol[i] = A[(long)i * nc + k];
        __syncthreads();
        for (long idx = threadIdx.x; idx < n2; idx += blockDim.x) {
            int i = (int)(idx / nc), j = (int)(idx % nc);
            if (i == k) continue;
            double f = fcol[i];
            A[idx] -= f * A[(long)k * nc + j];
            Ainv[idx] -= f * Ainv[(long)k * nc + j];
        }
        __syncthreads();
    }
}

__global__ void k_minmax(long n, const double *V, double *out) {
    __shared__ double mn[256];
    __shared__ int bad[256];
    double m = INFINITY;
    int b = 0;
    for (long p = threadIdx.x; p < n; p += blockDim.x) {
        double v = V[p];
        if (!isfinite(v)) b = 1;
        else m = fmin(m, v);
    }
    mn[threadIdx.x] = m;
    bad[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + w]);
            bad[threadIdx.x] |= bad[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = mn[0];
        out[1] = bad[0] ? 1.0 : 0.0;
    }
}

__global__ void k_d2f(size_t count, const double *in, float *out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void k_f2d(size_t count, const float *in, double *out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}
// The interface of an FP32 preconditioner inside an FP64 block PCG, fused
// into the PCG's own passes:
// k_pcg_xr_mg: x += alpha p, r -= alpha q, partial r.r (all FP64, the
// geometry of the FP64 level), and the V-cycle's entry: r32 = (float) r and
// its first damped-Jacobi sweep from zero z32 = wD32 r32 -- the values
// k_d2f and k_jacobi_first<float> would write.
template <int V>
__global__ void __launch_bounds__(256) k_pcg_xr_mg(long n, int N, int ppt,
                                                   const double *__restrict__ alpha,
                                                   const double *__restrict__ p_,
                                                   const double *__restrict__ q_,
                                                   double *__restrict__ x, double *__restrict__ r,
                                                   double *part, const float *__restrict__ wD32,
                                                   float *__restrict__ r32,
                                                   float *__restrict__ z32) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    double acc[V], a[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
        acc[v] = 0.0;
        a[v] = cv ? alpha[col + v] : 0.0;
    }
    const long base = (long)blockIdx.y * TY * ppt;
    for (int k = 0; k < ppt; k++) {
        long p = base + (long)k * TY + threadIdx.y;
        if (!cv || p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<double, V> pv = ldv<double, V>(p_ + e), qv = ldv<double, V>(q_ + e),
                      xv = ldv<double, V>(x + e), rv = ldv<double, V>(r + e);
#pragma unroll
        for (int v = 0; v < V; v++) {
            xv.v[v] += a[v] * pv.v[v];
            rv.v[v] -= a[v] * qv.v[v];
            acc[v] += rv.v[v] * rv.v[v];
        }
        stv<double, V>(x + e, xv);
        stv<double, V>(r + e, rv);
        const float w = wD32[p];
        VT<float, V> rf, zf;
#pragma unroll
        for (int v = 0; v < V; v++) {
            rf.v[v] = (float)rv.v[v];
            zf.v[v] = w * rf.v[v];
        }
        stv<float, V>(r32 + e, rf);
        stv<float, V>(z32 + e, zf);
    }
    block_col_reduce<V, double>(acc, red, part, N, col, cv);
}

// the V-cycle's last sweep on the finest FP32 level (k_jacobi<float>'s
// update) with the PCG's dot product formed in FP64 from the FP64 residual:
// partial sum of r64 . (double) z_out per column (the values k_widen_dot
// would add; its per-thread order differs)
template <int V>
__global__ void __launch_bounds__(256) k_jacobi_dot64(int m, long n, int N, int ppt,
                                                      const float *__restrict__ wD, float c,
                                                      float omw, const float *__restrict__ r,
                                                      const double *__restrict__ r64,
                                                      const float *__restrict__ zin,
                                                      float *__restrict__ zout, double *part) {
    __shared__ double red[1024];
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool cv = col < N;
    double acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 0.0;
    const size_t sx = (size_t)N, sy = (size_t)m * N, sz = (size_t)m * m * N;
    const long base = (long)blockIdx.y * TY * ppt;
    long p = base + threadIdx.y;
    int i, j, kk;
    grid_decomp((unsigned)p, (unsigned)m, i, j, kk);
    for (int k = 0; k < ppt; k++, p += TY, grid_advance(TY, m, i, j, kk)) {
        if (!cv || p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<float, V> zc = ldv<float, V>(zin + e), rv = ldv<float, V>(r + e);
        VT<float, V> sm = nbr_sum<float, V>(zin, e, i, j, kk, m, sx, sy, sz);
        VT<double, V> r8 = ldv<double, V>(r64 + e);
        const float w = wD[p];
        VT<float, V> o;
#pragma unroll
        for (int v = 0; v < V; v++) o.v[v] = omw * zc.v[v] + w * (rv.v[v] + c * sm.v[v]);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] += r8.v[v] * (double)o.v[v];
        stv<float, V>(zout + e, o);
    }
    block_col_reduce<V, double>(acc, red, part, N, col, cv);
}

// p = (double) z32 + beta p: the PCG's direction update from the FP32
// preconditioned residual (the value k_widen_dot then k_pcg_p would give)
template <int V>
__global__ void __launch_bounds__(256) k_pcg_p_mg(long n, int N, int ppt,
                                                  const double *__restrict__ beta,
                                                  const float *__restrict__ z32,
                                                  double *__restrict__ p_) {
    const int TY = blockDim.y;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (col >= N) return;
    double bt[V];
#pragma unroll
    for (int v = 0; v < V; v++) bt[v] = beta[col + v];
    const long base = (long)blockIdx.y * TY * ppt;
    for (int k = 0; k < ppt; k++) {
        long p = base + (long)k * TY + threadIdx.y;
        if (p >= n) continue;
        size_t e = (size_t)p * N + col;
        VT<float, V> zv = ldv<float, V>(z32 + e);
        VT<double, V> pv = ldv<double, V>(p_ + e);
#pragma unroll
        for (int v = 0; v < V; v++) pv.v[v] = (double)zv.v[v] + bt[v] * pv.v[v];
        stv<double, V>(p_ + e, pv);
    }
}

template <typename T>
__global__ void k_scale(size_t count, const double *factor, T *x) {
    T f = (T)factor[0];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline dim3 blk(const GridGeom &g) { return dim3(g.tx, g.ty); }
static inline dim3 grd(const GridGeom &g) { return dim3(g.gx, g.gy); }

#define HQ_VEC_DISPATCH(T, g, KERNEL, ...)                                       \
    do {                                                                         \
        if ((g).vec == 4) KERNEL<T, (sizeof(T) == 4 ? 4 : 2)>(__VA_ARGS__);       \
        else if ((g).vec == 2) KERNEL<T, 2>(__VA_ARGS__);                         \
        else KERNEL<T, 1>(__VA_ARGS__);                                           \
    } while (0)

// z-marching launch shape: nseg x-segments of TY points per y-row, m rows,
// zch z-chunks of mz planes; one CTA (and one partial row) per (segment,
// row, chunk)
static inline int zm_segments(const GridGeom &g) { return (g.m + g.ty - 1) / g.ty; }
static inline int zm_planes(const GridGeom &g) { return (g.m + g.zch - 1) / g.zch; }
static inline dim3 zm_grid(const GridGeom &g) {
    return dim3(g.gx, (unsigned)(zm_segments(g) * g.m * g.zch));
}

int part_rows(const GridGeom &g) {
    return g.zch > 0 ? zm_segments(g) * g.m * g.zch : g.gy;
}

template <typename T, int V>
static void run_apply(const GridGeom &g, const T *D, T c, const T *x, T *y, double *part,
                      cudaStream_t s) {
    const double el = (double)g.n * g.N;
    if (g.zch > 0) {
        const int ns = zm_segments(g), mz = zm_planes(g);
        if (part)
            HQ_LAUNCH_W(HQ_K_STENCIL, el, k_stencil_zm<T, V, 0, true><<<zm_grid(g), blk(g), 0, s>>>(
                                              g.m, g.N, ns, mz, D, c, x, nullptr, y, part, nullptr));
        else
            HQ_LAUNCH_W(HQ_K_STENCIL, el, k_stencil_zm<T, V, 0, false><<<zm_grid(g), blk(g), 0, s>>>(
                                              g.m, g.N, ns, mz, D, c, x, nullptr, y, part, nullptr));
        return;
    }
    if (part)
        HQ_LAUNCH_W(HQ_K_STENCIL, el, k_stencil<T, V, 0, true><<<grd(g), blk(g), 0, s>>>(
                                          g.m, g.n, g.N, g.ppt, D, c, x, nullptr, y, part, nullptr));
    else
        HQ_LAUNCH_W(HQ_K_STENCIL, el, k_stencil<T, V, 0, false><<<grd(g), blk(g), 0, s>>>(
                                          g.m, g.n, g.N, g.ppt, D, c, x, nullptr, y, part, nullptr));
}
template <typename T>
void launch_apply(const GridGeom &g, const T *D, T c, const T *x, T *y, double *part_xy,
                  cudaStream_t s) {
    HQ_VEC_DISPATCH(T, g, run_apply, g, D, c, x, y, part_xy, s);
}

template <typename T, int V>
static void run_resid(const GridGeom &g, const T *D, T c, const T *x, const T *b, T *y,
                      double *p1, double *p2, cudaStream_t s) {
    const double el = (double)g.n * g.N;
    if (p1)
        HQ_LAUNCH_W(HQ_K_RESIDUAL, el, k_stencil<T, V, 1, true><<<grd(g), blk(g), 0, s>>>(
                                           g.m, g.n, g.N, g.ppt, D, c, x, b, y, p1, p2));
    else
        HQ_LAUNCH_W(HQ_K_RESIDUAL, el, k_stencil<T, V, 1, false><<<grd(g), blk(g), 0, s>>>(
                                           g.m, g.n, g.N, g.ppt, D, c, x, b, y, p1, p2));
}
template <typename T, int V>
static void run_resid_zm(const GridGeom &g, const T *D, T c, const T *x, const T *b, T *y,
                         double *p1, double *p2, cudaStream_t s) {
    const double el = (double)g.n * g.N;
    const int ns = zm_segments(g), mz = zm_planes(g);
    if (p1)
        HQ_LAUNCH_W(HQ_K_RESIDUAL, el, k_stencil_zm<T, V, 1, true><<<zm_grid(g), blk(g), 0, s>>>(
                                           g.m, g.N, ns, mz, D, c, x, b, y, p1, p2));
    else
        HQ_LAUNCH_W(HQ_K_RESIDUAL, el, k_stencil_zm<T, V, 1, false><<<zm_grid(g), blk(g), 0, s>>>(
                                           g.m, g.N, ns, mz, D, c, x, b, y, p1, p2));
}
template <typename T>
void launch_resid(const GridGeom &g, const T *D, T c, const T *x, const T *b, T *y,
                  double *part_yy, double *part_bb, cudaStream_t s) {
    if (g.zch > 0) {
        HQ_VEC_DISPATCH(T, g, run_resid_zm, g, D, c, x, b, y, part_yy, part_bb, s);
        return;
    }
    HQ_VEC_DISPATCH(T, g, run_resid, g, D, c, x, b, y, part_yy, part_bb, s);
}

template <typename T, int V>
static void run_pcg_xr(const GridGeom &g, const double *alpha, const T *p, const T *q, T *x,
                       T *r, double *part, const T *wD, T *zf, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_VECTOR, (double)g.n * g.N, k_pcg_xr<T, V><<<grd(g), blk(g), 0, s>>>(g.m, g.n, g.N, g.ppt, alpha, p, q, x, r, part, wD,
                                             zf));
}
template <typename T>
void launch_pcg_xr(const GridGeom &g, const double *alpha, const T *p, const T *q, T *x, T *r,
                   double *part_rr, const T *wD, T *zf, cudaStream_t s) {
    HQ_VEC_DISPATCH(T, g, run_pcg_xr, g, alpha, p, q, x, r, part_rr, wD, zf, s);
}

template <typename T, int V>
static void run_pcg_p(const GridGeom &g, const double *beta, const T *z, T *p, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_VECTOR, (double)g.n * g.N, k_pcg_p<T, V><<<grd(g), blk(g), 0, s>>>(g.n, g.N, g.ppt, beta, z, p));
}
template <typename T>
void launch_pcg_p(const GridGeom &g, const double *beta, const T *z, T *p, cudaStream_t s) {
    HQ_VEC_DISPATCH(T, g, run_pcg_p, g, beta, z, p, s);
}

template <typename T, int V>
static void run_jacobi(const GridGeom &g, const T *wD, T c, T omw, const T *r, const T *zin,
                       T *zout, double *part, cudaStream_t s) {
    const double el = (double)g.n * g.N;
    if (part)
        HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi<T, V, true><<<grd(g), blk(g), 0, s>>>(
                                         g.m, g.n, g.N, g.ppt, wD, c, omw, r, zin, zout, part));
    else
        HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi<T, V, false><<<grd(g), blk(g), 0, s>>>(
                                         g.m, g.n, g.N, g.ppt, wD, c, omw, r, zin, zout, part));
}
template <typename T, int V>
static void run_jacobi_zm(const GridGeom &g, const T *wD, T c, T omw, const T *r, const T *zin,
                          T *zout, double *part, cudaStream_t s) {
    const double el = (double)g.n * g.N;
    const int ns = zm_segments(g), mz = zm_planes(g);
    if (part)
        HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi_zm<T, V, true><<<zm_grid(g), blk(g), 0, s>>>(
                                         g.m, g.N, ns, mz, wD, c, omw, r, zin, zout, part));
    else
        HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi_zm<T, V, false><<<zm_grid(g), blk(g), 0, s>>>(
                                         g.m, g.N, ns, mz, wD, c, omw, r, zin, zout, part));
}
template <typename T>
void launch_jacobi(const GridGeom &g, const T *D, const T *wD, T c, T omw, const T *r,
                   const T *zin, T *zout, double *part_rz, cudaStream_t s) {
    (void)D;
    if (g.zch > 0) {
        HQ_VEC_DISPATCH(T, g, run_jacobi_zm, g, wD, c, omw, r, zin, zout, part_rz, s);
        return;
    }
    HQ_VEC_DISPATCH(T, g, run_jacobi, g, wD, c, omw, r, zin, zout, part_rz, s);
}

// the sweep from the pre-scaled right-hand side (k_jacobi<..., RT = true>):
// wc = omega c / D per point, rt = wD r; r is read only with partials
template <typename T, int V>
static void run_jacobi_rt(const GridGeom &g, const T *wc, T omw, const T *r, const T *rt,
                          const T *zin, T *zout, double *part, cudaStream_t s) {
    const double el = (double)g.n * g.N;
    if (g.zch > 0) {
        const int ns = zm_segments(g), mz = zm_planes(g);
        if (part)
            HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi_zm<T, V, true, true><<<zm_grid(g), blk(g), 0, s>>>(
                                         g.m, g.N, ns, mz, wc, T(0), omw, r, zin, zout, part, rt));
        else
            HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi_zm<T, V, false, true><<<zm_grid(g), blk(g), 0, s>>>(
                                         g.m, g.N, ns, mz, wc, T(0), omw, r, zin, zout, part, rt));
        return;
    }
    if (part)
        HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi<T, V, true, true><<<grd(g), blk(g), 0, s>>>(
                                     g.m, g.n, g.N, g.ppt, wc, T(0), omw, r, zin, zout, part, rt));
    else
        HQ_LAUNCH_W(HQ_K_SMOOTH, el, k_jacobi<T, V, false, true><<<grd(g), blk(g), 0, s>>>(
                                     g.m, g.n, g.N, g.ppt, wc, T(0), omw, r, zin, zout, part, rt));
}
template <typename T>
void launch_jacobi_rt(const GridGeom &g, const T *wc, T omw, const T *r, const T *rt,
                      const T *zin, T *zout, double *part_rz, cudaStream_t s) {
    HQ_VEC_DISPATCH(T, g, run_jacobi_rt, g, wc, omw, r, rt, zin, zout, part_rz, s);
}

template <typename T, int V>
static void run_pcg_xr_mg(const GridGeom &g, const double *alpha, const double *p, const double *q,
                          double *x, double *r, double *part, const float *wD32, float *r32,
                          float *z32, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_VECTOR, (double)g.n * g.N,
                k_pcg_xr_mg<V><<<grd(g), blk(g), 0, s>>>(g.n, g.N, g.ppt, alpha, p, q, x, r, part,
                                                         wD32, r32, z32));
}
void launch_pcg_xr_mg(const GridGeom &g, const double *alpha, const double *p, const double *q,
                      double *x, double *r, double *part_rr, const float *wD32, float *r32,
                      float *z32, cudaStream_t s) {
    HQ_VEC_DISPATCH(double, g, run_pcg_xr_mg, g, alpha, p, q, x, r, part_rr, wD32, r32, z32, s);
}
template <typename T, int V>
static void run_jacobi_dot64(const GridGeom &g, const float *wD, float c, float omw,
                             const float *r, const double *r64, const float *zin, float *zout,
                             double *part, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_SMOOTH, (double)g.n * g.N,
                k_jacobi_dot64<V><<<grd(g), blk(g), 0, s>>>(g.m, g.n, g.N, g.ppt, wD, c, omw, r,
                                                            r64, zin, zout, part));
}
void launch_jacobi_dot64(const GridGeom &g, const float *wD, float c, float omw, const float *r,
                         const double *r64, const float *zin, float *zout, double *part,
                         cudaStream_t s) {
    HQ_VEC_DISPATCH(float, g, run_jacobi_dot64, g, wD, c, omw, r, r64, zin, zout, part, s);
}
template <typename T, int V>
static void run_pcg_p_mg(const GridGeom &g, const double *beta, const float *z32, double *p,
                         cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_VECTOR, (double)g.n * g.N,
                k_pcg_p_mg<V><<<grd(g), blk(g), 0, s>>>(g.n, g.N, g.ppt, beta, z32, p));
}
void launch_pcg_p_mg(const GridGeom &g, const double *beta, const float *z32, double *p,
                     cudaStream_t s) {
    HQ_VEC_DISPATCH(double, g, run_pcg_p_mg, g, beta, z32, p, s);
}

template <typename T, int V>
static void run_jacobi_first(const GridGeom &g, const T *wD, const T *r, T *z, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_VECTOR, (double)g.n * g.N, k_jacobi_first<T, V><<<grd(g), blk(g), 0, s>>>(g.n, g.N, g.ppt, wD, r, z));
}
template <typename T>
void launch_jacobi_first(const GridGeom &g, const T *wD, const T *r, T *z, cudaStream_t s) {
    HQ_VEC_DISPATCH(T, g, run_jacobi_first, g, wD, r, z, s);
}

GridGeom make_geom_pts(long npts, int N, int elem_bytes) {
    GridGeom g = make_geom(1, N, elem_bytes);
    g.m = 0;
    g.n = npts;
    long target_gy = std::max(1L, 152L * 16 / g.gx);
    long ppt = (npts + (long)g.ty * target_gy - 1) / ((long)g.ty * target_gy);
    g.ppt = (int)std::max(1L, ppt);
    g.gy = (int)((npts + (long)g.ty * g.ppt - 1) / ((long)g.ty * g.ppt));
    return g;
}

template <typename T, int V, int NT>
static void run_axis(const GridGeom &g, int o2, int o1, int o0, int ilen, int axis,
                     const int *idx, const double *wd, const float *wf, T scale, const T *in,
                     const T *add, T *out, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_TRANSFER, (double)g.n * g.N,
                k_axis_pass<T, V, NT><<<grd(g), blk(g), 0, s>>>(o2, o1, o0, ilen, axis, g.N, g.ppt,
                                                                idx, wd, wf, scale, in, add, out));
}

template <typename T, int NT>
static void axis_pass(int o2, int o1, int o0, int ilen, int axis, int N, const int *idx,
                      const double *wd, const float *wf, T scale, const T *in, const T *add, T *out,
                      cudaStream_t s) {
    GridGeom g = make_geom_pts((long)o2 * o1 * o0, N, (int)sizeof(T));
    if (g.vec == 4) run_axis<T, (sizeof(T) == 4 ? 4 : 2), NT>(g, o2, o1, o0, ilen, axis, idx, wd, wf, scale, in, add, out, s);
    else if (g.vec == 2) run_axis<T, 2, NT>(g, o2, o1, o0, ilen, axis, idx, wd, wf, scale, in, add, out, s);
    else run_axis<T, 1, NT>(g, o2, o1, o0, ilen, axis, idx, wd, wf, scale, in, add, out, s);
}

void launch_xfer_tables(int mf, int mc, const XferTab &t, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SETUP, k_xfer_tables<<<1, 256, 0, s>>>(mf, mc, t.ridx, t.rw, t.rwf, t.pidx,
                                                           t.pw, t.pwf));
}

// rc = ((mc+1)/(mf+1))^3 (Rz Ry Rx) rf : x pass (mf,mf,mf)->(mf,mf,mc),
// y pass ->(mf,mc,mc), z pass (scaled) ->(mc,mc,mc)
template <typename T>
void launch_restrict(int mf, int mc, int N, const XferTab &t, const T *rf, T *tmp1, T *tmp2,
                     T *rc, cudaStream_t s) {
    const double q = (double)(mc + 1) / (double)(mf + 1);
    axis_pass<T, XFER_RTAPS>(mf, mf, mc, mf, 0, N, t.ridx, t.rw, t.rwf, T(1), rf, nullptr, tmp1, s);
    axis_pass<T, XFER_RTAPS>(mf, mc, mc, mf, 1, N, t.ridx, t.rw, t.rwf, T(1), tmp1, nullptr, tmp2, s);
    axis_pass<T, XFER_RTAPS>(mc, mc, mc, mf, 2, N, t.ridx, t.rw, t.rwf, (T)(q * q * q), tmp2,
                             nullptr, rc, s);
}

// ef_out = ef_in + (Pz Py Px) ec : z pass (mc,mc,mc)->(mf,mc,mc), y pass
// ->(mf,mf,mc), x pass with the add ->(mf,mf,mf)
template <typename T>
void launch_prolong(int mf, int mc, int N, const XferTab &t, const T *ec, T *tmp1, T *tmp2,
                    const T *efin, T *efout, cudaStream_t s) {
    axis_pass<T, 2>(mf, mc, mc, mc, 2, N, t.pidx, t.pw, t.pwf, T(1), ec, nullptr, tmp2, s);
    axis_pass<T, 2>(mf, mf, mc, mc, 1, N, t.pidx, t.pw, t.pwf, T(1), tmp2, nullptr, tmp1, s);
    axis_pass<T, 2>(mf, mf, mf, mc, 0, N, t.pidx, t.pw, t.pwf, T(1), tmp1, efin, efout, s);
}

template <typename T, int V>
static void run_coarse_solve(const GridGeom &g, const double *Ainv, const T *r, T *z,
                             cudaStream_t s) {
    // one coarse point per CTA row: the FP64 products of the dense inverse
    // are spread over nc CTAs (GB300's per-SM FP64 rate is low)
    HQ_LAUNCH_W(HQ_K_COARSE, (double)g.n * g.N,
                k_coarse_solve<T, V><<<dim3(g.gx, (unsigned)g.n), dim3(g.tx, CS_Y), 0, s>>>(
                    g.n, g.N, Ainv, r, z));
}
template <typename T>
void launch_coarse_solve(const GridGeom &g, const double *Ainv, const T *r, T *z,
                         cudaStream_t s) {
    HQ_VEC_DISPATCH(T, g, run_coarse_solve, g, Ainv, r, z, s);
}

template <typename T, int V>
static void run_dot(const GridGeom &g, const T *x, const T *y, double *part, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_VECTOR, (double)g.n * g.N, k_dot<T, V><<<grd(g), blk(g), 0, s>>>(g.n, g.N, g.ppt, x, y, part));
}
template <typename T, int V>
static void run_widen_dot(const GridGeom &g, const float *z32, const double *r, double *z,
                          double *part, cudaStream_t s) {
    HQ_LAUNCH_W(HQ_K_VECTOR, (double)g.n * g.N,
                k_widen_dot<V><<<grd(g), blk(g), 0, s>>>(g.n, g.N, g.ppt, z32, r, z, part));
}
void launch_widen_dot(const GridGeom &g, const float *z32, const double *r, double *z,
                      double *part, cudaStream_t s) {
    HQ_VEC_DISPATCH(double, g, run_widen_dot, g, z32, r, z, part, s);
}

template <typename T>
void launch_dot(const GridGeom &g, const T *x, const T *y, double *part, cudaStream_t s) {
    HQ_VEC_DISPATCH(T, g, run_dot, g, x, y, part, s);
}

int finalize_chunks(int gy) { return (gy + FIN_ROWS - 1) / FIN_ROWS; }

void launch_finalize(int mode, int N, int gy, const double *part, const double *part2,
                     PcgScalars sc, double rtol, cudaStream_t s) {
    const dim3 grid((N + 31) / 32, finalize_chunks(gy));
    HQ_LAUNCH(HQ_K_REDUCE, k_finalize<<<grid, 256, 0, s>>>(mode, N, gy, part, part2, sc, rtol));
}

template <typename T>
void launch_fill_hash(long count, unsigned long long seed, T *out, cudaStream_t s) {
    const int blocks = (int)std::min<long>((count + 255) / 256, 152L * 8);
    HQ_LAUNCH(HQ_K_SETUP, k_fill_hash<T><<<blocks, 256, 0, s>>>(count, seed, out));
}
template void launch_fill_hash<float>(long, unsigned long long, float *, cudaStream_t);
template void launch_fill_hash<double>(long, unsigned long long, double *, cudaStream_t);

void launch_pcg_cond(const int *num_active, int *iter, int maxit, cudaGraphConditionalHandle h,
                     cudaStream_t s) {
    HQ_LAUNCH(HQ_K_REDUCE, k_pcg_cond<<<1, 1, 0, s>>>(num_active, iter, maxit, h));
}

void launch_pcg_cond_init(const int *num_active, int maxit, cudaGraphConditionalHandle hw,
                          cudaStream_t s) {
    HQ_LAUNCH(HQ_K_REDUCE, k_pcg_cond_init<<<1, 1, 0, s>>>(num_active, maxit, hw));
}
void launch_pcg_cond2(const int *num_active, int *iter, int maxit, cudaGraphConditionalHandle hw,
                      cudaGraphConditionalHandle hif, long long *counters, int *status,
                      int check_maxit, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_REDUCE, k_pcg_cond2<<<1, 1, 0, s>>>(num_active, iter, maxit, hw, hif, counters,
                                                        status, check_maxit));
}

void launch_coarse_potential(int mf, const double *Vf, int mc, double *Vc, cudaStream_t s) {
    long nc = (long)mc * mc * mc;
    int blocks = (int)std::min<long>((nc + 255) / 256, 4096);
    HQ_LAUNCH(HQ_K_SETUP, k_coarse_potential<<<blocks, 256, 0, s>>>(mf, Vf, mc, Vc));
}
void launch_level_diag(long n, const double *V, double sigma, double c, double omega,
                       double *D, double *wD, double *wcD, cudaStream_t s) {
    int blocks = (int)std::min<long>((n + 255) / 256, 4096);
    HQ_LAUNCH(HQ_K_SETUP, k_level_diag<<<blocks, 256, 0, s>>>(n, V, sigma, c, omega, D, wD, wcD));
}
void launch_assemble_dense(int mc, double c, const double *V, double sigma, double *A,
                           cudaStream_t s) {
    long nc = (long)mc * mc * mc;
    int blocks = (int)std::min<long>((nc * nc + 255) / 256, 4096);
    HQ_LAUNCH(HQ_K_SETUP, k_assemble_dense<<<blocks, 256, 0, s>>>(mc, c, V, sigma, A));
}
void launch_gauss_jordan(int nc, double *A, double *Ainv, int *status, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SETUP, k_gauss_jordan<<<1, 256, sizeof(double) * nc, s>>>(nc, A, Ainv, status));
}
void launch_minmax(long n, const double *V, double *out2, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_REDUCE, k_minmax<<<1, 256, 0, s>>>(n, V, out2));
}
void launch_convert_d2f(size_t count, const double *in, float *out, cudaStream_t s) {
    int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
    if (count) HQ_LAUNCH(HQ_K_VECTOR, k_d2f<<<blocks, 256, 0, s>>>(count, in, out));
}
void launch_convert_f2d(size_t count, const float *in, double *out, cudaStream_t s) {
    int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
    if (count) HQ_LAUNCH(HQ_K_VECTOR, k_f2d<<<blocks, 256, 0, s>>>(count, in, out));
}
template <typename T>
void launch_scale(size_t count, const double *factor, T *x, cudaStream_t s) {
    int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
    if (count) HQ_LAUNCH(HQ_K_VECTOR, k_scale<T><<<blocks, 256, 0, s>>>(count, factor, x));
}

#define HQ_INST(T)                                                                           \
    template void launch_apply<T>(const GridGeom &, const T *, T, const T *, T *, double *,   \
                                  cudaStream_t);                                             \
    template void launch_resid<T>(const GridGeom &, const T *, T, const T *, const T *, T *,  \
                                  double *, double *, cudaStream_t);                         \
    template void launch_pcg_xr<T>(const GridGeom &, const double *, const T *, const T *,    \
                                   T *, T *, double *, const T *, T *, cudaStream_t);        \
    template void launch_pcg_p<T>(const GridGeom &, const double *, const T *, T *,           \
                                  cudaStream_t);                                             \
    template void launch_jacobi<T>(const GridGeom &, const T *, const T *, T, T, const T *,   \
                                   const T *, T *, double *, cudaStream_t);                  \
    template void launch_jacobi_first<T>(const GridGeom &, const T *, const T *, T *,         \
                                         cudaStream_t);                                      \
    template void launch_jacobi_rt<T>(const GridGeom &, const T *, T, const T *, const T *,   \
                                      const T *, T *, double *, cudaStream_t);               \
    template void launch_restrict<T>(int, int, int, const XferTab &, const T *, T *, T *, T *, \
                                     cudaStream_t);                                          \
    template void launch_prolong<T>(int, int, int, const XferTab &, const T *, T *, T *,      \
                                    const T *, T *, cudaStream_t);                           \
    template void launch_coarse_solve<T>(const GridGeom &, const double *, const T *, T *,    \
                                         cudaStream_t);                                      \
    template void launch_dot<T>(const GridGeom &, const T *, const T *, double *,             \
                                cudaStream_t);                                               \
    template void launch_scale<T>(size_t, const double *, T *, cudaStream_t);

HQ_INST(double)
HQ_INST(float)

}  // namespace hq
