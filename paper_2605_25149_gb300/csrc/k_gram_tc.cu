// Inner-product matrices <A,B> = w A^T A of FP32 tall-skinny blocks on the
// 5th-generation tensor cores (tcgen05, kind::tf32), FP32-accurate by the
// 3xTF32 split: each FP32 value a = hi + lo with hi = rna_tf32(a) and
// lo = rna_tf32(a - hi), and A^T A ~ hi^T hi + hi^T lo + lo^T hi (the dropped
// lo^T lo term is below 2^-22 relative).
//
// Work decomposition: the (na x na) symmetric output is cut into 128 x 128
// tiles (upper triangle only) and the n grid points into chunks; one CTA
// computes one tile over one chunk, accumulating in TMEM (128 lanes x 128
// FP32 columns), and writes its partial tile; a second kernel reduces the
// chunk partials in FP64 in a fixed order (deterministic).
//
// Per 32-point K-slice the 128 threads copy the tile columns of 32 point rows
// (coalesced along the columns of the point-major block) into a raw
// shared-memory stage with cp.async, three slices ahead; they split a landed
// slice into tf32 hi/lo and store it K-major with the 128-byte swizzle into a
// double-buffered MMA stage; one thread issues 12 MMAs (4 K-steps of 8 x 3
// products, M = N = 128) and commits them to the stage's mbarrier.
// Every wait is bounded: on expiry the CTA sets an error flag, stops issuing
// and still releases its TMEM.
#include "hq_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace hq {

constexpr int TC_T = 128;        // output tile edge (M = N = 128)
constexpr int TC_K = 32;         // points per slice (128 bytes of tf32 per row)
constexpr int TC_THREADS = 128;  // 4 warps: each owns 32 TMEM lanes in the epilogue
constexpr int TC_TILE_BYTES = TC_T * TC_K * 4;   // 16 KB: one operand, one of hi / lo
constexpr int TC_RAW = 3;                          // raw FP32 slices in flight (cp.async)
constexpr int TC_RAW_BYTES = TC_K * TC_T * 4;      // 16 KB: one operand's raw slice
// instruction descriptor: D f32, A/B tf32, both K-major, M = N = 128
__host__ __device__ constexpr uint32_t idesc_tf32_128x128() {
    return (1u << 4)                 // D format: F32
           | (2u << 7)               // A format: TF32
           | (2u << 10)              // B format: TF32
           | ((uint32_t)(TC_T >> 3) << 17)   // N / 8
           | ((uint32_t)(TC_T >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

struct TcPlan {
    long n;
    int na, tiles, ntiles, chunks;
    long chunk_rows;
};

__device__ __forceinline__ void tc_tile_of(int t, int tiles, int &ta, int &tb) {
    int r = 0, rem = t;
    while (rem >= tiles - r) {
        rem -= tiles - r;
        r++;
    }
    ta = r;
    tb = r + rem;
}

__device__ __forceinline__ float tc_gat(const float *X1, int n1, const float *X2, int n2, long p,
                                        int c) {
    return c < n1 ? X1[(size_t)p * n1 + c] : X2[(size_t)p * n2 + (c - n1)];
}

// Shared memory (bytes): two MMA stages [A_hi | A_lo | B_hi | B_lo] of 16 KB
// each (1024-aligned), then TC_RAW raw stages [A | B] of 16 KB each.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gram_tf32x3(TcPlan P, const float *__restrict__ X1, int n1, const float *__restrict__ X2,
                  int n2, float *__restrict__ partials, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int ta, tb;
    tc_tile_of(blockIdx.x, P.tiles, ta, tb);
    const bool diag = (ta == tb);
    const int a0 = ta * TC_T, b0 = tb * TC_T;
    const long r0 = (long)blockIdx.y * P.chunk_rows;
    const long r1 = (P.n < r0 + P.chunk_rows) ? P.n : r0 + P.chunk_rows;
    const int nslices = (int)((r1 - r0 + TC_K - 1) / TC_K);

    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TC_T)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    // Raw FP32 slices (32 point rows x 128 columns, rows of 512 bytes) are
    // copied into shared memory with cp.async, three slices ahead of the one
    // being split, so the global-memory latency overlaps the split and the
    // MMAs.  Thread t copies 16-byte chunks q = t + 128 j: row = q / 32,
    // column quad = q % 32; chunks the vector path cannot take (ragged rows
    // or columns, unaligned blocks) are written with plain loads and stores.
    unsigned char *raw = smem + 2 * 4 * TC_TILE_BYTES;   // TC_RAW stages x (A | B)
    const bool vec4 = (n1 % 4 == 0) && (n2 % 4 == 0) &&
                      (((uintptr_t)X1 & 15) == 0) && (X2 == nullptr || ((uintptr_t)X2 & 15) == 0);
    auto issue_slice = [&](int sl, unsigned char *dst, int c0) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int q = tid + TC_THREADS * j;
            const int row = q >> 5, cq = (q & 31) * 4;
            const long p = r0 + (long)sl * TC_K + row;
            const int c = c0 + cq;
            float *d = reinterpret_cast<float *>(dst + (size_t)row * 512 + cq * 4);
            if (p < r1 && vec4 && c + 3 < P.na) {
                const float *src = c < n1 ? X1 + (size_t)p * n1 + c : X2 + (size_t)p * n2 + (c - n1);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(d)),
                             "l"(src)
                             : "memory");
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    d[u] = (p < r1 && c + u < P.na) ? tc_gat(X1, n1, X2, n2, p, c + u) : 0.f;
            }
        }
    };
    auto issue_raw = [&](int sl) {
        unsigned char *dst = raw + (size_t)(sl % TC_RAW) * 2 * TC_RAW_BYTES;
        issue_slice(sl, dst, a0);
        if (!diag) issue_slice(sl, dst + TC_RAW_BYTES, b0);
    };
    // split: raw element (point row k, column i) -> K-major tile row i, k.
    // Thread = (tile row i, quad of 4 consecutive points): four 4-byte reads
    // down a raw column (consecutive i across the lanes: no bank conflicts)
    // and one 16-byte store per half (a swizzled chunk of row i).
    auto split_slice = [&](const unsigned char *src, unsigned char *hi, unsigned char *lo) {
        const float *rf = reinterpret_cast<const float *>(src);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int q = tid + TC_THREADS * j;
            const int i = q & (TC_T - 1), kq = q >> 7;
            float h[4], l[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const float v = rf[(4 * kq + t) * TC_T + i];
                h[t] = tf32_rna(v);
                l[t] = tf32_rna(v - h[t]);
            }
            const uint32_t off = sw128_offset(i, 4 * kq);
            *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
    };

    const uint32_t idesc = idesc_tf32_128x128();
    for (int sl = 0; sl < TC_RAW; sl++) {
        if (sl < nslices) issue_raw(sl);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int s = 0; s < nslices; s++) {
        const int st = s & 1;
        unsigned char *base = smem + st * 4 * TC_TILE_BYTES;
        unsigned char *Ahi = base, *Alo = base + TC_TILE_BYTES;
        unsigned char *Bhi = diag ? Ahi : base + 2 * TC_TILE_BYTES;
        unsigned char *Blo = diag ? Alo : base + 3 * TC_TILE_BYTES;
        // slice s has landed once all but the TC_RAW - 1 newest groups are done
        asm volatile("cp.async.wait_group %0;" ::"n"(TC_RAW - 1) : "memory");
        if (s >= 2) {
            if (!mbar_wait(&mbar[st], (unsigned)(((s - 2) >> 1) & 1))) atomicExch(&abort_sh, 1);
        }
        __syncthreads();
        if (abort_sh) break;
        const unsigned char *rs = raw + (size_t)(s % TC_RAW) * 2 * TC_RAW_BYTES;
        split_slice(rs, Ahi, Alo);
        if (!diag) split_slice(rs + TC_RAW_BYTES, Bhi, Blo);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s + TC_RAW < nslices) issue_raw(s + TC_RAW);
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
            const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
#pragma unroll
            for (int kk = 0; kk < TC_K / 8; kk++) {
                const uint32_t ko = kk * 32;   // 8 tf32 = 32 bytes along K
                const uint64_t dah = make_desc_sw128(ahi + ko), dal = make_desc_sw128(alo + ko);
                const uint64_t dbh = make_desc_sw128(bhi + ko), dbl = make_desc_sw128(blo + ko);
                mma_tf32(tmem, dah, dbh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            mma_commit(&mbar[st]);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // wait for the last two commits (they complete in issue order)
    bool ok = !abort_sh;
    if (ok && nslices >= 1) {
        int s = nslices - 1;
        ok = mbar_wait(&mbar[s & 1], (unsigned)((s >> 1) & 1));
        if (ok && nslices >= 2) {
            s = nslices - 2;
            ok = mbar_wait(&mbar[s & 1], (unsigned)((s >> 1) & 1));
        }
    }
    if (!ok) atomicExch(&abort_sh, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_sh) {
        if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
    } else if (nslices > 0) {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (tile rows), 32 columns at a time
        float *dst = partials + ((size_t)blockIdx.y * P.ntiles + blockIdx.x) * TC_T * TC_T;
        const int row = warp * 32 + lane;
        for (int cb = 0; cb < TC_T; cb += 32) {
            float v[32];
            tmem_ld32<32>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
            for (int j = 0; j < 32; j++) dst[(size_t)row * TC_T + cb + j] = v[j];
        }
    } else {
        float *dst = partials + ((size_t)blockIdx.y * P.ntiles + blockIdx.x) * TC_T * TC_T;
        for (int e = tid; e < TC_T * TC_T; e += TC_THREADS) dst[e] = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_T)
                     : "memory");
}

// one thread per tile entry (grid: tiles x entry blocks), chunks summed in
// order in FP64
__global__ void k_gram_tc_reduce(TcPlan P, const float *partials, double w, double *out) {
    const int tile = blockIdx.x;
    int ta, tb;
    tc_tile_of(tile, P.tiles, ta, tb);
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= TC_T * TC_T) return;
    const int la = e / TC_T, lb = e % TC_T;
    const int a = ta * TC_T + la, b = tb * TC_T + lb;
    if (a >= P.na || b >= P.na) return;
    // within a diagonal tile the MMA accumulates (i,j) and (j,i) in different
    // orders: keep the upper entry and mirror it
    if (ta == tb && la > lb) return;
    double s = 0.0;
    for (int c = 0; c < P.chunks; c++)
        s += (double)partials[((size_t)c * P.ntiles + tile) * TC_T * TC_T + e];
    s *= w;
    out[(size_t)a * P.na + b] = s;
    if (a != b) out[(size_t)b * P.na + a] = s;
}

TcPlan make_tc_plan(long n, int na) {
    TcPlan p;
    p.n = n;
    p.na = na;
    p.tiles = (na + TC_T - 1) / TC_T;
    p.ntiles = p.tiles * (p.tiles + 1) / 2;
    long target = std::max(1L, (long)(2 * 152) / p.ntiles);
    long maxchunks = std::max(1L, (n + 4 * TC_K - 1) / (4 * TC_K));
    long chunks = std::min(target, maxchunks);
    long rows = (n + chunks - 1) / chunks;
    rows = (rows + TC_K - 1) / TC_K * TC_K;
    p.chunk_rows = rows;
    p.chunks = (int)((n + rows - 1) / rows);
    return p;
}

size_t gram_tc_partial_bytes(long n, int na) {
    TcPlan p = make_tc_plan(n, na);
    return sizeof(float) * (size_t)p.chunks * p.ntiles * TC_T * TC_T;
}

size_t gram_tc_smem_bytes() { return 2 * 4 * TC_TILE_BYTES + TC_RAW * 2 * TC_RAW_BYTES + 1024; }

void launch_gram_tc(long n, const float *X1, int n1, const float *X2, int n2, double w,
                    float *partials, double *out, int *status, cudaStream_t s) {
    TcPlan p = make_tc_plan(n, n1 + n2);
    const int smem = (int)gram_tc_smem_bytes();
    tc_prepare();
    HQ_LAUNCH(HQ_K_GRAM, k_gram_tf32x3<<<dim3(p.ntiles, p.chunks), TC_THREADS, smem, s>>>(
                             p, X1, n1, X2, n2, partials, status));
    HQ_LAUNCH(HQ_K_GRAM, k_gram_tc_reduce<<<dim3(p.ntiles, (TC_T * TC_T + 255) / 256), 256, 0, s>>>(
                             p, partials, w, out));
}



// ===========================================================================
// Block x small-matrix products on tcgen05:
//   Out (n x ncol) = [A1 A2] (n x (k1 + k2)) [M1; M2] (+ Cin), FP32 blocks,
//   FP64 small matrices, 3xTF32.
// D = A B with M = 128 grid points per CTA (tile rows), N = NT output columns
// (NT = min(256, ncol rounded up to 16)), K = the block's columns in slices
// of 32.  The point rows of a point-major block are already K-major, so an A
// slice (128 points x 32 columns) is loaded, split into tf32 hi / lo and
// stored with the 128-byte swizzle exactly as in the Gram kernel.  The small
// matrix is split once per call by k_split_small into the same swizzled
// shared-memory image (per column tile and K slice), which each CTA copies
// with plain 16-byte loads.  Accumulators: TMEM, 128 lanes x NT columns.
// ===========================================================================
constexpr int TT_M = 128;
// raw A slices in flight (cp.async) for wide tiles; tiles of NT <= 64 stage A
// through registers instead, which keeps their shared memory small enough
// for two CTAs per SM
template <int NT>
__host__ __device__ constexpr int tt_raw() { return NT >= 128 ? 2 : 0; }

struct TallTcPlan {
    long n;
    int k1, k2, kpad, nslices, ncol, nt, ctiles;
};

TallTcPlan make_tall_tc_plan(long n, int k1, int k2, int ncol) {
    TallTcPlan p;
    p.n = n;
    p.k1 = k1;
    p.k2 = k2;
    p.kpad = (k1 + k2 + TC_K - 1) / TC_K * TC_K;
    p.nslices = p.kpad / TC_K;
    p.ncol = ncol;
    // instantiated tile widths (multiples of 16 up to the M = 128 limit of 256)
    const int widths[6] = {16, 32, 48, 64, 128, 256};
    p.nt = 256;
    for (int i = 0; i < 6; i++)
        if (widths[i] >= ncol) {
            p.nt = widths[i];
            break;
        }
    p.ctiles = (ncol + p.nt - 1) / p.nt;
    return p;
}

size_t tall_tc_image_bytes(int k1, int k2, int ncol) {
    TallTcPlan p = make_tall_tc_plan(1, k1, k2, ncol);
    return (size_t)p.ctiles * p.nslices * 2 * p.nt * 128;
}

// image[(ct * nslices + s)] = { hi: nt rows x 128 B, lo: nt rows x 128 B },
// row = output column c (within the tile), 32 k values per row, swizzled.
__global__ void k_split_small(TallTcPlan P, const double *M1, const double *M2,
                              unsigned char *image) {
    const long total = (long)P.ctiles * P.nt * P.kpad;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int k = (int)(idx % P.kpad);
        const long q = idx / P.kpad;
        const int r = (int)(q % P.nt);
        const int ct = (int)(q / P.nt);
        const int c = ct * P.nt + r;
        double v = 0.0;
        if (c < P.ncol) {
            if (k < P.k1) v = M1[(size_t)k * P.ncol + c];
            else if (k < P.k1 + P.k2) v = M2[(size_t)(k - P.k1) * P.ncol + c];
        }
        const float f = (float)v;
        const float h = tf32_rna(f);
        const float l = tf32_rna(f - h);
        const int s = k / TC_K, kk = k % TC_K;
        unsigned char *blk = image + ((size_t)ct * P.nslices + s) * 2 * P.nt * 128;
        const uint32_t off = sw128_offset(r, kk);
        *reinterpret_cast<float *>(blk + off) = h;
        *reinterpret_cast<float *>(blk + (size_t)P.nt * 128 + off) = l;
    }
}

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <int NT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tall_tf32x3(TallTcPlan P, const float *__restrict__ A1, const float *__restrict__ A2,
                  const unsigned char *__restrict__ image, const float *__restrict__ Cin,
                  float *__restrict__ Out, double *part_sq, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    __shared__ double red[TC_THREADS];
    constexpr int ABYTES = TT_M * 128;           // one operand half (hi or lo): 16 KB
    constexpr int BBYTES = NT * 128;             // 32 KB for NT = 256
    constexpr int STAGE = 2 * ABYTES + 2 * BBYTES;
    constexpr uint32_t TCOLS = NT < 32 ? 32 : (NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256)));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long r0 = (long)blockIdx.x * TT_M;
    const int ct = blockIdx.y;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const bool vec4 = (P.k1 % 4 == 0) && (P.k2 % 4 == 0) && (((uintptr_t)A1 & 15) == 0) &&
                      (A2 == nullptr || ((uintptr_t)A2 & 15) == 0);

    if constexpr (tt_raw<NT>() == 0) {
    // A slice: 128 points x 32 columns; thread t takes float4 q = t + 128 j:
    // row = q / 8, column quad = (q % 8) * 4
    float4 ra[8];
    auto load_a = [&](int s) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int q = tid + TC_THREADS * j;
            const int row = q >> 3, kq = (q & 7) * 4;
            const long p = r0 + row;
            const int k = s * TC_K + kq;
            if (p < P.n && vec4 && k + 3 < P.k1 + P.k2) {
                const float *src = k < P.k1 ? A1 + (size_t)p * P.k1 + k
                                            : A2 + (size_t)p * P.k2 + (k - P.k1);
                ra[j] = *reinterpret_cast<const float4 *>(src);
            } else {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int kk = k + u;
                    v[u] = 0.f;
                    if (p < P.n && kk < P.k1) v[u] = A1[(size_t)p * P.k1 + kk];
                    else if (p < P.n && kk < P.k1 + P.k2) v[u] = A2[(size_t)p * P.k2 + (kk - P.k1)];
                }
                ra[j] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    };
    auto store_a = [&](unsigned char *hi, unsigned char *lo) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int q = tid + TC_THREADS * j;
            const int row = q >> 3, kq = (q & 7) * 4;
            const float v[4] = {ra[j].x, ra[j].y, ra[j].z, ra[j].w};
            float h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                h[u] = tf32_rna(v[u]);
                l[u] = tf32_rna(v[u] - h[u]);
            }
            // the four values form one 16-byte chunk of the swizzled row
            const uint32_t off = sw128_offset(row, kq);
            *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
    };
    auto copy_b = [&](int s, unsigned char *dst) {
        const uint4 *src = reinterpret_cast<const uint4 *>(
            image + ((size_t)ct * P.nslices + s) * 2 * (size_t)BBYTES);
        uint4 *d = reinterpret_cast<uint4 *>(dst);
        for (int i = tid; i < 2 * BBYTES / 16; i += TC_THREADS) d[i] = src[i];
    };

    const uint32_t idesc = idesc_tf32(TT_M, NT);
    if (P.nslices > 0) load_a(0);
    for (int s = 0; s < P.nslices; s++) {
        const int st = s & 1;
        unsigned char *base = smem + st * STAGE;
        unsigned char *Ahi = base, *Alo = base + ABYTES, *Bhi = base + 2 * ABYTES,
                      *Blo = base + 2 * ABYTES + BBYTES;
        if (s >= 2) {
            if (!mbar_wait(&mbar[st], (unsigned)(((s - 2) >> 1) & 1))) atomicExch(&abort_sh, 1);
        }
        __syncthreads();
        if (abort_sh) break;
        store_a(Ahi, Alo);
        copy_b(s, Bhi);
        if (s + 1 < P.nslices) load_a(s + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
            const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
#pragma unroll
            for (int kk = 0; kk < TC_K / 8; kk++) {
                const uint32_t ko = kk * 32;
                const uint64_t dah = make_desc_sw128(ahi + ko), dal = make_desc_sw128(alo + ko);
                const uint64_t dbh = make_desc_sw128(bhi + ko), dbl = make_desc_sw128(blo + ko);
                mma_tf32(tmem, dah, dbh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            mma_commit(&mbar[st]);
        }
    }
    } else {
    // A slices (128 points x 32 columns, rows of 128 bytes) are copied raw
    // into shared memory with cp.async two slices ahead and split into tf32
    // hi / lo from there; the B image of slice s + 1 is copied with cp.async
    // straight into its MMA stage as soon as the MMAs of slice s - 1 that used
    // the stage have completed.  Thread t copies / splits the 16-byte chunks
    // q = t + 128 j: row = q / 8, column quad = (q % 8) * 4.
    constexpr int TT_RAW = tt_raw<NT>();
    unsigned char *raw = smem + 2 * STAGE;   // TT_RAW slices x 16 KB
    auto issue_a = [&](int sl) {
        unsigned char *dst = raw + (size_t)(sl % TT_RAW) * ABYTES;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int q = tid + TC_THREADS * j;
            const int row = q >> 3, kq = (q & 7) * 4;
            const long p = r0 + row;
            const int k = sl * TC_K + kq;
            float *d = reinterpret_cast<float *>(dst + row * 128 + kq * 4);
            if (p < P.n && vec4 && k + 3 < P.k1 + P.k2) {
                const float *src = k < P.k1 ? A1 + (size_t)p * P.k1 + k
                                            : A2 + (size_t)p * P.k2 + (k - P.k1);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(d)),
                             "l"(src)
                             : "memory");
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int kk = k + u;
                    float v = 0.f;
                    if (p < P.n && kk < P.k1) v = A1[(size_t)p * P.k1 + kk];
                    else if (p < P.n && kk < P.k1 + P.k2) v = A2[(size_t)p * P.k2 + (kk - P.k1)];
                    d[u] = v;
                }
            }
        }
    };
    auto split_a = [&](int sl, unsigned char *hi, unsigned char *lo) {
        const unsigned char *src = raw + (size_t)(sl % TT_RAW) * ABYTES;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int q = tid + TC_THREADS * j;
            const int row = q >> 3, kq = (q & 7) * 4;
            const float4 v4 = *reinterpret_cast<const float4 *>(src + row * 128 + kq * 4);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
            float h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                h[u] = tf32_rna(v[u]);
                l[u] = tf32_rna(v[u] - h[u]);
            }
            // the four values form one 16-byte chunk of the swizzled row
            const uint32_t off = sw128_offset(row, kq);
            *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
    };
    auto issue_b = [&](int sl) {
        const unsigned char *src =
            image + ((size_t)ct * P.nslices + sl) * 2 * (size_t)BBYTES;
        unsigned char *dst = smem + (sl & 1) * STAGE + 2 * ABYTES;
        for (int i = tid; i < 2 * BBYTES / 16; i += TC_THREADS)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + 16 * i)),
                         "l"(src + 16 * (size_t)i)
                         : "memory");
    };
    auto commit = [&]() { asm volatile("cp.async.commit_group;" ::: "memory"); };

    const uint32_t idesc = idesc_tf32(TT_M, NT);
    // prologue: B(0) | A(0) | A(1)
    if (P.nslices > 0) issue_b(0);
    commit();
    for (int sl = 0; sl < TT_RAW; sl++) {
        if (sl < P.nslices) issue_a(sl);
        commit();
    }
    for (int s = 0; s < P.nslices; s++) {
        const int st = s & 1;
        unsigned char *base = smem + st * STAGE;
        unsigned char *Ahi = base, *Alo = base + ABYTES, *Bhi = base + 2 * ABYTES,
                      *Blo = base + 2 * ABYTES + BBYTES;
        // B(s) and A(s) have landed once only the newest TT_RAW - 1 groups
        // (A(s + 1)) may still be in flight
        asm volatile("cp.async.wait_group %0;" ::"n"(TT_RAW - 1) : "memory");
        __syncthreads();
        if (abort_sh) break;
        split_a(s, Ahi, Alo);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
            const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
#pragma unroll
            for (int kk = 0; kk < TC_K / 8; kk++) {
                const uint32_t ko = kk * 32;
                const uint64_t dah = make_desc_sw128(ahi + ko), dal = make_desc_sw128(alo + ko);
                const uint64_t dbh = make_desc_sw128(bhi + ko), dbl = make_desc_sw128(blo + ko);
                mma_tf32(tmem, dah, dbh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            mma_commit(&mbar[st]);
        }
        // the other stage is free once the MMAs of slice s - 1 are done: copy
        // B(s + 1) there, and A(s + 2) into the raw slot A(s) just left
        if (s >= 1) {
            if (!mbar_wait(&mbar[st ^ 1], (unsigned)(((s - 1) >> 1) & 1))) atomicExch(&abort_sh, 1);
        }
        if (s + 1 < P.nslices) issue_b(s + 1);
        commit();
        if (s + TT_RAW < P.nslices) issue_a(s + TT_RAW);
        commit();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    bool ok = !abort_sh;
    if (ok && P.nslices >= 1) {
        int s = P.nslices - 1;
        ok = mbar_wait(&mbar[s & 1], (unsigned)((s >> 1) & 1));
        // the register-staged variant has not yet waited for slice n - 2
        if (tt_raw<NT>() == 0 && ok && P.nslices >= 2) {
            s = P.nslices - 2;
            ok = mbar_wait(&mbar[s & 1], (unsigned)((s >> 1) & 1));
        }
    }
    if (!ok) atomicExch(&abort_sh, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    double sq = 0.0;
    if (abort_sh) {
        if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
    } else {
        // epilogue: thread = one point row (TMEM lane), 32 columns per load;
        // 16-byte loads / stores where the row segment allows, squares summed
        // in FP32 per 32 columns and in FP64 across segments (only when the
        // sum of squares is requested)
        const long p = r0 + warp * 32 + lane;
        const bool v4 = (P.ncol % 4 == 0) && (((uintptr_t)Out & 15) == 0) &&
                        (((uintptr_t)Cin & 15) == 0);
        for (int cb = 0; cb < NT; cb += 32) {
            float v[32];
            tmem_ld32<32>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
            if (p >= P.n) continue;
            const int c0 = ct * NT + cb;
            float sqf = 0.f;
            if (v4 && cb + 32 <= NT && c0 + 32 <= P.ncol) {
                const size_t e0 = (size_t)p * P.ncol + c0;
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    float4 o = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    if (Cin) {
                        const float4 ci = *reinterpret_cast<const float4 *>(Cin + e0 + j);
                        o.x += ci.x;
                        o.y += ci.y;
                        o.z += ci.z;
                        o.w += ci.w;
                    }
                    if (Out) *reinterpret_cast<float4 *>(Out + e0 + j) = o;
                    if (part_sq) sqf += (o.x * o.x + o.y * o.y) + (o.z * o.z + o.w * o.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const int c = c0 + j;
                    if (cb + j >= NT || c >= P.ncol) continue;
                    const size_t e = (size_t)p * P.ncol + c;
                    float o = v[j];
                    if (Cin) o += Cin[e];
                    if (Out) Out[e] = o;
                    if (part_sq) sqf += o * o;
                }
            }
            if (part_sq) sq += (double)sqf;
        }
    }
    if (part_sq) {
        red[tid] = sq;
        __syncthreads();
        for (int k = TC_THREADS / 2; k > 0; k >>= 1) {
            if (tid < k) red[tid] += red[tid + k];
            __syncthreads();
        }
        if (tid == 0) part_sq[(size_t)blockIdx.x * gridDim.y + blockIdx.y] = red[0];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                     : "memory");
}

template <int NT>
static void run_tall_tc(const TallTcPlan &p, const float *A1, const float *A2,
                        const unsigned char *image, const float *Cin, float *Out, double *part_sq,
                        int *status, cudaStream_t s) {
    const int smem = 2 * (2 * TT_M * 128 + 2 * NT * 128) + tt_raw<NT>() * TT_M * 128 + 1024;
    tc_prepare();
    const unsigned gx = (unsigned)((p.n + TT_M - 1) / TT_M);
    HQ_LAUNCH(HQ_K_BLOCKGEMM,
              k_tall_tf32x3<NT><<<dim3(gx, p.ctiles), TC_THREADS, smem, s>>>(p, A1, A2, image, Cin,
                                                                             Out, part_sq, status));
}

template <int NT>
static void prep_tall() {
    const int smem = 2 * (2 * TT_M * 128 + 2 * NT * 128) + tt_raw<NT>() * TT_M * 128 + 1024;
    cudaFuncSetAttribute(k_tall_tf32x3<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

void tc_prepare() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_gram_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)gram_tc_smem_bytes());
    prep_tall<16>();
    prep_tall<32>();
    prep_tall<48>();
    prep_tall<64>();
    prep_tall<128>();
    prep_tall<256>();
    done = true;
}

int tall_tc_partials(long n, int ncol) {
    TallTcPlan p = make_tall_tc_plan(n, 4, 0, ncol);
    return (int)(((n + TT_M - 1) / TT_M) * p.ctiles);
}

void launch_tall_tc(long n, const float *A1, int k1, const double *M1, const float *A2, int k2,
                    const double *M2, int ncol, const float *Cin, float *Out, double *part_sq,
                    unsigned char *image, int *status, cudaStream_t s) {
    TallTcPlan p = make_tall_tc_plan(n, k1, k2, ncol);
    const long total = (long)p.ctiles * p.nt * p.kpad;
    HQ_LAUNCH(HQ_K_BLOCKGEMM, k_split_small<<<(int)std::min<long>((total + 255) / 256, 4096), 256, 0,
                                             s>>>(p, M1, A2 ? M2 : nullptr, image));
    switch (p.nt) {
    case 16: run_tall_tc<16>(p, A1, A2, image, Cin, Out, part_sq, status, s); break;
    case 32: run_tall_tc<32>(p, A1, A2, image, Cin, Out, part_sq, status, s); break;
    case 48: run_tall_tc<48>(p, A1, A2, image, Cin, Out, part_sq, status, s); break;
    case 64: run_tall_tc<64>(p, A1, A2, image, Cin, Out, part_sq, status, s); break;
    case 128: run_tall_tc<128>(p, A1, A2, image, Cin, Out, part_sq, status, s); break;
    case 256: run_tall_tc<256>(p, A1, A2, image, Cin, Out, part_sq, status, s); break;
    }
}

}  // namespace hq
