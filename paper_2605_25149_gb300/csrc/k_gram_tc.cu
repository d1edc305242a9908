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
// Per 32-point K-slice the 512 threads copy the tile columns of 32 point rows
// (coalesced along the columns of the point-major block) into a raw
// shared-memory stage with cp.async, three slices ahead; they split a landed
// slice into tf32 hi/lo and store it K-major with the 128-byte swizzle into a
// double-buffered MMA stage; one thread issues 12 MMAs (4 K-steps of 8 x 3
// products, M = N = 128) and commits them to the stage's mbarrier.
//
// Accumulation.  The tensor core's FP32 accumulator truncates each addition
// relative to its own magnitude (measured on GB300: a 3xTF32 Gram diagonal
// accumulated over 70,000 points in one TMEM accumulator came out 5.7e-4 too
// small, the error growing linearly with the points summed).  So every
// slice accumulates into a fresh TMEM accumulator (two, alternating), the
// two small cross terms first, and the threads add the slice result into
// FP32 registers (round to nearest) once its MMAs have completed: the bias
// is that of one 32-point slice.
// Every wait is bounded: on expiry the CTA sets an error flag, stops issuing
// and still releases its TMEM.
#include "hq_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace hq {

constexpr int TC_T = 128;        // output tile edge (M = N = 128)
constexpr int TC_K = 32;         // points per slice (128 bytes of tf32 per row)
constexpr int TC_THREADS = 512;  // 16 warps; warp w reads TMEM lanes 32 (w % 4)
constexpr int TC_CW = TC_T / (TC_THREADS / 128);   // columns of a thread's share (32)
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

// One 32-deep K slice of the 3xTF32 product hi hi^T + hi lo^T + lo hi^T into
// a fresh accumulator d (shared-memory addresses of the four swizzled
// K-major operand halves): the cross terms first, while the accumulator is
// small, then hi hi^T.
__device__ __forceinline__ void mma_slice_3xtf32(uint32_t d, uint32_t ahi, uint32_t alo,
                                                 uint32_t bhi, uint32_t blo, uint32_t idesc) {
#pragma unroll
    for (int kk = 0; kk < TC_K / 8; kk++) {
        const uint32_t ko = kk * 32;   // 8 tf32 = 32 bytes along K
        mma_tf32(d, make_desc_sw128(ahi + ko), make_desc_sw128(blo + ko), idesc, kk > 0 ? 1u : 0u);
        mma_tf32(d, make_desc_sw128(alo + ko), make_desc_sw128(bhi + ko), idesc, 1u);
    }
#pragma unroll
    for (int kk = 0; kk < TC_K / 8; kk++) {
        const uint32_t ko = kk * 32;
        mma_tf32(d, make_desc_sw128(ahi + ko), make_desc_sw128(bhi + ko), idesc, 1u);
    }
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
                     "r"(2 * TC_T)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;   // accumulator of slice s: columns (s & 1) * 128 + 0..127
    // this thread's share of the tile: row wl + lane (its TMEM lane), columns
    // cbeg + 0..TC_CW-1, summed over the slices in FP32 registers
    const int wl = (warp & 3) * 32, cbeg = (warp >> 2) * TC_CW;
    const uint32_t tl = tmem + ((uint32_t)wl << 16) + (uint32_t)cbeg;
    float acc[TC_CW];
#pragma unroll
    for (int j = 0; j < TC_CW; j++) acc[j] = 0.f;

    // Raw FP32 slices (32 point rows x 128 columns, rows of 512 bytes) are
    // copied into shared memory with cp.async, three slices ahead of the one
    // being split, so the global-memory latency overlaps the split and the
    // MMAs.  Thread t copies 16-byte chunks q = t + 512 j: row = q / 32,
    // column quad = q % 32; chunks the vector path cannot take (ragged rows
    // or columns, unaligned blocks) are written with plain loads and stores.
    unsigned char *raw = smem + 2 * 4 * TC_TILE_BYTES;   // TC_RAW stages x (A | B)
    const bool vec4 = (n1 % 4 == 0) && (n2 % 4 == 0) &&
                      (((uintptr_t)X1 & 15) == 0) && (X2 == nullptr || ((uintptr_t)X2 & 15) == 0);
    auto issue_slice = [&](int sl, unsigned char *dst, int c0) {
#pragma unroll
        for (int j = 0; j < TC_K * TC_T / 4 / TC_THREADS; j++) {
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
        for (int j = 0; j < TC_K * TC_T / 4 / TC_THREADS; j++) {
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
            // the MMAs of slice s - 2 (this stage, this accumulator) are
            // done: add their result into the registers (a warp-uniform
            // decision: tcgen05.ld is a whole-warp instruction)
            const bool done = __all_sync(0xffffffffu, mbar_wait(&mbar[st], (unsigned)(((s - 2) >> 1) & 1)));
            if (!done) atomicExch(&abort_sh, 1);
            else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                tmem_add32<TC_CW / 32>(tl + (uint32_t)(st * TC_T), acc);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
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
            mma_slice_3xtf32(tmem + (uint32_t)(st * TC_T), smem_u32(Ahi), smem_u32(Alo),
                             smem_u32(Bhi), smem_u32(Blo), idesc);
            mma_commit(&mbar[st]);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last two slices (their MMAs complete in issue order): add them in
    // slice order
    bool ok = !abort_sh;
    if (ok && nslices >= 1) {
        const int s = nslices - 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&mbar[s & 1], (unsigned)((s >> 1) & 1)));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok && nslices >= 2) tmem_add32<TC_CW / 32>(tl + (uint32_t)(((s - 1) & 1) * TC_T), acc);
        if (ok) tmem_add32<TC_CW / 32>(tl + (uint32_t)((s & 1) * TC_T), acc);
    }
    if (!ok) atomicExch(&abort_sh, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_sh) {
        if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
    } else if (nslices > 0) {
        float *dst = partials + ((size_t)blockIdx.y * P.ntiles + blockIdx.x) * TC_T * TC_T +
                     (size_t)(wl + lane) * TC_T + cbeg;
#pragma unroll
        for (int j = 0; j < TC_CW; j += 4)
            *reinterpret_cast<float4 *>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
    } else {
        float *dst = partials + ((size_t)blockIdx.y * P.ntiles + blockIdx.x) * TC_T * TC_T;
        for (int e = tid; e < TC_T * TC_T; e += TC_THREADS) dst[e] = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * TC_T)
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
    double s = ordered_sum(partials + (size_t)tile * TC_T * TC_T + e, P.chunks,
                           (size_t)P.ntiles * TC_T * TC_T);
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
// Work item = 128 grid points (M, the TMEM lanes) x one NT-column tile (N);
// K = the block's columns in slices of 32.  The point rows of a point-major
// block are already K-major, so an A slice (128 points x 32 columns) is
// loaded, split into tf32 hi / lo and stored with the 128-byte swizzle as in
// the Gram kernel.  The small matrix is split once per call by
// k_split_small into the same swizzled image (per column tile and K slice),
// copied into shared memory with one bulk (TMA) copy per slice.
//
// Persistent and warp-specialised: one CTA per SM walks the work items.
// Eight worker warps load and split the A slices into a three-stage ring
// and add each finished slice accumulator into FP32 registers (per-slice
// accumulation, see the Gram kernel); one control thread copies the B
// images and issues the MMAs.  The roles meet only at mbarriers: A stage
// full (worker warps arrive), B stage full (bulk-copy bytes), stage empty
// and accumulator full (MMA commits), accumulator empty (worker warps), so
// the MMAs of one slice overlap the split of the next ones and the write-out
// of a finished work item.
// ===========================================================================
constexpr int TT_M = 128;
constexpr int TT_STAGES = 3;
constexpr int TT_WORKERS = 8;                       // worker warps
constexpr int TT_THREADS = 32 * (TT_WORKERS + 1);   // + the control warp
// TMEM columns of one accumulator (a power of two, at least 32)
template <int NT>
__host__ __device__ constexpr uint32_t tt_cols() {
    return NT <= 32 ? 32u : (NT <= 64 ? 64u : 128u);
}
template <int NT>
__host__ __device__ constexpr int tt_smem() {
    return TT_STAGES * (2 * TT_M * 128 + 2 * NT * 128) + 1024;
}
// column groups of the read-out: the two worker-warp quartets take one half
// each where NT is a multiple of 64, else quartet 0 takes all columns
template <int NT>
__host__ __device__ constexpr int tt_groups() { return NT % 64 == 0 ? 2 : 1; }

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
    // instantiated tile widths (multiples of 16); wider outputs take several
    // 128-column tiles, whose CTAs run next to each other and share the A
    // rows through L2 (two accumulators of NT columns per CTA, see the kernel)
    const int widths[5] = {16, 32, 48, 64, 128};
    p.nt = 128;
    for (int i = 0; i < 5; i++)
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
__global__ void __launch_bounds__(TT_THREADS, 1)
    k_tall_tf32x3(TallTcPlan P, int nitems, const float *__restrict__ A1,
                  const float *__restrict__ A2, const unsigned char *__restrict__ image,
                  const float *__restrict__ Cin, float *__restrict__ Out, double *part_sq,
                  int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int ABYTES = TT_M * 128;           // one A half (hi or lo): 16 KB
    constexpr int BBYTES = NT * 128;             // one B half
    constexpr int STAGE = 2 * ABYTES + 2 * BBYTES;
    constexpr int S = TT_STAGES;
    constexpr int AQ = TT_M * TC_K / 4 / (32 * TT_WORKERS);   // 16-byte A chunks per thread
    constexpr uint32_t TCOLS = tt_cols<NT>();
    constexpr int G = tt_groups<NT>();
    constexpr int CW = NT / G;                   // columns per worker thread
    constexpr int NCH = (CW + 31) / 32;          // 32-column TMEM loads per slice
    constexpr int OWNERS = 4 * G;                // worker warps holding columns
    __shared__ uint64_t full_a[S], full_b[S], empty[S], accf[2], acce[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ns = P.nslices;
    auto aborted = [&]() { return *(volatile int *)&abort_sh != 0; };
    // this CTA's work items: blockIdx.x + i gridDim.x; global slice g = i ns + s
    const int my_items = blockIdx.x < nitems ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long total = (long)my_items * ns;
    if (tid == 0) {
        for (int b = 0; b < S; b++) {
            mbar_init(&full_a[b], TT_WORKERS);
            mbar_init(&full_b[b], 1);
            mbar_init(&empty[b], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], OWNERS);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(2 * TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;   // accumulator of slice g: columns (g & 1) TCOLS + ..
    auto item_of = [&](long g, int &rb, int &ct) {
        const int it = blockIdx.x + (int)(g / ns) * gridDim.x;
        rb = it / P.ctiles;
        ct = it % P.ctiles;
    };
    auto fail = [&]() {
        atomicExch(&abort_sh, 1);
        atomicOr(status, ST_TC_TIMEOUT);
    };

    if (warp == TT_WORKERS) {
        // ----------------------------------------------------------------- control
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(TT_M, NT);
            long b_issued = 0, b_landed = 0;
            auto issue_b = [&](long g) {
                int rb, ct;
                item_of(g, rb, ct);
                const unsigned char *src =
                    image + ((size_t)ct * ns + (size_t)(g % ns)) * 2 * (size_t)BBYTES;
                const int st = (int)(g % S);
                unsigned char *dst = smem + st * STAGE + 2 * ABYTES;
                mbar_expect_tx(&full_b[st], 2 * BBYTES);
                bulk_g2s(dst, src, 2 * BBYTES, &full_b[st]);
                b_issued++;
            };
            for (long g = 0; g < S - 1 && g < total; g++) issue_b(g);
            for (long g = 0; g < total && !aborted(); g++) {
                const int st = (int)(g % S);
                const unsigned u = (unsigned)((g / S) & 1);
                if (!mbar_wait(&full_a[st], u) || !mbar_wait(&full_b[st], u)) { fail(); break; }
                b_landed++;
                // the accumulator of slice g - 2 has been read out
                if (g >= 2 && !mbar_wait(&acce[g & 1], (unsigned)(((g - 2) >> 1) & 1))) { fail(); break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char *base = smem + st * STAGE;
                mma_slice_3xtf32(tmem + (uint32_t)((g & 1) * TCOLS), smem_u32(base),
                                 smem_u32(base + ABYTES), smem_u32(base + 2 * ABYTES),
                                 smem_u32(base + 2 * ABYTES + BBYTES), idesc);
                mma_commit(&empty[st]);
                mma_commit(&accf[g & 1]);
                // the B half of stage (g - 1) % S is free once the MMAs of g - 1 are done
                if (g + S - 1 < total) {
                    if (g >= 1 && !mbar_wait(&empty[(g - 1) % S], (unsigned)(((g - 1) / S) & 1))) {
                        fail();
                        break;
                    }
                    issue_b(g + S - 1);
                }
            }
            // B copies still in flight after an abort: wait for them (bounded)
            for (; b_landed < b_issued; b_landed++)
                if (!mbar_wait(&full_b[b_landed % S], (unsigned)((b_landed / S) & 1))) break;
        }
    } else {
        // ----------------------------------------------------------------- workers
        const int wt = tid;                        // 0 .. 255
        const int wl = (warp & 3) * 32, grp = warp >> 2;
        const bool owner = grp < G;                // warp-uniform
        const uint32_t tl = tmem + ((uint32_t)wl << 16) + (uint32_t)(grp * CW);
        const bool vec4 = (P.k1 % 4 == 0) && (P.k2 % 4 == 0) && (((uintptr_t)A1 & 15) == 0) &&
                          (A2 == nullptr || ((uintptr_t)A2 & 15) == 0);
        const bool v4o = (P.ncol % 4 == 0) && (((uintptr_t)Out & 15) == 0) &&
                         (((uintptr_t)Cin & 15) == 0);
        float acc[NCH * 32];
#pragma unroll
        for (int j = 0; j < NCH * 32; j++) acc[j] = 0.f;
        float4 ra[AQ];
        // A slice g into registers: chunk q = wt + 256 j: row q / 8, column quad (q % 8) * 4
        auto load_a = [&](long g) {
            int rb, ct;
            item_of(g, rb, ct);
            const long r0 = (long)rb * TT_M;
            const int k0 = (int)(g % ns) * TC_K;
#pragma unroll
            for (int j = 0; j < AQ; j++) {
                const int q = wt + 32 * TT_WORKERS * j;
                const int row = q >> 3, kq = (q & 7) * 4;
                const long p = r0 + row;
                const int k = k0 + kq;
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
        // the accumulator of slice h into registers, then release it
        auto drain = [&](long h) -> bool {
            if (!owner) return true;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&accf[h & 1], (unsigned)((h >> 1) & 1)));
            if (!ok) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tmem_add32<NCH>(tl + (uint32_t)((h & 1) * TCOLS), acc);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[h & 1]);
            return true;
        };
        // write out the finished work item of slice h, reset the sums
        auto write_item = [&](long h) {
            int rb, ct;
            item_of(h, rb, ct);
            double sq = 0.0;
            const long p = (long)rb * TT_M + wl + lane;
            if (owner && p < P.n) {
#pragma unroll
                for (int c = 0; c < NCH; c++) {
                    const int cb = grp * CW + c * 32;   // column within the tile
                    const int c0 = ct * NT + cb;
                    float sqf = 0.f;
                    if (v4o && c * 32 + 32 <= CW && c0 + 32 <= P.ncol) {
                        const size_t e0 = (size_t)p * P.ncol + c0;
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 o = make_float4(acc[c * 32 + j], acc[c * 32 + j + 1],
                                                   acc[c * 32 + j + 2], acc[c * 32 + j + 3]);
                            if (Cin) {
                                const float4 ci = __ldcs(reinterpret_cast<const float4 *>(Cin + e0 + j));
                                o.x += ci.x;
                                o.y += ci.y;
                                o.z += ci.z;
                                o.w += ci.w;
                            }
                            if (Out) __stcs(reinterpret_cast<float4 *>(Out + e0 + j), o);
                            if (part_sq) sqf += (o.x * o.x + o.y * o.y) + (o.z * o.z + o.w * o.w);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; j++) {
                            const int c1 = c0 + j;
                            if (c * 32 + j >= CW || c1 >= P.ncol) continue;
                            const size_t e = (size_t)p * P.ncol + c1;
                            float o = acc[c * 32 + j];
                            if (Cin) o += Cin[e];
                            if (Out) Out[e] = o;
                            if (part_sq) sqf += o * o;
                        }
                    }
                    if (part_sq) sq += (double)sqf;
                }
            }
#pragma unroll
            for (int j = 0; j < NCH * 32; j++) acc[j] = 0.f;
            if (part_sq) {
                // fixed butterfly within the warp; one partial per worker warp
                // and work item (summed in order by the consumer)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
                if (lane == 0) part_sq[((size_t)rb * P.ctiles + ct) * TT_WORKERS + warp] = sq;
            }
        };
        if (total > 0) load_a(0);
        for (long g = 0; g < total; g++) {
            const int st = (int)(g % S);
            unsigned char *base = smem + st * STAGE;
            // the stage is free once the MMAs of slice g - S are done
            if (g >= S && !__all_sync(0xffffffffu, mbar_wait(&empty[st], (unsigned)((g / S - 1) & 1)))) {
                fail();
                break;
            }
            if (aborted()) break;
#pragma unroll
            for (int j = 0; j < AQ; j++) {
                const int q = wt + 32 * TT_WORKERS * j;
                const int row = q >> 3, kq = (q & 7) * 4;
                const float v[4] = {ra[j].x, ra[j].y, ra[j].z, ra[j].w};
                float h[4], l[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    h[u] = tf32_rna(v[u]);
                    l[u] = tf32_rna(v[u] - h[u]);
                }
                const uint32_t off = sw128_offset(row, kq);
                *reinterpret_cast<float4 *>(base + off) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4 *>(base + ABYTES + off) = make_float4(l[0], l[1], l[2], l[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_a[st]);
            if (g + 1 < total) load_a(g + 1);
            // read out slice g - 1; a work item ends with it: write the item
            if (g >= 1) {
                if (!drain(g - 1)) {
                    fail();
                    break;
                }
                if ((g - 1) % ns == ns - 1) write_item(g - 1);
            }
        }
        if (total > 0 && !aborted()) {
            if (drain(total - 1)) write_item(total - 1);
            else fail();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * TCOLS)
                     : "memory");
}

int tall_tc_ctas() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 152;
    }
    return n;
}

template <int NT>
static void run_tall_tc(const TallTcPlan &p, const float *A1, const float *A2,
                        const unsigned char *image, const float *Cin, float *Out, double *part_sq,
                        int *status, cudaStream_t s) {
    const int smem = tt_smem<NT>();
    tc_prepare();
    const long items = (p.n + TT_M - 1) / TT_M * p.ctiles;
    const int grid = (int)std::min<long>(items, tall_tc_ctas());
    HQ_LAUNCH(HQ_K_BLOCKGEMM,
              k_tall_tf32x3<NT><<<grid, TT_THREADS, smem, s>>>(p, (int)items, A1, A2, image, Cin,
                                                               Out, part_sq, status));
}

template <int NT>
static void prep_tall() {
    const int smem = tt_smem<NT>();
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
    done = true;
}

int tall_tc_partials(long n, int ncol) {
    TallTcPlan p = make_tall_tc_plan(n, 4, 0, ncol);
    return (int)(((n + TT_M - 1) / TT_M) * p.ctiles * TT_WORKERS);
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
    }
}

}  // namespace hq
