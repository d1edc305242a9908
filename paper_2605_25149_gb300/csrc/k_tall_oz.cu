// FP64 block x small-matrix products on the tcgen05 tensor cores by exact
// integer slicing (the splitting idea of Ozaki, Ogita, Oishi and Rump, 2012).
//
//   Out (n x ncol) = [A1 A2] (n x K) [M1; M2] (K x ncol) (+ Cin), all FP64.
//
// GB300 retires about two FP64 lane operations per clock per SM, so the FP64
// SIMT form of these products is bound by the FP64 pipe.  Here every value is
// written as a scaled sum of 8 signed 7-bit integer digits:
//   A[p][k] = 2^(e_p) * sgn * sum_{i=1..8} a_i 2^(-7i)   (+ below 2^-56 |row max|),
// with e_p taken from the largest exponent of row p (points) of [A1 A2], and
// likewise for each column c of [M1; M2].  Digits are integers 0..127, exact
// in bf16.  Products of digit pairs with the same i + j = t share the scale
// 2^(-7t) and are accumulated by kind::f16 MMAs into one FP32 TMEM
// accumulator D_t; every partial sum is an integer below
// 8 * K * 127^2 < 2^24 for K <= 128, so the accumulation is exact.  Pairs with
// t <= 9 are kept (the dropped ones are below 2^-53 of |row max| |column max|
// per term).  The epilogue combines D_2..D_9 in 64-bit fixed point, converts
// once to FP64, applies 2^(e_p + f_c), adds Cin and optionally sums squares.
//
// CTA = 128 points x 64 output columns, all K; per 64-wide K chunk the 256
// threads convert the FP64 rows into 8 digit planes (K-major, 128-byte
// swizzle) while bulk copies bring the 8 digit planes of the small matrix
// (prepared once per call by k_oz_split); one thread issues 36 MMAs per K
// step of 16.  TMEM: 8 accumulators x 64 columns = 512 columns.  The output
// tile is staged in the freed digit planes for whole-row Cin reads and Out
// writes.  Every wait is bounded.
#include "hq_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace hq {

namespace {

constexpr int OZ_M = 128;                 // points per CTA (TMEM lanes)
constexpr int OZ_NT = 64;                 // output columns per CTA
constexpr int OZ_KC = 64;                 // K per chunk: 128 bytes of bf16 per row
constexpr int OZ_S = 8;                   // digits per value
constexpr int OZ_BITS = 7;                // bits per digit
constexpr int OZ_THREADS = 256;           // 8 warps: warp w reads TMEM lanes 32 (w % 4)..
constexpr int OZ_APLANE = OZ_M * 128;     // one digit plane of the point rows: 16 KB
constexpr int OZ_BPLANE = OZ_NT * 128;    // one digit plane of the small matrix: 8 KB
constexpr int OZ_SMEM = OZ_S * (OZ_APLANE + OZ_BPLANE) + 1024;
constexpr int OZ_EBAD = 0x7FF;            // biased exponent of Inf / NaN
constexpr int OZ_FRAC = 40;               // fraction bits of the fixed-point combination
constexpr int OZ_SLD = OZ_NT + 1;         // row stride (doubles) of the staged output tile
static_assert(OZ_M * OZ_SLD * 8 <= OZ_S * OZ_APLANE, "output tile fits the digit planes");

// byte offset of 16-bit element (row r, k) in a K-major tile of 64-element
// rows with the 128-byte swizzle (16-byte chunk c of row r at c ^ (r & 7))
__device__ __forceinline__ uint32_t sw128_offset16(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) +
                      ((k & 7) << 1));
}

// instruction descriptor: D f32, A/B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ int biased_exp(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// |x| / 2^(emax - 1022) with 62 fraction bits (0 for zero, subnormal, Inf,
// NaN), and the sign bit of x in bit 31
__device__ __forceinline__ unsigned long long oz_fixed(double x, int emax, uint32_t &sgn) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    sgn = (uint32_t)(b >> 32) & 0x80000000u;
    if (ex == 0 || ex == OZ_EBAD || emax == OZ_EBAD) return 0ull;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 9 + ex - emax;   // <= 9 since ex <= emax
    return sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
}

// the 8 digits of two values of one row / column relative to the biased
// exponent emax, as bf16 bit patterns of the signed integers, packed in
// pairs plane by plane (x0 in the low half).  Digit i is bits
// 55 - 7i .. 61 - 7i of the fixed-point magnitude; the signed integer +-d
// comes from one float addition, (2^23 + d) - 2^23 with the sign of x on both
// terms (+0 for d = 0), and its bf16 pattern is the upper half of the float.
__device__ __forceinline__ void oz_digits2(double x0, double x1, int emax, uint32_t (&pk)[OZ_S]) {
    uint32_t s0, s1;
    const unsigned long long f0 = oz_fixed(x0, emax, s0), f1 = oz_fixed(x1, emax, s1);
    const uint32_t c0 = 0x4B000000u | s0, c1 = 0x4B000000u | s1;
    const float a0 = s0 ? 8388608.0f : -8388608.0f, a1 = s1 ? 8388608.0f : -8388608.0f;
#pragma unroll
    for (int i = 0; i < OZ_S; i++) {
        const uint32_t d0 = (uint32_t)(f0 >> (62 - OZ_BITS * (i + 1))) & 127u;
        const uint32_t d1 = (uint32_t)(f1 >> (62 - OZ_BITS * (i + 1))) & 127u;
        const float v0 = __uint_as_float(c0 | d0) + a0;
        const float v1 = __uint_as_float(c1 | d1) + a1;
        pk[i] = __byte_perm(__float_as_uint(v0), __float_as_uint(v1), 0x7632);
    }
}

__device__ __forceinline__ double pow2(int e) {
    // 2^e for |e| <= 2000 as a product of two normal powers of two
    const int e1 = e / 2, e2 = e - e1;
    return __longlong_as_double((long long)(e1 + 1023) << 52) *
           __longlong_as_double((long long)(e2 + 1023) << 52);
}

// Digit planes of the small matrix [M1; M2] (K x ncol) in the layout the MMA
// reads: image[((ct * kchunks + ch) * 8 + j) * 8 KB] holds digit j of rows =
// output columns ct*64 .. +63 and K = ch*64 .. +63; fexp[c] = the column's
// largest biased exponent.  CTA = one column tile; thread (kg, cl) takes
// column cl and the pairs k = 2 (kg + SPL_G i), 2 (kg + SPL_G i) + 1 (the
// column maxima are reduced over the SPL_G groups in shared memory first).
constexpr int SPL_G = 16;

__global__ void __launch_bounds__(OZ_NT * SPL_G) k_oz_split(int K, int k1, int ncol, int kchunks,
                                                            const double *M1, const double *M2,
                                                            unsigned char *image, int *fexp) {
    __shared__ int emx[SPL_G][OZ_NT];
    const int ct = blockIdx.x, cl = threadIdx.x % OZ_NT, kg = threadIdx.x / OZ_NT;
    const int c = ct * OZ_NT + cl;
    auto val = [&](int k) -> double {
        if (c >= ncol || k >= K) return 0.0;
        return k < k1 ? M1[(size_t)k * ncol + c] : M2[(size_t)(k - k1) * ncol + c];
    };
    const int npairs = kchunks * OZ_KC / 2;
    int em = 0;
    for (int q = kg; q < npairs; q += SPL_G)
        em = max(em, max(biased_exp(val(2 * q)), biased_exp(val(2 * q + 1))));
    emx[kg][cl] = em;
    __syncthreads();
    em = 0;
#pragma unroll
    for (int g = 0; g < SPL_G; g++) em = max(em, emx[g][cl]);
    if (kg == 0 && c < ncol) fexp[c] = em;
    for (int q = kg; q < npairs; q += SPL_G) {
        const int k = 2 * q, ch = k / OZ_KC, kl = k % OZ_KC;
        unsigned char *base = image + (size_t)(ct * kchunks + ch) * OZ_S * OZ_BPLANE;
        uint32_t pk[OZ_S];
        oz_digits2(val(k), val(k + 1), em, pk);
        const uint32_t off = sw128_offset16(cl, kl);
#pragma unroll
        for (int j = 0; j < OZ_S; j++)
            *reinterpret_cast<uint32_t *>(base + (size_t)j * OZ_BPLANE + off) = pk[j];
    }
}

// largest biased exponent of every point row of [A1 A2] (one warp per row)
__global__ void __launch_bounds__(256) k_oz_rowexp(long n, int k1, int k2, const double *A1,
                                                   const double *A2, int *erow) {
    const int lane = threadIdx.x & 31;
    const long p = (long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (p >= n) return;
    int em = 0;
    for (int k = lane; k < k1; k += 32) em = max(em, biased_exp(A1[(size_t)p * k1 + k]));
    for (int k = lane; k < k2; k += 32) em = max(em, biased_exp(A2[(size_t)p * k2 + k]));
    for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
    if (lane == 0) erow[p] = em;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_tall_oz(long n, int k1, int k2, int ncol, int kchunks, const double *__restrict__ A1,
              const double *__restrict__ A2, const unsigned char *__restrict__ image,
              const int *__restrict__ fexp, const int *__restrict__ erow_g,
              const double *__restrict__ Cin, double *__restrict__ Out, double *part_sq,
              int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *planesA = smem;
    unsigned char *planesB = smem + OZ_S * OZ_APLANE;
    __shared__ uint64_t mbar, bbar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int erow[OZ_M];
    __shared__ int abort_sh, pend_sh, tmem_free_sh;
    __shared__ double red[OZ_THREADS];
    constexpr uint32_t TCOLS = OZ_S * OZ_NT;   // 512

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long r0 = (long)blockIdx.x * OZ_M;
    const int ct = blockIdx.y;
    const int K = k1 + k2;
    if (tid == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&bbar, 1);
        abort_sh = 0;
        pend_sh = 0;
        tmem_free_sh = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    auto aval = [&](long p, int k) -> double {
        return k < k1 ? A1[(size_t)p * k1 + k] : A2[(size_t)p * k2 + (k - k1)];
    };
    // row exponents: from k_oz_rowexp when K spans several chunks, else
    // formed below from the chunk's values (erow_g null)
    if (erow_g)
        for (int r = tid; r < OZ_M; r += OZ_THREADS) erow[r] = (r0 + r < n) ? erow_g[r0 + r] : 0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t idesc = idesc_bf16(OZ_M, OZ_NT);

    for (int ch = 0; ch < kchunks; ch++) {
        if (ch > 0 && tid == 0) {
            if (!mbar_wait(&mbar, (unsigned)((ch - 1) & 1))) {
                abort_sh = 1;
                pend_sh = (ch - 1) & 1;
            }
        }
        // the chunk's digit planes of the small matrix (prepared by
        // k_oz_split) arrive by bulk copies while the threads convert A;
        // the previous chunk's MMAs, which read them, are complete here
        if (tid == 0 && !abort_sh) {
            const unsigned char *src = image + (size_t)(ct * kchunks + ch) * OZ_S * OZ_BPLANE;
            mbar_expect_tx(&bbar, (uint32_t)(OZ_S * OZ_BPLANE));
#pragma unroll
            for (int j = 0; j < OZ_S; j++)
                bulk_g2s(planesB + j * OZ_BPLANE, src + j * OZ_BPLANE, OZ_BPLANE, &bbar);
        }
        __syncthreads();
        if (abort_sh) break;
        // digit planes of the point rows for K = ch*64 .. ch*64+63: a warp owns
        // 16 rows, a lane the pair k = 2 lane, 2 lane + 1 of each (one 32-bit
        // store per plane; a warp's stores fill one 128-byte row); all 32
        // loads of a batch of 16 rows are issued before converting
        {
            constexpr int RPW = OZ_M / (OZ_THREADS / 32);   // rows per warp
            double xv[RPW][2];
#pragma unroll
            for (int q = 0; q < RPW; q++) {
                const int r = warp * RPW + q;
                const long p = r0 + r;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int kg = ch * OZ_KC + 2 * lane + h;
                    xv[q][h] = (p < n && kg < K) ? aval(p, kg) : 0.0;
                }
            }
#pragma unroll
            for (int q = 0; q < RPW; q++) {
                const int r = warp * RPW + q;
                int em;
                if (erow_g) {
                    em = erow[r];
                } else {
                    em = __reduce_max_sync(0xffffffffu, (unsigned)max(biased_exp(xv[q][0]),
                                                                      biased_exp(xv[q][1])));
                    if (lane == 0) erow[r] = em;
                }
                uint32_t pk[OZ_S];
                oz_digits2(xv[q][0], xv[q][1], em, pk);
                const uint32_t off = sw128_offset16(r, 2 * lane);
#pragma unroll
                for (int i = 0; i < OZ_S; i++)
                    *reinterpret_cast<uint32_t *>(planesA + i * OZ_APLANE + off) = pk[i];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !mbar_wait(&bbar, (unsigned)(ch & 1))) {
            // no MMA of this chunk is issued; the last commit (if any) was
            // waited for above
            abort_sh = 1;
            pend_sh = (ch + 1) & 1;
        } else if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < OZ_KC / 16; ks++) {
                const uint32_t ko = ks * 32;
#pragma unroll
                for (int t = 2; t <= OZ_S + 1; t++) {
                    const int ilo = t - OZ_S > 1 ? t - OZ_S : 1;
                    const int ihi = t - 1 < OZ_S ? t - 1 : OZ_S;
                    for (int i = ilo; i <= ihi; i++) {
                        const int j = t - i;
                        const uint64_t da = make_desc_sw128(smem_u32(planesA + (i - 1) * OZ_APLANE) + ko);
                        const uint64_t db = make_desc_sw128(smem_u32(planesB + (j - 1) * OZ_BPLANE) + ko);
                        const uint32_t acc = (ch > 0 || ks > 0 || i > ilo) ? 1u : 0u;
                        mma_bf16(tmem + (uint32_t)((t - 2) * OZ_NT), da, db, idesc, acc);
                    }
                }
            }
            mma_commit(&mbar);
        }
    }
    // the tile's rows and columns; Cin's tile is loaded (coalesced: a warp
    // reads 32 consecutive columns of one row) while the last MMAs run
    const int ncl = min(OZ_NT, ncol - ct * OZ_NT);
    const long nrw = min((long)OZ_M, n - r0);
    constexpr int EPT = OZ_M * OZ_NT / OZ_THREADS;   // tile elements per thread
    double cpre[EPT];
    if (Cin) {
#pragma unroll
        for (int u = 0; u < EPT; u++) {
            const int idx = tid + u * OZ_THREADS, rr = idx / OZ_NT, jj = idx % OZ_NT;
            cpre[u] = (rr < nrw && jj < ncl) ? Cin[(size_t)(r0 + rr) * ncol + ct * OZ_NT + jj]
                                             : 0.0;
        }
    }
    if (!abort_sh && tid == 0) {
        if (!mbar_wait(&mbar, (unsigned)((kchunks - 1) & 1))) {
            abort_sh = 1;
            pend_sh = (kchunks - 1) & 1;
        }
    }
    // after a wait that gave up, the MMAs of the last commit may still be
    // writing TMEM: one more bounded wait for them before the columns are
    // released; if they are still running, the columns stay allocated (only
    // the status word is meaningful after a timeout)
    if (abort_sh && tid == 0) tmem_free_sh = mbar_wait(&mbar, (unsigned)pend_sh) ? 1 : 0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    double sq = 0.0;
    if (abort_sh) {
        if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
    } else {
        // the digit planes are free once the MMAs are done: the output tile is
        // staged there (row stride OZ_SLD doubles: a half-warp's 8-byte
        // accesses to one column of 16 rows, or to 16 columns of one row,
        // fall in distinct banks), so Cin is read and Out written in whole
        // rows
        double *stg = reinterpret_cast<double *>(planesA);
        if (Cin) {
#pragma unroll
            for (int u = 0; u < EPT; u++) {
                const int idx = tid + u * OZ_THREADS;
                stg[(idx / OZ_NT) * OZ_SLD + idx % OZ_NT] = cpre[u];
            }
        }
        __syncthreads();
        // epilogue: thread = one point row (TMEM lane 32 (warp % 4) + lane) and
        // one half of the 64 output columns (warp / 4)
        const int r = (warp & 3) * 32 + lane;
        const long p = r0 + r;
        const int em = erow[r];
        {
            const int cb = (warp >> 2) * 32;
            // sum_t D_t 2^(-7(t-2)) as a 64-bit fixed-point integer with 40
            // fraction bits (|D_2| < 2^21: no overflow; the two smallest
            // scales lose at most 2^-39), so the FP64 pipe sees one
            // conversion per output instead of a Horner chain
            long long acc[32];
#pragma unroll
            for (int j = 0; j < 32; j++) acc[j] = 0;
#pragma unroll
            for (int t = 2; t <= OZ_S + 1; t++) {
                float v[32];
                tmem_ld32<32>(tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                  (uint32_t)((t - 2) * OZ_NT + cb), v);
                const int sh = OZ_FRAC - OZ_BITS * (t - 2);
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const long long d = (long long)__float2int_rn(v[j]);
                    acc[j] += sh >= 0 ? (d << sh) : (d >> (-sh));
                }
            }
            if (p < n) {
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int c = ct * OZ_NT + cb + j;
                if (c >= ncol) continue;
                const int fc = fexp[c];
                const int es = (em - 1022) + (fc - 1022) - 2 * OZ_BITS - OZ_FRAC;
                // the integer converts exactly or rounds once; the scaling by
                // 2^es is an add to the exponent field when the result stays
                // normal (one FP64 operation fewer per output), else a multiply
                const double a = (double)acc[j];
                const long long ab = __double_as_longlong(a);
                const int ea = (int)((ab >> 52) & 0x7FF) + es;
                double o;
                if (em == OZ_EBAD || fc == OZ_EBAD)
                    o = __longlong_as_double(0x7FF8000000000000ll);
                else if (ea - es != 0 && ea >= 1 && ea <= 2046)
                    o = __longlong_as_double(ab + (long long)es * (1ll << 52));
                else if (es >= -1022 && es <= 1023)
                    o = a * __longlong_as_double((long long)(es + 1023) << 52);
                else
                    o = a * pow2(es);
                double *sl = stg + r * OZ_SLD + cb + j;
                if (Cin) o += *sl;
                *sl = o;
                if (part_sq) sq = fma(o, o, sq);
            }
            }
        }
        if (Out) {
            __syncthreads();
#pragma unroll
            for (int u = 0; u < EPT; u++) {
                const int idx = tid + u * OZ_THREADS, rr = idx / OZ_NT, jj = idx % OZ_NT;
                if (rr < nrw && jj < ncl)
                    Out[(size_t)(r0 + rr) * ncol + ct * OZ_NT + jj] = stg[rr * OZ_SLD + jj];
            }
        }
    }
    if (part_sq) {
        red[tid] = sq;
        __syncthreads();
        for (int k = OZ_THREADS / 2; k > 0; k >>= 1) {
            if (tid < k) red[tid] += red[tid + k];
            __syncthreads();
        }
        if (tid == 0) part_sq[(size_t)blockIdx.x * gridDim.y + blockIdx.y] = red[0];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && tmem_free_sh)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                     : "memory");
}

// ---------------------------------------------------------------------------
// FP64 Gram <X, X> = w X^T X of X = [X1 X2] (n x na, na <= 128) by the same
// digit slicing, with per-column exponents over all points (k_oz_colexp).
// CTA = all na rows x 64 output columns over a chunk of points; the digit
// planes of a 32-point slice serve as both operands (the B operand is rows
// ct*64.. of the A planes; 64-byte rows, 64-byte swizzle).  The planes of
// OZ_GST slices are in flight: the converter warps fill slice s while the MMAs
// of slice s-1 run.  The exact-sum bound holds for 128 points, so every four
// slices the eight accumulators are read and added into 64-bit fixed-point
// registers (OZ_GFRAC fraction bits); the chunk's FP64 partial tile is
// summed over chunks in a fixed order by k_oz_gram_reduce.  D_t(i,j) and
// D_t(j,i) are the same integers, so the result is exactly symmetric.
// ---------------------------------------------------------------------------
constexpr int OZ_GFRAC = 32;
constexpr int OZ_GKC = 32;                       // points per slice: 64-byte rows
constexpr int OZ_GPLANE = OZ_M * 64;             // one digit plane of a slice: 8 KB
constexpr int OZ_GSTAGE = OZ_S * OZ_GPLANE;      // the eight planes: 64 KB
constexpr int OZ_GST = 3;                        // slices in flight
constexpr int OZ_GFLUSH = 128 / OZ_GKC;          // slices per exact accumulation
constexpr int OZ_GSMEM = OZ_GST * OZ_GSTAGE + 2048;   // + alignment slack

// byte offset of 16-bit element (row r, k) in a K-major tile of 32-element
// rows with the 64-byte swizzle (16-byte chunk c of row r at c ^ ((r >> 1) & 3))
__device__ __forceinline__ uint32_t sw64_offset16(int r, int k) {
    return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((k >> 3) ^ (r >> 1)) & 3) << 4) +
                      ((k & 7) << 1));
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle, SBO = 512 B
__device__ __forceinline__ uint64_t make_desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
    d |= (uint64_t)(1) << 16;                  // leading byte offset (unused, swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;           // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                    // descriptor version (sm_100 family)
    d |= (uint64_t)4 << 61;                    // swizzle mode: 64 B
    return d;
}

__global__ void __launch_bounds__(128) k_oz_colexp(long n, int n1, int n2, const double *X1,
                                                   const double *X2, int *colexp) {
    const int c = threadIdx.x, na = n1 + n2;
    if (c >= na) return;
    int em = 0;
    for (long p = blockIdx.x; p < n; p += gridDim.x)
        em = max(em, biased_exp(c < n1 ? X1[(size_t)p * n1 + c] : X2[(size_t)p * n2 + (c - n1)]));
    atomicMax(&colexp[c], em);
}

// 16 converter warps (digit planes, TMEM read-out, epilogue) and one warp
// whose first lane issues the MMAs; they meet only at mbarriers: full[st]
// (the planes of a slice are written), done[st] (its MMAs completed, the
// stage is free) and tfree (the accumulators were read out at a flush)
constexpr int OZ_GCONV = 512;
constexpr int OZ_GTHREADS = OZ_GCONV + 32;

__global__ void __launch_bounds__(OZ_GTHREADS, 1)
    k_gram_oz(long n, int n1, int n2, long chunk_rows, int ct0, const double *__restrict__ X1,
              const double *__restrict__ X2, const int *__restrict__ colexp,
              double *__restrict__ partials, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *planes = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[OZ_GST], done[OZ_GST], tfree;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int cexp[OZ_M];
    __shared__ volatile int abort_sh;
    __shared__ int last_sh, tmem_free_sh;
    constexpr uint32_t TCOLS = OZ_S * OZ_NT;   // 512
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int na = n1 + n2, ct = ct0 + blockIdx.x;   // output column tile
    const long p0 = (long)blockIdx.y * chunk_rows;
    const long p1 = (n < p0 + chunk_rows) ? n : p0 + chunk_rows;
    const int nslices = p1 > p0 ? (int)((p1 - p0 + OZ_GKC - 1) / OZ_GKC) : 0;
    if (tid == 0) {
        for (int i = 0; i < OZ_GST; i++) {
            mbar_init(&full[i], OZ_GCONV);
            mbar_init(&done[i], 1);
        }
        mbar_init(&tfree, OZ_GCONV);
        abort_sh = 0;
        last_sh = -1;   // last slice whose MMAs were committed
        tmem_free_sh = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int c = tid; c < OZ_M; c += OZ_GTHREADS) cexp[c] = c < na ? colexp[c] : 0;
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
    // completion of the MMAs of slice q: the (q / OZ_GST)-th commit on
    // done[q % OZ_GST].  No role can run a phase ahead of the one another
    // role waits for (each next arrival needs the awaited phase), so every
    // parity below is unambiguous.
    auto wait_done = [&](int q) -> bool {
        return mbar_wait(&done[q % OZ_GST], (unsigned)((q / OZ_GST) & 1));
    };
    // fixed-point sums: converter thread = TMEM lane 32 (warp % 4) + lane
    // (Gram row), 16 output columns (warp / 4)
    const int grow = (warp & 3) * 32 + lane, gcb = (warp >> 2) * 16;
    long long facc[16];
#pragma unroll
    for (int j = 0; j < 16; j++) facc[j] = 0;
    auto flush = [&]() {
#pragma unroll
        for (int t = 2; t <= OZ_S + 1; t++) {
            float v[16];
            tmem_ld32<16>(tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                              (uint32_t)((t - 2) * OZ_NT + gcb), v);
            const int sh = OZ_GFRAC - OZ_BITS * (t - 2);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const long long d = (long long)__float2int_rn(v[j]);
                facc[j] += sh >= 0 ? (d << sh) : (d >> (-sh));
            }
        }
    };
    if (warp == OZ_GCONV / 32) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(OZ_M, OZ_NT);
            for (int sl = 0; sl < nslices; sl++) {
                if (abort_sh) break;
                const int st = sl % OZ_GST;
                const bool fresh = sl % OZ_GFLUSH == 0;
                if (!mbar_wait(&full[st], (unsigned)((sl / OZ_GST) & 1)) ||
                    (fresh && sl > 0 && !mbar_wait(&tfree, (unsigned)((sl / OZ_GFLUSH - 1) & 1)))) {
                    abort_sh = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char *stage = planes + st * OZ_GSTAGE;
#pragma unroll
                for (int ks = 0; ks < OZ_GKC / 16; ks++) {
                    const uint32_t ko = ks * 32;
#pragma unroll
                    for (int t = 2; t <= OZ_S + 1; t++) {
                        const int ilo = t - OZ_S > 1 ? t - OZ_S : 1;
                        const int ihi = t - 1 < OZ_S ? t - 1 : OZ_S;
#pragma unroll
                        for (int i = ilo; i <= ihi; i++) {
                            const int j = t - i;
                            const uint64_t da =
                                make_desc_sw64(smem_u32(stage + (i - 1) * OZ_GPLANE) + ko);
                            const uint64_t db = make_desc_sw64(
                                smem_u32(stage + (j - 1) * OZ_GPLANE + ct * OZ_NT * 64) + ko);
                            const uint32_t acc = (!fresh || ks > 0 || i > ilo) ? 1u : 0u;
                            mma_bf16(tmem + (uint32_t)((t - 2) * OZ_NT), da, db, idesc, acc);
                        }
                    }
                }
                mma_commit(&done[st]);
                last_sh = sl;
            }
        }
    } else {
        // slice loads: thread t takes column c = t & 127 of the 8 consecutive
        // points 8 (t >> 7) + j (coalesced across the lanes for each j)
        const int lc = tid & (OZ_M - 1), lq = tid >> 7;
        double xv[8];
        auto load_slice = [&](int sl) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const long p = p0 + (long)sl * OZ_GKC + 8 * lq + j;
                xv[j] = (p < p1 && lc < na)
                            ? (lc < n1 ? X1[(size_t)p * n1 + lc] : X2[(size_t)p * n2 + (lc - n1)])
                            : 0.0;
            }
        };
        const int em = cexp[lc];
        if (nslices > 0) load_slice(0);
        for (int sl = 0; sl < nslices; sl++) {
            if (abort_sh) break;
            const int st = sl % OZ_GST;
            const bool fresh = sl % OZ_GFLUSH == 0;
            // the stage's previous slice is consumed
            if (sl >= OZ_GST && !wait_done(sl - OZ_GST)) {
                abort_sh = 1;
                break;
            }
            if (fresh && sl > 0) {
                // 128 points accumulated: every MMA so far is complete
                if (!wait_done(sl - 1)) {
                    abort_sh = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                flush();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&tfree);
            }
            // eight consecutive points of one column: one 16-byte chunk of
            // each digit plane
            {
                uint32_t pk[OZ_S][4];
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    uint32_t pp[OZ_S];
                    oz_digits2(xv[u], xv[u + 1], em, pp);
#pragma unroll
                    for (int i = 0; i < OZ_S; i++) pk[i][u >> 1] = pp[i];
                }
                unsigned char *stage = planes + st * OZ_GSTAGE;
                const uint32_t off = sw64_offset16(lc, 8 * lq);
#pragma unroll
                for (int i = 0; i < OZ_S; i++)
                    *reinterpret_cast<uint4 *>(stage + i * OZ_GPLANE + off) =
                        make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[st]);
            if (sl + 1 < nslices) load_slice(sl + 1);
        }
        if (!abort_sh && nslices > 0 && !wait_done(nslices - 1)) abort_sh = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // after a wait that gave up, one more bounded wait for the last commit
    // before the columns are released (if it fails too they stay allocated,
    // and only the status word is meaningful)
    if (tid == OZ_GCONV && abort_sh && last_sh >= 0) tmem_free_sh = wait_done(last_sh) ? 1 : 0;
    __syncthreads();
    if (abort_sh) {
        if (tid == 0) atomicOr(status, ST_TC_TIMEOUT);
    } else if (tid < OZ_GCONV) {
        if (nslices > 0) flush();
        double *dst = partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * OZ_M * OZ_NT;
        const int ea = cexp[grow];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int gc = ct * OZ_NT + gcb + j;
            double o = 0.0;
            if (grow < na && gc < na) {
                const int eb = cexp[gc];
                const int es = (ea - 1022) + (eb - 1022) - 2 * OZ_BITS - OZ_GFRAC;
                if (ea == OZ_EBAD || eb == OZ_EBAD) o = __longlong_as_double(0x7FF8000000000000ll);
                else if (es >= -1022 && es <= 1023)
                    o = (double)facc[j] * __longlong_as_double((long long)(es + 1023) << 52);
                else
                    o = (double)facc[j] * pow2(es);
            }
            dst[(size_t)grow * OZ_NT + gcb + j] = o;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && tmem_free_sh)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                     : "memory");
}

// out[i][j] = w * sum over chunks (in order) of the chunk partials, for the
// columns of the ctiles tiles from tile ct0 on (the others are not written)
__global__ void k_oz_gram_reduce(int na, int ct0, int ctiles, int chunks, const double *partials,
                                 double w, double *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= na * na) return;
    const int i = e / na, j = e % na, ct = j / OZ_NT - ct0, jl = j % OZ_NT;
    if (ct < 0) return;
    const double s = ordered_sum(partials + ((size_t)ct * OZ_M + i) * OZ_NT + jl, chunks,
                                 (size_t)ctiles * OZ_M * OZ_NT);
    out[e] = w * s;
}

}  // namespace

bool tall_oz_supported(int k1, int k2) { return k1 + k2 >= 1 && k1 + k2 <= 128; }

size_t tall_oz_image_bytes(long n, int K, int ncol) {
    const int kchunks = (K + OZ_KC - 1) / OZ_KC;
    const int ctiles = (ncol + OZ_NT - 1) / OZ_NT;
    return (size_t)ctiles * kchunks * OZ_S * OZ_BPLANE + sizeof(int) * (size_t)(ncol + 64 + n);
}

int tall_oz_partials(long n, int ncol) {
    return (int)(((n + OZ_M - 1) / OZ_M) * ((ncol + OZ_NT - 1) / OZ_NT));
}

void oz_prepare() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_tall_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    cudaFuncSetAttribute(k_gram_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_GSMEM);
    done = true;
}

bool gram_oz_supported(int na) { return na >= 1 && na <= OZ_M; }

namespace {
struct OzGramPlan {
    int ctiles, chunks;
    long chunk_rows;
};
OzGramPlan make_oz_gram_plan(long n, int na) {
    OzGramPlan g;
    g.ctiles = (na + OZ_NT - 1) / OZ_NT;
    // at most 16384 points per chunk: the 64-bit fixed-point sums then stay
    // below 2^60 (2^53 per 128-point flush)
    long chunks = std::max((long)(2 * 152) / g.ctiles, (n + 16383) / 16384);
    chunks = std::max(1L, std::min(chunks, (n + OZ_KC - 1) / OZ_KC));
    long rows = (n + chunks - 1) / chunks;
    rows = (rows + OZ_KC - 1) / OZ_KC * OZ_KC;
    g.chunk_rows = rows;
    g.chunks = (int)((n + rows - 1) / rows);
    return g;
}
}  // namespace

size_t gram_oz_scratch_bytes(long n, int na) {
    OzGramPlan g = make_oz_gram_plan(n, na);
    return sizeof(double) * (size_t)g.chunks * g.ctiles * OZ_M * OZ_NT + sizeof(int) * OZ_M;
}

void launch_gram_oz(long n, const double *X1, int n1, const double *X2, int n2, double w,
                    double *scratch, double *out, int *status, cudaStream_t s, int col0) {
    if (!X2) n2 = 0;
    const int na = n1 + n2;
    OzGramPlan g = make_oz_gram_plan(n, na);
    // output columns from the tile holding column col0 on
    const int ct0 = std::min(std::max(col0, 0) / OZ_NT, g.ctiles - 1), nt = g.ctiles - ct0;
    double *partials = scratch;
    int *colexp = reinterpret_cast<int *>(scratch + (size_t)g.chunks * g.ctiles * OZ_M * OZ_NT);
    cudaMemsetAsync(colexp, 0, sizeof(int) * OZ_M, s);
    HQ_LAUNCH(HQ_K_GRAM, k_oz_colexp<<<1024, 128, 0, s>>>(n, n1, n2, X1, n2 ? X2 : nullptr, colexp));
    HQ_LAUNCH(HQ_K_GRAM, k_gram_oz<<<dim3(nt, g.chunks), OZ_GTHREADS, OZ_GSMEM, s>>>(
                             n, n1, n2, g.chunk_rows, ct0, X1, n2 ? X2 : nullptr, colexp, partials,
                             status));
    HQ_LAUNCH(HQ_K_GRAM, k_oz_gram_reduce<<<(na * na + 255) / 256, 256, 0, s>>>(
                             na, ct0, nt, g.chunks, partials, w, out));
}

void launch_tall_oz(long n, const double *A1, int k1, const double *M1, const double *A2, int k2,
                    const double *M2, int ncol, const double *Cin, double *Out, double *part_sq,
                    unsigned char *image, int *status, cudaStream_t s) {
    if (!A2) k2 = 0;
    const int K = k1 + k2;
    const int kchunks = (K + OZ_KC - 1) / OZ_KC;
    const int ctiles = (ncol + OZ_NT - 1) / OZ_NT;
    int *fexp = reinterpret_cast<int *>(image + (size_t)ctiles * kchunks * OZ_S * OZ_BPLANE);
    int *erow = fexp + ncol + 64;
    HQ_LAUNCH(HQ_K_BLOCKGEMM, k_oz_split<<<ctiles, OZ_NT * SPL_G, 0, s>>>(K, k1, ncol, kchunks, M1,
                                                                   k2 ? M2 : nullptr, image, fexp));
    // one K chunk: the product kernel forms the row exponents from the values
    // it converts; more: a pass over the rows first
    if (kchunks > 1)
        HQ_LAUNCH(HQ_K_BLOCKGEMM, k_oz_rowexp<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(
                                      n, k1, k2, A1, k2 ? A2 : nullptr, erow));
    const unsigned gx = (unsigned)((n + OZ_M - 1) / OZ_M);
    HQ_LAUNCH(HQ_K_BLOCKGEMM,
              k_tall_oz<<<dim3(gx, ctiles), OZ_THREADS, OZ_SMEM, s>>>(
                  n, k1, k2, ncol, kchunks, A1, k2 ? A2 : nullptr, image, fexp,
                  kchunks > 1 ? erow : nullptr, Cin, Out,
                  part_sq, status));
}

}  // namespace hq
