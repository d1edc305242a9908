// hq_gram_static: the inner-product matrix w A^T B of two FP64 point-major
// blocks for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is
// being captured with a relaxed allocation policy, allocator-free plugin
// hosts that only hand out pre-registered buffers, and real-time loops that
// forbid allocation after start-up.  hq_gram (the context entry point) takes
// its split-K partial sums from the workspace the caller allocated for a
// context; this entry point needs no context and no workspace: its partials
// live in one file-scope device array of fixed size, HQ_GRAM_STATIC_SCRATCH
// doubles (4 MiB), which every GPU that loads the library keeps until the
// process exits.
//
// The host never uses the array's name as a device address (in host code
// that name is only a stand-in): the first call on each device, with that
// device current, asks the runtime for the array's device address with
// cudaGetSymbolAddress, checks the result and caches it for that device.  The
// cached address belongs to that device's context: after cudaDeviceReset the
// entry point must not be called again in the same process.
#include <mutex>

#include "../../include/hq.h"
#include "hq_internal.cuh"

namespace {

constexpr size_t HQ_GRAM_STATIC_SCRATCH = (size_t)1 << 19;   // doubles (4 MiB)
constexpr int HQ_GRAM_STATIC_MAXCOL = 512;
constexpr int HQ_MAX_DEVICES = 64;

static __device__ __align__(256) double g_gram_scratch[HQ_GRAM_STATIC_SCRATCH];

std::mutex g_static_mu;
double *g_static_ptr[HQ_MAX_DEVICES] = {};

// device address of g_gram_scratch on the current device (set up once)
hq_status static_scratch(double **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= HQ_MAX_DEVICES) return HQ_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess || p == nullptr)
            return HQ_ERR_CUDA;
        g_static_ptr[dev] = (double *)p;
    }
    *out = g_static_ptr[dev];
    return HQ_OK;
}

}  // namespace

extern "C" hq_status hq_gram_static(const double *A, int Na, const double *B, int Nb, long n,
                                    double w, double *out, void *cuda_stream) {
    using namespace hq;
    if (!A || !B || !out || n < 1 || Na < 1 || Nb < 1 || Na > HQ_GRAM_STATIC_MAXCOL ||
        Nb > HQ_GRAM_STATIC_MAXCOL)
        return HQ_ERR_ARG;
    GramPlan p = make_gram_plan(n, Na, Nb, A == B && Na == Nb);
    // fit the split over grid points into the fixed scratch
    const size_t per_chunk = (size_t)p.ntiles * 64 * 64;
    const long max_chunks = (long)(HQ_GRAM_STATIC_SCRATCH / per_chunk);
    if (max_chunks < 1) return HQ_ERR_ARG;
    if (p.chunks > max_chunks) {
        long rows = (n + max_chunks - 1) / max_chunks;
        rows = (rows + 15) / 16 * 16;
        p.chunk_rows = rows;
        p.chunks = (int)((n + rows - 1) / rows);
    }
    if ((size_t)p.chunks * per_chunk > HQ_GRAM_STATIC_SCRATCH) return HQ_ERR_ARG;
    // an error left pending by the caller's earlier work is not this call's:
    // report it without launching and without clearing it
    if (cudaPeekAtLastError() != cudaSuccess) return HQ_ERR_CUDA;
    double *scratch = nullptr;
    hq_status st = static_scratch(&scratch);
    if (st != HQ_OK) return st;
    // every partial tile is written before it is read: nothing to clear
    launch_gram<double>(p, A, Na, nullptr, 0, B, Nb, nullptr, 0, w, scratch, out,
                        (cudaStream_t)cuda_stream);
    // the slate was clean on entry, so an error now comes from these launches
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return HQ_ERR_CUDA;
    }
    return HQ_OK;
}
