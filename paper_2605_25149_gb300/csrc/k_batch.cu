// Device side of the batched form: the time loop of Algorithm 1 for many
// independent problems inside one CUDA graph.  Each problem keeps eight
// 64-bit words of loop state in its own workspace (BS_* in hq_internal.cuh);
// the kernels below read and write only those words and set the
// conditional-node handles that skip finished problems and end the loop.
#include <cuda_runtime.h>

#include "hq_internal.cuh"

namespace hq {

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_batch_init(BatchArgs a, cudaGraphConditionalHandle hT) {
    const int k = threadIdx.x;
    if (k < a.count) {
        long long *sl = a.slot[k];
        sl[BS_STEPS] = 0;
        sl[BS_DONE] = BD_RUNNING;
        sl[BS_AEXEC] = 0;
    }
    if (k == 0) {
        if (a.count > 0) a.slot[0][BS_T0] = (long long)global_ns();
        cudaGraphSetConditional(hT, a.count > 0 ? 1u : 0u);
    }
}

__global__ void k_batch_arm(BatchArgs a) {
    const int k = threadIdx.x;
    if (k >= a.count) return;
    long long *sl = a.slot[k];
    long long done = sl[BS_DONE];
    if (done == BD_RUNNING && sl[BS_MODE] == 1 && sl[BS_STEPS] >= sl[BS_MAXSTEPS]) {
        done = BD_MAXSTEPS;
        sl[BS_DONE] = done;
    }
    cudaGraphSetConditional(a.h[k], done == BD_RUNNING ? 1u : 0u);
}

__global__ void k_batch_check(long long *sl, const double *g, const int *st1, const int *st2,
                              cudaGraphConditionalHandle hB) {
    const double gv = g[0];
    const double eps = __longlong_as_double(sl[BS_EPS]);
    sl[BS_AEXEC] += 1;
    long long code = BD_RUNNING;
    if (st1[0] != 0 || st2[0] != 0 || !isfinite(gv)) code = BD_ERROR;
    else if (sl[BS_MODE] == 0 && gv < eps) code = BD_CONVERGED;
    else if (sl[BS_STEPS] >= sl[BS_MAXSTEPS]) code = BD_MAXSTEPS;
    sl[BS_DONE] = code;
    cudaGraphSetConditional(hB, code == BD_RUNNING ? 1u : 0u);
}

__global__ void k_batch_count(long long *sl) { sl[BS_STEPS] += 1; }

__global__ void k_batch_cond(BatchArgs a, cudaGraphConditionalHandle hT) {
    const int k = threadIdx.x;
    bool timed_out = false;
    if (a.count > 0) {
        const long long lim = a.slot[0][BS_TIMEOUT];
        timed_out = lim > 0 && (long long)global_ns() - a.slot[0][BS_T0] > lim;
    }
    bool running = false;
    if (k < a.count) {
        long long *sl = a.slot[k];
        if (sl[BS_DONE] == BD_RUNNING) {
            if (timed_out) sl[BS_DONE] = BD_TIMEOUT;
            else running = true;
        }
    }
    const int any = __syncthreads_or(running ? 1 : 0);
    if (k == 0) {
        if (a.count > 0) a.slot[0][BS_ITERS] += 1;
        cudaGraphSetConditional(hT, any ? 1u : 0u);
    }
}

int threads_for(int count) { return ((count + 31) / 32) * 32; }

}  // namespace

void launch_batch_init(const BatchArgs &a, cudaGraphConditionalHandle hT, cudaStream_t s) {
    k_batch_init<<<1, threads_for(a.count > 0 ? a.count : 1), 0, s>>>(a, hT);
}

void launch_batch_arm(const BatchArgs &a, cudaStream_t s) {
    k_batch_arm<<<1, threads_for(a.count > 0 ? a.count : 1), 0, s>>>(a);
}

void launch_batch_check(long long *slot, const double *g, const int *st1, const int *st2,
                        cudaGraphConditionalHandle hB, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_batch_check<<<1, 1, 0, s>>>(slot, g, st1, st2, hB));
}

void launch_batch_count(long long *slot, cudaStream_t s) {
    HQ_LAUNCH(HQ_K_SMALL, k_batch_count<<<1, 1, 0, s>>>(slot));
}

void launch_batch_cond(const BatchArgs &a, cudaGraphConditionalHandle hT, cudaStream_t s) {
    k_batch_cond<<<1, threads_for(a.count > 0 ? a.count : 1), 0, s>>>(a, hT);
}

}  // namespace hq
