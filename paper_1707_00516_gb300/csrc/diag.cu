// Diagnostics: the bounded device wait and its status report, on a flag the
// caller owns (see fastid_wait_flag in fastid.h).  The compare kernels bound
// every wait the same way: past the limit they record ST_TIMEOUT and a site
// code in the context's status word, return, and leave the context usable.
#include <string>

#include "common.cuh"
#include "internal.h"

namespace fastid {

namespace {

constexpr uint32_t SITE_WAIT_FLAG = 10;

__global__ void wait_flag_kernel(const uint32_t *flag, uint64_t limit_ns, uint32_t *status) {
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0) return;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            atomicOr(status, ST_TIMEOUT);
            atomicExch(status + 1, SITE_WAIT_FLAG);
            return;
        }
        __nanosleep(1000);
    }
}

// Read-and-clear of the status word in one step (so that a condition a
// kernel on another stream records meanwhile is never lost between a read
// and a clear): snap[i] = atomicExch(status[i], 0) for the 4 words.
__global__ void status_take_kernel(uint32_t *status, uint32_t *snap) {
    const int i = threadIdx.x;
    if (i < 4) snap[i] = atomicExch(status + i, 0u);
}

}  // namespace

cudaError_t launch_status_take(uint32_t *status, uint32_t *snap, cudaStream_t s) {
    status_take_kernel<<<1, 32, 0, s>>>(status, snap);
    return cudaGetLastError();
}

}  // namespace fastid

using namespace fastid;

extern "C" fastid_status fastid_wait_flag(fastid_ctx *ctx, const uint32_t *flag_dev, int32_t wait_ms,
                                          fastid_stream stream) {
    FASTID_RANGE();
    if (!ctx) return FASTID_EINVAL;
    if (!flag_dev) {
        ctx->last_error = "flag is NULL";
        return FASTID_EINVAL;
    }
    if (wait_ms < 1 || wait_ms > 10000) {
        ctx->last_error = "wait_ms out of range (1 .. 10000)";
        return FASTID_EINVAL;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) {
        wait_flag_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(flag_dev, (uint64_t)wait_ms * 1000000ull,
                                                            ctx->dev_status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        ctx->last_error = std::string("wait_flag: ") + cudaGetErrorString(e);
        return FASTID_ECUDA;
    }
    ctx->launches += 1;
    return FASTID_OK;
}
