// selftest.cu -- the failure path of the bounded device waits, exercised
// without a fault: one thread waits on an mbarrier that nothing arrives at,
// with the try-wait / deadline loop the pipelined kernels use, then records
// a timeout in the context's error word and returns.  Also the FP32 FMA
// throughput microbenchmark that gives the SIMT roofline of the FP32 form.
#include <algorithm>

#include "pg_internal.cuh"

namespace {

__global__ void k_wait_selftest(unsigned long long limit_ns, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(0u)
            : "memory");
        if (ok) return;
        __nanosleep(1000);
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            record_error(err, DERR_TIMEOUT, -1);
            return;
        }
    }
}

// Eight independent FMA chains per thread; every SM full (2048 threads).
// The result is stored only under a condition the caller makes false, so
// the chains stay live without a store per iteration.
__global__ void __launch_bounds__(512, 4) k_fma_peak(float *out, int iters, float a, float b,
                                                  float never) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += x[k];
    if (t == never) out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

extern "C" pg_status pg_measure_fp32_peak(pg_ctx *ctx, double *host_tflops) {
    if (!ctx || !host_tflops) return PG_ERR_INVALID_ARG;
    const int per_sm = 4, threads = 512, iters = 1 << 18;
    const int blocks = ctx->num_sms * per_sm;
    Scratch<float> out;
    PG_TRY(out.alloc(ctx, (size_t)blocks * threads));
    cudaEvent_t e0, e1;
    PG_TRY_CUDA(ctx, cudaEventCreate(&e0));
    PG_TRY_CUDA(ctx, cudaEventCreate(&e1));
    double best = 0.0;
    pg_status st = PG_OK;
    for (int rep = 0; rep < 4 && st == PG_OK; ++rep) {
        cudaEventRecord(e0, ctx->stream);
        k_fma_peak<<<blocks, threads, 0, ctx->stream>>>(out.p, iters, 0.999f, 1e-4f, -1.f);
        cudaError_t e = cudaGetLastError();
        ctx->launches++;
        cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) st = pg_cuda_fail(ctx, e, "fp32 peak");
        else if (rep > 0 && ms > 0.f)  // the first launch warms up
            best = std::max(best, 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *host_tflops = best;
    return st;
}

extern "C" pg_status pg_selftest_wait_timeout(pg_ctx *ctx, double seconds) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!(seconds > 0.0 && seconds <= 5.0))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 0 < seconds <= 5");
    k_wait_selftest<<<1, 32, 0, ctx->stream>>>((unsigned long long)(seconds * 1e9), ctx->d_err);
    PG_LAUNCHED(ctx);
    return pg_sync_check(ctx, "pg_selftest_wait_timeout");
}
