// selftest.cu -- the failure path of the bounded device waits, exercised
// without a fault: one thread waits on an mbarrier that nothing arrives at,
// with the try-wait / deadline loop the pipelined kernels use, then records
// a timeout in the context's error word and returns.
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

}  // namespace

extern "C" pg_status pg_selftest_wait_timeout(pg_ctx *ctx, double seconds) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    if (!(seconds > 0.0 && seconds <= 5.0))
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "need 0 < seconds <= 5");
    k_wait_selftest<<<1, 32, 0, ctx->stream>>>((unsigned long long)(seconds * 1e9), ctx->d_err);
    PG_LAUNCHED(ctx);
    return pg_sync_check(ctx, "pg_selftest_wait_timeout");
}
