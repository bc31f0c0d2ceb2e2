// ctx.cu -- context lifetime, stream-ordered scratch with an HBM budget,
// error reporting, statistics counters and per-dataset arithmetic facts.
#include <cstdarg>
#include <cstring>
#include <cmath>

#include <algorithm>

#include "pg_internal.cuh"

pg_status pg_fail(pg_ctx *ctx, pg_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

pg_status pg_cuda_fail(pg_ctx *ctx, cudaError_t e, const char *what) {
    pg_status st = (e == cudaErrorMemoryAllocation) ? PG_ERR_OOM : PG_ERR_CUDA;
    return pg_fail(ctx, st, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" void pg_default_params(pg_build_params *p) {
    if (!p) return;
    p->metric = PG_METRIC_L2SQ;
    p->precision = PG_PREC_FP32;
    p->K = 64;
    p->L = 200;
    p->R = 32;
    p->M = 16;
    p->alpha_deg = 66.0;
    p->alpha_final_deg = 60.0;
    p->iters = 2;
    p->connect_final = 1;
    p->route_layers = 1;
    p->seed = 0;
    p->reuse_pruning = 1;
    p->quality_target = 0.0;
    p->quality_eps = 0.6;
    p->quality_k = 0;
    p->connect_replace = 1;
    p->knn_descent_iters = -1;
}

extern "C" pg_status pg_ctx_create(void *cuda_stream, size_t hbm_budget_bytes, pg_ctx **out) {
    if (!out) return PG_ERR_INVALID_ARG;
    *out = nullptr;
    pg_ctx *ctx = new (std::nothrow) pg_ctx();
    if (!ctx) return PG_ERR_OOM;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->budget = hbm_budget_bytes;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, 4 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->d_counters, PG_CNT_SLOTS * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMallocHost(&ctx->h_pinned, PG_CNT_SLOTS * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_err, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, 4 * sizeof(int), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->d_counters, 0, PG_CNT_SLOTS * sizeof(unsigned long long),
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        pg_ctx_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? PG_ERR_OOM : PG_ERR_CUDA;
    }
    *out = ctx;
    return PG_OK;
}

const char *const pg_timer_names[TM_SLOTS] = {"knn",    "prune",          "union",
                                               "connect", "search",        "medoid",
                                               "connect_select", "connect_fast",
                                               "connect_scan",   "connect_commit"};

static cudaEvent_t take_event(pg_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void pg_timer_begin(pg_ctx *ctx, int slot) {
    if (!ctx->timing) return;
    pg_ctx::TimedPair t{slot, take_event(ctx), take_event(ctx)};
    cudaEventRecord(t.a, ctx->stream);
    ctx->pending.push_back(t);
}

void pg_timer_end(pg_ctx *ctx, int slot, double work) {
    if (!ctx->timing || ctx->pending.empty()) return;
    ctx->timer_work[slot] += work;
    for (auto it = ctx->pending.rbegin(); it != ctx->pending.rend(); ++it) {
        if (it->slot == slot) {
            cudaEventRecord(it->b, ctx->stream);
            ctx->timer_launches[slot] += 1;
            return;
        }
    }
}

void pg_timer_resolve(pg_ctx *ctx) {
    if (ctx->pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &t : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) ctx->timer_ms[t.slot] += ms;
        ctx->event_pool.push_back(t.a);
        ctx->event_pool.push_back(t.b);
    }
    ctx->pending.clear();
    cudaGetLastError();
}

extern "C" pg_status pg_ctx_set_timing(pg_ctx *ctx, int enable) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    pg_timer_resolve(ctx);
    ctx->timing = enable ? 1 : 0;
    for (int i = 0; i < TM_SLOTS; ++i) {
        ctx->timer_ms[i] = 0.0;
        ctx->timer_launches[i] = 0;
        ctx->timer_work[i] = 0.0;
    }
    // the device work counters restart with the timers
    return pg_reset_counters(ctx);
}

extern "C" pg_status pg_ctx_set_tie_count(pg_ctx *ctx, int enable) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    ctx->count_ties = enable ? 1 : 0;
    return PG_OK;
}

extern "C" pg_status pg_ctx_kernel_work(pg_ctx *ctx, const char *name, double *work) {
    if (!ctx || !name || !work) return PG_ERR_INVALID_ARG;
    pg_timer_resolve(ctx);
    for (int i = 0; i < TM_SLOTS; ++i) {
        if (strcmp(name, pg_timer_names[i]) == 0) {
            *work = ctx->timer_work[i];
            return PG_OK;
        }
    }
    return pg_fail(ctx, PG_ERR_INVALID_ARG, "unknown timer %s", name);
}

extern "C" pg_status pg_ctx_kernel_time(pg_ctx *ctx, const char *name, double *total_ms,
                                        int64_t *launches) {
    if (!ctx || !name) return PG_ERR_INVALID_ARG;
    pg_timer_resolve(ctx);
    for (int i = 0; i < TM_SLOTS; ++i) {
        if (strcmp(name, pg_timer_names[i]) == 0) {
            if (total_ms) *total_ms = ctx->timer_ms[i];
            if (launches) *launches = ctx->timer_launches[i];
            return PG_OK;
        }
    }
    return pg_fail(ctx, PG_ERR_INVALID_ARG, "unknown timer %s", name);
}

extern "C" pg_status pg_ctx_counter(pg_ctx *ctx, const char *name, int64_t *value) {
    if (!ctx || !name || !value) return PG_ERR_INVALID_ARG;
    if (strcmp(name, "connect_edges") == 0) *value = ctx->connect_edges;
    else if (strcmp(name, "connect_full_rounds") == 0) *value = ctx->connect_full_rounds;
    else if (strcmp(name, "connect_conflicts") == 0) *value = ctx->connect_why_full;
    else if (strcmp(name, "connect_free_nodes") == 0) *value = ctx->connect_free;
    else {
        static const struct {
            const char *name;
            int slot;
        } dev[] = {{"search_expansions", CNT_SEARCH_EXP}, {"search_evaluations", CNT_SEARCH_EVAL},
                   {"prune_rows", CNT_ROWS},           {"prune_candidates", CNT_CANDS},
                   {"prune_scanned", CNT_SCANNED},     {"prune_occlusion_tests", CNT_OCCL},
                   {"search_bytes", CNT_SEARCH_BYTES}, {"prune_bytes", CNT_PRUNE_BYTES},
                   {"prune_fp64_rechecks", CNT_RECHECK}, {"prune_fp64_flips", CNT_FLIP},
                   {"prune_near_ties", CNT_NEAR_TIE},  {"prune_edges", CNT_EDGES},
                   {"knn_fallback_rows", CNT_KNN_FALLBACK}, {"knn_fp64_rechecks", CNT_KNN_RECHECK}};
        for (const auto &e : dev) {
            if (strcmp(name, e.name) == 0) {
                unsigned long long c[PG_CNT_SLOTS];
                PG_TRY(pg_read_counters(ctx, c));
                *value = (int64_t)c[e.slot];
                return PG_OK;
            }
        }
        return pg_fail(ctx, PG_ERR_INVALID_ARG, "unknown counter %s", name);
    }
    return PG_OK;
}

extern "C" void pg_ctx_destroy(pg_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    pg_timer_resolve(ctx);
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_counters) cudaFree(ctx->d_counters);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    delete ctx;
}

extern "C" const char *pg_last_error(const pg_ctx *ctx) {
    return ctx ? ctx->last_error.c_str() : "null context";
}

extern "C" int64_t pg_ctx_launches(const pg_ctx *ctx) { return ctx ? ctx->launches : 0; }

pg_status pg_alloc(pg_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return pg_fail(ctx, PG_ERR_BUDGET, "scratch of %zu bytes exceeds the HBM budget "
                       "(%zu in use of %zu)", bytes, ctx->in_use, ctx->budget);
    cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return pg_cuda_fail(ctx, e, "cudaMallocAsync");
    }
    ctx->in_use += bytes;
    return PG_OK;
}

void pg_free(pg_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    cudaFreeAsync(p, ctx->stream);
    ctx->in_use -= bytes;
}

pg_status pg_sync_check(pg_ctx *ctx, const char *where) {
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_err, ctx->d_err, 4 * sizeof(int),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PG_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int err[4];
    memcpy(err, ctx->h_err, sizeof err);
    ctx->last_derr = err[0];
    if (err[0] != DERR_NONE) {
        long long info = (long long)(unsigned)err[2] | ((long long)err[3] << 32);
        ctx->last_err_info = info;
        PG_TRY_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, 4 * sizeof(int), ctx->stream));
        PG_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        switch (err[0]) {
        case DERR_BAD_ID:
            return pg_fail(ctx, PG_ERR_DEVICE_CHECK, "%s: id out of range at %lld", where, info);
        case DERR_CAPACITY:
            return pg_fail(ctx, PG_ERR_CAPACITY, "%s: capacity exceeded (%lld)", where, info);
        case DERR_TIMEOUT:
            return pg_fail(ctx, PG_ERR_TIMEOUT, "%s: a bounded device wait expired (block %lld)",
                           where, info);
        case DERR_NO_SLOT:
            return pg_fail(ctx, PG_ERR_CAPACITY,
                           "%s: connectivity found no reached node with a free slot "
                           "(unreached node %lld)", where, info);
        default:
            return pg_fail(ctx, PG_ERR_INTERNAL, "%s: internal device check %d (%lld)", where,
                           err[0], info);
        }
    }
    return PG_OK;
}

extern "C" pg_status pg_ctx_sync(pg_ctx *ctx) {
    if (!ctx) return PG_ERR_INVALID_ARG;
    return pg_sync_check(ctx, "pg_ctx_sync");
}

pg_status pg_reset_counters(pg_ctx *ctx) {
    PG_TRY_CUDA(ctx, cudaMemsetAsync(ctx->d_counters, 0,
                                     PG_CNT_SLOTS * sizeof(unsigned long long), ctx->stream));
    return PG_OK;
}

pg_status pg_read_counters(pg_ctx *ctx, unsigned long long *host32) {
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, ctx->d_counters,
                                     PG_CNT_SLOTS * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PG_TRY(pg_sync_check(ctx, "counters"));
    memcpy(host32, ctx->h_pinned, PG_CNT_SLOTS * sizeof(unsigned long long));
    return PG_OK;
}

// ------------------------------------------------------------ data facts
// Per block: [0] all integer-valued (1/0), [1] min, [2] max, [3] max row norm^2
__global__ void k_data_facts(const float *__restrict__ D, int64_t n, int d, float *blk_out) {
    __shared__ float s_min[8], s_max[8], s_nrm[8];
    __shared__ int s_int[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float mn = INFINITY, mx = -INFINITY, nrm = 0.f;
    int integral = 1;
    // one warp per row, grid-stride over rows
    for (int64_t r = (int64_t)blockIdx.x * 8 + wid; r < n; r += (int64_t)gridDim.x * 8) {
        const float *row = D + r * d;
        float acc = 0.f;
        for (int c = lane; c < d; c += 32) {
            float x = row[c];
            mn = fminf(mn, x);
            mx = fmaxf(mx, x);
            acc = fmaf(x, x, acc);
            if (x != rintf(x)) integral = 0;
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        nrm = fmaxf(nrm, acc);
    }
    for (int o = 16; o; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        nrm = fmaxf(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
        integral &= __shfl_xor_sync(0xffffffffu, integral, o);
    }
    if (lane == 0) {
        s_min[wid] = mn;
        s_max[wid] = mx;
        s_nrm[wid] = nrm;
        s_int[wid] = integral;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            mn = fminf(mn, s_min[w]);
            mx = fmaxf(mx, s_max[w]);
            nrm = fmaxf(nrm, s_nrm[w]);
            integral &= s_int[w];
        }
        blk_out[blockIdx.x * 4 + 0] = (float)integral;
        blk_out[blockIdx.x * 4 + 1] = mn;
        blk_out[blockIdx.x * 4 + 2] = mx;
        blk_out[blockIdx.x * 4 + 3] = nrm;
    }
}

DataFacts pg_reduce_facts(const float *blk, int blocks, int64_t n, int32_t d, pg_metric metric) {
    int integral = 1;
    float mn = INFINITY, mx = -INFINITY, nrm = 0.f;
    for (int b = 0; b < blocks; ++b) {
        integral &= blk[b * 4] != 0.f;
        mn = fminf(mn, blk[b * 4 + 1]);
        mx = fmaxf(mx, blk[b * 4 + 2]);
        nrm = fmaxf(nrm, blk[b * 4 + 3]);
    }
    DataFacts f;
    f.max_norm2 = nrm;
    f.max_abs = fmaxf(fabsf(mn), fabsf(mx));
    f.min_v = mn;
    f.max_v = mx;
    // Exact FP32 distances need integer rows whose every partial sum stays
    // below 2^24: d*(max-min)^2 for the difference form, 2*d*max|x|^2 for
    // the norm form |x|^2 + |y|^2 - 2<x,y>.
    const double range = (double)mx - (double)mn;
    const double lim = 16777216.0;
    f.bf16_exact = integral && f.max_abs <= 256.f;
    f.u8_exact = integral && n > 0 && mn >= 0.f && mx <= 255.f;
    f.exact = metric == PG_METRIC_L2SQ && integral && n > 0 && (double)d * range * range < lim &&
              2.0 * (double)d * (double)f.max_abs * (double)f.max_abs < lim;
    return f;
}

pg_status pg_data_facts(pg_ctx *ctx, const float *D, int64_t n, int32_t d, pg_metric metric,
                        DataFacts *out) {
    int blocks = ctx->num_sms * 4;
    Scratch<float> blk;
    PG_TRY(blk.alloc(ctx, (size_t)blocks * 4));
    k_data_facts<<<blocks, 256, 0, ctx->stream>>>(D, n, d, blk.p);
    PG_LAUNCHED(ctx);
    std::vector<float> h((size_t)blocks * 4);
    PG_TRY_CUDA(ctx, cudaMemcpyAsync(h.data(), blk.p, h.size() * sizeof(float),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PG_TRY(pg_sync_check(ctx, "data facts"));
    *out = pg_reduce_facts(h.data(), blocks, n, d, metric);
    return PG_OK;
}

pg_status pg_query_facts(pg_ctx *ctx, const float *Q, int64_t nq, int32_t d, pg_metric metric,
                         DataFacts *f) {
    if (nq <= 0) return PG_OK;
    DataFacts fq;
    PG_TRY(pg_data_facts(ctx, Q, nq, d, metric, &fq));
    const double lo = std::min(f->min_v, fq.min_v), hi = std::max(f->max_v, fq.max_v);
    const double mab = std::max(f->max_abs, fq.max_abs);
    f->exact = f->exact && fq.exact && (double)d * (hi - lo) * (hi - lo) < 16777216.0 &&
               2.0 * (double)d * mab * mab < 16777216.0;
    f->bf16_exact = f->bf16_exact && fq.bf16_exact;
    f->u8_exact = f->u8_exact && fq.u8_exact;
    f->max_norm2 = std::max(f->max_norm2, fq.max_norm2);
    f->max_abs = (float)mab;
    f->min_v = (float)lo;
    f->max_v = (float)hi;
    return PG_OK;
}

bool pg_u8_usable(const DataFacts &f, pg_metric metric, int d, pg_precision precision) {
    return precision == PG_PREC_BF16_SCREEN && metric == PG_METRIC_L2SQ && f.exact && f.u8_exact &&
           d % 16 == 0;
}

__global__ void k_to_u8(const float *__restrict__ D, int64_t count, uint8_t *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // 4 values per thread
    if (t * 4 >= count) return;
    const float4 v = reinterpret_cast<const float4 *>(D)[t];
    const unsigned w = (unsigned)v.x | ((unsigned)v.y << 8) | ((unsigned)v.z << 16) |
                       ((unsigned)v.w << 24);
    reinterpret_cast<unsigned *>(out)[t] = w;
}

pg_status pg_make_u8(pg_ctx *ctx, const float *D, int64_t n, int32_t d, Scratch<uint8_t> &out) {
    const int64_t count = n * d;  // d % 16 == 0
    PG_TRY(out.alloc(ctx, (size_t)count));
    k_to_u8<<<(unsigned)((count / 4 + 255) / 256), 256, 0, ctx->stream>>>(D, count, out.p);
    PG_LAUNCHED(ctx);
    return PG_OK;
}

ErrModel pg_err_model(pg_metric metric, int d, const DataFacts &f, bool gemm_form) {
    ErrModel m;
    const double u = 5.9604644775390625e-08;  // 2^-24
    if (metric == PG_METRIC_L2SQ) {
        m.metric = 0;
        if (f.exact) {
            m.rel = 0.f;
        } else if (gemm_form) {
            // |x|^2+|y|^2-2<x,y>: error relative to |x|^2+|y|^2, not to s;
            // callers of the norm form use a per-pair bound instead.
            m.rel = (float)((d + 8) * u * 1.01 + 1e-12);
        } else {
            // the gathers sum in teams of eight lanes (each lane a strided
            // sequence of at most ceil(d / 8) + 3 terms, then three butterfly
            // additions) or in 32 strided lanes and five additions: at most
            // ceil(d / 8) + 8 roundings on any term's path
            m.rel = (float)((double)((d + 7) / 8 + 8) * u * 1.01 + 1e-12);
        }
    } else {
        m.metric = 1;
        double nm = f.max_norm2 > 0.f ? (double)f.max_norm2 : 1.0;
        m.abs_ = (float)((2.0 * ((d + 7) / 8 + 8) * u * nm + u * (2.0 + 2.0 * nm)) * 1.01 + 1e-12);
    }
    return m;
}
